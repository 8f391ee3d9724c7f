"""The seeded synthetic workloads (paper_0704_0043_gb300/inputs.py) on the CPU:
reproducible from their seeds, and with the shapes and distributions they are
stated to have (arrival rate, request mix, sizes, step counts, Reynolds
numbers), so a bench or test line names a definite input."""
import math

import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs


def test_serving_trace_is_reproducible_and_has_its_stated_mix():
    a = inputs.serving_trace(seed=11, n_requests=2000)
    b = inputs.serving_trace(seed=11, n_requests=2000)
    assert [(t, w.name, w.steps) for t, w in a] == [(t, w.name, w.steps) for t, w in b]
    t = np.array([x for x, _ in a])
    assert (np.diff(t) > 0).all()
    assert 1.0 / np.diff(t).mean() == pytest.approx(200.0, rel=0.08)  # Poisson arrivals at 200 / s
    cav = [w for _, w in a if w.lattice == 2]
    tube = [w for _, w in a if w.lattice == 1]
    assert len(cav) / len(a) == pytest.approx(0.7, abs=0.04)
    assert all(100 <= w.nx <= 1024 and w.nx == w.ny for w in cav)
    assert all(2000.0 <= w.extra["re"] <= 7500.0 for w in cav)
    assert all(800 <= w.nx <= 1_000_000 and w.ny == 1 and 0.25 <= w.rho_right <= 0.5 for w in tube)
    steps = np.array([w.steps for _, w in a])
    assert steps.min() >= 1000 and steps.max() <= 100000
    # log-uniform: the median sits near the geometric mean of the range
    assert np.median(steps) == pytest.approx(math.sqrt(1000 * 100000), rel=0.15)


def test_batched_cavities_are_reproducible_and_in_range():
    a = inputs.batched_cavities()
    b = inputs.batched_cavities()
    assert len(a) == 256 and [w.nx for w in a] == [w.nx for w in b]
    assert all(64 <= w.nx <= 512 and w.nx == w.ny for w in a)
    assert {w.limiters for w in a} == {inputs.LIM_POSITIVITY, inputs.LIM_EHRENFEST, inputs.LIM_MEDIAN}
    assert all(0.5 < w.beta < 1.0 for w in a)


def test_shock_tube_and_rest_states():
    rho, u = inputs.shock_tube(800)
    assert rho.shape == (800,) and (rho[:400] == 1.0).all() and (rho[400:] == 0.5).all() and (u == 0).all()
    rho, ux, uy = inputs.cavity_rest(7, 5, 2.7)
    assert rho.shape == (5, 7) and (rho == 2.7).all() and (ux == 0).all() and (uy == 0).all()


def test_random_populations_positive_unless_kicked():
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = inputs.random_populations(3, 9, 20, 30, w, 0.2)
    assert f.shape == (9, 20, 30) and (f > 0).all()
    assert np.array_equal(f, inputs.random_populations(3, 9, 20, 30, w, 0.2))
    g = inputs.random_populations(3, 9, 20, 30, w, 0.2, neg_frac=0.1)
    frac = (g < 0).any(axis=0).mean()
    assert 0.05 < frac < 0.15


def test_viscosity_conventions():
    # beta = 1 / (6 nu + 1) (c_s^2 = 1/3); the printed beta = 1 / (2 nu + 1) on request
    assert inputs.beta_from_nu(0.1) == pytest.approx(1.0 / 1.6)
    assert inputs.beta_from_nu(0.1, "paper") == pytest.approx(1.0 / 1.2)
    assert inputs.cavity_nu(100, 0.1, 5000.0) == pytest.approx(100 * 0.1 / 5000.0)
