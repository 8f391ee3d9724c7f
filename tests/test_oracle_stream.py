"""Pins of the oracle's free flight and wall rules.

With beta = 0 the LBGK collision is the identity (Sec. 2), so a step is pure
free flight f_k(x + v_k) <- f_k(x) (Sec. 2), and a marked population can be
followed site by site; the velocity table and the opposite map come from the
trigonometric definition of Sec. 4.1, not from the oracle.  Halfway
bounce-back (Sec. 4.4.1) reflects a population leaving the lattice into the
opposite direction at the same site one step later.  Mass conservation,
mirror symmetry and the exact factor-2 scaling of the whole step (every
operation is homogeneous of degree one in f, rho_wall and the thresholds) are
checked on full runs with all limiters on.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_V3, PAPER_W3, PAPER_W9, moments_np, opposite, paper_velocities_d2q9

V9 = paper_velocities_d2q9()
OPP9 = opposite(V9)
ALL = oracle.LIM_POSITIVITY | oracle.LIM_EHRENFEST | oracle.LIM_MEDIAN


def _background(q, ny, nx):
    w = PAPER_W9 if q == 9 else PAPER_W3
    return np.broadcast_to(w.reshape(q, 1, 1), (q, ny, nx)).copy()


@pytest.mark.parametrize("k", range(9))
def test_free_flight_moves_each_direction_by_its_velocity(k):
    nx, ny, eps = 7, 5, 1e-2
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_PERIODIC, beta=0.0)
    f = _background(9, ny, nx)
    bg = f.copy()
    i0, j0 = 2, 3
    f[k, j0, i0] += eps
    for t in range(1, 12):
        f = oracle.step(cfg, f).f
        want = bg.copy()
        want[k, (j0 + t * V9[k, 1]) % ny, (i0 + t * V9[k, 0]) % nx] += eps
        np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_bounce_back_reflects_into_the_opposite_direction(k):
    """A marked population sent straight at a still wall comes back at the same
    site in direction opp(k) and then travels along -v_k."""
    nx, ny, eps = 6, 6, 1e-2
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS, beta=0.0,
                        u_lid=0.0)
    vx, vy = V9[k]
    # start on the wall the population is heading for (a corner for diagonals)
    i0 = nx - 1 if vx > 0 else (0 if vx < 0 else 2)
    j0 = ny - 1 if vy > 0 else (0 if vy < 0 else 2)
    f = _background(9, ny, nx)
    bg = f.copy()
    f[k, j0, i0] += eps
    f = oracle.step(cfg, f).f
    want = bg.copy()
    want[OPP9[k], j0, i0] += eps
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)
    f = oracle.step(cfg, f).f
    want = bg.copy()
    want[OPP9[k], j0 - vy, i0 - vx] += eps
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)


def test_d1q3_free_flight_and_closed_ends():
    n, eps = 9, 1e-2
    cfg = oracle.Config(lattice=oracle.D1Q3, nx=n, ny=1, boundary=oracle.BC_WALLS, beta=0.0)
    f = _background(3, 1, n)
    bg = f.copy()
    f[2, 0, 6] += eps  # right-moving population (v = +1)
    pos, k = 6, 2
    for _ in range(12):
        f = oracle.step(cfg, f).f
        nxt = pos + PAPER_V3[k]
        if 0 <= nxt < n:
            pos = nxt
        else:
            k = 1 if k == 2 else 2  # reflected into the opposite direction
        want = bg.copy()
        want[k, 0, pos] += eps
        np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)


def _perturbed_cavity(nx, ny, seed, rho0=1.0):
    rho, ux, uy = inputs.random_moments(seed, nx, ny, rho0=rho0, drho=0.05, umax=0.05)
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny)
    f = oracle.init(cfg, rho, ux, uy)
    rng = np.random.default_rng(seed + 1)
    return f * (1 + 0.05 * rng.uniform(-1, 1, f.shape))


def test_mass_conserved_in_closed_cavity_with_lid_and_all_limiters():
    """The lid terms of the two diagonal links through the lid cancel at every
    node, bounce-back returns every population, collisions and limiters keep
    rho: total mass is constant up to FP64 rounding."""
    nx, ny = 12, 10
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS, beta=0.95,
                        u_lid=0.1, rho_wall=1.0, limiters=ALL, delta_median=1e-6,
                        delta_ehrenfest=1e-4, k_max=3)
    f = _perturbed_cavity(nx, ny, 7)
    m0 = f.sum()
    acted = 0
    for _ in range(300):
        r = oracle.step(cfg, f)
        f = r.f
        acted += r.stats["n_med"] + r.stats["n_ehr"]
    assert acted > 0
    assert abs(f.sum() - m0) <= 1e-13 * m0
    assert abs(r.stats["mass"] - m0) <= 1e-13 * m0


def test_step_is_homogeneous_of_degree_one_bitwise():
    """Doubling every population, rho_wall and both thresholds doubles the
    next state exactly: no operation of the step carries a hidden scale."""
    nx, ny = 10, 9
    base = dict(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS, beta=0.97,
                u_lid=0.1, limiters=ALL, k_max=4)
    c1 = oracle.Config(rho_wall=1.0, delta_median=1e-5, delta_ehrenfest=1e-4, **base)
    c2 = oracle.Config(rho_wall=2.0, delta_median=2e-5, delta_ehrenfest=2e-4, **base)
    f = _perturbed_cavity(nx, ny, 11)
    rng = np.random.default_rng(3)
    f[rng.integers(1, 9), 4, 4] *= 6.0  # an over-full population: f' < 0 after collision
    f1, f2 = f.copy(), 2 * f
    acted = {"n_pos": 0, "n_med": 0, "n_ehr": 0}
    for _ in range(25):
        r1, r2 = oracle.step(c1, f1), oracle.step(c2, f2)
        f1, f2 = r1.f, r2.f
        for key in acted:
            acted[key] += r1.stats[key]
        np.testing.assert_array_equal(f2, 2 * f1)
        np.testing.assert_array_equal(r2.selected, r1.selected)
    assert all(v > 0 for v in acted.values()), acted


def test_d1q3_tube_mirror_symmetry():
    n = 64
    rho = np.where(np.abs(np.arange(n) - (n - 1) / 2) < 10, 1.0, 0.5)
    cfg = oracle.Config(lattice=oracle.D1Q3, nx=n, ny=1, boundary=oracle.BC_WALLS, beta=0.99,
                        limiters=oracle.LIM_POSITIVITY | oracle.LIM_MEDIAN, delta_median=1e-6)
    f = oracle.init(cfg, rho, np.zeros(n))
    f, st, rc = oracle.run(cfg, f, 150)
    assert rc == 0
    r, u = moments_np(f[:, 0, :], PAPER_V3)
    np.testing.assert_allclose(r, r[::-1], rtol=1e-13)
    np.testing.assert_allclose(u, -u[::-1], rtol=0, atol=1e-13)


def test_d2q9_cavity_mirror_symmetry_without_lid():
    nx, ny = 11, 9
    rng = np.random.default_rng(5)
    rho = 1 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    rho = 0.5 * (rho + rho[:, ::-1])
    ux = 0.03 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.5 * (ux - ux[:, ::-1])
    uy = 0.03 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.5 * (uy + uy[:, ::-1])
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS, beta=0.95,
                        limiters=oracle.LIM_POSITIVITY | oracle.LIM_MEDIAN, delta_median=1e-7)
    f = oracle.init(cfg, rho, ux, uy)
    f, _, _ = oracle.run(cfg, f, 100)
    r, a, b = moments_np(f, V9)
    np.testing.assert_allclose(r, r[:, ::-1], rtol=1e-13)
    np.testing.assert_allclose(a, -a[:, ::-1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b, b[:, ::-1], rtol=0, atol=1e-13)
