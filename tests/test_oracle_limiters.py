"""Pins of the oracle's limiters (Sec. 3) against independent computations.

* every limiter is f -> f* + phi (f - f*) and keeps rho and rho u (Sec. 1,
  Eq. LimGenF); phi = 1 leaves the state untouched, bit for bit;
* positivity rule (Sec. 3.1): the result is the point of the line through f
  and f* closest to f with no negative population, so its smallest population
  is exactly zero, and phi is the largest feasible value;
* median filter (Sec. 3.5, Sec. 4.4 wall rules): the median is compared with
  numpy.median over the stencil, phi with the homothety sqrt(dS_t / dS) of
  Eq. entrHom; a lone spike on a smooth field is the only site filtered (the
  "salt and pepper" case of Sec. 3.5);
* Ehrenfests' trimming (Sec. 3.2, Sec. 4.3.2): the equilibrated set is the k
  largest dS > delta, ties to the lower site index, checked against a
  brute-force sort with planted ties; the chosen sites end at f*;
* dissipativity 0 <= phi <= 1 (Sec. 3.8) and the limiter entropy production
  sum (1 - phi^2) dS (+ phi^2 dS at Ehrenfests' sites) of Sec. 3.4.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_V3, PAPER_W9, moments_np, paper_velocities_d2q9

V9 = paper_velocities_d2q9()
ALL = oracle.LIM_POSITIVITY | oracle.LIM_EHRENFEST | oracle.LIM_MEDIAN


def _cavity_cfg(nx, ny, **kw):
    base = dict(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS, beta=0.97,
                u_lid=0.1, rho_wall=1.0)
    base.update(kw)
    return oracle.Config(**base)


def _noisy_field(nx, ny, seed, eps=0.08, neg_frac=0.0):
    return inputs.random_populations(seed, 9, ny, nx, PAPER_W9, eps, neg_frac=neg_frac)


def _feq_field(f):
    r, a, b = moments_np(f, V9)
    out = np.empty_like(f)
    for j in range(f.shape[1]):
        for i in range(f.shape[2]):
            out[:, j, i] = oracle.feq(oracle.D2Q9, r[j, i], a[j, i], b[j, i])
    return out


def test_limiters_keep_moments_and_phi_in_unit_interval():
    nx, ny = 12, 10
    cfg = _cavity_cfg(nx, ny, limiters=ALL, delta_median=0.0, delta_ehrenfest=1e-3, k_max=5)
    f = _noisy_field(nx, ny, 1, neg_frac=0.1)
    r = oracle.limit(cfg, f, ALL)
    assert r.stats["n_pos"] > 0 and r.stats["n_med"] > 0 and r.stats["n_ehr"] == 5
    m0, m1 = moments_np(f, V9), moments_np(r.f, V9)
    for a, b in zip(m0, m1):
        np.testing.assert_allclose(b, a, rtol=0, atol=2e-15)
    assert (r.phi >= 0).all() and (r.phi <= 1).all()
    # the same through a full step
    s0 = oracle.step(_cavity_cfg(nx, ny), f)          # no limiters: f_out = f'
    s1 = oracle.step(cfg, f)
    for a, b in zip(moments_np(s0.f, V9), moments_np(s1.f, V9)):
        np.testing.assert_allclose(b, a, rtol=0, atol=2e-15)


def test_phi_one_is_the_identity_bitwise():
    nx, ny = 12, 10
    f = _noisy_field(nx, ny, 2)
    plain = oracle.step(_cavity_cfg(nx, ny), f)
    idle = oracle.step(_cavity_cfg(nx, ny, limiters=ALL, delta_median=np.inf,
                                   delta_ehrenfest=np.inf, k_max=10), f)
    assert idle.stats["n_pos"] == 0 and idle.stats["n_med"] == 0 and idle.stats["n_ehr"] == 0
    np.testing.assert_array_equal(idle.f, plain.f)
    assert idle.stats["dS_lim"] == 0.0


def test_positivity_rule_lands_on_the_positivity_boundary():
    nx, ny = 9, 8
    cfg = _cavity_cfg(nx, ny)
    f = _noisy_field(nx, ny, 3, neg_frac=0.3)
    fs = _feq_field(f)
    assert (fs > 0).all()
    r = oracle.limit(cfg, f, oracle.LIM_POSITIVITY)
    neg = (f < 0).any(axis=0)
    assert neg.sum() > 5
    # untouched where nothing was negative
    np.testing.assert_array_equal(r.f[:, ~neg], f[:, ~neg])
    # on the line f* + phi (f - f*), at its first zero crossing
    lam = np.where(f < 0, fs / (fs - f), np.inf).min(axis=0)
    np.testing.assert_allclose(r.phi[neg], lam[neg], rtol=1e-15)
    np.testing.assert_allclose(r.f[:, neg], (fs + lam * (f - fs))[:, neg], rtol=0, atol=1e-16)
    assert r.f.min() >= -1e-17
    np.testing.assert_allclose(r.f[:, neg].min(axis=0), 0.0, atol=1e-17)
    assert r.stats["n_pos"] == neg.sum()


def _stencil(dS, i, j):
    """Wall rules of Sec. 4.4 for walls half a link outside the lattice: a
    node next to one wall uses itself and its two neighbours along that wall,
    a corner node itself and its inward x and y neighbours, every other node
    the 3 x 3 block."""
    ny, nx = dS.shape
    nearx, neary = i in (0, nx - 1), j in (0, ny - 1)
    if nearx and neary:
        ii = 1 if i == 0 else nx - 2
        jj = 1 if j == 0 else ny - 2
        return np.array([dS[j, i], dS[j, ii], dS[jj, i]])
    if neary:
        return dS[j, i - 1:i + 2]
    if nearx:
        return dS[j - 1:j + 2, i]
    return dS[j - 1:j + 2, i - 1:i + 2].ravel()


@pytest.mark.parametrize("mode", [oracle.MEDIAN_THRESHOLD, oracle.MEDIAN_GATE])
@pytest.mark.parametrize("delta", [0.0, 3e-4])
def test_median_filter_matches_numpy_median(mode, delta):
    nx, ny = 11, 9
    cfg = _cavity_cfg(nx, ny, delta_median=delta, median_mode=mode)
    f = _noisy_field(nx, ny, 4, eps=0.05)
    r = oracle.limit(cfg, f, oracle.LIM_MEDIAN)
    dS = r.dS
    want = np.ones_like(dS)
    for j in range(ny):
        for i in range(nx):
            st = _stencil(dS, i, j)
            med = float(np.median(st))
            x = dS[j, i]
            if mode == oracle.MEDIAN_THRESHOLD:
                t = max(med, delta)
                if x > t:
                    want[j, i] = np.sqrt(t / x)
            elif x > delta and med < x:
                want[j, i] = np.sqrt(med / x)
    np.testing.assert_allclose(r.phi, want, rtol=1e-15)
    assert 0 < r.stats["n_med"] == (want < 1).sum()
    fs = _feq_field(f)
    np.testing.assert_allclose(r.f, fs + want * (f - fs), rtol=0, atol=1e-16)


def _field_with_dS(target, seed):
    """A D2Q9 field whose dS equals `target` (up to rounding): one fixed
    nonequilibrium direction d about one f*, scaled per site."""
    base = _noisy_field(1, 1, seed, eps=0.1)
    fs = _feq_field(base)
    d = base - fs
    ds0 = (((d) ** 2) / fs).sum()
    x = np.sqrt(np.asarray(target) / ds0)
    return fs + x[None] * d


def test_median_removes_a_lone_spike_only():
    nx, ny = 12, 10
    flat = np.full((ny, nx), 1e-4)
    flat[5, 6] = 5e-3                             # salt-and-pepper spike
    f = _field_with_dS(flat, 5)
    cfg = _cavity_cfg(nx, ny, delta_median=0.0)
    r = oracle.limit(cfg, f, oracle.LIM_MEDIAN)
    assert r.stats["n_med"] == 1 and r.phi[5, 6] < 1
    # after the homothety the spike carries the median of its 3 x 3 block
    after = oracle.limit(cfg, r.f, 0).dS
    np.testing.assert_allclose(after[5, 6], np.median(r.dS[4:7, 5:8]), rtol=1e-12)
    # on a smooth ramp below the tolerance only the spike is above dS_t
    jj, ii = np.mgrid[0:ny, 0:nx]
    ramp = 1e-4 * (1 + 0.1 * ii + 0.07 * jj)
    ramp[5, 6] = 5e-3
    cfg = _cavity_cfg(nx, ny, delta_median=4e-4)
    r = oracle.limit(cfg, _field_with_dS(ramp, 5), oracle.LIM_MEDIAN)
    assert r.stats["n_med"] == 1 and r.phi[5, 6] < 1
    np.testing.assert_allclose(r.phi[5, 6] ** 2, 4e-4 / r.dS[5, 6], rtol=1e-14)


def test_d1q3_three_point_median_spike():
    n = 40
    target = 1e-5 * (1 + 0.05 * np.arange(n))
    target[17] = 1e-3
    rng = np.random.default_rng(6)
    f0 = np.array([2 / 3, 1 / 6, 1 / 6]) * (1 + 0.1 * rng.uniform(-1, 1, 3))
    fs = oracle.feq(oracle.D1Q3, *moments_np(f0, PAPER_V3))
    d = f0 - fs
    x = np.sqrt(target / ((d ** 2) / fs).sum())
    f = (fs[:, None] + x[None] * d[:, None]).reshape(3, 1, n)
    cfg = oracle.Config(lattice=oracle.D1Q3, nx=n, ny=1, boundary=oracle.BC_WALLS, beta=1.0,
                        delta_median=0.0)
    r = oracle.limit(cfg, f, oracle.LIM_MEDIAN)
    assert r.stats["n_med"] == 1 and r.phi[0, 17] < 1
    np.testing.assert_allclose(r.phi[0, 17] ** 2, max(r.dS[0, 16], r.dS[0, 18]) / r.dS[0, 17],
                               rtol=1e-14)


def test_ehrenfests_top_k_with_ties_matches_brute_force():
    nx, ny, k = 12, 10, 7
    f = _noisy_field(nx, ny, 7, eps=0.1)
    dS0 = oracle.limit(_cavity_cfg(nx, ny), f, 0).dS.ravel()
    order = np.argsort(-dS0, kind="stable")
    # plant exact ties with the 3rd largest site at lower and higher indices
    src = order[2]
    for dst in (order[40], order[50], order[60]):
        f[:, dst // nx, dst % nx] = f[:, src // nx, src % nx]
    delta = float(np.sort(dS0)[len(dS0) // 2])
    cfg = _cavity_cfg(nx, ny, delta_ehrenfest=delta, k_max=k)
    r = oracle.limit(cfg, f, oracle.LIM_EHRENFEST)
    dS = r.dS.ravel()
    cands = [s for s in range(nx * ny) if dS[s] > delta]
    want = sorted(cands, key=lambda s: (-dS[s], s))[:k]
    assert list(r.selected) == want
    assert r.stats["n_cand"] == len(cands)
    tied = [s for s in range(nx * ny) if dS[s] == dS[src]]
    assert len(tied) == 4
    # the chosen sites are at equilibrium afterwards, the others untouched
    after = oracle.limit(cfg, r.f, 0).dS.ravel()
    assert after[want].max() < 1e-28
    rest = np.setdiff1d(np.arange(nx * ny), want)
    np.testing.assert_array_equal(r.f.reshape(9, -1)[:, rest], f.reshape(9, -1)[:, rest])
    # threshold is strict and k larger than the candidate count takes them all
    cfg2 = _cavity_cfg(nx, ny, delta_ehrenfest=float(dS[want[0]]), k_max=10 ** 6)
    r2 = oracle.limit(cfg2, f, oracle.LIM_EHRENFEST)
    assert want[0] not in list(r2.selected)
    assert list(r2.selected) == sorted([s for s in range(nx * ny) if dS[s] > dS[want[0]]],
                                       key=lambda s: (-dS[s], s))


def test_limiter_entropy_production_bookkeeping():
    nx, ny = 12, 10
    cfg = _cavity_cfg(nx, ny, limiters=ALL, delta_median=1e-5, delta_ehrenfest=2e-3, k_max=4)
    f = _noisy_field(nx, ny, 8, eps=0.1, neg_frac=0.05)
    r = oracle.step(cfg, f)
    sel = np.zeros(nx * ny, bool)
    sel[r.selected] = True
    phi, dS = r.phi.ravel(), r.dS.ravel()
    want = ((1 - phi ** 2) * dS).sum() + ((phi ** 2) * dS)[sel].sum()
    assert r.stats["dS_lim"] >= 0
    np.testing.assert_allclose(r.stats["dS_lim"], want, rtol=1e-13)
    np.testing.assert_allclose(r.stats["sum_dS"], dS.sum(), rtol=1e-13)
    assert r.stats["n_ehr"] == len(r.selected) == 4
    np.testing.assert_allclose(r.stats["mass"], f.sum(), rtol=1e-14)
