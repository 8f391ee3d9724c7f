"""Pins of the oracle's entropic quasiequilibria (Eq. entropiceq1d, Eq. maxwellian)
and its exact nonequilibrium entropy (Eq. DelS), against properties the
mathematics fixes rather than a second copy of the formulas:

* f* has the moments it is built from (Eq. macro_dis), and f*(rho, 0) = rho W;
* f* is the conditional maximum of the lattice entropy of Sec. 4.1: ln(f*_k / W_k)
  lies in the span of the collision invariants {1, v_x, v_y} (Lagrange condition),
  and every moment-preserving perturbation lowers S;
* the D2Q9 formula is the tensor product of the D1Q3 one (W_k = W_{k_x} W_{k_y}
  and the product over j of Eq. maxwellian), which ties the two printed formulas
  together and fixes the velocity sign of the D1Q3 movers;
* dS = S(f*) - S(f) for f with the moments of f* (Eq. DelS, with S computed from
  the weights W, not from f*); dS >= 0 (Gibbs); dS -> half the quadratic form for
  small deviations (the quadratic approximation of Sec. 3.6);
* the step: entropic f* is a fixed point of the collision; mass is conserved; the
  statistics equal entropy differences S(f') - S(f_in) computed from S; the
  Ehrenfests' sites end at the entropic f* of their own moments.
"""
import math

import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_V3, PAPER_W3, PAPER_W9, moments_np, paper_velocities_d2q9

V9 = paper_velocities_d2q9()


def _invariants(lattice):
    if lattice == oracle.D1Q3:
        return np.stack([np.ones(3), PAPER_V3.astype(float)])
    return np.stack([np.ones(9), V9[:, 0].astype(float), V9[:, 1].astype(float)])


def _random_states(n, seed, umax=0.6):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.3, 3.0, n), rng.uniform(-umax, umax, n), rng.uniform(-umax, umax, n)


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_entropic_feq_has_its_moments(lattice):
    rho, ux, uy = _random_states(200, 1, umax=0.9)
    for r, a, b in zip(rho, ux, uy):
        if lattice == oracle.D1Q3:
            b = 0.0
        f = oracle.feq_entropic(lattice, r, a, b)
        assert f is not None and (f > 0).all()
        m = _invariants(lattice) @ f
        assert m[0] == pytest.approx(r, rel=1e-14)
        assert m[1] == pytest.approx(r * a, abs=1e-14 * r)
        if lattice == oracle.D2Q9:
            assert m[2] == pytest.approx(r * b, abs=1e-14 * r)


def test_entropic_feq_at_rest_is_rho_w():
    for r in (0.5, 1.0, 2.7):
        assert np.array_equal(oracle.feq_entropic(oracle.D2Q9, r, 0.0, 0.0), r * PAPER_W9)
        np.testing.assert_allclose(oracle.feq_entropic(oracle.D1Q3, r, 0.0), r * PAPER_W3, rtol=2e-16, atol=0)


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_entropic_feq_satisfies_the_lagrange_condition(lattice):
    # conditional entropy maximum: ln(f*_k / W_k) = mu . (1, v_k)  (Sec. 3.6)
    W = PAPER_W3 if lattice == oracle.D1Q3 else PAPER_W9
    M = _invariants(lattice).T
    rho, ux, uy = _random_states(100, 2, umax=0.8)
    for r, a, b in zip(rho, ux, uy):
        f = oracle.feq_entropic(lattice, r, a, 0.0 if lattice == oracle.D1Q3 else b)
        y = np.log(f / W)
        mu, *_ = np.linalg.lstsq(M, y, rcond=None)
        assert np.abs(M @ mu - y).max() < 1e-14


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_entropic_feq_maximises_the_entropy(lattice):
    rng = np.random.default_rng(3)
    M = _invariants(lattice)
    _, _, vt = np.linalg.svd(M)
    null = vt[M.shape[0]:]  # moment-preserving directions
    rho, ux, uy = _random_states(40, 4)
    for r, a, b in zip(rho, ux, uy):
        f = oracle.feq_entropic(lattice, r, a, 0.0 if lattice == oracle.D1Q3 else b)
        s0 = oracle.entropy(lattice, f)
        for _ in range(5):
            d = rng.standard_normal(null.shape[0]) @ null
            for eps in (1e-3, -1e-3):
                g = f + eps * f.min() * d / np.abs(d).max()
                assert oracle.entropy(lattice, g) < s0


def test_d2q9_entropic_feq_is_the_tensor_product_of_d1q3():
    rho, ux, uy = _random_states(100, 5, umax=0.9)
    for r, a, b in zip(rho, ux, uy):
        fx = oracle.feq_entropic(oracle.D1Q3, 1.0, a)
        fy = oracle.feq_entropic(oracle.D1Q3, 1.0, b)
        f = oracle.feq_entropic(oracle.D2Q9, r, a, b)
        ix = [0 if v == 0 else (1 if v < 0 else 2) for v in V9[:, 0]]
        iy = [0 if v == 0 else (1 if v < 0 else 2) for v in V9[:, 1]]
        expect = r * fx[ix] * fy[iy]
        np.testing.assert_allclose(f, expect, rtol=1e-12, atol=0)  # the D1Q3 movers cancel at |u| -> 1


def test_entropic_feq_exists_only_inside_the_velocity_hull():
    assert oracle.feq_entropic(oracle.D1Q3, 1.0, 1.0) is None
    assert oracle.feq_entropic(oracle.D1Q3, 1.0, -1.2) is None
    assert oracle.feq_entropic(oracle.D2Q9, 1.0, 0.2, 1.0) is None
    assert oracle.feq_entropic(oracle.D2Q9, 1.0, -1.0, 0.0) is None
    assert oracle.feq_entropic(oracle.D2Q9, 1.0, 0.99, -0.99) is not None


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_relative_entropy_is_the_entropy_difference(lattice):
    # Eq. DelS: dS = S(f*) - S(f) when f and f* share their moments
    rng = np.random.default_rng(6)
    M = _invariants(lattice)
    _, _, vt = np.linalg.svd(M)
    null = vt[M.shape[0]:]
    rho, ux, uy = _random_states(60, 7)
    for r, a, b in zip(rho, ux, uy):
        fs = oracle.feq_entropic(lattice, r, a, 0.0 if lattice == oracle.D1Q3 else b)
        d = rng.standard_normal(null.shape[0]) @ null
        f = fs + 0.3 * fs.min() * d / np.abs(d).max()
        ds = oracle.rel_entropy(f, fs)
        ref = oracle.entropy(lattice, fs) - oracle.entropy(lattice, f)
        assert ds > 0
        assert ds == pytest.approx(ref, abs=2e-14 * r)


def test_relative_entropy_is_nonnegative_and_quadratic_for_small_deviations():
    rng = np.random.default_rng(8)
    M = _invariants(oracle.D2Q9)
    _, _, vt = np.linalg.svd(M)
    null = vt[3:]
    fs = oracle.feq_entropic(oracle.D2Q9, 1.2, 0.1, -0.05)
    assert oracle.rel_entropy(fs, fs) == 0.0
    for _ in range(20):
        d = rng.standard_normal(6) @ null
        d *= fs.min() / np.abs(d).max()
        q = ((d ** 2) / fs).sum()
        for eps in (1e-2, 1e-3):
            x = oracle.rel_entropy(fs + eps * d, fs)
            assert x > 0
            # sum f ln(f/f*) = sum (f - f*)^2 / (2 f*) + O(eps^3)
            assert x / (eps * eps) == pytest.approx(0.5 * q, rel=3 * eps)


def test_relative_entropy_domain_conventions():
    fs = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = fs.copy()
    f[3] = -1e-300
    assert oracle.rel_entropy(f, fs) == math.inf
    f[3] = 0.0
    f[1] += fs[3]  # keep the mass
    assert math.isfinite(oracle.rel_entropy(f, fs))


def _periodic_cfg(nx, ny, **kw):
    base = dict(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_PERIODIC, beta=0.9,
                equilibrium=oracle.EQ_ENTROPIC)
    base.update(kw)
    return oracle.Config(**base)


def test_entropic_equilibrium_is_a_fixed_point_of_the_step():
    cfg = _periodic_cfg(6, 5)
    rho = np.full(cfg.sites, 1.3)
    f0 = oracle.init(cfg, rho, np.full(cfg.sites, 0.12), np.full(cfg.sites, -0.07))
    r = oracle.step(cfg, f0)
    np.testing.assert_allclose(r.f, f0, rtol=4e-15, atol=0)
    assert np.abs(r.dS).max() < 1e-15


def test_entropic_init_is_entropic_feq_per_site():
    cfg = _periodic_cfg(4, 3)
    rng = np.random.default_rng(9)
    rho, ux, uy = rng.uniform(0.5, 2, 12), rng.uniform(-0.3, 0.3, 12), rng.uniform(-0.3, 0.3, 12)
    f = oracle.init(cfg, rho, ux, uy).reshape(9, -1)
    for s in range(12):
        assert np.array_equal(f[:, s], oracle.feq_entropic(oracle.D2Q9, rho[s], ux[s], uy[s]))


def _pull_periodic(f):
    return np.stack([np.roll(f[k], (V9[k, 1], V9[k, 0]), axis=(0, 1)) for k in range(9)])


def test_entropic_step_statistics_are_entropy_differences():
    # periodic lattice, no limiters: f_in is a roll of f; the collision's entropy
    # production is S(f') - S(f_in) summed over sites, with S from the weights W
    cfg = _periodic_cfg(7, 6, beta=0.8)
    f = inputs.random_populations(10, 9, 6, 7, PAPER_W9, 0.2)
    r = oracle.step(cfg, f)
    fin = _pull_periodic(f)
    a = 2 * cfg.beta - 1
    s_lbgk = 0.0
    s_sum = 0.0
    for j in range(6):
        for i in range(7):
            x = fin[:, j, i]
            rho, ux, uy = oracle.site_moments(oracle.D2Q9, x)
            fs = oracle.feq_entropic(oracle.D2Q9, rho, ux, uy)
            fp = fs + a * (fs - x)
            s_lbgk += oracle.entropy(oracle.D2Q9, fp) - oracle.entropy(oracle.D2Q9, x)
            s_sum += oracle.entropy(oracle.D2Q9, fs) - oracle.entropy(oracle.D2Q9, fp)
            np.testing.assert_allclose(r.f[:, j, i], fp, rtol=1e-15, atol=1e-17)
    assert r.stats["dS_lbgk"] > 0
    assert r.stats["dS_lbgk"] == pytest.approx(s_lbgk, rel=1e-9)
    assert r.stats["sum_dS"] == pytest.approx(s_sum, rel=1e-9)
    assert r.stats["mass"] == pytest.approx(f.sum(), rel=1e-15)


def test_entropic_step_conserves_mass_in_the_cavity():
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=12, ny=10, boundary=oracle.BC_WALLS, beta=0.95,
                        u_lid=0.1, rho_wall=1.0, equilibrium=oracle.EQ_ENTROPIC,
                        limiters=oracle.LIM_MEDIAN | oracle.LIM_POSITIVITY)
    f = oracle.init(cfg, np.ones(cfg.sites), np.zeros(cfg.sites), np.zeros(cfg.sites))
    m0 = f.sum()
    f2, st, rc = oracle.run(cfg, f, 200)
    assert rc == 0
    assert f2.sum() == pytest.approx(m0, rel=1e-13)
    rho, ux, uy = oracle.moments(cfg, f2)
    assert ux[-1].mean() > 0.01  # the lid drags the top row


def test_entropic_ehrenfest_sites_end_at_their_entropic_feq_and_add_their_entropy():
    cfg = _periodic_cfg(9, 8, beta=0.95, limiters=oracle.LIM_EHRENFEST, k_max=5, delta_ehrenfest=1e-4)
    f = inputs.random_populations(11, 9, 8, 9, PAPER_W9, 0.25)
    r = oracle.step(cfg, f)
    assert len(r.selected) == 5
    free = oracle.step(oracle.Config(**{**cfg.__dict__, "limiters": 0}), f)
    order = sorted(range(cfg.sites), key=lambda s: (-free.dS.reshape(-1)[s], s))
    assert list(r.selected) == [s for s in order if free.dS.reshape(-1)[s] > 1e-4][:5]
    add = 0.0
    out = r.f.reshape(9, -1)
    pre = free.f.reshape(9, -1)
    for s in r.selected:
        rho, ux, uy = oracle.site_moments(oracle.D2Q9, pre[:, s])
        fs = oracle.feq_entropic(oracle.D2Q9, rho, ux, uy)
        assert np.array_equal(out[:, s], fs)
        add += oracle.entropy(oracle.D2Q9, fs) - oracle.entropy(oracle.D2Q9, pre[:, s])
    assert r.stats["dS_lim"] == pytest.approx(add, rel=1e-9)


def test_entropic_negative_population_gives_infinite_dS_without_flagging():
    cfg = _periodic_cfg(6, 6, beta=1.0, limiters=oracle.LIM_POSITIVITY | oracle.LIM_MEDIAN)
    f = inputs.random_populations(12, 9, 6, 6, PAPER_W9, 0.9)
    r = oracle.step(cfg, f)
    free = oracle.step(oracle.Config(**{**cfg.__dict__, "limiters": 0}), f)
    neg = (free.f < 0).any(axis=0)
    assert neg.any() and r.rc == 0 and r.stats["n_bad"] == 0
    assert np.isinf(r.dS[neg]).all() and np.isfinite(r.dS[~neg]).all()
    assert r.f.min() >= -1e-16
    assert r.stats["n_pos"] == neg.sum()


def test_entropic_site_without_equilibrium_is_flagged():
    cfg = _periodic_cfg(4, 4, beta=0.9)
    f = oracle.init(cfg, np.ones(16), np.zeros(16), np.zeros(16))
    f[3, 2, 2] = -0.6  # arrives at (1, 2) with rho = 0.289, u_x = 2.46
    r = oracle.step(cfg, f)
    assert r.rc == 1 and r.stats["n_bad"] >= 1


def test_entropic_shock_tube_keeps_mass_and_mirror_symmetry():
    # D1Q3 closed tube, mirror-symmetric density step: the entropic step keeps
    # the mirror image f_left(x) = f_right(n - 1 - x) and the total mass
    n = 64
    cfg = oracle.Config(lattice=oracle.D1Q3, nx=n, ny=1, boundary=oracle.BC_WALLS, beta=0.999,
                        equilibrium=oracle.EQ_ENTROPIC, limiters=oracle.LIM_POSITIVITY | oracle.LIM_MEDIAN)
    x = np.arange(n)
    rho = np.where((x < n // 4) | (x >= n - n // 4), 1.0, 0.5)
    f = oracle.init(cfg, rho, np.zeros(n))
    m0 = f.sum()
    f2, st, rc = oracle.run(cfg, f, 40)
    assert rc == 0
    assert f2.sum() == pytest.approx(m0, rel=1e-14)
    f2 = f2.reshape(3, n)
    np.testing.assert_allclose(f2[1], f2[2][::-1], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f2[0], f2[0][::-1], rtol=1e-12, atol=1e-15)
