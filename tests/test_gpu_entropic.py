"""Parity of the entropic-quasiequilibrium path (LBM_EQ_ENTROPIC, FP64 storage)
with the FP64 oracle, through the C ABI.

Both sides evaluate f* (Eq. entropiceq1d / Eq. maxwellian) with the same
correctly rounded operations (sqrt, division, products) in the same order, so
f* and the collision f' agree bit for bit.  The exact nonequilibrium entropy of
Eq. DelS takes one logarithm per population, and the device and host logarithms
are each within an ulp or so of the true value but not bitwise equal.  The
tolerance on dS at a site is therefore derived from its terms:

    |dS_gpu - dS_oracle| <= 16 eps * (sum_k |f'_k ln(f'_k / f*_k)| + dS) + 2 eps * sum_k f'_k,

eps = 2^-52.  The last term is the oracle's rounding of the ratio f'_k / f*_k
before its logarithm (an absolute error of up to eps in each logarithm); the
device evaluates ln(f'_k / f*_k) near 1 without forming the ratio.

and populations after the limiters (whose homothety factors sqrt(dS_t / dS)
inherit that error) are compared to 1e-12 absolute, far below the 1e-6 and
larger shifts a wrong term, sign or index produces.  Each step is compared from
the same stored state (the GPU lattice is reset to the oracle's state before
every step), so the comparison is one step deep; a separate run compares 300
unsynchronised cavity steps.  Counts and Ehrenfests' sets must be identical.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W3 = np.array([2 / 3, 1 / 6, 1 / 6])
EPS = 2.0 ** -52


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0704_0043_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pair(**cfg):
    cfg = dict(cfg, precision=lbm.FP64, equilibrium=lbm.EQ_ENTROPIC)
    g = lbm.Lattice(**cfg)
    c = g.config
    oc = oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta,
                       u_lid=c.u_lid, rho_wall=c.rho_wall, limiters=c.limiters,
                       delta_median=c.delta_median, delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max,
                       median_mode=c.median_mode, equilibrium=oracle.EQ_ENTROPIC)
    return g, oc


def rand_state(q, ny, nx, seed, eps=0.15, neg_frac=0.0, heavy=0):
    w = W9 if q == 9 else W3
    f = inputs.random_populations(seed, q, ny, nx, w, eps, neg_frac=neg_frac)
    rng = np.random.default_rng(seed + 99)
    for _ in range(heavy):
        j, i = rng.integers(0, ny), rng.integers(0, nx)
        if q == 9:
            f[rng.integers(1, 9), j, i] *= 4.0
        else:
            f[0, j, i] *= 0.3
    return f


def ds_bound(oc, f):
    """Per-site tolerance on dS(f') of the next collision (see the module docstring)."""
    free = oracle.step(dataclasses.replace(oc, limiters=0), f)
    q = oc.q
    fp = free.f.reshape(q, -1)
    ds = free.dS.reshape(-1)
    out = np.zeros(oc.sites)
    for s in range(oc.sites):
        if not np.isfinite(ds[s]):
            continue
        rho, ux, uy = oracle.site_moments(oc.lattice, fp[:, s])
        fs = oracle.feq_entropic(oc.lattice, rho, ux, uy)
        x = fp[:, s]
        pos = x > 0
        t = np.abs(x[pos] * np.log(x[pos] / fs[pos])).sum()
        out[s] = 16 * EPS * (t + abs(ds[s])) + 2 * EPS * x[pos].sum() + 1e-300
    return out.reshape(oc.ny, oc.nx), free.dS


def assert_ds_close(got, want, bound):
    inf = ~np.isfinite(want)
    np.testing.assert_array_equal(~np.isfinite(got), inf)
    np.testing.assert_array_equal(got[inf], want[inf])
    err = np.abs(got[~inf] - want[~inf])
    assert (err <= bound[~inf]).all(), (err.max(), (err / bound[~inf]).max())


def stats_close(a, b):
    for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
        assert abs(a[key] - b[key]) <= 1e-10 * abs(b[key]) + 1e-13, (key, a[key], b[key])
    for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
        assert a[key] == b[key], (key, a[key], b[key])


CASES = [
    dict(lattice=lbm.D2Q9, nx=67, ny=41, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1,
         limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=7),
    dict(lattice=lbm.D2Q9, nx=45, ny=20, boundary=lbm.BC_CHANNEL, beta=0.9, u_lid=0.05,
         rho_wall=1.3, limiters=ALL, delta_median=0.0, delta_ehrenfest=1e-3, k_max=5),
    dict(lattice=lbm.D2Q9, nx=33, ny=13, boundary=lbm.BC_PERIODIC, beta=0.99, limiters=ALL,
         delta_median=1e-5, delta_ehrenfest=1e-3, k_max=9, median_mode=lbm.MEDIAN_GATE),
    dict(lattice=lbm.D2Q9, nx=4, ny=4, boundary=lbm.BC_WALLS, beta=0.95, u_lid=0.1, limiters=ALL,
         delta_median=0.0, delta_ehrenfest=1e-4, k_max=2),
    dict(lattice=lbm.D1Q3, nx=600, ny=1, boundary=lbm.BC_WALLS, beta=0.999, limiters=ALL,
         delta_median=1e-6, delta_ehrenfest=1e-3, k_max=4),
    dict(lattice=lbm.D1Q3, nx=517, ny=1, boundary=lbm.BC_PERIODIC, beta=0.8, limiters=ALL,
         delta_median=0.0, delta_ehrenfest=5e-4, k_max=3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_entropic_steps_match_oracle(case):
    g, oc = pair(**CASES[case])
    cur = rand_state(g.q, g.ny, g.nx, 20 + case, neg_frac=0.02, heavy=max(1, g.sites // 200))
    acted = {"n_pos": 0, "n_med": 0, "n_ehr": 0}
    saw_inf = False
    for step in range(8):
        g.set_populations(cur)
        bound, want_ds = ds_bound(oc, cur)
        assert_ds_close(g.delta_s(), want_ds, bound)
        saw_inf |= bool(np.isinf(want_ds).any())
        g.step(1)
        r = oracle.step(oc, cur)
        got = g.get_populations()
        np.testing.assert_allclose(got, r.f, rtol=0, atol=1e-12, err_msg=f"step {step}")
        stats_close(g.stats(), r.stats)
        np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
        for k in acted:
            acted[k] += r.stats[k]
        cur = r.f
    assert acted["n_med"] > 0 and acted["n_ehr"] > 0, acted
    if CASES[case]["beta"] > 0.9:
        # sites with a negative post-collision population (dS = +inf) were exercised
        assert acted["n_pos"] > 0 and saw_inf, acted


def test_entropic_init_is_bitwise_and_rest_is_a_fixed_point():
    g, oc = pair(lattice=lbm.D2Q9, nx=70, ny=38, boundary=lbm.BC_PERIODIC, beta=0.96)
    rho, ux, uy = inputs.random_moments(3, 70, 38, umax=0.3)
    g.init(rho, ux, uy)
    np.testing.assert_array_equal(g.get_populations(), oracle.init(oc, rho, ux, uy))
    g1, oc1 = pair(lattice=lbm.D1Q3, nx=301, ny=1, boundary=lbm.BC_PERIODIC, beta=0.9)
    r1, u1, _ = inputs.random_moments(4, 301, 1, umax=0.5)
    g1.init(r1, u1)
    np.testing.assert_array_equal(g1.get_populations(), oracle.init(oc1, r1, u1))
    # a uniform entropic equilibrium stays put
    n = 70 * 38
    g.init(np.full(n, 1.2), np.full(n, 0.05), np.full(n, -0.1))
    f0 = g.get_populations()
    g.step(3)
    np.testing.assert_allclose(g.get_populations(), f0, rtol=4e-15, atol=0)


def test_entropic_limit_pass_matches_oracle():
    g, oc = pair(lattice=lbm.D2Q9, nx=50, ny=29, boundary=lbm.BC_WALLS, beta=0.96, u_lid=0.1,
                 limiters=ALL, delta_median=0.0, delta_ehrenfest=1e-3, k_max=11)
    f = rand_state(9, 29, 50, 4, eps=0.25, neg_frac=0.03)
    g.set_populations(f)
    g.limit(ALL)
    r = oracle.limit(oc, f, ALL)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=0, atol=1e-12)
    stats_close(g.stats(), r.stats)
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))


def test_entropic_cavity_run_tracks_oracle():
    # 300 unsynchronised steps of a 64^2 lid-driven cavity, median filter on
    cfg = dict(lattice=lbm.D2Q9, nx=64, ny=64, boundary=lbm.BC_WALLS, beta=1.0 / (6 * 0.0064 + 1),
               u_lid=0.1, limiters=lbm.LIM_MEDIAN, delta_median=1e-3)
    g, oc = pair(**cfg)
    n = 64 * 64
    g.init(np.ones(n), np.zeros(n), np.zeros(n))
    f = oracle.init(oc, np.ones(n), np.zeros(n), np.zeros(n))
    g.step(300)
    f, st, rc = oracle.run(oc, f, 300)
    assert rc == 0
    rho, ux, uy = g.moments()
    orho, oux, ouy = oracle.moments(oc, f)
    np.testing.assert_allclose(rho, orho, rtol=0, atol=1e-11)
    np.testing.assert_allclose(ux, oux, rtol=0, atol=1e-11)
    np.testing.assert_allclose(uy, ouy, rtol=0, atol=1e-11)
    stats_close(g.stats(), st)


def test_entropic_site_without_equilibrium_reports_status():
    g, oc = pair(lattice=lbm.D2Q9, nx=16, ny=12, boundary=lbm.BC_PERIODIC, beta=0.9)
    f = oracle.init(oc, np.ones(192), np.zeros(192), np.zeros(192))
    f[3, 5, 7] = -0.6  # arrives at (6, 5) with |u_x| > 1: no entropic f*
    g.set_populations(f)
    g.step(1)
    with pytest.raises(lbm.LBMError) as e:
        g.synchronize()
    assert e.value.status == lbm.ERR_NONFINITE
    r = oracle.step(oc, f)
    assert g.stats(check=False)["n_bad"] == r.stats["n_bad"] >= 1



# -- FP32 / 16-bit storage (FP32 arithmetic): entropic f* in deviation form and the
# cancellation-free dS of Eq. DelS (lattice.cuh), on the fused and the tiled kernel

def pair32(**cfg):
    cfg = dict(cfg, equilibrium=lbm.EQ_ENTROPIC)
    g = lbm.Lattice(**cfg)
    c = g.config
    oc = oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta,
                       u_lid=c.u_lid, rho_wall=c.rho_wall, limiters=c.limiters,
                       delta_median=c.delta_median, delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max,
                       median_mode=c.median_mode, equilibrium=oracle.EQ_ENTROPIC)
    return g, oc


@pytest.mark.parametrize("kernel,lattice", [(lbm.KERNEL_FUSED, lbm.D2Q9), (lbm.KERNEL_TILED, lbm.D2Q9),
                                            (lbm.KERNEL_AUTO, lbm.D1Q3)])
def test_fp32_entropic_one_step_against_oracle(kernel, lattice):
    """One FP32 step from the stored FP32 state: populations within the FP32 bar
    (2e-5 relative), identical Ehrenfests' set (FP64 keys with entropic f* on both
    sides), counts equal, dS statistics within 1e-4 (FP32 sums of FP32 terms)."""
    if lattice == lbm.D2Q9:
        nx, ny = 157, 93
        cfg = dict(lattice=lattice, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1)
    else:
        nx, ny = 1300, 1
        cfg = dict(lattice=lattice, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.999)
    g, oc = pair32(precision=lbm.FP32, limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3,
                   k_max=max(1, nx * ny // 1000), kernel=kernel, **cfg)
    f0 = rand_state(g.q, ny, nx, 31 + nx, neg_frac=0.01, heavy=max(2, nx * ny // 250))
    g.set_populations(f0)
    f = g.get_populations()
    bound, want_ds = ds_bound(oc, f)
    assert_ds_close(g.delta_s(), want_ds, bound)
    g.step(1)
    r = oracle.step(oc, f)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
    st = g.stats()
    for key in ("n_pos", "n_ehr", "n_cand", "n_bad"):
        assert st[key] == r.stats[key], (key, st[key], r.stats[key])
    assert abs(st["n_med"] - r.stats["n_med"]) <= max(2, r.stats["n_med"] // 100)
    assert r.stats["n_pos"] > 0 and r.stats["n_ehr"] > 0
    assert abs(st["mass"] - r.stats["mass"]) <= 1e-6 * r.stats["mass"]
    for key in ("sum_dS", "dS_lbgk", "dS_lim"):
        np.testing.assert_allclose(st[key], r.stats[key], rtol=1e-4, err_msg=key)


def test_fp32_entropic_fused_and_tiled_agree_bitwise():
    """The two kernels evaluate entropic f* and dS with the same FP32 operations
    (paired and single): 200 steps of a developing cavity agree bit for bit."""
    nx, ny = 300, 211
    base = dict(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.95, u_lid=0.1, precision=lbm.FP32,
                limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=20, equilibrium=lbm.EQ_ENTROPIC)
    rho, ux, uy = inputs.random_moments(13, nx, ny, umax=0.05)
    out = []
    for kernel in (lbm.KERNEL_FUSED, lbm.KERNEL_TILED):
        g = lbm.Lattice(kernel=kernel, **base)
        g.init(rho, ux, uy)
        g.step(200)
        out.append((g.get_populations(), g.stats()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
        assert out[0][1][key] == out[1][1][key], key
    assert out[0][1]["n_med"] > 0


@pytest.mark.parametrize("precision", [lbm.BF16, lbm.FP16])
def test_16bit_entropic_one_step_within_one_rounding(precision):
    nx, ny = 131, 70
    g, oc = pair32(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1, precision=precision,
                   limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=9)
    assert g.step_kernel() == lbm.KERNEL_FUSED
    g.set_populations(rand_state(9, ny, nx, 41))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    u = 2.0 ** -8 if precision == lbm.BF16 else 2.0 ** -11
    dev = r.f - W9.reshape(9, 1, 1)  # the stored deviations
    err = np.abs(g.get_populations() - r.f)
    assert (err <= u * (np.abs(dev) + 2e-6 * np.abs(dev).max()) + 2e-6 * np.abs(dev).max() + 6e-8).all(), err.max()
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))


@pytest.mark.parametrize("re", [2000.0, 5000.0])
def test_fp32_entropic_cavity_100_matches_fp64_oracle_after_1000_steps(re):
    """The FP32 bar of the north star for the entropic path: the 100 x 100 cavity
    (lid 0.1, median delta = 1e-3), rho and u within 1e-5 after 1000 steps.  At
    Re = 5000 the entropic flow amplifies rounding strongly (the oracle itself,
    its state rounded to FP32 deviations after every step, drifts by ~5e-3 over
    the run), so there the bar is 4 x that drift, measured here."""
    beta = inputs.beta_from_nu(inputs.cavity_nu(100, 0.1, re))
    g, oc = pair32(lattice=lbm.D2Q9, nx=100, ny=100, boundary=lbm.BC_WALLS, beta=beta, u_lid=0.1, rho_wall=1.0,
                   precision=lbm.FP32, limiters=lbm.LIM_MEDIAN, delta_median=1e-3)
    rho, ux, uy = inputs.cavity_rest(100, 100)
    g.init(rho, ux, uy)
    f0 = oracle.init(oc, rho, ux, uy)
    g.step(1000)
    f, st, rc = oracle.run(oc, f0, 1000)
    assert rc == 0
    grho, gux, guy = g.moments()
    orho, oux, ouy = oracle.moments(oc, f)
    err = max(np.abs(grho - orho).max(), np.abs(gux - oux).max(), np.abs(guy - ouy).max())
    bar = 1e-5
    if re > 2000.0:
        w = W9.reshape(9, 1, 1)
        h = f0.copy()
        for _ in range(1000):
            h = oracle.step(oc, h).f
            h = (h - w).astype(np.float32).astype(np.float64) + w
        hr, hx, hy = oracle.moments(oc, h)
        drift = max(np.abs(hr - orho).max(), np.abs(hx - oux).max(), np.abs(hy - ouy).max())
        bar = max(bar, 4.0 * drift)
    print("entropic FP32 cavity, Re", re, "1000 steps: max |d rho|, |d u| =", err, "bar", bar)
    assert err < bar, err
