"""Parity of the ensemble-dependent limiters (LBM_LIM_SMOOTH, LBM_LIM_THRESHOLD)
with the FP64 oracle, through the C ABI.

Both limiters use E(dS), the mean of dS(f') over the lattice.  The GPU adds
the same dS values as the oracle (bitwise in FP64) but in another order, so E
differs by a rounding; the limiter's pow / sqrt on the device and on the host
differ by an ulp or so.  The homothety factor phi then agrees to ~1e-15
relative, and populations are compared to 1e-13 absolute in FP64 (values
~0.01..0.5; a wrong exponent, sign or mean shifts them by 1e-4 and more).
Counts, dS fields and Ehrenfests' sets must be identical.  FP32 storage is
compared after one step from the same stored state, to the FP32 bar of the
other limiters (2e-5 relative), on the fused kernel and on the tiled kernel,
which must also agree with each other bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ENS = lbm.LIM_SMOOTH | lbm.LIM_THRESHOLD
ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN | ENS
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W3 = np.array([2 / 3, 1 / 6, 1 / 6])


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0704_0043_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def pair(**cfg):
    g = lbm.Lattice(**cfg)
    c = g.config
    oc = oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta,
                       u_lid=c.u_lid, rho_wall=c.rho_wall, limiters=c.limiters,
                       delta_median=c.delta_median, delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max,
                       median_mode=c.median_mode, equilibrium=c.equilibrium, smooth_delta=c.smooth_delta,
                       smooth_k=c.smooth_k, threshold_c=c.threshold_c, threshold_delta=c.threshold_delta)
    return g, oc


def rand_state(q, ny, nx, seed, eps=0.15, neg_frac=0.0):
    return inputs.random_populations(seed, q, ny, nx, W9 if q == 9 else W3, eps, neg_frac=neg_frac)


def stats_close(a, b, rtol=1e-10):
    for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
        assert abs(a[key] - b[key]) <= rtol * abs(b[key]) + 1e-13, (key, a[key], b[key])
    for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
        assert a[key] == b[key], (key, a[key], b[key])


CASES = [
    dict(lattice=lbm.D2Q9, nx=67, ny=41, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1, limiters=ALL,
         delta_median=1e-4, delta_ehrenfest=2e-3, k_max=7, smooth_delta=0.05, threshold_c=4.0),
    dict(lattice=lbm.D2Q9, nx=45, ny=20, boundary=lbm.BC_PERIODIC, beta=0.9, limiters=lbm.LIM_SMOOTH,
         smooth_delta=0.5, smooth_k=1.0),
    dict(lattice=lbm.D2Q9, nx=33, ny=13, boundary=lbm.BC_CHANNEL, beta=0.99, u_lid=0.05,
         limiters=lbm.LIM_THRESHOLD, threshold_c=2.0, threshold_delta=1e-4),
    dict(lattice=lbm.D1Q3, nx=800, ny=1, boundary=lbm.BC_WALLS, beta=0.999, limiters=lbm.LIM_SMOOTH,
         smooth_delta=0.01, smooth_k=0.5),
    dict(lattice=lbm.D1Q3, nx=517, ny=1, boundary=lbm.BC_PERIODIC, beta=0.95,
         limiters=lbm.LIM_THRESHOLD | lbm.LIM_POSITIVITY, threshold_c=5.0),
    dict(lattice=lbm.D2Q9, nx=40, ny=30, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1,
         limiters=ENS | lbm.LIM_EHRENFEST, smooth_delta=0.1, threshold_c=3.0, k_max=4,
         delta_ehrenfest=1e-3, equilibrium=lbm.EQ_ENTROPIC),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_ensemble_limiters_match_oracle(case):
    g, oc = pair(**dict(CASES[case], precision=lbm.FP64))
    cur = rand_state(g.q, g.ny, g.nx, 40 + case, neg_frac=0.01)
    limited = 0.0
    for step in range(6):
        g.set_populations(cur)
        if oc.equilibrium == oracle.EQ_POLYNOMIAL:
            np.testing.assert_array_equal(g.delta_s(), oracle.delta_s(oc, cur))
        g.step(1)
        r = oracle.step(oc, cur)
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=0, atol=1e-13, err_msg=f"step {step}")
        stats_close(g.stats(), r.stats)
        np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
        limited += r.stats["dS_lim"]
        cur = r.f
    assert limited > 0


def test_fp64_ensemble_shock_tube_run_tracks_oracle():
    # the paper's smooth-limiter shock tube (Sec. 4.3.2): 800 sites, nu = 1e-9,
    # k = 1/2, delta = 0.01; 200 unsynchronised steps
    cfg = dict(lattice=lbm.D1Q3, nx=800, ny=1, boundary=lbm.BC_WALLS, beta=1.0 / (6e-9 + 1),
               limiters=lbm.LIM_SMOOTH, smooth_delta=0.01, smooth_k=0.5, precision=lbm.FP64)
    g, oc = pair(**cfg)
    x = np.arange(800)
    rho = np.where(x < 400, 1.0, 0.5)
    g.init(rho, np.zeros(800))
    f = oracle.init(oc, rho, np.zeros(800))
    g.step(200)
    f, st, rc = oracle.run(oc, f, 200)
    assert rc == 0 and st["dS_lim"] > 0
    grho, gux, _ = g.moments()
    orho, oux, _ = oracle.moments(oc, f)
    # E couples every site each step, so summation-order differences travel;
    # 1e-8 is far below the limiter's own effect (dS_lim > 0, phi ~ 1 - 1e-3)
    np.testing.assert_allclose(grho, orho, rtol=0, atol=1e-8)
    np.testing.assert_allclose(gux, oux, rtol=0, atol=1e-8)


def test_fp64_ensemble_limit_pass_matches_oracle():
    g, oc = pair(lattice=lbm.D2Q9, nx=50, ny=29, boundary=lbm.BC_WALLS, beta=0.96, u_lid=0.1,
                 precision=lbm.FP64, limiters=ENS, smooth_delta=0.2, threshold_c=1.5)
    f = rand_state(9, 29, 50, 4, eps=0.25)
    for lim in (lbm.LIM_SMOOTH, lbm.LIM_THRESHOLD, ENS):
        g.set_populations(f)
        g.limit(lim)
        r = oracle.limit(oc, f, lim)
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=0, atol=1e-13)
        stats_close(g.stats(), r.stats)


@pytest.mark.parametrize("precision,kernel", [(lbm.FP32, lbm.KERNEL_AUTO), (lbm.FP32, lbm.KERNEL_TILED),
                                              (lbm.BF16, lbm.KERNEL_AUTO), (lbm.FP16, lbm.KERNEL_AUTO)])
def test_lowprec_ensemble_limiters_one_step(precision, kernel):
    g, oc = pair(lattice=lbm.D2Q9, nx=130, ny=70, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1,
                 precision=precision, limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=9,
                 smooth_delta=0.05, threshold_c=4.0, kernel=kernel)
    # the walled cavity takes the fused kernel unless the tiled one is asked for
    assert g.step_kernel() == (lbm.KERNEL_TILED if kernel == lbm.KERNEL_TILED else lbm.KERNEL_FUSED)
    g.set_populations(rand_state(9, 70, 130, 9))
    f = g.get_populations()  # the exact stored state
    g.step(1)
    r = oracle.step(oc, f)
    if precision == lbm.FP32:
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)
    else:
        # one 16-bit rounding of the stored deviation (2^-8 / 2^-11 relative) plus the FP32 arithmetic
        u = 2.0 ** -8 if precision == lbm.BF16 else 2.0 ** -11
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=0, atol=u * np.abs(r.f).max() + 1e-6)
    st = g.stats()
    np.testing.assert_allclose(st["dS_lim"], r.stats["dS_lim"], rtol=2e-3)
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))


@pytest.mark.parametrize("limiters,eq", [(ALL, lbm.EQ_POLYNOMIAL), (ALL & ~lbm.LIM_MEDIAN, lbm.EQ_POLYNOMIAL),
                                         (ALL & ~lbm.LIM_MEDIAN, lbm.EQ_ENTROPIC)])
def test_fused_and_tiled_ensemble_limiters_agree_bitwise(limiters, eq):
    """The fused kernel applies the ensemble-dependent limiters with the tiled
    kernel's FP32 operations (the same E(dS) and alpha from the same reduction):
    60 steps of a developing cavity with every limiter but Eq. EntThresh (whose
    atomically added sums are reproducible to rounding only) agree bit for bit.
    Without the median the fused kernel stores the limited update at once
    instead of overwriting the row one row later: the same bits."""
    nx, ny = 301, 203
    base = dict(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.95, u_lid=0.1, precision=lbm.FP32,
                limiters=limiters, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=20, smooth_delta=0.05,
                threshold_c=3.0, equilibrium=eq)
    rho, ux, uy = inputs.random_moments(12, nx, ny, umax=0.05)
    runs = []
    for kernel in (lbm.KERNEL_FUSED, lbm.KERNEL_TILED):
        g = lbm.Lattice(kernel=kernel, **base)
        g.init(rho, ux, uy)
        g.step(60)
        runs.append((g.get_populations(), g.stats()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
        assert runs[0][1][key] == runs[1][1][key], key
    assert runs[0][1]["dS_lim"] > 0


def test_ensemble_limiters_refused_where_not_available():
    b = lbm.Batch()
    with pytest.raises(lbm.LBMError):
        b.add(lattice=lbm.D2Q9, nx=64, ny=64, precision=lbm.FP32, limiters=lbm.LIM_THRESHOLD)
