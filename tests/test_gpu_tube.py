"""The D1Q3 tube kernel (LBM_KERNEL_TUBE) through the C ABI.

It evaluates every site with the same device functions as the tiled kernel,
so with FP64 storage its populations, Ehrenfests' sets and counts equal the
FP64 oracle's bit for bit (sums: 1e-12 relative), and with FP32 storage its
populations equal the tiled kernel's bit for bit; its sums are added in
another order (FP32: dS sums within 1e-6 and the mass within 1e-9 relative of
the tiled kernel's; FP64 1e-12).
Lattice sizes cover every launch shape: one site per lane with one warp per
block (short tubes), 16-byte vectors with several warps per block, grids
above one chunk of the tail's reduction, and ragged last chunks.  Random
states with a few negative populations may hold a site with rho <= 0 (counted
in n_bad by both sides), so the statistics are read without raising.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

W3 = np.array([2 / 3, 1 / 6, 1 / 6])
ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0704_0043_gb300 import build
    build.build()


def ocfg(g):
    c = g.config
    return oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta, u_lid=c.u_lid,
                         rho_wall=c.rho_wall, limiters=c.limiters, delta_median=c.delta_median,
                         delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max, median_mode=c.median_mode,
                         equilibrium=c.equilibrium, collision=c.collision, phi_rule=c.phi_rule)


def state(nx, seed, eps=0.1, kicks=0):
    f = inputs.random_populations(seed, 3, 1, nx, W3, eps, neg_frac=0.003)
    rng = np.random.default_rng(seed + 5)
    for _ in range(kicks):  # strongly nonequilibrium sites: Ehrenfests' candidates and medians
        f[0, 0, rng.integers(0, nx)] *= 0.02
    return f


def tube(nx, precision, boundary=lbm.BC_WALLS, kernel=lbm.KERNEL_AUTO, **kw):
    cfg = dict(lattice=lbm.D1Q3, nx=nx, ny=1, boundary=boundary, precision=precision, beta=0.99,
               limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=max(1, nx // 200), kernel=kernel)
    cfg.update(kw)
    return lbm.Lattice(**cfg)


# sizes: 3 and 5 sites, a ragged short tube, the largest one-site-per-lane tube
# (32 x 4 x 152), the first vector shapes above it, and grids above 256 blocks
SIZES = [3, 5, 1000, 19456, 19457, 20000, 300001]


@pytest.mark.parametrize("nx", SIZES)
@pytest.mark.parametrize("boundary", [lbm.BC_WALLS, lbm.BC_PERIODIC])
def test_fp64_tube_kernel_bitwise_equal_to_oracle(nx, boundary):
    if boundary == lbm.BC_WALLS and nx < 3:
        pytest.skip("closed tube needs 3 sites")
    g = tube(nx, lbm.FP64, boundary)
    assert g.step_kernel() == lbm.KERNEL_TUBE
    oc = ocfg(g)
    cur = state(nx, 11 + nx, kicks=max(2, nx // 300))
    steps = 3 if nx > 100000 else 6
    for step in range(steps):
        g.set_populations(cur)
        g.step(1)
        r = oracle.step(oc, cur)
        np.testing.assert_array_equal(g.get_populations(), r.f, err_msg=f"step {step}")
        st = g.stats(check=False)
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert st[key] == r.stats[key], (step, key, st[key], r.stats[key])
        for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
            assert abs(st[key] - r.stats[key]) <= 1e-12 * abs(r.stats[key]) + 1e-300, (step, key)
        np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
        cur = r.f


@pytest.mark.parametrize("case", ["entropic", "elbm", "phi_entropy", "gate"])
def test_fp64_tube_kernel_variants_bitwise_equal_to_tiled(case):
    """Entropic f*, ELBM and the Sec. 3.7 solve use the device logarithm, so they
    are checked against the tiled kernel (itself checked against the oracle to
    the logarithm's rounding): the same device functions give the same bits."""
    kw = dict(equilibrium=lbm.EQ_ENTROPIC)
    if case == "elbm":
        kw.update(collision=lbm.COLL_ELBM)
    elif case == "phi_entropy":
        kw.update(phi_rule=lbm.PHI_ENTROPY)
    elif case == "gate":
        kw = dict(median_mode=lbm.MEDIAN_GATE)
    nx = 3001
    a = tube(nx, lbm.FP64, **kw)
    b = tube(nx, lbm.FP64, kernel=lbm.KERNEL_TILED, **kw)
    assert a.step_kernel() == lbm.KERNEL_TUBE and b.step_kernel() == lbm.KERNEL_TILED
    f0 = state(nx, 5, eps=0.05, kicks=8)
    a.set_populations(f0)
    b.set_populations(f0)
    for _ in range(5):
        a.step(1)
        b.step(1)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
        sa, sb = a.stats(check=False), b.stats(check=False)
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert sa[key] == sb[key], key
        for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
            assert abs(sa[key] - sb[key]) <= 1e-12 * abs(sb[key]) + 1e-300, key
        np.testing.assert_array_equal(a.limited_sites(), b.limited_sites())


@pytest.mark.parametrize("nx", SIZES)
@pytest.mark.parametrize("boundary", [lbm.BC_WALLS, lbm.BC_PERIODIC])
@pytest.mark.parametrize("eq", [lbm.EQ_POLYNOMIAL, lbm.EQ_ENTROPIC])
def test_fp32_tube_kernel_bitwise_equal_to_tiled(nx, boundary, eq):
    a = tube(nx, lbm.FP32, boundary, equilibrium=eq)
    b = tube(nx, lbm.FP32, boundary, kernel=lbm.KERNEL_TILED, equilibrium=eq)
    assert a.step_kernel() == lbm.KERNEL_TUBE
    f0 = state(nx, 21 + nx, kicks=max(2, nx // 300))
    a.set_populations(f0)
    b.set_populations(f0)
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    for step in range(40):
        a.step(1)
        b.step(1)
        if step % 8 == 7 or step == 0:
            np.testing.assert_array_equal(a.get_populations(), b.get_populations(), err_msg=f"step {step}")
            sa, sb = a.stats(check=False), b.stats(check=False)
            for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
                assert sa[key] == sb[key], (step, key)
            # FP32 sums of rho - rho_ref over other groups of sites (the sites of a
            # warp differ between the kernels): 1e-9 relative, as between batched
            # and lone lattices
            assert abs(sa["mass"] - sb["mass"]) <= 1e-9 * sb["mass"]
            for key in ("sum_dS", "dS_lbgk", "dS_lim"):
                assert abs(sa[key] - sb[key]) <= 1e-6 * abs(sb[key]) + 1e-30, (step, key, sa[key], sb[key])
            np.testing.assert_array_equal(a.limited_sites(), b.limited_sites())


def test_fp32_tube_kernel_one_step_against_oracle_at_scale():
    """300,001 sites (a grid above one chunk of the tail's reduction): one FP32
    step from the stored state within 2e-5 relative of the oracle, the same
    Ehrenfests' set (FP64 keys on both sides) and counts."""
    nx = 300001
    g = tube(nx, lbm.FP32)
    oc = ocfg(g)
    g.set_populations(state(nx, 99, kicks=2000))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
    st = g.stats(check=False)
    for key in ("n_ehr", "n_cand", "n_pos", "n_bad"):
        assert st[key] == r.stats[key], key
    assert abs(st["n_med"] - r.stats["n_med"]) <= max(2, r.stats["n_med"] // 100)
    assert abs(st["mass"] - r.stats["mass"]) <= 1e-8 * r.stats["mass"]
    for key in ("sum_dS", "dS_lbgk", "dS_lim"):
        np.testing.assert_allclose(st[key], r.stats[key], rtol=1e-6, err_msg=key)


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_tube_kernel_limiter_pass(precision):
    """lbm_limit (no collision) on the tube kernel: the oracle's limiter pass
    (FP64 bit for bit; FP32 equal to the tiled kernel's)."""
    nx = 5000
    a = tube(nx, precision)
    f0 = state(nx, 7, eps=0.3, kicks=40)
    a.set_populations(f0)
    f = a.get_populations()
    a.limit(ALL)
    if precision == lbm.FP64:
        r = oracle.limit(ocfg(a), f, ALL)
        np.testing.assert_array_equal(a.get_populations(), r.f)
        np.testing.assert_array_equal(a.limited_sites(), np.sort(r.selected))
    else:
        b = tube(nx, precision, kernel=lbm.KERNEL_TILED)
        b.set_populations(f0)
        b.limit(ALL)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
        np.testing.assert_array_equal(a.limited_sites(), b.limited_sites())


def test_shock_tube_on_the_tube_kernel_matches_the_oracle_over_400_steps():
    """The 1:2 shock tube of Sec. 4.3 (800 sites, nu = 1e-9, Ehrenfests' delta =
    1e-3, k = 4), FP64: populations equal the oracle's after 400 steps."""
    w = inputs.shock_tube_workload(800)
    g = lbm.Lattice(lattice=lbm.D1Q3, nx=w.nx, ny=1, boundary=lbm.BC_WALLS, precision=lbm.FP64, beta=w.beta,
                    limiters=w.limiters, delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max)
    assert g.step_kernel() == lbm.KERNEL_TUBE
    rho, ux = inputs.shock_tube(w.nx, 1.0, w.rho_right)
    g.init(rho, ux, None)
    oc = ocfg(g)
    f0 = oracle.init(oc, rho, ux)
    g.step(400)
    f, st, rc = oracle.run(oc, f0, 400)
    assert rc == 0
    np.testing.assert_array_equal(g.get_populations(), f)
