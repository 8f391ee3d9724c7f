"""The threshold filter with dS_0 from Eq. EntThresh on the GPU (LBM_LIM_ENTTHRESH),
against the FP64 oracle's exact solve on the sorted dS values, through the C ABI.

The GPU finds dS_0 by a radix descent over the dS field's bit patterns and adds
the sums of Eq. EntThresh by atomics, so dS_0 agrees with the oracle's to the
rounding of sums over many values, and t = (S_m - rhs) / m can lose a few more
digits to the difference S_m - rhs: phi = sqrt(dS_t / dS) then agrees to about
1e-12 relative.  FP64 populations are compared to 1e-11 absolute (values
~0.01..0.5), FP32 storage after one step from the same stored state to the FP32
bar of the other limiters (2e-5 relative).  A site whose dS lies within that
rounding of dS_t may be limited on one side only; its phi is then within 1e-12
of 1, inside the same bound.  Counts other than the filter's are identical.

Eq. LimEntLim is met with equality when the filter acts alone: the entropy the
limiter adds, sum over limited sites of (1 - phi^2) dS = sum max(dS - dS_t, 0),
equals delta_0 (1 - (2 beta - 1)^2) sum dS.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W3 = np.array([2 / 3, 1 / 6, 1 / 6])
ENT = lbm.LIM_ENTTHRESH


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0704_0043_gb300 import build
    build.build()


def pair(**cfg):
    g = lbm.Lattice(**cfg)
    c = g.config
    oc = oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta,
                       u_lid=c.u_lid, rho_wall=c.rho_wall, limiters=c.limiters,
                       delta_median=c.delta_median, delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max,
                       median_mode=c.median_mode, equilibrium=c.equilibrium, threshold_c=c.threshold_c,
                       threshold_delta=c.threshold_delta, entthresh_delta0=c.entthresh_delta0,
                       phi_rule=c.phi_rule)
    return g, oc


CASES = [
    dict(lattice=lbm.D2Q9, nx=67, ny=41, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1,
         limiters=ENT | lbm.LIM_MEDIAN | lbm.LIM_EHRENFEST, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=7,
         entthresh_delta0=0.1),
    dict(lattice=lbm.D2Q9, nx=120, ny=77, boundary=lbm.BC_NODE_WALLS, beta=0.95, u_lid=0.1, limiters=ENT,
         entthresh_delta0=0.3, threshold_delta=1e-5),
    dict(lattice=lbm.D1Q3, nx=800, ny=1, boundary=lbm.BC_WALLS, beta=0.999, limiters=ENT, entthresh_delta0=0.05),
    dict(lattice=lbm.D2Q9, nx=40, ny=30, boundary=lbm.BC_PERIODIC, beta=0.97, limiters=ENT | lbm.LIM_POSITIVITY,
         entthresh_delta0=0.2, equilibrium=lbm.EQ_ENTROPIC, phi_rule=lbm.PHI_ENTROPY),
    # delta_0 = 0: the right side vanishes and nothing is limited (dS_0 = +inf)
    dict(lattice=lbm.D2Q9, nx=50, ny=20, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1, limiters=ENT,
         entthresh_delta0=0.0),
    # a right side above sum dS: dS_0 = 0, every site above threshold_delta is brought to it
    dict(lattice=lbm.D2Q9, nx=50, ny=20, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1, limiters=ENT,
         entthresh_delta0=1e3, threshold_delta=1e-6),
]


def _state(q, ny, nx, seed):
    return inputs.random_populations(seed, q, ny, nx, W9 if q == 9 else W3, 0.15, neg_frac=0.005)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_entthresh_matches_oracle(case):
    g, oc = pair(**dict(CASES[case], precision=lbm.FP64))
    cur = _state(g.q, g.ny, g.nx, 70 + case)
    limited = 0.0
    for step in range(5):
        g.set_populations(cur)
        if oc.equilibrium == oracle.EQ_POLYNOMIAL:  # the same dS field, bit for bit
            np.testing.assert_array_equal(g.delta_s(), oracle.delta_s(oc, cur))
        g.step(1)
        r = oracle.step(oc, cur)
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=0, atol=1e-11, err_msg=f"step {step}")
        st = g.stats()
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert st[key] == r.stats[key], (key, st[key], r.stats[key])
        for key in ("mass", "sum_dS", "dS_lbgk"):
            assert abs(st[key] - r.stats[key]) <= 1e-10 * abs(r.stats[key]) + 1e-13, key
        assert abs(st["dS_lim"] - r.stats["dS_lim"]) <= 1e-9 * abs(r.stats["dS_lim"]) + 1e-14
        np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
        limited += r.stats["dS_lim"]
        cur = r.f
    if CASES[case]["entthresh_delta0"] == 0.0:
        assert limited == 0.0
    else:
        assert limited > 0.0


def test_entthresh_alone_meets_eq_limentlim_with_equality():
    """sum (1 - phi^2) dS over the limited sites = delta_0 (1 - (2 beta - 1)^2) sum dS."""
    for precision in (lbm.FP64, lbm.FP32):
        g, oc = pair(lattice=lbm.D2Q9, nx=300, ny=200, boundary=lbm.BC_PERIODIC, beta=0.95, limiters=ENT,
                     entthresh_delta0=0.1, precision=precision)
        g.set_populations(_state(9, 200, 300, 81))
        g.step(1)
        st = g.stats()
        a = 2 * 0.95 - 1
        want = 0.1 * (1 - a * a) * st["sum_dS"]
        rtol = 1e-12 if precision == lbm.FP64 else 1e-4
        np.testing.assert_allclose(st["dS_lim"], want, rtol=rtol)


def test_fp32_entthresh_one_step_against_oracle():
    nx, ny = 257, 131
    g, oc = pair(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_WALLS, beta=0.97, u_lid=0.1, precision=lbm.FP32,
                 limiters=ENT | lbm.LIM_EHRENFEST | lbm.LIM_POSITIVITY, delta_ehrenfest=2e-3, k_max=20,
                 entthresh_delta0=0.1)
    g.set_populations(_state(9, ny, nx, 82))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
    st = g.stats()
    assert st["n_ehr"] == r.stats["n_ehr"] and st["n_pos"] == r.stats["n_pos"]
    np.testing.assert_allclose(st["dS_lim"], r.stats["dS_lim"], rtol=1e-4)


def test_entthresh_needs_the_bit_at_create():
    g = lbm.Lattice(lattice=lbm.D2Q9, nx=20, ny=20, boundary=lbm.BC_WALLS, precision=lbm.FP64, beta=0.9)
    g.init(*inputs.cavity_rest(20, 20))
    with pytest.raises(lbm.LBMError) as e:
        g.limit(ENT)
    assert e.value.status == lbm.ERR_INVALID_ARG
