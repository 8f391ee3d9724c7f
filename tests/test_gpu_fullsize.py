"""Parity at full size: the 4096 x 4096 cavity workload (Re = 7500, lid 0.05,
median delta = 1e-3 plus Ehrenfests' delta = 1e-3 with k = 1677), in the
launch configuration the benchmark times (the default kernel choice, i.e. the
row-streaming fused kernel), one step from a stored state against one oracle
step over the whole lattice.

The state is a random near-equilibrium field (3 % population noise) with 5000
strongly nonequilibrium sites, so the median filter acts widely and the
Ehrenfests' candidates outnumber k (a real top-k of the 16.7M sites).  FP32:
populations within 2e-5 relative (2e-7 absolute) of the oracle and the
identical Ehrenfests' set.  BF16 / FP16 storage: within one rounding of the
format (see test_gpu_lowprec.py) and the identical set.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs, lbm

from test_gpu_parity import pair, rand_state

pytestmark = pytest.mark.gpu

UNIT = {lbm.BF16: 2.0 ** -8, lbm.FP16: 2.0 ** -11}
SUBNORMAL_HALF = {lbm.BF16: 0.0, lbm.FP16: 2.0 ** -25}
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def state():
    w = inputs.cavity4096_workload()
    f0 = rand_state(9, w.ny, w.nx, 4096, eps=0.03, heavy=5000)
    return w, f0


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.BF16, lbm.FP16])
def test_cavity4096_one_step_against_oracle(state, precision):
    w, f0 = state
    g, oc = pair(lattice=lbm.D2Q9, nx=w.nx, ny=w.ny, boundary=lbm.BC_WALLS, beta=w.beta, u_lid=w.u_lid,
                 rho_wall=w.rho0, precision=precision, limiters=w.limiters, delta_median=w.delta_median,
                 delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max)
    assert g.step_kernel() == lbm.KERNEL_FUSED
    g.set_populations(f0)
    f = g.get_populations()  # the stored state, as FP64
    g.step(1)
    g.synchronize()
    r = oracle.step(oc, f)
    got = g.get_populations()
    st = g.stats()
    assert r.stats["n_cand"] > w.k_max and st["n_ehr"] == w.k_max
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
    assert st["n_cand"] == r.stats["n_cand"]
    assert abs(st["n_med"] - r.stats["n_med"]) <= max(2, r.stats["n_med"] // 1000)
    assert abs(st["mass"] - r.stats["mass"]) <= 1e-8 * r.stats["mass"]
    if precision == lbm.FP32:
        err = np.abs(got - r.f)
        assert np.all(err <= 2e-5 * np.abs(r.f) + 2e-7), float(err.max())
    else:
        dev = r.f - W9[:, None, None]
        e = 2e-6 * np.abs(dev).max()
        bound = UNIT[precision] * (np.abs(dev) + e) + e + SUBNORMAL_HALF[precision]
        excess = np.abs(got - r.f) - bound
        assert excess.max() <= 0, float(excess.max())
    print("precision", precision, "max |f - f_oracle|", float(np.abs(got - r.f).max()),
          "limited", st["n_med"], "Ehrenfests'", st["n_ehr"], "of", st["n_cand"])
