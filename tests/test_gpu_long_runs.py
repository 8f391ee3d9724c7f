"""Long high-Re cavity runs on the GPU against the oracle's own long runs.

The 100 x 100 cavity as Sec. 4.4.1 sets it up (boundary nodes on the walls with
bounce-back and a constant lid profile, density 2.7, lid 0.1, polynomial f*,
median filter delta = 1e-3) runs 2e5 steps in FP32 on the GPU at Re = 5000 and
Re = 7500.  Each vortex centre must lie within one cell (1/99) of the oracle's
FP64 run of the same length (tests/golden/cavity100_long_oracle.txt, itself
within one cell of the paper's Table vort), and the mass the lattice carries
must be conserved to the FP32 bound (1e-6 relative).  Unregularised LBGK at
Re = 7500 must blow up (the oracle's run reports a nonfinite site at step 569).
"""
import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs, lbm
from tests.helpers import vortex_centres_nodes
from tests.test_oracle_cavity_table import CELL, NAMES, read_oracle_runs

pytestmark = pytest.mark.gpu

N, U0, RHO0, STEPS = 100, 0.1, 2.7, 200000


def _lattice(re, limiters, delta):
    beta = inputs.beta_from_nu(inputs.cavity_nu(N - 1, U0, re))
    g = lbm.Lattice(lattice=lbm.D2Q9, nx=N, ny=N, boundary=lbm.BC_NODE_WALLS, precision=lbm.FP32, beta=beta,
                    u_lid=U0, rho_wall=RHO0, rho_ref=RHO0, limiters=limiters, delta_median=delta)
    g.init(*inputs.cavity_rest(N, N, RHO0))
    g.set_graph(1000)
    return g


@pytest.mark.parametrize("re", [5000, 7500])
def test_fp32_long_run_vortex_centres_and_mass_match_the_oracle(re):
    want = read_oracle_runs()[(re, "median", 1e-3)]
    g = _lattice(float(re), lbm.LIM_MEDIAN, 1e-3)
    g.step(1)
    m0 = g.stats()["mass"]
    g.step(STEPS - 1)
    st = g.stats()
    rho, ux, uy = g.moments()
    got = vortex_centres_nodes(ux, N, NAMES)
    drift = (st["mass"] - m0) / m0
    print("Re", re, "centres", got, "mass drift", drift, "n_med", st["n_med"])
    assert st["n_bad"] == 0 and st["step"] == STEPS
    assert abs(drift) < 1e-6, drift
    for v, name in enumerate(NAMES):
        assert np.all(np.abs(np.array(got[name]) - want["centres"][v]) <= CELL + 1e-4), (name, got[name],
                                                                                       want["centres"][v])


def test_unregularised_lbgk_blows_up_at_re_7500():
    g = _lattice(7500.0, 0, 0.0)
    g.step(20000)
    with pytest.raises(lbm.LBMError) as e:
        g.synchronize()
    assert e.value.status == lbm.ERR_NONFINITE
