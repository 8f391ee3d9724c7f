"""The control-point record (the monitoring point of Sec. 4.4.2) through the C ABI.

After every step the tail kernel stores rho, u_x, u_y of one site; those must be
the values lbm_moments gives for that site after the same step (bit for bit),
the ring keeps the most recent `capacity` samples, and a lattice recorded inside
a batch gives the same samples as alone.
"""
import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_probe_samples_equal_the_moments_after_each_step(precision):
    nx, ny = 40, 30
    g = lbm.Lattice(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_DIFFUSIVE, precision=precision, beta=0.95,
                    u_lid=0.1, limiters=lbm.LIM_MEDIAN, delta_median=1e-4)
    g.init(*inputs.cavity_rest(nx, ny))
    g.step(5)
    i, j = nx // 16, 13 * ny // 16
    g.probe(j * nx + i, 4)
    want = []
    for _ in range(10):
        g.step(1)
        rho, ux, uy = g.moments()
        want.append((rho[j, i], ux[j, i], uy[j, i]))
    got = g.probe_read(100)
    assert got.shape == (4, 3)  # the ring keeps the last four
    np.testing.assert_array_equal(got, np.array(want[-4:]))
    g.probe(-1)
    with pytest.raises(lbm.LBMError):
        g.probe_read(4)


def test_probe_in_a_batch_equals_probe_alone():
    cfg = dict(lattice=lbm.D2Q9, nx=50, ny=50, boundary=lbm.BC_DIFFUSIVE, precision=lbm.FP32, beta=0.97, u_lid=0.1,
               limiters=lbm.LIM_MEDIAN, delta_median=1e-3)
    site = 40 * 50 + 3
    g = lbm.Lattice(**cfg)
    g.init(*inputs.cavity_rest(50, 50))
    g.probe(site, 64)
    g.step(60)
    b = lbm.Batch()
    s0 = b.add(**cfg)
    s1 = b.add(**dict(cfg, beta=0.9))
    for s in (s0, s1):
        b.init(s, *inputs.cavity_rest(50, 50))
    b.probe(s0, site, 64)
    b.set_graph(20)
    b.step(60)
    np.testing.assert_array_equal(b.probe_read(s0, 64), g.probe_read(64))
    assert b.probe_read(s0, 64).shape == (60, 3)
