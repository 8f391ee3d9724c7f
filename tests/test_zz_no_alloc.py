"""lbm_step_noalloc: the step for callers that cannot allocate device memory.

A framework that owns all device memory through its own pool, or a host that
allows no allocation once running, can still take limited LBGK steps: it owns
the population arrays and the library takes its scratch from a fixed static
device array.  The result must be that of an ordinary LBM_FP64 context, bit
for bit, on two calls in a row (the second call starts from the scratch the
first one left behind).  This file is collected last so that a failure here
never hides another test.
"""
import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _cfg(nx, ny):
    return dict(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_WALLS, precision=lbm.FP64,
                beta=0.97, u_lid=0.1, limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3,
                k_max=9)


def test_noalloc_step_matches_context_step_twice():
    import torch
    from paper_0704_0043_gb300 import build
    build.build()
    nx, ny = 97, 61
    cfg = _cfg(nx, ny)
    f0 = inputs.random_populations(77, 9, ny, nx, W9, 0.15)
    f0[1, 5, 7] *= 8.0  # make the positivity rule act
    ref = lbm.Lattice(**cfg)
    ref.set_populations(f0)
    want = []
    for _ in range(2):
        ref.step(1)
        want.append((ref.get_populations(), ref.stats()))
    a = torch.from_numpy(f0.copy()).cuda()
    b = torch.empty_like(a)
    got = []
    for _ in range(2):
        st = lbm.step_noalloc(a, b, **cfg)
        torch.cuda.synchronize()
        got.append((b.cpu().numpy().copy(), st))
        a, b = b, a
    for (fw, sw), (fg, sg) in zip(want, got):
        np.testing.assert_array_equal(fg, fw)
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert sg[key] == sw[key], key
        for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
            assert abs(sg[key] - sw[key]) <= 1e-12 * abs(sw[key]), key
        assert sg["step"] == 1
    assert want[0][1]["n_pos"] + want[1][1]["n_pos"] > 0 and want[0][1]["n_ehr"] > 0


def test_noalloc_rejects_lattices_beyond_the_scratch():
    import torch
    cfg = _cfg(1024, 1024)  # above LBM_NOALLOC_MAX_SITES
    a = torch.zeros(9 * 1024 * 1024, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(lbm.LBMError) as e:
        lbm.step_noalloc(a, b, **cfg)
    assert e.value.status == lbm.ERR_INVALID_ARG
    assert "LBM_NOALLOC_MAX_SITES" in str(e.value)
