"""lbm_step_noalloc: the step for callers that cannot allocate device memory.

A framework that owns all device memory through its own pool, or a host that
allows no allocation once running, can still take limited LBGK steps: it owns
the population arrays and the library takes its scratch from a fixed static
device array.  The result must be that of an ordinary LBM_FP64 context, bit
for bit, on two calls in a row (the second call starts from the scratch the
first one left behind), for every lattice kind the entry point accepts, and
the calls must not change the device's free memory.  This file is collected
last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W3 = np.array([2 / 3, 1 / 6, 1 / 6])


def _case(name):
    """(config, initial populations) of one lattice kind."""
    if name == "walls":
        cfg = dict(lattice=lbm.D2Q9, nx=97, ny=61, boundary=lbm.BC_WALLS, precision=lbm.FP64,
                   beta=0.97, u_lid=0.1, limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=9)
        f0 = inputs.random_populations(77, 9, 61, 97, W9, 0.15)
        f0[1, 5, 7] *= 8.0  # make the positivity rule act
        return cfg, f0
    if name == "periodic":
        cfg = dict(lattice=lbm.D2Q9, nx=70, ny=45, boundary=lbm.BC_PERIODIC, precision=lbm.FP64,
                   beta=0.95, limiters=ALL, delta_median=1e-4, delta_ehrenfest=2e-3, k_max=6)
        f0 = inputs.random_populations(78, 9, 45, 70, W9, 0.15, neg_frac=0.01)
        return cfg, f0
    if name == "tube":
        # D1Q3 tiles finish 62 sites each: 1000 sites give 17 tiles, the last one ragged
        cfg = dict(lattice=lbm.D1Q3, nx=1000, ny=1, boundary=lbm.BC_WALLS, precision=lbm.FP64,
                   beta=0.99, limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=4)
        f0 = inputs.random_populations(79, 3, 1, 1000, W3, 0.1, neg_frac=0.005)
        return cfg, f0
    assert name == "entropic"
    cfg = dict(lattice=lbm.D2Q9, nx=64, ny=40, boundary=lbm.BC_WALLS, precision=lbm.FP64,
               equilibrium=lbm.EQ_ENTROPIC, beta=0.97, u_lid=0.1, limiters=ALL, delta_median=1e-4,
               delta_ehrenfest=2e-3, k_max=5)
    f0 = inputs.random_populations(80, 9, 40, 64, W9, 0.1)
    return cfg, f0


@pytest.mark.parametrize("name", ["walls", "periodic", "tube", "entropic"])
def test_noalloc_step_matches_context_step_twice(name):
    import torch
    from paper_0704_0043_gb300 import build
    build.build()
    cfg, f0 = _case(name)
    ref = lbm.Lattice(**cfg)
    ref.set_populations(f0)
    want = []
    for _ in range(2):
        ref.step(1)
        want.append((ref.get_populations(), ref.stats()))
    a = torch.from_numpy(f0.copy()).cuda()
    b = torch.empty_like(a)
    lbm.step_noalloc(a, b, **cfg)  # set-up call (looks up the scratch address once)
    a.copy_(torch.from_numpy(f0))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = []
    for _ in range(2):
        st = lbm.step_noalloc(a, b, **cfg)
        torch.cuda.synchronize()
        got.append((b.cpu().numpy().copy(), st))
        a, b = b, a
    # the calls allocate nothing: the device's free memory is unchanged
    assert torch.cuda.mem_get_info()[0] == free0
    for (fw, sw), (fg, sg) in zip(want, got):
        np.testing.assert_array_equal(fg.reshape(fw.shape), fw)
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert sg[key] == sw[key], key
        for key in ("mass", "sum_dS", "dS_lbgk", "dS_lim"):
            assert abs(sg[key] - sw[key]) <= 1e-12 * abs(sw[key]), key
        assert sg["step"] == 1
    assert want[0][1]["n_med"] + want[1][1]["n_med"] > 0


def test_noalloc_rejects_lattices_beyond_the_scratch():
    import torch
    cfg, _ = _case("walls")
    cfg.update(nx=1024, ny=1024)  # above LBM_NOALLOC_MAX_SITES
    a = torch.zeros(9 * 1024 * 1024, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(lbm.LBMError) as e:
        lbm.step_noalloc(a, b, **cfg)
    assert e.value.status == lbm.ERR_INVALID_ARG
    assert "LBM_NOALLOC_MAX_SITES" in str(e.value)


def test_noalloc_rejects_host_and_overlapping_arrays():
    import torch
    cfg, f0 = _case("walls")
    n = f0.size
    dev = torch.zeros(n, dtype=torch.float64, device="cuda")
    host = np.zeros(n)
    # the binding accepts CUDA tensors of the current device only
    with pytest.raises(ValueError):
        lbm.step_noalloc(host, dev, **cfg)
    # the C entry point itself checks the pointers before it launches anything
    c = lbm.default_config(**cfg)
    st = lbm.StepStats()
    s = lbm.lib().lbm_step_noalloc(ctypes.byref(c), ctypes.c_void_p(host.ctypes.data),
                                   ctypes.c_void_p(dev.data_ptr()), ctypes.byref(st), ctypes.c_void_p(0))
    assert s == lbm.ERR_INVALID_ARG
    assert b"device memory" in lbm.lib().lbm_last_error(None)
    big = torch.zeros(n + 9, dtype=torch.float64, device="cuda")
    s = lbm.lib().lbm_step_noalloc(ctypes.byref(c), ctypes.c_void_p(big.data_ptr()),
                                   ctypes.c_void_p(big.data_ptr() + 72), ctypes.byref(st), ctypes.c_void_p(0))
    assert s == lbm.ERR_INVALID_ARG
    assert b"overlap" in lbm.lib().lbm_last_error(None)
