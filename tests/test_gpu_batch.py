"""The batch engine: many lattices advanced by shared launches.

Each lattice of a batch must evolve exactly as it does alone (same per-site
arithmetic; bit for bit), whatever the mix of sizes, lattices and limiters,
with or without CUDA-graph replay, and across the autotuner (which must
restore every lattice's state).
"""
import numpy as np
import pytest

from paper_0704_0043_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

ALL = lbm.LIM_POSITIVITY | lbm.LIM_EHRENFEST | lbm.LIM_MEDIAN


def _mix():
    rng = np.random.default_rng(5)
    cfgs = []
    for i, side in enumerate([64, 100, 257, 130, 77]):
        lim = [lbm.LIM_MEDIAN, lbm.LIM_EHRENFEST, lbm.LIM_POSITIVITY, ALL, lbm.LIM_MEDIAN][i]
        cfgs.append(dict(lattice=lbm.D2Q9, nx=side, ny=side + 3 * i, boundary=lbm.BC_WALLS,
                         precision=lbm.FP32, beta=float(rng.uniform(0.9, 0.99)), u_lid=0.1,
                         limiters=lim, delta_median=1e-4, delta_ehrenfest=1e-3,
                         k_max=max(1, side * side // 1000)))
    cfgs.append(dict(lattice=lbm.D1Q3, nx=3000, ny=1, boundary=lbm.BC_WALLS, precision=lbm.FP32,
                     beta=0.999, limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=4))
    cfgs.append(dict(lattice=lbm.D2Q9, nx=90, ny=40, boundary=lbm.BC_CHANNEL, precision=lbm.FP32,
                     beta=0.95, u_lid=0.05, limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-3,
                     k_max=3))
    return cfgs


def _ic(cfg, seed):
    if cfg["lattice"] == lbm.D1Q3:
        rho, ux = inputs.shock_tube(cfg["nx"])
        return rho, ux, None
    return inputs.random_moments(seed, cfg["nx"], cfg["ny"], umax=0.05)


@pytest.mark.parametrize("graph", [0, 8])
def test_batch_matches_lone_runs_bitwise(graph):
    cfgs = _mix()
    steps = 37
    alone = []
    for i, c in enumerate(cfgs):
        g = lbm.Lattice(**c)
        g.init(*_ic(c, i))
        g.step(steps)
        alone.append((g.get_populations(), g.stats(), g.limited_sites()))
    b = lbm.Batch()
    slots = [b.add(**c) for c in cfgs]
    for i, (c, s) in enumerate(zip(cfgs, slots)):
        b.init(s, *_ic(c, i))
    if graph:
        b.set_graph(graph)
    b.step(10)
    b.step(steps - 10)
    b.synchronize()
    for i, s in enumerate(slots):
        f, st, sel = alone[i]
        np.testing.assert_array_equal(b.get_populations(s), f, err_msg=f"lattice {i}")
        bs = b.stats(s)
        assert bs["step"] == steps
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert bs[key] == st[key], (i, key)
        assert abs(bs["mass"] - st["mass"]) <= 1e-9 * st["mass"]
        np.testing.assert_array_equal(b.limited_sites(s), sel)
    assert b.launch_count() > 0


def test_batch_add_remove_and_tune_keep_states():
    cfgs = _mix()[:4]
    b = lbm.Batch()
    slots = [b.add(**c) for c in cfgs]
    for i, (c, s) in enumerate(zip(cfgs, slots)):
        b.init(s, *_ic(c, i))
    b.step(5)
    before = [b.get_populations(s) for s in slots]
    ms = b.tune(2)
    assert ms > 0
    for s, f in zip(slots, before):
        np.testing.assert_array_equal(b.get_populations(s), f)
        assert b.stats(s)["step"] == 5
    b.remove(slots[1])
    assert b.size() == 3
    b.step(4)
    # the remaining lattices continue exactly as alone
    for i in (0, 2, 3):
        g = lbm.Lattice(**cfgs[i])
        g.init(*_ic(cfgs[i], i))
        g.step(9)
        np.testing.assert_array_equal(b.get_populations(slots[i]), g.get_populations())


@pytest.mark.parametrize("seg_rows,waves", [(0, 1), (16, 2), (0, 4), (64, 1), (8, 8), (4, 2)])
def test_batch_shape_never_changes_results(seg_rows, waves):
    """The fused kernel's segment length and work-item budget change the work
    split only: every lattice matches its lone run bit for bit."""
    cfgs = [c for c in _mix() if c["lattice"] == lbm.D2Q9 and c["boundary"] == lbm.BC_WALLS]
    steps = 12
    alone = []
    for i, c in enumerate(cfgs):
        g = lbm.Lattice(**c)
        g.init(*_ic(c, i))
        g.step(steps)
        alone.append(g.get_populations())
    b = lbm.Batch()
    b.set_shape(seg_rows, waves)
    slots = [b.add(**c) for c in cfgs]
    for i, (c, s) in enumerate(zip(cfgs, slots)):
        b.init(s, *_ic(c, i))
    b.step(steps)
    b.synchronize()
    for i, s in enumerate(slots):
        np.testing.assert_array_equal(b.get_populations(s), alone[i], err_msg=f"lattice {i}")


def test_batched_tubes_match_lone_runs():
    """D1Q3 lattices of a batch run on the tube kernel in groups of 1024 sites
    handed out from one counter (a tube of many groups is shared between many
    warps), and a lone tube on the tube kernel with its own launch shape: the
    populations agree bit for bit, the counts exactly, the sums to the
    rounding of their other grouping."""
    sizes = [(800, lbm.BC_WALLS), (5003, lbm.BC_PERIODIC), (20001, lbm.BC_WALLS), (130000, lbm.BC_WALLS),
             (3, lbm.BC_WALLS)]
    cfgs = [dict(lattice=lbm.D1Q3, nx=n, ny=1, boundary=bc, precision=lbm.FP32, beta=0.999,
                 limiters=ALL, delta_median=1e-5, delta_ehrenfest=1e-4, k_max=max(1, n // 500)) for n, bc in sizes]
    steps = 60
    alone = []
    for c in cfgs:
        g = lbm.Lattice(**c)
        assert g.step_kernel() == lbm.KERNEL_TUBE
        g.init(*_ic(c, 0))
        g.step(steps)
        alone.append((g.get_populations(), g.stats(check=False), g.limited_sites()))
    b = lbm.Batch()
    slots = [b.add(**c) for c in cfgs]
    for c, s in zip(cfgs, slots):
        b.init(s, *_ic(c, 0))
    b.step(steps)
    try:
        b.synchronize()
    except lbm.LBMError as e:
        assert e.status == lbm.ERR_NONFINITE
    for i, s in enumerate(slots):
        f, st, sel = alone[i]
        np.testing.assert_array_equal(b.get_populations(s), f, err_msg=f"tube {i}")
        bs = b.stats(s)
        for key in ("n_pos", "n_med", "n_ehr", "n_cand", "n_bad"):
            assert bs[key] == st[key], (i, key)
        # FP32 sums of rho - rho_ref (-0.5 on half of a shock tube) over chunks of
        # 32 or 128 sites: each chunk total carries a rounding of up to 2^-24 of
        # its magnitude, so the two groupings agree to ~1e-8 relative
        assert abs(bs["mass"] - st["mass"]) <= 1e-7 * st["mass"]
        for key in ("sum_dS", "dS_lbgk", "dS_lim"):
            assert abs(bs[key] - st[key]) <= 1e-6 * abs(st[key]) + 1e-30, (i, key)
        np.testing.assert_array_equal(b.limited_sites(s), sel)
