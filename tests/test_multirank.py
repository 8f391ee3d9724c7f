"""The N > 1 path of bench.py on the CPU: replicas only (each rank runs its own
lattice, no collective on the data path), so the host logic is the barrier,
the maximum of the ranks' timed regions and the whole-job value.  Two gloo
ranks, spawned as separate processes, each report a different elapsed time;
both must see the maximum, and the value must count both replicas' sites."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        elapsed = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        q.put((rank, elapsed, bench.whole_job_mlups(world, 1_000_000, 20, elapsed)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica_and_count_both():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert all(abs(o[2] - 2 * 1_000_000 * 20 / 2.5 / 1e6) < 1e-9 for o in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, None, "cpu") == 0.25
    assert bench.whole_job_mlups(1, 4096 * 4096, 100, 0.5) == 4096 * 4096 * 100 / 0.5 / 1e6
