"""Host logic of the continuous-batching server (paper_0704_0043_gb300/serve.py)
on the CPU, with a stand-in batch that records what the server asks of it:
admission by device footprint within the memory budget, first come first
served; every lattice advanced exactly its step count (rounds never overshoot
a resident lattice); a lattice that meets a nonfinite site retired as failed
while the others carry on; a request larger than the budget refused.  The
footprints come from the C library's lbm_footprint_bytes (validation only, no
GPU).  The same loop over the real batch runs in tests/test_gpu_serve.py."""
import numpy as np
import pytest

from paper_0704_0043_gb300 import build as lbm_build
from paper_0704_0043_gb300 import inputs, lbm, serve


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lbm_build.build()
    lbm.lib()


class FakeBatch:
    def __init__(self, poison=()):
        self.slots = {}
        self.next = 0
        self.poison = set(poison)  # nx of lattices that blow up on their first round
        self.log = []

    def set_graph(self, n):
        pass

    def add(self, **cfg):
        s = self.next
        self.next += 1
        self.slots[s] = {"cfg": cfg, "steps": 0, "bad": False}
        self.log.append(("add", s, cfg["nx"]))
        return s

    def init(self, s, rho, ux, uy):
        assert np.all(np.isfinite(rho))

    def step(self, n):
        assert n > 0
        for s, d in self.slots.items():
            d["steps"] += n
            if d["cfg"]["nx"] in self.poison:
                d["bad"] = True
        self.log.append(("step", n, sorted(self.slots)))

    def synchronize(self):
        if any(d["bad"] for d in self.slots.values()):
            raise lbm.LBMError(lbm.ERR_NONFINITE, "nonfinite")

    def lattice_status(self, s):
        return lbm.ERR_NONFINITE if self.slots[s]["bad"] else lbm.OK

    def moments(self, s):
        cfg = self.slots[s]["cfg"]
        z = np.zeros((cfg["ny"], cfg["nx"]))
        return z, z, z

    def stats(self, s):
        return {"step": self.slots[s]["steps"]}

    def remove(self, s):
        self.log.append(("remove", s, self.slots[s]["steps"]))
        del self.slots[s]

    def close(self):
        pass


def _cavity(side, steps):
    return inputs.Workload(f"cavity{side}", 2, side, side, 0.99, 0.1, 1.0, lbm.LIM_MEDIAN, steps=steps)


def _requests(sides_steps):
    return [serve.Request(i, 0.001 * i, _cavity(s, n)) for i, (s, n) in enumerate(sides_steps)]


def _footprint(side):
    return lbm.footprint_bytes(**serve.lattice_config(_cavity(side, 1)))


def test_admission_stays_within_the_memory_budget_first_come_first_served():
    reqs = _requests([(64, 700), (64, 300), (64, 1200), (64, 100), (64, 900)])
    budget = int(2.5 * _footprint(64))
    fb = FakeBatch()
    srv = serve.Server(budget, quantum=250, batch=fb)
    peaks = []
    res = srv.run(reqs, realtime=False, on_round=lambda s, active: peaks.append(sum(a[3] for a in active.values())))
    assert len(res) == 5 and all(r.status == "ok" for r in res)
    assert max(peaks) <= budget
    adds = [e for e in fb.log if e[0] == "add"]
    assert [a[1] for a in adds] == sorted(a[1] for a in adds)  # slots taken in arrival order
    admitted = sorted(res, key=lambda r: r.rid)
    assert all(a.admitted <= b.admitted for a, b in zip(admitted, admitted[1:]))
    # never more than two resident at once: every step round covers at most two slots
    assert max(len(e[2]) for e in fb.log if e[0] == "step") == 2


def test_every_lattice_runs_exactly_its_step_count():
    steps = [700, 300, 1250, 100, 901, 2]
    reqs = _requests([(32 + 8 * i, n) for i, n in enumerate(steps)])
    fb = FakeBatch()
    srv = serve.Server(10 ** 12, quantum=256, batch=fb)
    res = srv.run(reqs, realtime=False)
    removed = {e[1]: e[2] for e in fb.log if e[0] == "remove"}
    assert sorted(removed.values()) == sorted(steps)
    for r in res:
        assert r.steps == steps[r.rid] and r.stats["step"] == steps[r.rid]
    # a round is never longer than the quantum or than any resident lattice's remaining steps
    assert all(e[1] <= 256 for e in fb.log if e[0] == "step")
    assert srv.steps_run == sum(e[1] for e in fb.log if e[0] == "step")


def test_a_blown_up_lattice_retires_as_failed_and_the_others_finish():
    reqs = _requests([(40, 600), (48, 600), (56, 600)])
    fb = FakeBatch(poison={48})
    res = serve.Server(10 ** 12, quantum=200, batch=fb).run(reqs, realtime=False)
    by = {r.rid: r for r in res}
    assert by[1].status == "nonfinite" and by[1].rho is None
    assert by[0].status == "ok" and by[2].status == "ok"
    assert by[0].steps == 600 and by[2].steps == 600
    s = serve.summarize(res, 1.0, 10)
    assert s["requests"] == 3 and s["failed"] == 1


def test_a_request_above_the_budget_is_refused():
    reqs = _requests([(256, 10)])
    with pytest.raises(ValueError):
        serve.Server(_footprint(256) - 1, batch=FakeBatch()).run(reqs, realtime=False)
