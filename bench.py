"""Benchmark of the limited LBGK step: prints one JSON line.

Default workload: the 4096 x 4096 lid-driven cavity (D2Q9, Re = 7500, lid
0.05, median filter delta = 1e-3 plus Ehrenfests' trimming delta = 1e-3 with
k = 1677 = 0.01 % of the sites), FP32 populations, FP64 sums.  A bench step is
one limited LBGK step of the whole lattice (free flight, collision, dS,
positivity / median / Ehrenfests' limiters, FP64 sums) through lbm_step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the step does not shard across GPUs here); value = all ranks'
site updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_SITE = {("d2q9", "fp32"): 72, ("d2q9", "bf16"): 36, ("d2q9", "fp16"): 36, ("d2q9", "fp64"): 144, ("d1q3", "fp32"): 24,
                  ("d1q3", "fp64"): 48}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity4096",
                    choices=["cavity4096", "cavity100", "tube", "batched", "serve", "hopf"],
                    help="cavity4096: the 4096^2 cavity (default); cavity100: the 100^2 cavity at Re 5000; "
                         "tube: the 800-site D1Q3 shock tube (FP64); batched: 256 cavities of sides "
                         "64..512; serve: Poisson-arriving solves through the continuous-batching server")
    ap.add_argument("--graph", type=int, default=0,
                    help="single lattices: CUDA-graph replay of runs of this many steps (even; 0 = off)")
    ap.add_argument("--state", default="developed", choices=["developed", "active"],
                    help="developed: the flow after --develop steps from rest; active: every site "
                         "out of equilibrium (limiters act widely)")
    ap.add_argument("--tube-sites", type=int, default=800, help="tube: lattice sites")
    ap.add_argument("--hopf-re", default="7000,7125,7250,7375,7500,7625,7750,7875",
                    help="hopf: Reynolds numbers of the sweep (one lattice each)")
    ap.add_argument("--hopf-steps", type=int, default=0,
                    help="hopf: steps per lattice (default 5000 L / u0, the paper's protocol)")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests in the trace")
    ap.add_argument("--develop", type=int, default=-1,
                    help="untimed steps before warm-up so the flow has left the rest state "
                         "(default: the 4096^2 cavity's full 1e4 steps; 0 for the small workloads)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tiled", "fused", "tube"])
    ap.add_argument("--limiters", default="median+ehrenfest",
                    choices=["median+ehrenfest", "smooth+ehrenfest", "threshold+ehrenfest", "entthresh+ehrenfest"],
                    help="smooth / threshold: the ensemble-dependent limiters (tiled kernel, E(dS) reduction first)")
    ap.add_argument("--equilibrium", default="polynomial", choices=["polynomial", "entropic"],
                    help="entropic: Eq. maxwellian f* with the exact dS of Eq. DelS")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp16", "fp64"],
                    help="population storage (FP32 arithmetic for the 32- and 16-bit forms); default "
                         "fp32, fp64 for the shock tube")
    ap.add_argument("--side", type=int, default=4096,
                    help="cavity side (4096 is the workload; smaller sides are for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock, power and throttle reasons, every 50 ms,
    while the GPU is busy.  The sampler runs from the first untimed step (the flow's
    development and the warm-up) to the end of the timed region, so that a timed
    region of a few milliseconds still has a clock record of the load it sits in;
    `in_timed` counts the samples taken inside the timed region itself."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t_timed = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS), "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def timed_begin(self):
        self.t_timed = (time.perf_counter(), None)

    def timed_end(self):
        if self.t_timed is not None:
            self.t_timed = (self.t_timed[0], time.perf_counter())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(2 * self.INTERVAL_MS / 1e3)  # the sample that covers the region's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons, inside = [], [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.t_timed if self.t_timed else (None, None)
        for ts, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            if t0 is not None and t1 is not None and t0 <= ts <= t1 + self.INTERVAL_MS / 1e3:
                inside += 1
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm), "in_timed": inside,
                "interval_ms": self.INTERVAL_MS,
                "window": "development + warm-up + timed steps (GPU busy throughout)"}


# The sources each step kernel is compiled from (its .cu file and every header
# it includes): a recorded ncu figure stays valid while these are unchanged.
KERNEL_SOURCES = {
    "fused": ["paper_0704_0043_gb300/csrc/step_fused.cu", "paper_0704_0043_gb300/csrc/keys.cuh",
              "paper_0704_0043_gb300/csrc/lattice.cuh", "paper_0704_0043_gb300/csrc/internal.h",
              "include/lbm.h"],
    "tube": ["paper_0704_0043_gb300/csrc/step_tube.cu", "paper_0704_0043_gb300/csrc/lattice.cuh",
             "paper_0704_0043_gb300/csrc/internal.h", "include/lbm.h"],
    "tiled": ["paper_0704_0043_gb300/csrc/step_tiled.cu", "paper_0704_0043_gb300/csrc/lattice.cuh",
              "paper_0704_0043_gb300/csrc/internal.h", "include/lbm.h"],
}


def _code_only(text: str) -> str:
    """Source text without comments and whitespace: what the compiler sees."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def source_hash(kernel: str, read=None) -> str:
    """Hash of the code (comments and whitespace dropped) of the sources the
    kernel is compiled from; `read(rel)` returns a file's text (default: the tree)."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        if read is None:
            with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(rel)
        h.update(rel.encode() + _code_only(text).encode())
    return h.hexdigest()[:16]


def _profile_entry(kernel_name: str):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    ent = d.get(kernel_name)
    if not ent or ent.get("src_hash") != source_hash(kernel_name.split("_")[0]):
        return None
    return ent


def fp64_flops_from_profile(kernel_name: str, sites: int):
    """Executed FP64 FLOPs per launch (dadd + dmul + 2 dfma per thread
    instruction, from ncu) scaled to this lattice; None when the kernel's
    sources changed since the count was taken."""
    ent = _profile_entry(kernel_name)
    if not ent or "fp64_flops_per_site" not in ent:
        return None
    return ent["fp64_flops_per_site"] * sites


def traffic_from_profile(kernel_name: str, sites: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    scaled to this lattice; None when the kernel's sources changed since."""
    ent = _profile_entry(kernel_name)
    if not ent:
        return None
    return ent["dram_bytes_per_site"] * sites


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks of the default process group (x itself
    when there is none): the timed region ends when the slowest replica does."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, sites: int, steps: int, elapsed_s: float) -> float:
    """Site updates of all replicas (each runs its own lattice) per second, in millions."""
    return world * sites * steps / elapsed_s / 1e6


def timing_every(steps: int) -> int:
    """The step and tail kernels are timed with CUDA events on one step in this
    many: events between two kernels delay the next launch by a few microseconds,
    so long runs sample one step in 8, short ones (a few dozen steps) every second
    step so that the kernel average still rests on several launches."""
    return 2 if steps < 200 else 8


def workload(side: int = 4096):
    from paper_0704_0043_gb300 import inputs
    w = inputs.cavity4096_workload()
    if side != w.nx:
        w.nx = w.ny = side
        w.name = f"cavity_d2q9_{side}_re7500"
        w.k_max = int(1e-4 * side * side)
    return w


def lattice_kwargs(w, kernel: str, precision: str = "fp32", equilibrium: str = "polynomial"):
    from paper_0704_0043_gb300 import lbm
    km = {"auto": lbm.KERNEL_AUTO, "tiled": lbm.KERNEL_TILED, "fused": lbm.KERNEL_FUSED, "tube": lbm.KERNEL_TUBE}[kernel]
    pm = {"fp32": lbm.FP32, "bf16": lbm.BF16, "fp16": lbm.FP16, "fp64": lbm.FP64}[precision]
    em = {"polynomial": lbm.EQ_POLYNOMIAL, "entropic": lbm.EQ_ENTROPIC}[equilibrium]
    return dict(lattice=lbm.D2Q9, nx=w.nx, ny=w.ny, boundary=lbm.BC_WALLS, precision=pm,
                beta=w.beta, u_lid=w.u_lid, rho_wall=w.rho0, limiters=w.limiters,
                delta_median=w.delta_median, delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max,
                kernel=km, equilibrium=em)


def oracle_cfg(w, side: int, equilibrium: str = "polynomial"):
    import oracle
    return oracle.Config(lattice=oracle.D2Q9, nx=side, ny=side, boundary=oracle.BC_WALLS,
                         beta=w.beta, u_lid=w.u_lid, rho_wall=w.rho0, limiters=w.limiters,
                         delta_median=w.delta_median, delta_ehrenfest=w.delta_ehrenfest,
                         k_max=max(1, int(1e-4 * side * side)),
                         equilibrium=oracle.EQ_ENTROPIC if equilibrium == "entropic" else oracle.EQ_POLYNOMIAL)


def cpu_baseline(w, steps: int = 1, equilibrium: str = "polynomial"):
    """The FP64 oracle as it stands, single-threaded, on `steps` full-size steps."""
    import oracle
    from paper_0704_0043_gb300 import inputs
    oc = oracle_cfg(w, w.nx, equilibrium)
    rho, ux, uy = inputs.cavity_rest(w.nx, w.ny, w.rho0)
    f = oracle.init(oc, rho, ux, uy)
    t0 = time.perf_counter()
    f, _, _ = oracle.run(oc, f, steps)
    dt = time.perf_counter() - t0
    return {"value": w.sites * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} step(s) of the full {w.nx}x{w.ny} cavity, FP64, one thread, "
                      f"{dt:.1f} s"}


def run_reference(args):
    """The oracle timed as it stands on the host, K steps of a 1024^2 sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_0704_0043_gb300 import inputs
    w = workload()
    side = 1024
    oc = oracle_cfg(w, side)
    rho, ux, uy = inputs.cavity_rest(side, side, w.rho0)
    f = oracle.init(oc, rho, ux, uy)
    f, _, _ = oracle.run(oc, f, args.warmup)
    t0 = time.perf_counter()
    f, _, _ = oracle.run(oc, f, args.steps)
    dt = time.perf_counter() - t0
    v = side * side * args.steps / dt / 1e6
    sample = (f"{side}x{side} cavity with the {w.nx}^2 workload's parameters (Re 7500, lid 0.05, "
              f"median + Ehrenfests' k = 0.01 % of sites), one oracle step per bench step")
    out = {"impl": "reference", "metric": "limited-LBM MLUPS", "value": v, "unit": "MLUPS",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "sample_side": side},
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(args):
    """256 cavities (sides U{64..512}, Re U[2000, 7500], lid 0.1, one limiter each
    drawn from positivity / Ehrenfests' / median), FP32, advanced together by the
    batch engine (shared launches, CUDA-graph replay, autotuned tiles), against
    the same lattices stepped one after another through lbm_step."""
    import torch
    from paper_0704_0043_gb300 import build as lbm_build
    from paper_0704_0043_gb300 import inputs, lbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lbm_build.build()
    ws = inputs.batched_cavities()
    sites = sum(w.sites for w in ws)
    def kw(w):
        return dict(lattice=lbm.D2Q9, nx=w.nx, ny=w.ny, boundary=lbm.BC_WALLS, precision=lbm.FP32,
                    beta=w.beta, u_lid=w.u_lid, rho_wall=w.rho0, limiters=w.limiters,
                    delta_median=w.delta_median, delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max)
    b = lbm.Batch()
    slots = [b.add(**kw(w)) for w in ws]
    for s, w in zip(slots, ws):
        b.init(s, *inputs.cavity_rest(w.nx, w.ny, w.rho0))
    graph = 50
    b.set_graph(graph)
    tuned_ms = b.tune(3)
    def sync_batch():
        try:
            b.synchronize()
        except lbm.LBMError as e:  # lattices that blew up keep their (equal-cost) steps
            if e.status != lbm.ERR_NONFINITE:
                raise
    b.step(max(args.warmup, 2 * graph))
    sync_batch()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_batch = ev0.elapsed_time(ev1) / 1e3
    launches = b.launch_count() - l0
    sync_batch()
    nonfinite = sum(b.lattice_status(s) != lbm.OK for s in slots)
    # the same lattices one by one (plain per-instance launches)
    plain_steps = max(20, args.steps // 10)
    lats = []
    for w in ws:
        g = lbm.Lattice(**kw(w))
        g.init(*inputs.cavity_rest(w.nx, w.ny, w.rho0))
        g.step(2)
        lats.append(g)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(plain_steps):
        for g in lats:
            g.step(1)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_plain = ev0.elapsed_time(ev1) / 1e3
    v = sites * args.steps / t_batch / 1e6
    vp = sites * plain_steps / t_plain / 1e6
    peak, kind = peaks()
    out = {"metric": "batched limited-LBM MLUPS", "value": v, "unit": "MLUPS", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "batched_cavities_256", "lattices": len(ws), "sites": sites,
                      "sides": "U{64..512}", "graph_steps": graph, "tuned_ms_per_step": tuned_ms},
           "plain_value": vp, "plain_steps": plain_steps, "batched_over_plain": v / vp,
           "nonfinite_lattices": nonfinite,
           "roofline": {"bound": "hbm", "achieved": 72 * sites * args.steps / t_batch / 1e9,
                        "peak": peak, "unit": "GB/s", "frac": 72 * sites * args.steps / t_batch / 1e9 / peak,
                        "peak_kind": kind, "note": "whole batched step (all launches), not one kernel"},
           "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)
    b.close()


def hopf_energy(u, L, u0):
    """E_u^2 of Sec. 4.4.2 (Eq. energy): E_u = || sqrt(L / (u0 |u|)) (u - mean(u)) ||_2 over the
    final 1 % of the control-point signal u, |u| its length, so E_u^2 = (L / u0) var(u)."""
    import numpy as np
    u = np.asarray(u, dtype=np.float64)
    return float((L / u0) * np.mean((u - u.mean()) ** 2))


def hopf_fit(res, e2):
    """Re_c of Sec. 4.4.2: E_u^2 grows linearly with Re past a Hopf bifurcation, so a
    line fitted through the points clearly above the steady level (E_u^2 above a
    tenth of the largest) meets E_u^2 = 0 at the critical Re.  None with fewer than
    two such points."""
    import numpy as np
    res, e2 = np.asarray(res, float), np.asarray(e2, float)
    up = e2 > 0.1 * e2.max() if e2.max() > 0 else np.zeros_like(e2, bool)
    if up.sum() < 2:
        return None
    a, b = np.polyfit(res[up], e2[up], 1)
    return float(-b / a) if a > 0 else None


def dominant_frequency(u, L, u0):
    """Frequency of the largest non-zero Fourier mode of the control-point signal,
    in cycles per non-dimensional time unit L / u0 (one sample per step)."""
    import numpy as np
    u = np.asarray(u, float) - np.mean(u)
    spec = np.abs(np.fft.rfft(u * np.hanning(len(u))))
    freq = np.fft.rfftfreq(len(u), d=u0 / L)  # d = non-dimensional time per step
    k = 1 + int(np.argmax(spec[1:]))
    return float(freq[k])


def run_hopf(args):
    """The first Hopf bifurcation of the lid-driven cavity (Sec. 4.4.2): 100 x 100,
    boundary nodes on the walls with the diffusive Maxwell wall, lid 0.1, density 1,
    median filter delta = 1e-3, polynomial f* in FP32 (the paper finds no
    significant difference between polynomial and entropic f* in the cavity,
    Sec. 4.4.1), one lattice per Re of the sweep, all in one batch with graph
    replay.  Each lattice records u at the control point (L/16, 13L/16) every step;
    E_u^2 of the final 1 % of 5000 non-dimensional time units (5000 L / u0 steps)
    gives Re_c by the line fit of Sec. 4.4.2."""
    import numpy as np
    import torch
    from paper_0704_0043_gb300 import build as lbm_build
    from paper_0704_0043_gb300 import inputs, lbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lbm_build.build()
    n, u0 = 100, 0.1
    L = n - 1  # between the wall nodes
    res = [float(r) for r in args.hopf_re.split(",")]
    steps = args.hopf_steps if args.hopf_steps > 0 else int(round(5000 * L / u0))
    rec = max(2, steps // 100)
    ci, cj = int(round(L / 16)), int(round(13 * L / 16))
    b = lbm.Batch()
    slots = []
    for re in res:
        s = b.add(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_DIFFUSIVE, precision=lbm.FP32,
                  beta=inputs.beta_from_nu(inputs.cavity_nu(L, u0, re)), u_lid=u0, rho_wall=1.0,
                  limiters=lbm.LIM_MEDIAN, delta_median=1e-3)
        b.init(s, *inputs.cavity_rest(n, n))
        b.probe(s, cj * n + ci, rec)
        slots.append(s)
    b.set_graph(1000)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count()
    torch.cuda.synchronize()
    sampler.timed_begin()
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.timed_end()
    clocks = sampler.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    failed = []
    try:
        b.synchronize()
    except lbm.LBMError:
        pass
    e2, freqs = [], []
    for re, s in zip(res, slots):
        if b.lattice_status(s) != lbm.OK:
            failed.append(re)
            e2.append(float("nan"))
            freqs.append(float("nan"))
            continue
        sig = b.probe_read(s, rec)[:, 1]  # u_x at the control point, final 1 %
        e2.append(hopf_energy(sig, L, u0))
        freqs.append(dominant_frequency(sig, L, u0))
    ok = [i for i, v in enumerate(e2) if np.isfinite(v)]
    re_c = hopf_fit([res[i] for i in ok], [e2[i] for i in ok])
    sites = len(res) * n * n
    v = sites * steps / t / 1e6
    out = {"metric": "batched limited-LBM MLUPS", "value": v, "unit": "MLUPS", "n_gpus": 1, "steps": steps,
           "warmup": 0, "ms_per_step": t * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "hopf_sweep_cavity100_diffusive", "lattices": len(res), "nx": n, "ny": n,
                      "walls": "diffusive Maxwell (boundary nodes)", "u_lid": u0, "rho0": 1.0,
                      "limiters": "median", "delta": 1e-3, "equilibrium": "polynomial", "storage": "fp32",
                      "control_point": [ci, cj], "record_steps": rec, "graph_steps": 1000,
                      "l2": "lattices resident in L2 (no flush: the workload itself is that small)"},
           "hopf": {"re": res, "E_u2": e2, "re_c_fit": re_c, "dominant_frequency": freqs,
                    "frequency_unit": "cycles per L/u0", "failed_re": failed,
                    "paper": {"re_c": 7135, "omega_at_7375": 0.525}},
           "gpu_launches": b.launch_count() - l0, "clocks": clocks}
    print(json.dumps(out), flush=True)
    b.close()


def run_serve(args):
    """Poisson arrivals (200/s): 70 % cavities of side 100..1024, 30 % shock
    tubes of 800..1e6 sites (density ratio 1:2..1:4), 1e3..1e5 steps each,
    served by continuous batching with admission by HBM footprint.  The 200/s
    trace offers far more work than one GPU can do (an overload run); the same
    requests are then replayed at about 70 % of the measured capacity."""
    import torch
    from paper_0704_0043_gb300 import build as lbm_build
    from paper_0704_0043_gb300 import inputs, serve
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    lbm_build.build()
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.7)
    trace = inputs.serving_trace(n_requests=args.requests)
    work = sum(w.sites * w.steps for _, w in trace)
    out_runs = {}
    for label, scale in (("overload_200hz", 1.0), ("capacity_70pct", None)):
        if scale is None:
            cap_rps = out_runs["overload_200hz"]["aggregate_mlups"] * 1e6 / (work / len(trace))
            rate = 0.7 * cap_rps
            scale = 200.0 / rate
        reqs = serve.requests_from_trace([(t * scale, w) for t, w in trace])
        srv = serve.Server(memory_bytes=budget, quantum=1000, graph_steps=0)
        t0 = time.perf_counter()
        res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        s = serve.summarize(res, wall, srv.site_updates)
        s["arrival_rate_hz"] = 200.0 / scale
        s["rounds"] = srv.rounds
        out_runs[label] = s
        srv.close()
    o = out_runs["overload_200hz"]
    print(json.dumps({"metric": "served limited-LBM MLUPS", "value": o["aggregate_mlups"], "unit": "MLUPS",
                      "n_gpus": 1, "steps": None, "warmup": 0, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "serving_trace_7040044", "requests": len(trace),
                                 "site_updates": work, "memory_budget_bytes": budget,
                                 "quantum_steps": 1000},
                      "p50_latency_s": o["p50_latency_s"], "p99_latency_s": o["p99_latency_s"],
                      "runs": out_runs}), flush=True)


def single_workload(args, lbm, inputs):
    """(workload, lattice kwargs, lattice kind, storage) of the single-lattice lines."""
    if args.workload == "tube":
        # the 1:2 shock tube of Sec. 4.3: 800 sites, nu = 1e-9, Ehrenfests' delta = 1e-3, k = 4, FP64
        w = inputs.shock_tube_workload(args.tube_sites)
        prec = args.precision or "fp64"
        kw = dict(lattice=lbm.D1Q3, nx=w.nx, ny=1, boundary=lbm.BC_WALLS,
                  precision={"fp32": lbm.FP32, "fp64": lbm.FP64}[prec], beta=w.beta, limiters=w.limiters,
                  delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max,
                  kernel={"auto": lbm.KERNEL_AUTO, "tiled": lbm.KERNEL_TILED, "tube": lbm.KERNEL_TUBE}[args.kernel])
        return w, kw, "d1q3", prec
    if args.workload == "cavity100":
        # the 100 x 100 cavity at Re = 5000 (lid 0.1), median filter, FP32
        w = inputs.cavity100_workload()
        kw = lattice_kwargs(w, args.kernel, args.precision, args.equilibrium)
        kw["rho_ref"] = w.rho0
        kw["boundary"] = w.boundary  # boundary nodes on the walls (tiled kernel)
        return w, kw, "d2q9", args.precision
    w = workload(args.side)
    if args.limiters != "median+ehrenfest":
        # Eq. smooth1 with k = 1/2, delta = 0.01, or the threshold filter with dS_t = 10 E(dS)
        # or Eq. EntThresh's dS_0 with delta_0 = 0.1
        kind = {"smooth": lbm.LIM_SMOOTH, "threshold": lbm.LIM_THRESHOLD, "entthresh": lbm.LIM_ENTTHRESH}
        w.limiters = kind[args.limiters.split("+")[0]] | lbm.LIM_EHRENFEST
        w.name = w.name + "_" + args.limiters.split("+")[0]
    if args.equilibrium == "entropic":
        w.name = w.name.replace("cavity_d2q9", "cavity_d2q9_entropic")
    return w, lattice_kwargs(w, args.kernel, args.precision, args.equilibrium), "d2q9", args.precision


def initial_fields(w, inputs):
    if w.lattice == 1:
        rho, ux = inputs.shock_tube(w.nx, 1.0, w.rho_right)
        return rho, ux, None
    return inputs.cavity_rest(w.nx, w.ny, w.rho0)


def main():
    args = parse()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "tube" else "fp32"
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "hopf":
        run_hopf(args)
        return
    import numpy as np
    import torch

    from paper_0704_0043_gb300 import build as lbm_build
    from paper_0704_0043_gb300 import inputs, lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        lbm_build.build()
    if dist is not None:
        dist.barrier()
    lbm.lib()

    w, kw, lat_kind, prec = single_workload(args, lbm, inputs)
    entropic = args.equilibrium == "entropic"
    develop = args.develop if args.develop >= 0 else (10000 if args.workload == "cavity4096" else 0)
    lat = lbm.Lattice(**kw)
    if args.graph:
        lat.set_graph(args.graph)
    fields = initial_fields(w, inputs)
    sampler = ClockSampler(local)
    sampler.start()
    lat.init(*fields)
    f_act = None
    if args.state == "active":
        # every site out of equilibrium, the full-size parity state: seeded random
        # deviations of the rest state, W_k (1 + 0.15 U(-1, 1)), and 5000 sites with
        # one population raised eightfold, so that the median filter forms its
        # stencil in every row and Ehrenfests' candidates outnumber k.  The flow
        # relaxes such a state within a few steps, so every timed step starts from
        # it: it is reloaded on the device (untimed) before each step.
        wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4) if lat_kind == "d2q9" else np.array([2 / 3, 1 / 6, 1 / 6])
        fa = inputs.random_populations(704, len(wts), w.ny, w.nx, w.rho0 * wts, 0.15)
        rng = np.random.default_rng(705)
        for _ in range(5000):
            fa[rng.integers(1, len(wts)), rng.integers(0, w.ny), rng.integers(0, w.nx)] *= 8.0
        f_act = torch.from_numpy(fa).cuda()
        del fa
        lat.set_populations(f_act)
        develop = 0
    lat.step(develop + args.warmup)
    lat.synchronize()

    stream = torch.cuda.current_stream()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lat.launch_count()
    every = timing_every(args.steps)
    # per-kernel events on one step in `every` (events between the kernels delay
    # the next launch, so timing every step would slow the measured run); graph
    # replay is off while they are recorded, so the graph line times the steps alone
    if f_act is not None:
        every = 1  # each timed step is its own launch pair
    if not args.graph:
        lat.timing(True, every=every)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.timed_begin()
    if f_act is None:
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed = ev0.elapsed_time(ev1) / 1e3
    else:
        # one step at a time from the active state, each timed by its own events
        elapsed = 0.0
        for _ in range(args.steps):
            lat.set_populations(f_act)
            ev0.record(stream)
            lat.step(1)
            ev1.record(stream)
            torch.cuda.synchronize()
            elapsed += ev0.elapsed_time(ev1) / 1e3
        launches0 += args.steps  # the reloads are not steps
    sampler.timed_end()
    launches = lat.launch_count() - launches0
    step_ms, tail_ms, timed = lat.timing_read() if not args.graph else (0.0, 0.0, 0)
    lat.timing(False)
    clocks = sampler.stop()
    st = lat.stats()
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    mlups = whole_job_mlups(world, w.sites, args.steps, elapsed)

    # roofline of the step kernel (the dominant launch): algorithmic bytes / event time
    bps = BYTES_PER_SITE[(lat_kind, prec)]
    ensemble = args.limiters != "median+ehrenfest" and args.workload == "cavity4096"
    if ensemble:
        # the pass first reads every population once more for E(dS) (k_ens_partial);
        # the library's events bracket that reduction and the step kernel together
        bps += bps // 2
        if args.limiters.startswith("entthresh"):
            bps += 8  # Eq. EntThresh: the dS field written once and read once (FP32)
    if timed:
        kern_s = step_ms / 1e3 / timed
    else:  # graph replay: the whole step (step kernel + tail) from the run's own events
        kern_s = elapsed / args.steps
    achieved = bps * w.sites / kern_s / 1e9
    peak, peak_kind = peaks()
    kname = {lbm.KERNEL_FUSED: "fused", lbm.KERNEL_TUBE: "tube"}.get(lat.step_kernel(), "tiled")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": traffic_from_profile(f"{kname}_{prec}", w.sites),
            "kernel": kname if timed else "whole step (graph replay)", "kernel_ms": kern_s * 1e3,
            "tail_kernel_ms": tail_ms / max(timed, 1), "timed_launches": timed, "timed_every": every,
            "bytes_per_site": bps}
    if w.sites * bps < 100e6:
        roof["note"] = ("the lattice lives in L2 (%.1f MB of populations); the step is launch- and "
                        "latency-bound, so this fraction is no HBM claim" % (w.sites * bps / 1e6))
    if ensemble:
        # E(dS) by the fused kernel's row streaming (nothing stored) for FP32
        # cavities, by k_ens_partial otherwise
        epass = "k_fused E(dS) pass + k_ens_fx" if prec == "fp32" else "k_ens_partial + k_ens_mean"
        roof["kernel"] = epass + " + " + ("EntThresh solve + " if args.limiters.startswith("entthresh")
                                           else "") + ("k_fused" if kname == "fused" else "k_tiled")
        roof["traffic"] = traffic_from_profile("fused_fp32_ensemble" if prec == "fp32" else "tiled_fp32_ensemble",
                                               w.sites)

    if entropic and prec == "fp64":
        # The entropic step is bound by FP64 arithmetic (a logarithm per population
        # and sqrt / divisions for f*), not by HBM: the roofline is the FP64 pipe
        # (152 SMs x 2 FP64 FMA per clock x 2 FLOP at the sampled SM clock), and
        # the executed FP64 FLOPs per site come from one ncu count of the kernel's
        # FP64 instructions (profiles/traffic.json).
        fl = fp64_flops_from_profile("tiled_fp64_entropic", w.sites)
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        fpeak = 152 * 2 * 2 * mhz * 1e6 / 1e9
        roof_hbm = dict(roof)
        roof = {"bound": "alu", "unit": "GFLOP/s", "peak": fpeak,
                "peak_kind": "derived: 152 SMs x 4 FP64 FLOP/clk x sampled SM clock",
                "achieved": fl / kern_s / 1e9 if fl else None,
                "frac": (fl / kern_s / 1e9) / fpeak if fl else None,
                "fp64_flops_per_site": fl / w.sites if fl else None,
                "traffic": traffic_from_profile("tiled_fp64_entropic", w.sites), "kernel": kname,
                "kernel_ms": kern_s * 1e3,
                "tail_kernel_ms": roof_hbm["tail_kernel_ms"], "timed_launches": timed,
                "timed_every": every, "hbm": {k: roof_hbm[k] for k in ("achieved", "peak", "frac", "bytes_per_site")}}

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(lat, w, args.steps, torch, fields)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_for(args, w, kw)
    if args.workload == "cavity4096":
        cfg = {"workload": w.name, "nx": w.nx, "ny": w.ny, "reynolds": 7500,
               "u_lid": w.u_lid, "beta": w.beta, "limiters": args.limiters,
               "delta": 1e-3, "k_max": w.k_max, "storage": prec, "sums": "fp64",
               "equilibrium": args.equilibrium}
    elif args.workload == "cavity100":
        cfg = {"workload": w.name, "nx": w.nx, "ny": w.ny, "reynolds": 5000, "u_lid": w.u_lid,
               "rho0": w.rho0, "beta": w.beta, "walls": "boundary nodes on the walls, bounce-back",
               "limiters": "median", "delta": w.delta_median,
               "storage": prec, "sums": "fp64", "equilibrium": args.equilibrium}
    else:
        cfg = {"workload": w.name if w.nx == 800 else f"shock_tube_d1q3_{w.nx}", "sites": w.nx,
               "density_ratio": "1:2", "nu": 1e-9, "beta": w.beta, "limiters": "ehrenfest",
               "delta": w.delta_ehrenfest, "k_max": w.k_max, "storage": prec}
    cfg.update({"kernel": kname, "develop_steps": develop, "state": args.state,
                "graph_steps": args.graph,
                "l2": ("inputs larger than L2 (%.2f GB population buffers vs 129 MB L2)" % (w.sites * bps / 2 / 1e9)
                       if w.sites * bps / 2 > 129e6 else
                       "lattice resident in L2 (%.2f MB of populations); no flush: the workload itself is that small"
                       % (w.sites * bps / 1e6)),
                "parallelism": f"replicas{world}" if world > 1 else "single"})
    out = {"metric": "limited-LBM MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": elapsed * 1e3 / args.steps, "us_per_step": elapsed * 1e6 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic", "config": cfg,
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "clocks": clocks,
           "last_step_stats": {k: st[k] for k in ("step", "mass", "sum_dS", "dS_lim", "n_pos", "n_med",
                                                   "n_ehr", "n_cand")}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    lat.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline_for(args, w, kw):
    """The oracle as it stands, one thread, on a bounded sample of the workload."""
    import oracle
    from paper_0704_0043_gb300 import inputs
    if args.workload == "cavity4096":
        return cpu_baseline(w, 1, args.equilibrium)
    oc = oracle.Config(lattice=kw["lattice"], nx=w.nx, ny=w.ny, boundary=kw.get("boundary", 0), beta=w.beta,
                       u_lid=w.u_lid, rho_wall=w.rho0, limiters=w.limiters, delta_median=w.delta_median,
                       delta_ehrenfest=w.delta_ehrenfest, k_max=w.k_max)
    f = oracle.init(oc, *initial_fields(w, inputs))
    steps = 400 if args.workload == "tube" else 1000
    t0 = time.perf_counter()
    f, _, _ = oracle.run(oc, f, steps)
    dt = time.perf_counter() - t0
    return {"value": w.sites * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the full workload ({w.nx}x{w.ny}), FP64, one thread, {dt:.2f} s"}


def end_to_end(lat, w, steps, torch, fields):
    """Same metric through the public API with pinned host buffers: upload the
    initial density/velocity fields, run `steps` steps, read the moments and
    the stats back; the copies are inside the timed region."""
    import numpy as np
    rho, ux, uy = fields
    hin = [torch.from_numpy(a.reshape(-1).copy()).pin_memory() for a in (rho, ux, uy) if a is not None]
    nout = 3 if uy is not None else 2
    hout = [torch.empty(w.sites, dtype=torch.float64).pin_memory() for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.init(*hin)
    lat.step(steps)
    lat.moments(out=tuple(hout))
    st = lat.stats()
    dt = time.perf_counter() - t0
    assert np.isfinite(st["mass"])
    h2d = len(hin) * 8 * w.sites
    d2h = nout * 8 * w.sites + 96
    return {"value": w.sites * steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "request": f"init from host rho/u, {steps} steps, moments + stats to host"}


if __name__ == "__main__":
    main()
