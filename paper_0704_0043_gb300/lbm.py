"""Thin ctypes binding over liblbm's C ABI (include/lbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
they must be contiguous float64 of the documented size.  PyTorch supplies the
CUDA stream (``torch.cuda.current_stream()``) when it is importable.

The library must have been built (``paper_0704_0043_gb300.build.build()`` or
``__graft_entry__.build()``); loading raises otherwise -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

D1Q3, D2Q9 = 1, 2
FP64, FP32, BF16, FP16 = 0, 1, 2, 3
BC_WALLS, BC_PERIODIC, BC_CHANNEL, BC_NODE_WALLS, BC_DIFFUSIVE = 0, 1, 2, 3, 4
LIM_POSITIVITY, LIM_EHRENFEST, LIM_MEDIAN, LIM_SMOOTH, LIM_THRESHOLD, LIM_ENTTHRESH = 1, 2, 4, 8, 16, 32
MEDIAN_THRESHOLD, MEDIAN_GATE = 0, 1
EQ_POLYNOMIAL, EQ_ENTROPIC = 0, 1
KERNEL_AUTO, KERNEL_TILED, KERNEL_FUSED, KERNEL_TUBE = 0, 1, 2, 3
COLL_LBGK, COLL_ELBM = 0, 1
PHI_HOMOTHETY, PHI_ENTROPY = 0, 1

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = range(7)


class Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("boundary", ctypes.c_int32), ("precision", ctypes.c_int32), ("limiters", ctypes.c_uint32),
        ("median_mode", ctypes.c_int32), ("kernel", ctypes.c_int32), ("beta", ctypes.c_double),
        ("u_lid", ctypes.c_double), ("rho_wall", ctypes.c_double), ("delta_median", ctypes.c_double),
        ("delta_ehrenfest", ctypes.c_double), ("k_max", ctypes.c_int64),
        ("stats_history", ctypes.c_int32), ("equilibrium", ctypes.c_int32), ("rho_ref", ctypes.c_double),
        ("smooth_delta", ctypes.c_double), ("smooth_k", ctypes.c_double), ("threshold_c", ctypes.c_double),
        ("threshold_delta", ctypes.c_double), ("collision", ctypes.c_int32), ("phi_rule", ctypes.c_int32),
        ("entthresh_delta0", ctypes.c_double),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("mass", ctypes.c_double), ("sum_dS", ctypes.c_double),
        ("dS_lbgk", ctypes.c_double), ("dS_lim", ctypes.c_double), ("n_pos", ctypes.c_int64),
        ("n_med", ctypes.c_int64), ("n_ehr", ctypes.c_int64), ("n_cand", ctypes.c_int64),
        ("n_bad", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


_LIB = None


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """The loaded liblbm (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm is not built ({path} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        cfgp = ctypes.POINTER(Config)
        L.lbm_config_default.argtypes = [cfgp]
        L.lbm_config_default.restype = None
        L.lbm_create.argtypes = [cfgp, vp, ctypes.POINTER(vp)]
        L.lbm_destroy.argtypes = [vp]
        L.lbm_init.argtypes = [vp, vp, vp, vp]
        L.lbm_step.argtypes = [vp, ctypes.c_int64]
        L.lbm_delta_s.argtypes = [vp, vp]
        L.lbm_limit.argtypes = [vp, ctypes.c_uint32]
        L.lbm_moments.argtypes = [vp, vp, vp, vp]
        L.lbm_stats.argtypes = [vp, ctypes.POINTER(StepStats)]
        L.lbm_stats_history.argtypes = [vp, ctypes.POINTER(StepStats), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64)]
        L.lbm_limited_sites.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_get_populations.argtypes = [vp, vp]
        L.lbm_set_populations.argtypes = [vp, vp]
        L.lbm_synchronize.argtypes = [vp]
        L.lbm_get_config.argtypes = [vp, cfgp]
        L.lbm_device_bytes.argtypes = [vp]
        L.lbm_device_bytes.restype = ctypes.c_int64
        L.lbm_footprint_bytes.argtypes = [cfgp]
        L.lbm_footprint_bytes.restype = ctypes.c_int64
        L.lbm_timing.argtypes = [vp, ctypes.c_int32]
        L.lbm_timing_read.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_step_kernel.argtypes = [vp]
        L.lbm_step_kernel.restype = ctypes.c_int32
        L.lbm_launch_count.argtypes = [vp]
        L.lbm_launch_count.restype = ctypes.c_int64
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_status_string.argtypes = [ctypes.c_int]
        L.lbm_status_string.restype = ctypes.c_char_p
        L.lbm_abi_version.restype = ctypes.c_int32
        L.lbm_probe.argtypes = [vp, ctypes.c_int64, ctypes.c_int64]
        L.lbm_probe.restype = ctypes.c_int
        L.lbm_probe_read.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_probe_read.restype = ctypes.c_int
        L.lbm_set_graph.argtypes = [vp, ctypes.c_int32]
        L.lbm_set_graph.restype = ctypes.c_int
        L.lbm_step_noalloc.argtypes = [cfgp, vp, vp, ctypes.POINTER(StepStats), vp]
        L.lbm_step_noalloc.restype = ctypes.c_int
        i32p, i64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        batch_sigs = {
            "lbm_batch_create": [vp, ctypes.POINTER(vp)], "lbm_batch_destroy": [vp],
            "lbm_batch_add": [vp, cfgp, i32p], "lbm_batch_remove": [vp, ctypes.c_int32],
            "lbm_batch_init": [vp, ctypes.c_int32, vp, vp, vp],
            "lbm_batch_set_populations": [vp, ctypes.c_int32, vp],
            "lbm_batch_get_populations": [vp, ctypes.c_int32, vp],
            "lbm_batch_moments": [vp, ctypes.c_int32, vp, vp, vp],
            "lbm_batch_stats": [vp, ctypes.c_int32, ctypes.POINTER(StepStats)],
            "lbm_batch_limited_sites": [vp, ctypes.c_int32, vp, ctypes.c_int64, i64p],
            "lbm_batch_step": [vp, ctypes.c_int64], "lbm_batch_synchronize": [vp],
            "lbm_batch_set_graph": [vp, ctypes.c_int32],
            "lbm_batch_set_shape": [vp, ctypes.c_int32, ctypes.c_int32],
            "lbm_batch_lattice_status": [vp, ctypes.c_int32],
            "lbm_batch_tune": [vp, ctypes.c_int32, dp],
            "lbm_batch_probe": [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64],
            "lbm_batch_probe_read": [vp, ctypes.c_int32, vp, ctypes.c_int64, i64p],
        }
        for name, args in batch_sigs.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = ctypes.c_int
        L.lbm_batch_size.argtypes = [vp]
        L.lbm_batch_size.restype = ctypes.c_int32
        L.lbm_batch_device_bytes.argtypes = [vp]
        L.lbm_batch_device_bytes.restype = ctypes.c_int64
        L.lbm_batch_launch_count.argtypes = [vp]
        L.lbm_batch_launch_count.restype = ctypes.c_int64
        L.lbm_batch_last_error.argtypes = [vp]
        L.lbm_batch_last_error.restype = ctypes.c_char_p
        for name in ("lbm_create", "lbm_destroy", "lbm_init", "lbm_step", "lbm_delta_s", "lbm_limit",
                     "lbm_moments", "lbm_stats", "lbm_stats_history", "lbm_limited_sites",
                     "lbm_get_populations", "lbm_set_populations", "lbm_synchronize",
                     "lbm_get_config", "lbm_timing", "lbm_timing_read"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _status_name(s: int) -> str:
    try:
        return lib().lbm_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _check(status: int, handle=None):
    if status != OK:
        msg = lib().lbm_last_error(handle).decode(errors="replace")
        raise LBMError(status, msg)


def current_stream_handle() -> int:
    """cudaStream_t of torch's current stream (0 if torch/CUDA is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _ptr(a, count: int, writable: bool):
    """(address, keepalive) of a float64 buffer of `count` elements."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):  # torch tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != count:
            raise ValueError(f"expected a contiguous float64 tensor of {count} elements")
        return a.data_ptr(), a
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or arr.size != count:
        if writable:
            raise ValueError(f"expected a contiguous float64 array of {count} elements")
        arr = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
        if arr.size != count:
            raise ValueError(f"expected {count} elements, got {arr.size}")
    return arr.ctypes.data, arr


def default_config(**kw) -> Config:
    c = Config()
    lib().lbm_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise TypeError(f"unknown config field {k}")
        setattr(c, k, v)
    return c


def footprint_bytes(**kw) -> int:
    c = default_config(**kw)
    n = lib().lbm_footprint_bytes(ctypes.byref(c))
    if n == 0:
        raise LBMError(ERR_INVALID_ARG, lib().lbm_last_error(None).decode())
    return n


def step_noalloc(f_in, f_out, stream: int | None = None, **cfg) -> dict:
    """lbm_step_noalloc: one FP64 limited step from device array f_in into
    device array f_out (torch CUDA tensors, q * nx * ny float64 each), with no
    device allocation by the library.  Returns the step's stats."""
    import torch
    c = default_config(**cfg)
    q = 3 if c.lattice == D1Q3 else 9
    n = q * c.nx * c.ny
    dev = torch.cuda.current_device()
    for name, t in (("f_in", f_in), ("f_out", f_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous float64 tensor of {n} elements")
    pi, ki = _ptr(f_in, n, False)
    po, ko = _ptr(f_out, n, True)
    nbytes = 8 * n
    if pi < po + nbytes and po < pi + nbytes:
        raise ValueError("f_in and f_out must not overlap")
    st = StepStats()
    s = current_stream_handle() if stream is None else stream
    _check(lib().lbm_step_noalloc(ctypes.byref(c), ctypes.c_void_p(pi), ctypes.c_void_p(po),
                                  ctypes.byref(st), ctypes.c_void_p(s)))
    return st.as_dict()


class Lattice:
    """One lattice owned by liblbm (lbm_create ... lbm_destroy)."""

    def __init__(self, stream: int | None = None, **cfg):
        self.config = default_config(**cfg)
        self.q = 3 if self.config.lattice == D1Q3 else 9
        self.nx, self.ny = self.config.nx, self.config.ny
        self.sites = self.nx * self.ny
        self.stream = current_stream_handle() if stream is None else stream
        h = ctypes.c_void_p()
        _check(lib().lbm_create(ctypes.byref(self.config), ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self._h = h

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- the C ABI, one method per entry point --------------------------------
    def init(self, rho, ux, uy=None):
        p1, k1 = _ptr(rho, self.sites, False)
        p2, k2 = _ptr(ux, self.sites, False)
        p3, k3 = _ptr(uy, self.sites, False)
        _check(lib().lbm_init(self._h, p1, p2, p3), self._h)

    def step(self, nsteps: int = 1):
        _check(lib().lbm_step(self._h, int(nsteps)), self._h)

    def limit(self, limiters: int):
        _check(lib().lbm_limit(self._h, int(limiters)), self._h)

    def delta_s(self, out=None):
        if out is None:
            out = np.empty((self.ny, self.nx))
        p, k = _ptr(out, self.sites, True)
        _check(lib().lbm_delta_s(self._h, p), self._h)
        return out

    def moments(self, out=None, check: bool = True):
        if out is None:
            out = tuple(np.empty((self.ny, self.nx)) for _ in range(3))
        rho, ux, uy = out
        a, ka = _ptr(rho, self.sites, True)
        b, kb = _ptr(ux, self.sites, True)
        c, kc = _ptr(uy, self.sites, True)
        s = lib().lbm_moments(self._h, a, b, c)
        if check:
            _check(s, self._h)
        return rho, ux, uy

    def stats(self, check: bool = True) -> dict:
        st = StepStats()
        s = lib().lbm_stats(self._h, ctypes.byref(st))
        if check:
            _check(s, self._h)
        return st.as_dict()

    def stats_history(self, cap: int):
        arr = (StepStats * cap)()
        n = ctypes.c_int64()
        _check(lib().lbm_stats_history(self._h, arr, cap, ctypes.byref(n)), self._h)
        return [arr[i].as_dict() for i in range(n.value)]

    def limited_sites(self) -> np.ndarray:
        cap = max(1, int(self.config.k_max))
        out = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int64()
        _check(lib().lbm_limited_sites(self._h, out.ctypes.data, cap, ctypes.byref(n)), self._h)
        return out[:min(n.value, cap)].copy()

    def get_populations(self, out=None):
        if out is None:
            out = np.empty((self.q, self.ny, self.nx))
        p, k = _ptr(out, self.q * self.sites, True)
        _check(lib().lbm_get_populations(self._h, p), self._h)
        return out

    def set_populations(self, f):
        p, k = _ptr(f, self.q * self.sites, False)
        _check(lib().lbm_set_populations(self._h, p), self._h)

    def synchronize(self):
        _check(lib().lbm_synchronize(self._h), self._h)

    def probe(self, site: int, capacity: int = 1):
        """Record rho, u_x, u_y of `site` (j * nx + i) after every step (ring of
        `capacity` samples); site = -1 stops."""
        _check(lib().lbm_probe(self._h, int(site), int(capacity)), self._h)

    def probe_read(self, cap: int) -> np.ndarray:
        """The most recent samples of the control point, oldest first: (n, 3) array."""
        out = np.zeros((max(1, cap), 3))
        n = ctypes.c_int64()
        _check(lib().lbm_probe_read(self._h, out.ctypes.data, int(cap), ctypes.byref(n)), self._h)
        return out[:n.value].copy()

    def set_graph(self, steps_per_graph: int):
        """CUDA-graph replay of runs of steps_per_graph steps (even, >= 2; 0 = off)."""
        _check(lib().lbm_set_graph(self._h, int(steps_per_graph)), self._h)

    def timing(self, enable: bool, every: int = 1):
        """Per-kernel event timing on (one step in `every`) or off."""
        _check(lib().lbm_timing(self._h, max(1, int(every)) if enable else 0), self._h)

    def timing_read(self):
        """(step-kernel ms, tail-kernel ms, timed steps) since timing was enabled."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(lib().lbm_timing_read(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)), self._h)
        return a.value, b.value, n.value

    def device_bytes(self) -> int:
        return lib().lbm_device_bytes(self._h)

    def step_kernel(self) -> int:
        """KERNEL_TILED, KERNEL_FUSED or KERNEL_TUBE: the kernel lbm_step launches."""
        return lib().lbm_step_kernel(self._h)

    def launch_count(self) -> int:
        return lib().lbm_launch_count(self._h)


def _bcheck(status: int, handle):
    if status != OK:
        raise LBMError(status, lib().lbm_batch_last_error(handle).decode(errors="replace"))


class Batch:
    """Many lattices stepped together (include/lbm_batch.h)."""

    def __init__(self, stream: int | None = None):
        self.stream = current_stream_handle() if stream is None else stream
        h = ctypes.c_void_p()
        _check(lib().lbm_batch_create(ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self._h = h
        self.shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, **cfg) -> int:
        c = default_config(**cfg)
        slot = ctypes.c_int32()
        _bcheck(lib().lbm_batch_add(self._h, ctypes.byref(c), ctypes.byref(slot)), self._h)
        q = 3 if c.lattice == D1Q3 else 9
        self.shapes[slot.value] = (q, c.ny, c.nx)
        return slot.value

    def remove(self, slot: int):
        _bcheck(lib().lbm_batch_remove(self._h, slot), self._h)
        self.shapes.pop(slot, None)

    def size(self) -> int:
        return lib().lbm_batch_size(self._h)

    def device_bytes(self) -> int:
        return lib().lbm_batch_device_bytes(self._h)

    def init(self, slot: int, rho, ux, uy=None):
        q, ny, nx = self.shapes[slot]
        p1, k1 = _ptr(rho, nx * ny, False)
        p2, k2 = _ptr(ux, nx * ny, False)
        p3, k3 = _ptr(uy, nx * ny, False)
        _bcheck(lib().lbm_batch_init(self._h, slot, p1, p2, p3), self._h)

    def set_populations(self, slot: int, f):
        q, ny, nx = self.shapes[slot]
        p, k = _ptr(f, q * ny * nx, False)
        _bcheck(lib().lbm_batch_set_populations(self._h, slot, p), self._h)

    def get_populations(self, slot: int, out=None):
        q, ny, nx = self.shapes[slot]
        if out is None:
            out = np.empty((q, ny, nx))
        p, k = _ptr(out, q * ny * nx, True)
        _bcheck(lib().lbm_batch_get_populations(self._h, slot, p), self._h)
        return out

    def moments(self, slot: int, out=None):
        q, ny, nx = self.shapes[slot]
        if out is None:
            out = tuple(np.empty((ny, nx)) for _ in range(3))
        ptrs = [_ptr(a, nx * ny, True) for a in out]
        _bcheck(lib().lbm_batch_moments(self._h, slot, ptrs[0][0], ptrs[1][0], ptrs[2][0]), self._h)
        return out

    def stats(self, slot: int) -> dict:
        st = StepStats()
        _bcheck(lib().lbm_batch_stats(self._h, slot, ctypes.byref(st)), self._h)
        return st.as_dict()

    def limited_sites(self, slot: int, cap: int = 4096) -> np.ndarray:
        out = np.zeros(max(1, cap), dtype=np.int64)
        n = ctypes.c_int64()
        _bcheck(lib().lbm_batch_limited_sites(self._h, slot, out.ctypes.data, cap, ctypes.byref(n)), self._h)
        return out[:min(n.value, cap)].copy()

    def step(self, nsteps: int = 1):
        _bcheck(lib().lbm_batch_step(self._h, int(nsteps)), self._h)

    def synchronize(self):
        _bcheck(lib().lbm_batch_synchronize(self._h), self._h)

    def lattice_status(self, slot: int) -> int:
        """Status of one lattice as collected by the last synchronize (OK = 0)."""
        st = lib().lbm_batch_lattice_status(self._h, int(slot))
        if st == ERR_INVALID_ARG:
            raise LBMError(st, "no lattice in that slot")
        return st

    def set_graph(self, steps_per_graph: int):
        _bcheck(lib().lbm_batch_set_graph(self._h, int(steps_per_graph)), self._h)

    def probe(self, slot: int, site: int, capacity: int = 1):
        """Record rho, u_x, u_y of `site` of lattice `slot` after every step."""
        _bcheck(lib().lbm_batch_probe(self._h, int(slot), int(site), int(capacity)), self._h)

    def probe_read(self, slot: int, cap: int) -> np.ndarray:
        out = np.zeros((max(1, cap), 3))
        n = ctypes.c_int64()
        _bcheck(lib().lbm_batch_probe_read(self._h, int(slot), out.ctypes.data, int(cap), ctypes.byref(n)),
                self._h)
        return out[:n.value].copy()

    def set_shape(self, seg_rows: int = 0, waves: int = 8):
        """Fused work split: rows per work item (0: automatic, else >= 4); with automatic
        segments about `waves` (1 .. 64) work items per resident warp."""
        _bcheck(lib().lbm_batch_set_shape(self._h, int(seg_rows), int(waves)), self._h)

    def tune(self, trial_steps: int = 5) -> float:
        ms = ctypes.c_double()
        _bcheck(lib().lbm_batch_tune(self._h, int(trial_steps), ctypes.byref(ms)), self._h)
        return ms.value

    def launch_count(self) -> int:
        return lib().lbm_batch_launch_count(self._h)
