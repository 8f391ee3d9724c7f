"""FP64 CPU oracle for the entropy-limited LBGK step -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library: the C source here (``lbm_oracle.c``) is compiled on its own with gcc
into ``_build/liblbm_oracle.so`` and loaded with ctypes; nothing in
``paper_0704_0043_gb300`` is imported.

Each function cites the part of Brownlee, Gorban & Levesley (Physica A 2007)
it follows; the C file lists the step order (Eq. lbgkLB with the limiter as a
post-processing routine after the collision, Sec. 4.3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")

D1Q3, D2Q9 = 1, 2
BC_WALLS, BC_PERIODIC, BC_CHANNEL, BC_NODE_WALLS, BC_DIFFUSIVE = 0, 1, 2, 3, 4
LIM_POSITIVITY, LIM_EHRENFEST, LIM_MEDIAN = 1, 2, 4
LIM_SMOOTH, LIM_THRESHOLD, LIM_ENTTHRESH = 8, 16, 32
MEDIAN_THRESHOLD, MEDIAN_GATE = 0, 1
EQ_POLYNOMIAL, EQ_ENTROPIC = 0, 1
COLL_LBGK, COLL_ELBM = 0, 1
PHI_HOMOTHETY, PHI_ENTROPY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("boundary", ctypes.c_int), ("beta", ctypes.c_double), ("u_lid", ctypes.c_double),
        ("rho_wall", ctypes.c_double), ("limiters", ctypes.c_uint),
        ("delta_median", ctypes.c_double), ("delta_ehrenfest", ctypes.c_double),
        ("k_max", ctypes.c_longlong), ("median_mode", ctypes.c_int), ("equilibrium", ctypes.c_int),
        ("smooth_delta", ctypes.c_double), ("smooth_k", ctypes.c_double),
        ("threshold_c", ctypes.c_double), ("threshold_delta", ctypes.c_double),
        ("entthresh_delta0", ctypes.c_double), ("collision", ctypes.c_int), ("phi_rule", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("sum_dS", ctypes.c_double), ("dS_lbgk", ctypes.c_double),
        ("dS_lim", ctypes.c_double), ("n_pos", ctypes.c_longlong), ("n_med", ctypes.c_longlong),
        ("n_ehr", ctypes.c_longlong), ("n_cand", ctypes.c_longlong), ("n_bad", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        llp = ctypes.POINTER(ctypes.c_longlong)
        cp = ctypes.POINTER(_Config)
        sp = ctypes.POINTER(Stats)
        lib.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_feq_entropic.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_feq_entropic.restype = ctypes.c_int
        lib.orc_entropy.argtypes = [ctypes.c_int, dp]
        lib.orc_entropy.restype = ctypes.c_double
        lib.orc_rel_entropy.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_rel_entropy.restype = ctypes.c_double
        lib.orc_elbm_alpha.argtypes = [ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.orc_elbm_alpha.restype = ctypes.c_double
        lib.orc_phi_entropy.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double]
        lib.orc_phi_entropy.restype = ctypes.c_double
        lib.orc_site_moments.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        lib.orc_init.argtypes = [cp, dp, dp, dp, dp]
        lib.orc_moments.argtypes = [cp, dp, dp, dp, dp]
        lib.orc_step.argtypes = [cp, dp, dp, dp, dp, llp, llp, sp]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_run.argtypes = [cp, dp, ctypes.c_longlong, sp]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_delta_s.argtypes = [cp, dp, dp]
        lib.orc_delta_s.restype = ctypes.c_int
        lib.orc_limit.argtypes = [cp, ctypes.c_uint, dp, dp, dp, dp, llp, llp, sp]
        lib.orc_limit.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Config:
    """Parameters of one lattice (see oracle/lbm_oracle.h for each field)."""
    lattice: int = D2Q9
    nx: int = 100
    ny: int = 100
    boundary: int = BC_WALLS
    beta: float = 1.0
    u_lid: float = 0.0
    rho_wall: float = 1.0
    limiters: int = 0
    delta_median: float = 1e-3
    delta_ehrenfest: float = 1e-3
    k_max: int = 0
    median_mode: int = MEDIAN_THRESHOLD
    equilibrium: int = EQ_POLYNOMIAL
    smooth_delta: float = 1e-2
    smooth_k: float = 0.5
    threshold_c: float = 10.0
    threshold_delta: float = 0.0
    entthresh_delta0: float = 0.1
    collision: int = COLL_LBGK
    phi_rule: int = PHI_HOMOTHETY

    @property
    def q(self) -> int:
        return 3 if self.lattice == D1Q3 else 9

    @property
    def sites(self) -> int:
        return self.nx * self.ny

    def shape(self):
        return (self.q, self.ny, self.nx)

    def _c(self) -> _Config:
        return _Config(self.lattice, self.nx, self.ny, self.boundary, self.beta, self.u_lid,
                       self.rho_wall, self.limiters, self.delta_median, self.delta_ehrenfest,
                       self.k_max, self.median_mode, self.equilibrium, self.smooth_delta,
                       self.smooth_k, self.threshold_c, self.threshold_delta, self.entthresh_delta0,
                       self.collision, self.phi_rule)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def feq(lattice: int, rho: float, ux: float, uy: float = 0.0) -> np.ndarray:
    """Polynomial quasiequilibrium at one site (Eq. polyeq1d / Eq. polyeq2d)."""
    out = np.zeros(3 if lattice == D1Q3 else 9)
    _load().orc_feq(lattice, rho, ux, uy, _dp(out))
    return out


def feq_entropic(lattice: int, rho: float, ux: float, uy: float = 0.0):
    """Entropic quasiequilibrium at one site (Eq. entropiceq1d / Eq. maxwellian), or None
    where it does not exist (|u_j| >= 1)."""
    out = np.zeros(3 if lattice == D1Q3 else 9)
    if _load().orc_feq_entropic(lattice, rho, ux, uy, _dp(out)):
        return None
    return out


def entropy(lattice: int, f) -> float:
    """Lattice entropy S(f) of one site (Sec. 4.1)."""
    f = _f64(f)
    return _load().orc_entropy(lattice, _dp(f))


def rel_entropy(f, fs) -> float:
    """sum_k f_k ln(f_k / fs_k) (Eq. DelS); +inf if some f_k < 0."""
    f = _f64(f)
    fs = _f64(fs)
    return _load().orc_rel_entropy(len(f), _dp(f), _dp(fs))


def elbm_alpha(f, fs):
    """ELBM's alpha for one site (Eq. entropy_estimate) and whether the positivity boundary was taken."""
    f = _f64(f)
    fs = _f64(fs)
    pos = ctypes.c_int(0)
    a = _load().orc_elbm_alpha(len(f), _dp(f), _dp(fs), ctypes.byref(pos))
    return a, bool(pos.value)


def phi_entropy(fp, fs, target) -> float:
    """The phi of Sec. 3.7: dS(fs + phi (fp - fs)) = target (Eq. DelS), by bisection."""
    fp = _f64(fp)
    fs = _f64(fs)
    return _load().orc_phi_entropy(len(fp), _dp(fp), _dp(fs), float(target))


def site_moments(lattice: int, f) -> tuple:
    """rho, ux, uy of one site's populations (Eq. macro_dis)."""
    f = _f64(f)
    r, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_site_moments(lattice, _dp(f), ctypes.byref(r), ctypes.byref(a), ctypes.byref(b))
    return r.value, a.value, b.value


def init(cfg: Config, rho, ux, uy=None) -> np.ndarray:
    """Populations at equilibrium (the configured f*) for the given density and velocity fields."""
    rho = _f64(rho, (cfg.sites,))
    ux = _f64(ux, (cfg.sites,))
    uy = None if uy is None else _f64(uy, (cfg.sites,))
    f = np.zeros(cfg.shape())
    _load().orc_init(ctypes.byref(cfg._c()), _dp(rho), _dp(ux), _dp(uy), _dp(f))
    return f


def moments(cfg: Config, f):
    """(rho, ux, uy) fields of a stored population field, each shaped (ny, nx)."""
    f = _f64(f, cfg.shape())
    rho = np.zeros((cfg.ny, cfg.nx))
    ux = np.zeros((cfg.ny, cfg.nx))
    uy = np.zeros((cfg.ny, cfg.nx))
    _load().orc_moments(ctypes.byref(cfg._c()), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


@dataclass
class StepResult:
    f: np.ndarray
    dS: np.ndarray
    phi: np.ndarray
    selected: np.ndarray
    stats: dict
    rc: int


def step(cfg: Config, f) -> StepResult:
    """One limited LBGK step (free flight, collision, limiters) -- see lbm_oracle.c."""
    f = _f64(f, cfg.shape())
    out = np.empty_like(f)
    dS = np.empty((cfg.ny, cfg.nx))
    phi = np.empty((cfg.ny, cfg.nx))
    cap = max(1, min(cfg.k_max, cfg.sites))
    sel = np.zeros(cap, dtype=np.int64)
    nsel = ctypes.c_longlong(0)
    st = Stats()
    rc = _load().orc_step(ctypes.byref(cfg._c()), _dp(f), _dp(out), _dp(dS), _dp(phi),
                          sel.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                          ctypes.byref(nsel), ctypes.byref(st))
    return StepResult(out, dS, phi, sel[:nsel.value].copy(), st.as_dict(), rc)


def limit(cfg: Config, f, limiters: int) -> StepResult:
    """Limiters on the stored field alone (f' := f, f* := f*(m(f)))."""
    f = _f64(f, cfg.shape())
    out = np.empty_like(f)
    dS = np.empty((cfg.ny, cfg.nx))
    phi = np.empty((cfg.ny, cfg.nx))
    cap = max(1, min(cfg.k_max, cfg.sites))
    sel = np.zeros(cap, dtype=np.int64)
    nsel = ctypes.c_longlong(0)
    st = Stats()
    rc = _load().orc_limit(ctypes.byref(cfg._c()), limiters, _dp(f), _dp(out), _dp(dS), _dp(phi),
                           sel.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                           ctypes.byref(nsel), ctypes.byref(st))
    return StepResult(out, dS, phi, sel[:nsel.value].copy(), st.as_dict(), rc)


def run(cfg: Config, f, nsteps: int):
    """nsteps limited steps; returns (f, stats of the last step, rc)."""
    f = _f64(f, cfg.shape()).copy()
    st = Stats()
    rc = _load().orc_run(ctypes.byref(cfg._c()), _dp(f), nsteps, ctypes.byref(st))
    return f, st.as_dict(), rc


def delta_s(cfg: Config, f) -> np.ndarray:
    """dS(f') field of the collision the next step performs (no limiters)."""
    f = _f64(f, cfg.shape())
    out = np.empty((cfg.ny, cfg.nx))
    _load().orc_delta_s(ctypes.byref(cfg._c()), _dp(f), _dp(out))
    return out
