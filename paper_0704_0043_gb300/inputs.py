"""Seeded synthetic inputs and workload parameters.

This module is the one piece of code that both the CUDA path and the FP64
oracle are fed from.  It holds none of the method's arithmetic: it produces
density and velocity fields, plain random numbers and the parameters of each
workload (lattice sizes, relaxation parameter, limiter thresholds), never a
population, an equilibrium or an entropy.  Each side turns these into
populations with its own code.

Workloads follow the paper's numerical experiments (Brownlee, Gorban &
Levesley, Physica A 2007, Sec. 4): the 1:2 athermal shock tube (Sec. 4.3) and
the lid-driven cavity (Sec. 4.4), plus batched and served mixes of both.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LIM_POSITIVITY, LIM_EHRENFEST, LIM_MEDIAN = 1, 2, 4


def beta_from_nu(nu: float, convention: str = "lattice") -> float:
    """Relaxation parameter beta for kinematic viscosity nu (lattice units).

    The paper writes beta = 1/(2 nu + 1) next to Eq. lbgkLB.  With the lattice
    sound speed c_s^2 = 1/3 of both D1Q3 and D2Q9 the LBGK viscosity is
    nu = (1/3)(1/(2 beta) - 1/2), i.e. beta = 1/(6 nu + 1); that is the
    reading used for every workload ("lattice"), because the paper's
    Reynolds numbers (Sec. 4.4, Re = L u0 / nu) reproduce the literature's
    vortex centres and Hopf point only with physical viscosity.  The printed
    form is available as convention="paper".
    """
    if convention == "paper":
        return 1.0 / (2.0 * nu + 1.0)
    return 1.0 / (6.0 * nu + 1.0)


def cavity_nu(side: int, u_lid: float, reynolds: float) -> float:
    """nu = L u0 / Re with L the number of nodes across the cavity (Sec. 4.4)."""
    return side * u_lid / reynolds


def shock_tube(n: int = 800, rho_left: float = 1.0, rho_right: float = 0.5, split: float = 0.5):
    """Density and velocity of the athermal shock tube (Sec. 4.3): sites
    s < split * n hold rho_left, the rest rho_right; the fluid is at rest."""
    s = np.arange(n)
    rho = np.where(s < int(round(split * n)), rho_left, rho_right).astype(np.float64)
    return rho, np.zeros(n)


def cavity_rest(nx: int, ny: int, rho0: float = 1.0):
    """Uniform density rho0, fluid at rest (Sec. 4.4); fields shaped (ny, nx)."""
    return np.full((ny, nx), rho0), np.zeros((ny, nx)), np.zeros((ny, nx))


def random_moments(seed: int, nx: int, ny: int, rho0: float = 1.0, drho: float = 0.05,
                   umax: float = 0.1):
    """Smooth-plus-noise density and velocity fields for parity tests."""
    rng = np.random.default_rng(seed)
    rho = rho0 * (1.0 + drho * rng.uniform(-1.0, 1.0, (ny, nx)))
    ux = umax * rng.uniform(-1.0, 1.0, (ny, nx))
    uy = umax * rng.uniform(-1.0, 1.0, (ny, nx))
    return rho, ux, uy


def random_populations(seed: int, q: int, ny: int, nx: int, scale, eps: float,
                       neg_frac: float = 0.0):
    """Positive random populations plane by plane: scale[k] * (1 + eps * U(-1, 1)).

    ``scale`` is supplied by the caller (one number per direction).  With
    ``neg_frac`` > 0 that fraction of sites gets one population pushed
    below zero after a collision-size kick, to exercise the positivity rule.
    Returns an array shaped (q, ny, nx).
    """
    rng = np.random.default_rng(seed)
    scale = np.asarray(scale, dtype=np.float64).reshape(q, 1, 1)
    f = scale * (1.0 + eps * rng.uniform(-1.0, 1.0, (q, ny, nx)))
    if neg_frac > 0.0:
        hit = rng.uniform(0.0, 1.0, (ny, nx)) < neg_frac
        k = rng.integers(1, q, (ny, nx))
        jj, ii = np.nonzero(hit)
        f[k[jj, ii], jj, ii] = -0.2 * scale[k[jj, ii], 0, 0] * rng.uniform(0.0, 1.0, jj.size)
    return f


@dataclass
class Workload:
    """One lattice of a workload, with every parameter the step needs."""
    name: str
    lattice: int            # 1 = D1Q3, 2 = D2Q9
    nx: int
    ny: int
    beta: float
    u_lid: float
    rho0: float
    limiters: int
    delta_median: float = 1e-3
    delta_ehrenfest: float = 1e-3
    k_max: int = 0
    steps: int = 1
    rho_right: float = 0.5  # shock tubes only
    boundary: int = 0       # 0: walls half a link outside the lattice; 3: boundary nodes on the walls
    extra: dict = field(default_factory=dict)

    @property
    def sites(self) -> int:
        return self.nx * self.ny


def shock_tube_workload(n: int = 800, steps: int = 400) -> Workload:
    """1:2 shock tube, nu = 1e-9, Ehrenfests' delta = 1e-3 with k = 4 (FP64)."""
    return Workload("shock_tube_d1q3_800", 1, n, 1, beta_from_nu(1e-9), 0.0, 1.0,
                    LIM_EHRENFEST, delta_ehrenfest=1e-3, k_max=4, steps=steps)


def cavity100_workload(steps: int = 200000) -> Workload:
    """100 x 100 cavity as Sec. 4.4.1 sets it up: boundary nodes on the walls with
    bounce-back and a constant lid profile, lid 0.1, Re = 5000 with L = 99 (the
    distance between the wall nodes), median filter; initial density 1.  The
    paper's runs start from density 2.7 with delta = 1e-3; the step is
    homogeneous of degree one in the populations, rho_wall and delta, so density
    1 takes delta = 1e-3 / 2.7 for the same flow."""
    nu = cavity_nu(99, 0.1, 5000.0)
    return Workload("cavity_d2q9_100_re5000", 2, 100, 100, beta_from_nu(nu), 0.1, 1.0,
                    LIM_MEDIAN, delta_median=1e-3 / 2.7, steps=steps, boundary=3)


def cavity4096_workload(steps: int = 10000) -> Workload:
    """4096^2 cavity, lid 0.05, Re = 7500, median (delta 1e-3) + Ehrenfests'
    (delta 1e-3, k = 0.01 % of the sites = 1677)."""
    side = 4096
    nu = cavity_nu(side, 0.05, 7500.0)
    return Workload("cavity_d2q9_4096_re7500", 2, side, side, beta_from_nu(nu), 0.05, 1.0,
                    LIM_MEDIAN | LIM_EHRENFEST, delta_median=1e-3, delta_ehrenfest=1e-3,
                    k_max=int(math.floor(1e-4 * side * side)), steps=steps)


def batched_cavities(seed: int = 7040043, count: int = 256, lo: int = 64, hi: int = 512,
                     steps: int = 50000):
    """256 independent cavities: side ~ U{64..512}, Re ~ U[2000, 7500], lid 0.1,
    limiter drawn uniformly from positivity / Ehrenfests' / median."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, count)
    res = rng.uniform(2000.0, 7500.0, count)
    lim_choice = rng.integers(0, 3, count)
    lims = [LIM_POSITIVITY, LIM_EHRENFEST, LIM_MEDIAN]
    out = []
    for b in range(count):
        side = int(sides[b])
        nu = cavity_nu(side, 0.1, float(res[b]))
        lim = lims[int(lim_choice[b])]
        out.append(Workload(f"cavity{b}_{side}", 2, side, side, beta_from_nu(nu), 0.1, 1.0, lim,
                            delta_median=1e-3, delta_ehrenfest=1e-3,
                            k_max=max(1, int(math.floor(1e-4 * side * side))), steps=steps,
                            extra={"re": float(res[b])}))
    return out


def serving_trace(seed: int = 7040044, n_requests: int = 1000, rate_hz: float = 200.0,
                  cavity_frac: float = 0.7, min_steps: int = 1000, max_steps: int = 100000,
                  max_cavity: int = 1024, max_tube: int = 1000000):
    """Poisson arrivals (mean rate_hz) of cavity (side U{100..max_cavity}) and
    shock-tube (n U{800..max_tube}, density ratio 1:U[2, 4]) solves with
    log-uniform step counts.  Returns [(arrival_s, Workload)]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    lims = [LIM_POSITIVITY, LIM_EHRENFEST, LIM_MEDIAN]
    out = []
    for r in range(n_requests):
        steps = int(round(math.exp(rng.uniform(math.log(min_steps), math.log(max_steps)))))
        lim = lims[int(rng.integers(0, 3))]
        if rng.uniform() < cavity_frac:
            side = int(rng.integers(100, max_cavity + 1))
            re = float(rng.uniform(2000.0, 7500.0))
            nu = cavity_nu(side, 0.1, re)
            w = Workload(f"req{r}_cavity{side}", 2, side, side, beta_from_nu(nu), 0.1, 1.0, lim,
                         k_max=max(1, int(1e-4 * side * side)), steps=steps, extra={"re": re})
        else:
            n = int(rng.integers(800, max_tube + 1))
            ratio = float(rng.uniform(2.0, 4.0))
            w = Workload(f"req{r}_tube{n}", 1, n, 1, beta_from_nu(1e-9), 0.0, 1.0, lim,
                         k_max=4, steps=steps, rho_right=1.0 / ratio)
        out.append((float(t[r]), w))
    return out
