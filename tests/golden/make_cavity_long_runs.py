"""Writes tests/golden/cavity100_long_oracle.txt: the FP64 oracle's own long runs
of the 100 x 100 lid-driven cavity as Sec. 4.4.1 sets it up: D2Q9 LBGK,
polynomial f*, boundary nodes on the walls with bounce-back and a constant lid
profile (ORC_BC_NODE_WALLS), lid u0 = 0.1, initial density 2.7, median filter
delta = 1e-3 (Table vort rows (b)) and 1e-4 (rows (c)); from rest, 2e5 steps
at Re = 5000 and Re = 7500, and the unregularised run at Re = 7500 up to the
step at which it first reports a nonfinite site (row (a)).  Re = L u0 / nu with
L = 99, the distance between the wall nodes.

Only oracle/ computes the flow; the vortex centres are read off the oracle's
velocity field with the stream-function extrema of tests/helpers.py.

    python tests/golden/make_cavity_long_runs.py        (about 10 minutes, 5 processes)
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

OUT = os.path.join(HERE, "cavity100_long_oracle.txt")
N, U0, RHO0, STEPS, CHUNK = 100, 0.1, 2.7, 200000, 10000
NAMES = ("primary", "lower_left", "lower_right", "top_left")


def case(args):
    re, limiters, delta = args
    import numpy as np
    import oracle
    import helpers
    nu = (N - 1) * U0 / re               # Re = L u0 / nu, L = N - 1 between the wall nodes (Sec. 4.4)
    beta = 1.0 / (6.0 * nu + 1.0)         # nu = (1/3)(1/(2 beta) - 1/2)
    oc = oracle.Config(lattice=oracle.D2Q9, nx=N, ny=N, boundary=oracle.BC_NODE_WALLS, beta=beta,
                       u_lid=U0, rho_wall=RHO0, limiters=limiters, delta_median=delta)
    f0 = oracle.init(oc, np.full((N, N), RHO0), np.zeros((N, N)), np.zeros((N, N)))
    f = f0.copy()
    m0 = None
    done = 0
    while done < STEPS:
        f, st, rc = oracle.run(oc, f, CHUNK)
        if rc != 0 or not np.isfinite(f).all():
            # locate the first failing step inside the chunk
            f2, _, _ = oracle.run(oc, f0, done)
            for t in range(CHUNK):
                r = oracle.step(oc, f2)
                if r.rc != 0 or not np.isfinite(r.f).all():
                    return (re, limiters, delta, done + t + 1, None, None)
                f2 = r.f
        if m0 is None:
            _, st0, _ = oracle.run(oc, f0, 1)
            m0 = st0["mass"]  # mass carried by the lattice (boundary nodes: their live populations)
        done += CHUNK
    rho, ux, uy = oracle.moments(oc, f)
    c = helpers.vortex_centres_nodes(ux, N, NAMES)
    return (re, limiters, delta, done, c, (st["mass"] - m0) / m0)


def main():
    cases = [(5000.0, oracle_median(), 1e-3), (5000.0, oracle_median(), 1e-4), (7500.0, oracle_median(), 1e-3),
             (7500.0, oracle_median(), 1e-4), (7500.0, 0, 0.0)]
    with mp.get_context("spawn").Pool(len(cases)) as pool:
        res = pool.map(case, cases)
    lines = ["# FP64 oracle runs of the 100 x 100 cavity (Sec. 4.4.1): D2Q9 LBGK, polynomial f*, boundary",
             "# nodes on the walls with bounce-back and a constant lid profile, lid u0 = 0.1, rho = 2.7, from rest;",
             "# beta = 1/(6 nu + 1), nu = 99 u0 / Re.",
             "# Written by: python tests/golden/make_cavity_long_runs.py (oracle/ only).",
             "# Columns: Re limiter delta steps primary_x primary_y lowerleft_x lowerleft_y lowerright_x",
             "#          lowerright_y topleft_x topleft_y mass_drift_rel   (node coordinates i/99)",
             "# limiter: median = median filter (Sec. 3.5); none = unregularised LBGK, whose row gives the",
             "# first step with a nonfinite site (nan centres)."]
    for re, lim, delta, steps, c, drift in res:
        name = "median" if lim else "none"
        if c is None:
            lines.append(f"{int(re)} {name} {delta:g} {steps} " + " ".join(["nan"] * 8) + " nan")
        else:
            vals = " ".join(f"{c[k][0]:.4f} {c[k][1]:.4f}" for k in NAMES)
            lines.append(f"{int(re)} {name} {delta:g} {steps} {vals} {drift:.3e}")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


def oracle_median():
    return 4  # LIM_MEDIAN bit of oracle/lbm_oracle.h


if __name__ == "__main__":
    main()
