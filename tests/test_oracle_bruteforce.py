"""High-precision brute force of whole limited steps on tiny lattices.

An independent restatement of the step in Python's ``decimal`` arithmetic at
50 significant digits (no rounding question can hide behind it), written from
the paper's equations: free flight (Sec. 2) with halfway bounce-back and the
moving-lid momentum (Sec. 4.4.1), Eq. macro_dis, Eq. polyeq1d / polyeq2d,
Eq. lbgkLB, the quadratic dS of Sec. 3.6, the positivity rule (Sec. 3.1), the
median filter with the wall rules of Sec. 4.4 (Sec. 3.5) and Ehrenfests'
trimming (Sec. 3.2).  The FP64 oracle must agree to rounding level after
several steps, with every limiter active, on every boundary kind.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_V3, paper_velocities_d2q9

getcontext().prec = 50
D = Decimal
V9 = [tuple(int(c) for c in v) for v in paper_velocities_d2q9()]
W9 = [D(4) / 9] + [D(1) / 9] * 4 + [D(1) / 36] * 4
V3 = [(int(v), 0) for v in PAPER_V3]
OPP9 = [V9.index((-a, -b)) for a, b in V9]
OPP3 = [V3.index((-a, 0)) for a, _ in V3]


def feq(q, rho, ux, uy):
    if q == 3:
        u = ux
        return [D(2) * rho / 3 * (1 - D(3) * u * u / 2), rho / 6 * (1 - 3 * u + 3 * u * u),
                rho / 6 * (1 + 3 * u + 3 * u * u)]
    out = []
    for k in range(9):
        c = V9[k][0] * ux + V9[k][1] * uy
        out.append(rho * W9[k] * (1 + 3 * c + D(9) * c * c / 2 - D(3) * (ux * ux + uy * uy) / 2))
    return out


def moments(q, f):
    v = V3 if q == 3 else V9
    rho = sum(f, D(0))
    jx = sum((v[k][0] * f[k] for k in range(q)), D(0))
    jy = sum((v[k][1] * f[k] for k in range(q)), D(0))
    return rho, jx / rho, jy / rho


def step(p, f):
    """f: dict (k, j, i) -> Decimal.  Returns the next stored field."""
    q, nx, ny, bc = p["q"], p["nx"], p["ny"], p["bc"]
    v, opp = (V3, OPP3) if q == 3 else (V9, OPP9)
    a = 2 * D(p["beta"]) - 1
    fs, fp, dS = {}, {}, {}
    for j in range(ny):
        for i in range(nx):
            fin = []
            for k in range(q):
                si, sj = i - v[k][0], j - v[k][1]
                if bc == "periodic" or (bc == "channel" and q == 9):
                    si %= nx
                if bc == "periodic":
                    sj %= ny
                if 0 <= si < nx and 0 <= sj < ny:
                    fin.append(f[(k, sj, si)])
                else:
                    val = f[(opp[k], j, i)]
                    if q == 9 and sj > ny - 1:
                        val += 6 * W9[k] * D(p["rho_wall"]) * (v[k][0] * D(p["u_lid"]))
                    fin.append(val)
            rho, ux, uy = moments(q, fin)
            s = feq(q, rho, ux, uy)
            pr = [s[k] + a * (s[k] - fin[k]) for k in range(q)]
            for k in range(q):
                fs[(k, j, i)], fp[(k, j, i)] = s[k], pr[k]
            dS[(j, i)] = sum(((pr[k] - s[k]) ** 2 / s[k] for k in range(q)), D(0))
    out = {}
    phi = {}
    for j in range(ny):
        for i in range(nx):
            pp, pm = D(1), D(1)
            if p["lim"] & oracle.LIM_POSITIVITY:
                for k in range(q):
                    if fp[(k, j, i)] < 0:
                        pp = min(pp, fs[(k, j, i)] / (fs[(k, j, i)] - fp[(k, j, i)]))
            if p["lim"] & oracle.LIM_MEDIAN:
                st = stencil(p, dS, i, j)
                if st:
                    med = sorted(st)[len(st) // 2]
                    t = max(med, D(p["delta_m"]))
                    if dS[(j, i)] > t:
                        pm = (t / dS[(j, i)]).sqrt()
            ph = min(pp, pm)
            phi[(j, i)] = ph
            for k in range(q):
                out[(k, j, i)] = fs[(k, j, i)] + ph * (fp[(k, j, i)] - fs[(k, j, i)])
    if p["lim"] & oracle.LIM_EHRENFEST:
        cand = [(j * nx + i) for j in range(ny) for i in range(nx) if dS[(j, i)] > D(p["delta_e"])]
        cand.sort(key=lambda s: (-dS[(s // nx, s % nx)], s))
        for s in cand[:p["k"]]:
            j, i = divmod(s, nx)
            rho, ux, uy = moments(q, [out[(k, j, i)] for k in range(q)])
            e = feq(q, rho, ux, uy)
            for k in range(q):
                out[(k, j, i)] = e[k]
    return out


def stencil(p, dS, i, j):
    nx, ny, q, bc = p["nx"], p["ny"], p["q"], p["bc"]
    if q == 3:
        if bc == "periodic":
            return [dS[(0, (i - 1) % nx)], dS[(0, i)], dS[(0, (i + 1) % nx)]]
        if i in (0, nx - 1):
            return None
        return [dS[(0, i - 1)], dS[(0, i)], dS[(0, i + 1)]]
    wallx, wally = bc == "walls", bc != "periodic"
    nearx, neary = wallx and i in (0, nx - 1), wally and j in (0, ny - 1)
    if nearx and neary:
        return [dS[(j, i)], dS[(j, 1 if i == 0 else nx - 2)], dS[(1 if j == 0 else ny - 2, i)]]
    if neary:
        return [dS[(j, (i + d) % nx)] for d in (-1, 0, 1)]
    if nearx:
        return [dS[(j + d, i)] for d in (-1, 0, 1)]
    return [dS[((j + b) % ny, (i + a) % nx)] for b in (-1, 0, 1) for a in (-1, 0, 1)]


CASES = [
    dict(q=9, nx=5, ny=5, bc="walls", beta=0.96, u_lid=0.1, rho_wall=1.0, lim=7, delta_m=1e-5,
         delta_e=2e-3, k=2),
    dict(q=9, nx=6, ny=4, bc="channel", beta=0.9, u_lid=0.05, rho_wall=1.3, lim=7, delta_m=0.0,
         delta_e=1e-3, k=3),
    dict(q=9, nx=4, ny=4, bc="periodic", beta=0.99, u_lid=0.0, rho_wall=1.0, lim=7, delta_m=1e-6,
         delta_e=1e-3, k=1),
    dict(q=3, nx=7, ny=1, bc="walls", beta=0.999, u_lid=0.0, rho_wall=1.0, lim=7, delta_m=1e-6,
         delta_e=1e-3, k=2),
    dict(q=3, nx=6, ny=1, bc="periodic", beta=0.8, u_lid=0.0, rho_wall=1.0, lim=7, delta_m=0.0,
         delta_e=5e-4, k=1),
]
BC = {"walls": oracle.BC_WALLS, "periodic": oracle.BC_PERIODIC, "channel": oracle.BC_CHANNEL}


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_matches_50_digit_brute_force(case):
    p = CASES[case]
    q, nx, ny = p["q"], p["nx"], p["ny"]
    scale = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4 if q == 9 else [2 / 3, 1 / 6, 1 / 6]
    f = inputs.random_populations(100 + case, q, ny, nx, scale, 0.25, neg_frac=0.0)
    # a strongly nonequilibrium site so the positivity rule acts: an over-full
    # moving population (D2Q9) or an emptied rest population (D1Q3)
    if q == 9:
        f[1, 0, nx // 2] *= 8.0
    else:
        f[0, 0, nx // 2] *= 0.02
    cfg = oracle.Config(lattice=oracle.D1Q3 if q == 3 else oracle.D2Q9, nx=nx, ny=ny,
                        boundary=BC[p["bc"]], beta=p["beta"], u_lid=p["u_lid"],
                        rho_wall=p["rho_wall"], limiters=p["lim"], delta_median=p["delta_m"],
                        delta_ehrenfest=p["delta_e"], k_max=p["k"])
    exact = {(k, j, i): D(float(f[k, j, i])) for k in range(q) for j in range(ny) for i in range(nx)}
    cur = f.copy()
    acted = {"n_pos": 0, "n_med": 0, "n_ehr": 0}
    for _ in range(4):
        r = oracle.step(cfg, cur)
        for key in acted:
            acted[key] += r.stats[key]
        cur = r.f
        exact = step(p, exact)
        want = np.array([[[float(exact[(k, j, i)]) for i in range(nx)] for j in range(ny)]
                         for k in range(q)])
        np.testing.assert_allclose(cur, want, rtol=0, atol=2e-14)
    assert acted["n_pos"] > 0 and acted["n_med"] > 0 and acted["n_ehr"] > 0, acted
