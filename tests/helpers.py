"""Test helpers: lattice definitions rebuilt from the paper's text (not from
either implementation), and small utilities shared by the test files."""
from __future__ import annotations

import math

import numpy as np


def paper_velocities_d2q9():
    """D2Q9 velocities from the trigonometric definition of Sec. 4.1:
    v_0 = 0; v_i = (cos((i-1) pi/2), sin((i-1) pi/2)) for i = 1..4;
    v_i = sqrt(2) (cos((i-5) pi/2 + pi/4), sin((i-5) pi/2 + pi/4)) for i = 5..8."""
    v = [(0, 0)]
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        v.append((round(math.cos(a)), round(math.sin(a))))
    for i in range(5, 9):
        a = (i - 5) * math.pi / 2 + math.pi / 4
        v.append((round(math.sqrt(2) * math.cos(a)), round(math.sqrt(2) * math.sin(a))))
    return np.array(v, dtype=np.int64)


# Sec. 4.1: W_0 = 4/9, W_1..4 = 1/9, W_5..8 = 1/36.
PAPER_W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
# Sec. 4.1: D1Q3 velocities {0, -1, 1} for the static, left and right populations.
PAPER_V3 = np.array([0, -1, 1], dtype=np.int64)
PAPER_W3 = np.array([2 / 3, 1 / 6, 1 / 6])


def opposite(v):
    """Index of -v_k for each k."""
    v = np.asarray(v)
    out = []
    for k in range(len(v)):
        out.append(int(np.nonzero((v == -v[k]).all(axis=-1) if v.ndim > 1 else v == -v[k])[0][0]))
    return out


def moments_np(f, v):
    """rho and u of population fields f (q, ...) with velocity table v."""
    f = np.asarray(f, dtype=np.float64)
    rho = f.sum(axis=0)
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 1:
        j = np.tensordot(v, f, axes=(0, 0))
        return rho, j / rho
    jx = np.tensordot(v[:, 0], f, axes=(0, 0))
    jy = np.tensordot(v[:, 1], f, axes=(0, 0))
    return rho, jx / rho, jy / rho


def quad_dS(f, fs):
    """Quadratic nonequilibrium entropy sum_k (f_k - f*_k)^2 / f*_k (Sec. 3.6)."""
    return (((f - fs) ** 2) / fs).sum(axis=0)


def stream_function(ux, n):
    """psi(x, y) = integral of u_x dy from the bottom wall (psi = 0 there), by
    Simpson's rule on the half-cell-shifted grid (wall at y = 0, nodes at
    (j + 1/2)/n): the stream function of Sec. 4.4.1's steady-state procedure."""
    h = 1.0 / n
    psi = np.zeros_like(ux)
    # first node: trapezoid from the wall (u = 0) to y = h/2
    psi[0] = 0.5 * (0.0 + ux[0]) * (0.5 * h)
    for j in range(1, n):
        if j >= 2:
            # Simpson over [y_{j-2}, y_j]
            psi[j] = psi[j - 2] + (h / 3.0) * (ux[j - 2] + 4 * ux[j - 1] + ux[j])
        else:
            psi[j] = psi[j - 1] + 0.5 * h * (ux[j - 1] + ux[j])
    return psi


def extremum(psi, xs, ys, region, sign, valid=None):
    """Node coordinates of the largest sign * psi inside region ((x0, x1), (y0, y1))
    (among the nodes where `valid` is true, if given)."""
    (x0, x1), (y0, y1) = region
    mask = (xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1)
    if valid is not None:
        mask &= valid
    vals = np.where(mask, sign * psi, -np.inf)
    j, i = np.unravel_index(np.argmax(vals), psi.shape)
    return xs[j, i], ys[j, i]


# Search regions of the cavity's vortices (unit square, lid on top).
VORTEX_REGIONS = {
    "primary": ((0.2, 0.8), (0.2, 0.8)),
    "lower_left": ((0.0, 0.3), (0.0, 0.3)),
    "lower_right": ((0.6, 1.0), (0.0, 0.4)),
    "top_left": ((0.0, 0.3), (0.7, 1.0)),
}


def vortex_centres(ux, n, names=("primary", "lower_left", "lower_right")):
    """Centres of the cavity's vortices from the x-velocity field (n x n, nodes at
    (i + 1/2)/n): the primary vortex is the extremum of psi of the sign it takes at
    the cavity centre, the corner vortices the extrema of the opposite sign."""
    psi = stream_function(ux, n)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n))
    xs, ys = (ii + 0.5) / n, (jj + 0.5) / n
    sign = -np.sign(psi[n // 2, n // 2])
    out = {}
    for name in names:
        out[name] = extremum(psi, xs, ys, VORTEX_REGIONS[name], -sign if name == "primary" else sign)
    return out


def stream_function_nodes(ux, n):
    """psi(x, y) = integral of u_x dy from the bottom wall for boundary nodes on the
    walls (nodes at j/(n-1), u_x = 0 on the bottom row): Simpson's rule over pairs of
    cells, the trapezoid rule for the last cell of an odd count (Sec. 4.4.1)."""
    h = 1.0 / (n - 1)
    psi = np.zeros_like(ux)
    for j in range(1, n):
        if j >= 2:
            psi[j] = psi[j - 2] + (h / 3.0) * (ux[j - 2] + 4 * ux[j - 1] + ux[j])
        else:
            psi[j] = psi[j - 1] + 0.5 * h * (ux[j - 1] + ux[j])
    return psi


def vortex_centres_nodes(ux, n, names=("primary", "lower_left", "lower_right")):
    """As vortex_centres, for lattices whose outer nodes lie on the walls (node i at i/(n-1))."""
    psi = stream_function_nodes(ux, n)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n))
    xs, ys = ii / (n - 1.0), jj / (n - 1.0)
    fluid = (ii > 0) & (ii < n - 1) & (jj > 0) & (jj < n - 1)  # vortex centres lie off the walls
    sign = -np.sign(psi[n // 2, n // 2])
    out = {}
    for name in names:
        out[name] = extremum(psi, xs, ys, VORTEX_REGIONS[name], -sign if name == "primary" else sign, fluid)
    return out
