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
