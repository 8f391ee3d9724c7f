"""Pins of the oracle's quasiequilibria and collision against closed forms.

Nothing here re-calls the oracle's formulas: the expected values come from
the moment conditions the quasiequilibrium must satisfy (Sec. 2: f* has the
moments M of f), from exact rational evaluation of the printed D1Q3 formula
(Eq. polyeq1d), and from the special values of beta that Sec. 2 names for the
LBGK collision (Eq. collLBGK).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import PAPER_V3, PAPER_W3, PAPER_W9, moments_np, paper_velocities_d2q9

V9 = paper_velocities_d2q9()
RNG = np.random.default_rng(12345)
CASES = [(1.0, 0.0, 0.0), (2.7, 0.1, 0.0), (0.5, -0.07, 0.13)] + [
    (float(RNG.uniform(0.3, 3.0)), float(RNG.uniform(-0.3, 0.3)), float(RNG.uniform(-0.3, 0.3)))
    for _ in range(20)
]


@pytest.mark.parametrize("rho,ux,uy", CASES)
def test_d2q9_feq_moments_through_second_order(rho, ux, uy):
    """Polynomial f* (Eq. polyeq2d) reproduces rho, rho u and the Euler stress
    rho c_s^2 delta_ab + rho u_a u_b with c_s^2 = 1/3, using the velocity set
    rebuilt from the trigonometric definition of Sec. 4.1."""
    fs = oracle.feq(oracle.D2Q9, rho, ux, uy)
    v = V9.astype(np.float64)
    assert abs(fs.sum() - rho) <= 1e-15 * rho * 4
    assert abs((v[:, 0] * fs).sum() - rho * ux) <= 1e-15 * rho * 4
    assert abs((v[:, 1] * fs).sum() - rho * uy) <= 1e-15 * rho * 4
    u = (ux, uy)
    for a in range(2):
        for b in range(2):
            pab = (v[:, a] * v[:, b] * fs).sum()
            want = rho * (1.0 / 3.0) * (a == b) + rho * u[a] * u[b]
            assert abs(pab - want) <= 4e-15 * rho, (a, b, pab, want)


def test_d2q9_feq_at_rest_is_weights():
    """At u = 0, f*_i = rho W_i with the weights printed in Sec. 4.1."""
    for rho in (1.0, 2.7, 0.25):
        fs = oracle.feq(oracle.D2Q9, rho, 0.0, 0.0)
        np.testing.assert_allclose(fs, rho * PAPER_W9, rtol=2e-16, atol=0)
    assert abs(PAPER_W9.sum() - 1.0) < 1e-15


def _polyeq1d_exact(rho, u):
    rho, u = Fraction(rho), Fraction(u)
    return [Fraction(2, 3) * rho * (1 - Fraction(3, 2) * u * u),
            rho / 6 * (1 - 3 * u + 3 * u * u),
            rho / 6 * (1 + 3 * u + 3 * u * u)]


@pytest.mark.parametrize("rho,u", [(1.0, 0.0), (1.0, 0.1), (0.5, -0.25), (2.7, 0.3)] + [
    (float(RNG.uniform(0.3, 3.0)), float(RNG.uniform(-0.4, 0.4))) for _ in range(20)])
def test_d1q3_feq_matches_printed_formula_exactly(rho, u):
    """Eq. polyeq1d evaluated in exact rational arithmetic; the FP64 oracle is
    within a few ulp, and the moments of Sec. 4.1 hold (v = {0, -1, 1})."""
    fs = oracle.feq(oracle.D1Q3, rho, u)
    exact = _polyeq1d_exact(rho, u)
    for k in range(3):
        assert abs(Fraction(fs[k]) - exact[k]) <= abs(exact[k]) * Fraction(1, 2 ** 50) + Fraction(1, 2 ** 60)
    v = PAPER_V3.astype(np.float64)
    assert abs(fs.sum() - rho) <= 4e-16 * rho
    assert abs((v * fs).sum() - rho * u) <= 4e-16 * rho
    assert abs((v * v * fs).sum() - (rho / 3 + rho * u * u)) <= 4e-16 * rho
    # Same structure as D2Q9: rho W_k (1 + 3 v u + 9 (v u)^2 / 2 - 3 u^2 / 2).
    want = rho * PAPER_W3 * (1 + 3 * v * u + 4.5 * (v * u) ** 2 - 1.5 * u * u)
    np.testing.assert_allclose(fs, want, rtol=1e-14)


def _one_site(lattice, beta, limiters=0):
    # A 1 x 1 periodic lattice: free flight returns every population to the
    # same site, so a step is the collision (and limiter) alone.
    return oracle.Config(lattice=lattice, nx=1, ny=1, boundary=oracle.BC_PERIODIC, beta=beta,
                         limiters=limiters)


def _random_site(q, seed):
    rng = np.random.default_rng(seed)
    w = PAPER_W9 if q == 9 else PAPER_W3
    return (w * (1 + 0.3 * rng.uniform(-1, 1, q))).reshape(q, 1, 1)


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_collision_special_betas(lattice):
    """Sec. 2 after Eq. collLBGK: beta = 0 leaves f unchanged, beta = 1/2 is the
    Ehrenfests' step f -> f*, beta = 1 is the point reflection 2 f* - f."""
    q = 3 if lattice == oracle.D1Q3 else 9
    v = PAPER_V3 if q == 3 else V9
    for seed in range(5):
        f = _random_site(q, seed)
        m = moments_np(f[:, 0, 0], v)
        fs = oracle.feq(lattice, m[0], m[1], m[2] if q == 9 else 0.0)
        for beta, want in ((0.0, f[:, 0, 0]), (0.5, fs), (1.0, 2 * fs - f[:, 0, 0])):
            out = oracle.step(_one_site(lattice, beta), f).f[:, 0, 0]
            np.testing.assert_allclose(out, want, rtol=0, atol=4e-16)


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_collision_conserves_moments_and_fixes_equilibrium(lattice):
    """m(F(f)) = m(f) (Sec. 2) and f* is the fixed point of the collision."""
    q = 3 if lattice == oracle.D1Q3 else 9
    v = PAPER_V3 if q == 3 else V9
    for seed in range(5):
        beta = 0.5 + 0.5 * (seed + 1) / 6
        f = _random_site(q, 100 + seed)
        out = oracle.step(_one_site(lattice, beta), f).f
        m0 = moments_np(f[:, 0, 0], v)
        m1 = moments_np(out[:, 0, 0], v)
        np.testing.assert_allclose(m1, m0, rtol=0, atol=2e-15)
        fs = oracle.feq(lattice, m0[0], m0[1], m0[2] if q == 9 else 0.0).reshape(q, 1, 1)
        # Equal up to the rounding of re-deriving rho, u from f* (a few ulp).
        np.testing.assert_allclose(oracle.step(_one_site(lattice, beta), fs).f, fs, rtol=4e-15,
                                   atol=0)
