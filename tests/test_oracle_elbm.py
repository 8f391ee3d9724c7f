"""Pins of the oracle's ELBM collision (Sec. 3.7, Eq. elbm, Eq. entropy_estimate,
the bisection of Sec. 4.2), and of the filters' factor from the entropy itself
(Sec. 3.7: phi with S(f* + phi (f - f*)) = S(f*) - dS_t).

* alpha is the nontrivial root of S(f + alpha (f* - f)) = S(f): checked with the
  lattice entropy S computed from the weights W (not from f*), within the
  bisection's bracket, and never on the entropy-decreasing side;
* for small deviations alpha -> 2, the LBGK step (Sec. 3.7), and the ELBM step
  differs from LBGK by O(eps^2);
* where the entropy is still above S(f) at the positivity boundary of the line,
  alpha is that boundary: one population is exactly zero (the positivity rule);
* free flight permutes populations, so the lattice's total entropy is the same
  before and after it: with beta = 1 an ELBM step conserves the total entropy
  and with beta < 1 raises it; moments are conserved.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_W9, paper_velocities_d2q9

V9 = paper_velocities_d2q9()


def _null():
    M = np.stack([np.ones(9), V9[:, 0].astype(float), V9[:, 1].astype(float)])
    return np.linalg.svd(M)[2][3:]


def _site(seed, scale):
    rng = np.random.default_rng(seed)
    fs = oracle.feq_entropic(oracle.D2Q9, rng.uniform(0.7, 1.5), rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2))
    d = rng.standard_normal(6) @ _null()
    return fs + scale * fs.min() * d / np.abs(d).max(), fs


def test_alpha_is_the_entropy_conserving_root():
    for seed in range(40):
        f, fs = _site(seed, 0.5)
        a, pos = oracle.elbm_alpha(f, fs)
        assert not pos and 1.0 < a < 4.0
        s0 = oracle.entropy(oracle.D2Q9, f)
        lo = oracle.entropy(oracle.D2Q9, f + a * (fs - f))
        hi = oracle.entropy(oracle.D2Q9, f + (a + 2e-15 * 8) * (fs - f))
        assert lo >= s0 - 1e-13  # no entropy decrease at the returned alpha
        assert hi <= s0 + 1e-13  # the root lies within the bracket


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_alpha_tends_to_two_for_small_deviations(eps):
    worst = 0.0
    for seed in range(20):
        f, fs = _site(100 + seed, eps)
        a, _ = oracle.elbm_alpha(f, fs)
        worst = max(worst, abs(a - 2.0))
    assert worst < 4 * eps


def test_alpha_takes_the_positivity_boundary_when_no_root_exists():
    found = 0
    for seed in range(200):
        # deviations beyond the smallest f*_k: the mirror image f* - (f - f*) can leave the cone
        f, fs = _site(200 + seed, 1.0 + 4.0 * (seed % 5) / 4.0)
        if f.min() <= 0.0:
            continue
        a, pos = oracle.elbm_alpha(f, fs)
        if not pos:
            continue
        found += 1
        g = f + a * (fs - f)
        assert np.abs(g).min() < 1e-15 and g.min() > -1e-15  # one population at zero
        assert oracle.entropy(oracle.D2Q9, np.maximum(g, 0.0)) >= oracle.entropy(oracle.D2Q9, f) - 1e-13
    assert found > 0


def test_alpha_at_equilibrium_is_two():
    fs = oracle.feq_entropic(oracle.D2Q9, 1.1, 0.05, -0.1)
    assert oracle.elbm_alpha(fs, fs)[0] == 2.0


def _cfg(beta, collision):
    return oracle.Config(lattice=oracle.D2Q9, nx=11, ny=9, boundary=oracle.BC_PERIODIC, beta=beta,
                         equilibrium=oracle.EQ_ENTROPIC, collision=collision)


def _total_entropy(f):
    q, ny, nx = f.shape
    return sum(oracle.entropy(oracle.D2Q9, f[:, j, i]) for j in range(ny) for i in range(nx))


def test_elbm_step_conserves_the_total_entropy_at_beta_one():
    f = inputs.random_populations(3, 9, 9, 11, PAPER_W9, 0.3)
    r = oracle.step(_cfg(1.0, oracle.COLL_ELBM), f)
    assert r.rc == 0
    assert _total_entropy(r.f) == pytest.approx(_total_entropy(f), abs=1e-11)
    assert r.f.sum() == pytest.approx(f.sum(), rel=1e-14)
    # LBGK's mirror step does not conserve it
    r2 = oracle.step(_cfg(1.0, oracle.COLL_LBGK), f)
    assert abs(_total_entropy(r2.f) - _total_entropy(f)) > 1e-7


def test_elbm_step_with_beta_below_one_raises_the_entropy():
    f = inputs.random_populations(4, 9, 9, 11, PAPER_W9, 0.3)
    r = oracle.step(_cfg(0.8, oracle.COLL_ELBM), f)
    assert _total_entropy(r.f) > _total_entropy(f) + 1e-6


def test_elbm_step_approaches_lbgk_for_small_deviations():
    diffs = []
    for eps in (1e-2, 1e-3):
        f = inputs.random_populations(5, 9, 9, 11, PAPER_W9, eps)
        e = oracle.step(_cfg(0.9, oracle.COLL_ELBM), f).f
        g = oracle.step(_cfg(0.9, oracle.COLL_LBGK), f).f
        diffs.append(np.abs(e - g).max())
    # O(eps^2): a tenfold smaller deviation gives a ~hundredfold smaller difference
    assert diffs[1] < diffs[0] / 30


# -- Sec. 3.7: the filters' factor from the entropy itself ------------------------------------------

def _dS_mp(f, fs):
    """sum_k f_k ln(f_k / f*_k) (Eq. DelS) at 50 digits."""
    import mpmath
    mpmath.mp.dps = 50
    return sum(mpmath.mpf(float(a)) * mpmath.log(mpmath.mpf(float(a)) / mpmath.mpf(float(b)))
               for a, b in zip(f, fs) if a > 0)


def test_phi_solves_the_entropy_equation_of_sec_3_7():
    """phi in [0, 1] with dS(f* + phi (f - f*)) = dS_t: the returned phi gives at
    most dS_t, and phi + 4e-15 already exceeds it (checked at 50 digits), up to
    the FP64 evaluation of Eq. DelS, whose terms cancel to second order: its
    error is a few ulps of sum_k |f_k ln(f_k / f*_k)|, plus f_k times the
    rounding of each ratio f_k / f*_k before its logarithm."""
    import mpmath
    for seed in range(25):
        f, fs = _site(seed, 0.6)
        ds = float(_dS_mp(f, fs))
        for frac in (0.9, 0.3, 0.01):
            t = frac * ds
            phi = oracle.phi_entropy(f, fs, t)
            assert 0.0 <= phi <= 1.0
            g = fs + phi * (f - fs)
            terms = float(sum(abs(mpmath.mpf(float(a)) * mpmath.log(mpmath.mpf(float(a)) / mpmath.mpf(float(b))))
                              for a, b in zip(g, fs)))
            tol = 2.0 ** -52 * (16 * terms + 4 * g.sum())  # + the rounding of f / f* before its logarithm
            lo = _dS_mp(g, fs)
            hi = _dS_mp(fs + (phi + 4e-15) * (f - fs), fs)
            assert lo <= t + tol and hi >= t - tol, (seed, frac, float(lo), float(hi), t, tol)


def test_phi_tends_to_the_homothety_for_small_deviations():
    """In the quadratic approximation dS(f* + phi n) = phi^2 dS(f* + n), so the
    solve tends to sqrt(dS_t / dS) (Eq. entrHom) as the deviation shrinks."""
    for seed in range(10):
        errs = []
        for scale in (1e-2, 1e-3):
            f, fs = _site(seed, scale)
            ds = oracle.rel_entropy(f, fs)
            phi = oracle.phi_entropy(f, fs, 0.25 * ds)
            errs.append(abs(phi / 0.5 - 1.0))
        assert errs[1] < 2e-3 and errs[1] < errs[0] / 5, errs


def test_entropic_median_pass_with_the_exact_solve_lands_on_the_target():
    """A median pass with entropic f* and the solve of Sec. 3.7: every filtered
    site ends with dS = dS_t = max(median, delta) of its stencil (the entropy of
    the limited state is S(f*) - dS_t), moments unchanged."""
    nx, ny = 12, 10
    cfg = oracle.Config(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_WALLS,
                        equilibrium=oracle.EQ_ENTROPIC, phi_rule=oracle.PHI_ENTROPY, delta_median=1e-5)
    rho, ux, uy = inputs.random_moments(14, nx, ny, umax=0.1)
    fs = oracle.init(cfg, rho, ux, uy)
    rng = np.random.default_rng(15)
    f = fs * (1 + 0.08 * rng.uniform(-1, 1, fs.shape))
    r = oracle.limit(cfg, f, oracle.LIM_MEDIAN)
    after = oracle.limit(cfg, r.f, 0).dS
    hit = r.phi < 1
    assert hit.sum() > 10
    homothety = oracle.limit(oracle.Config(**{**cfg.__dict__, "phi_rule": oracle.PHI_HOMOTHETY}), f,
                             oracle.LIM_MEDIAN)
    np.testing.assert_array_equal(homothety.phi < 1, hit)  # the same sites are filtered
    for j, i in zip(*np.nonzero(hit)):
        # the target: the stencil median (R7 rules) or delta; recover it from the homothety's phi
        t = homothety.phi[j, i] ** 2 * r.dS[j, i]
        np.testing.assert_allclose(after[j, i], t, rtol=1e-9)
    r0, a0, b0 = oracle.moments(cfg, f)
    r1, a1, b1 = oracle.moments(cfg, r.f)
    np.testing.assert_allclose(r1, r0, rtol=1e-14)
    np.testing.assert_allclose(a1, a0, rtol=0, atol=1e-14)
