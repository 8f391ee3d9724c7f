"""Pins of the oracle's ensemble-dependent limiters (Sec. 3.3, Sec. 3.4, Sec. 4.3.2):
the smooth limiter of Eq. smooth1 with alpha = delta / E(dS)^k and the
threshold filter with dS_t = max(c E(dS), delta).  The checks are properties
the definitions fix, not the formulas retyped:

* ensemble dependence: phi depends on dS / E(dS) only, so scaling every site's
  nonequilibrium part by the same factor leaves every phi unchanged;
* a uniform field has dS = E everywhere, which gives closed forms: phi = 1/(1 + delta)
  for the smooth limiter (any k) and phi = sqrt(c) for the threshold filter with c < 1;
* delta = 0 (smooth), or no site above the threshold, leaves the
  state untouched bit for bit;
* the smooth limiter with k = 1/2 is double monotonic in the quadratic entropy
  (Sec. 3.8): phi falls and phi^2 dS rises with dS;
* the threshold filter brings every limited site's quadratic dS exactly to dS_t
  and leaves the others bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import inputs
from tests.helpers import PAPER_W9, quad_dS


def _cfg(nx, ny, limiters, **kw):
    base = dict(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=oracle.BC_PERIODIC, beta=0.9,
                limiters=limiters)
    base.update(kw)
    return oracle.Config(**base)


def _feq_field(f):
    q, ny, nx = f.shape
    out = np.empty_like(f)
    for j in range(ny):
        for i in range(nx):
            rho, ux, uy = oracle.site_moments(oracle.D2Q9, f[:, j, i])
            out[:, j, i] = oracle.feq(oracle.D2Q9, rho, ux, uy)
    return out


def _state(seed, nx=13, ny=11, eps=0.1):
    return inputs.random_populations(seed, 9, ny, nx, PAPER_W9, eps)


@pytest.mark.parametrize("lim", [oracle.LIM_SMOOTH, oracle.LIM_THRESHOLD])
def test_phi_depends_on_dS_over_its_mean_only(lim):
    f = _state(1)
    fs = _feq_field(f)
    cfg = _cfg(13, 11, lim, smooth_delta=0.3, smooth_k=0.5, threshold_c=1.5)
    r1 = oracle.limit(cfg, f, lim)
    r2 = oracle.limit(cfg, fs + 0.25 * (f - fs), lim)  # every dS scales by 1/16
    assert (r1.phi < 1).any()
    np.testing.assert_allclose(r2.phi, r1.phi, rtol=1e-12, atol=0)


def _uniform_state(nx=8, ny=6):
    rng = np.random.default_rng(5)
    site = PAPER_W9 * (1 + 0.1 * rng.uniform(-1, 1, 9))
    return np.repeat(np.repeat(site[:, None, None], ny, axis=1), nx, axis=2)


@pytest.mark.parametrize("k", [0.5, 1.0, 2.0])
def test_smooth_limiter_on_a_uniform_field(k):
    f = _uniform_state()
    fs = _feq_field(f)
    delta = 0.7
    r = oracle.limit(_cfg(8, 6, oracle.LIM_SMOOTH, smooth_delta=delta, smooth_k=k), f, oracle.LIM_SMOOTH)
    np.testing.assert_allclose(r.phi, 1 / (1 + delta), rtol=1e-14)
    np.testing.assert_allclose(r.f, fs + (f - fs) / (1 + delta), rtol=1e-14, atol=1e-16)


def test_threshold_filter_on_a_uniform_field():
    f = _uniform_state()
    r = oracle.limit(_cfg(8, 6, oracle.LIM_THRESHOLD, threshold_c=0.36), f, oracle.LIM_THRESHOLD)
    np.testing.assert_allclose(r.phi, 0.6, rtol=1e-14)
    r = oracle.limit(_cfg(8, 6, oracle.LIM_THRESHOLD, threshold_c=1.0), f, oracle.LIM_THRESHOLD)
    assert (r.phi == 1.0).all() and np.array_equal(r.f, f)


def test_smooth_limiter_with_zero_delta_is_the_identity():
    f = _state(2)
    r = oracle.limit(_cfg(13, 11, oracle.LIM_SMOOTH, smooth_delta=0.0), f, oracle.LIM_SMOOTH)
    assert np.array_equal(r.f, f) and r.stats["dS_lim"] == 0.0


def test_smooth_limiter_is_double_monotonic_for_k_one_half():
    f = _state(3, nx=20, ny=15, eps=0.3)
    fs = _feq_field(f)
    r = oracle.limit(_cfg(20, 15, oracle.LIM_SMOOTH, smooth_delta=0.5, smooth_k=0.5), f, oracle.LIM_SMOOTH)
    ds = quad_dS(f, fs).reshape(-1)
    out = quad_dS(r.f, fs).reshape(-1)
    order = np.argsort(ds)
    phi = r.phi.reshape(-1)[order]
    assert (np.diff(phi) <= 1e-15).all()
    assert (np.diff(out[order]) >= -1e-15).all()
    assert (phi < 1).all()


def test_threshold_filter_brings_limited_sites_to_the_threshold():
    f = _state(4, nx=20, ny=15, eps=0.3)
    fs = _feq_field(f)
    c = 1.2
    r = oracle.limit(_cfg(20, 15, oracle.LIM_THRESHOLD, threshold_c=c), f, oracle.LIM_THRESHOLD)
    ds = quad_dS(f, fs)
    t = c * ds.mean()
    hit = ds > t
    assert hit.any() and (~hit).any()
    np.testing.assert_allclose(quad_dS(r.f, fs)[hit], t, rtol=1e-12)
    assert np.array_equal(r.f[:, ~hit], f[:, ~hit])
    # dS_t = max(c E, delta): a delta above every dS switches the filter off
    r2 = oracle.limit(_cfg(20, 15, oracle.LIM_THRESHOLD, threshold_c=c, threshold_delta=10 * ds.max()), f,
                      oracle.LIM_THRESHOLD)
    assert np.array_equal(r2.f, f)


def test_ensemble_limiters_compose_with_the_others_as_the_minimum():
    f = _state(6, nx=16, ny=12, eps=0.3)
    lims = [oracle.LIM_MEDIAN, oracle.LIM_SMOOTH, oracle.LIM_THRESHOLD]
    cfg = _cfg(16, 12, 0, smooth_delta=0.2, threshold_c=2.0, delta_median=0.0)
    phis = [oracle.limit(cfg, f, lim).phi for lim in lims]
    both = oracle.limit(cfg, f, sum(lims)).phi
    np.testing.assert_array_equal(both, np.minimum.reduce(phis))


# Eq. EntThresh: dS_0 solves sum_s max(dS_s - dS_0, 0) = delta_0 [1 - (2 beta - 1)^2] sum_s dS_s on the
# ensemble's own distribution.  In the quadratic entropy the homothety sqrt(dS_t / dS) brings each limited
# site to dS_t, so the limiter's entropy production equals the right-hand side: Eq. LimEntLim holds with
# equality, delta_lim S = delta_0 [1 - (2 beta - 1)^2] sum dS.

@pytest.mark.parametrize("delta0", [0.05, 0.3, 0.9])
def test_entthresh_limiter_spends_exactly_its_entropy_budget(delta0):
    f = _state(7, nx=24, ny=17, eps=0.3)
    cfg = _cfg(24, 17, oracle.LIM_ENTTHRESH, beta=0.93, entthresh_delta0=delta0)
    r = oracle.step(cfg, f)
    a = 2 * cfg.beta - 1
    assert 0 < r.stats["dS_lim"]
    assert r.stats["dS_lim"] == pytest.approx(delta0 * (1 - a * a) * r.stats["sum_dS"], rel=1e-12)
    # the limited sites are exactly those above one common threshold
    hit = r.phi < 1
    assert hit.any() and (~hit).any()
    assert r.dS[hit].min() > r.dS[~hit].max()


def test_entthresh_limiter_on_a_uniform_field():
    f = _uniform_state()
    cfg = _cfg(8, 6, oracle.LIM_ENTTHRESH, beta=0.9, entthresh_delta0=0.5)
    a = 2 * cfg.beta - 1
    r = oracle.limit(cfg, f, oracle.LIM_ENTTHRESH)
    # every dS equal: dS_0 = dS (1 - delta_0 [1 - a^2]), phi = sqrt of that ratio
    np.testing.assert_allclose(r.phi, np.sqrt(1 - 0.5 * (1 - a * a)), rtol=1e-14)


def test_entthresh_limiter_switched_off():
    f = _state(8)
    r = oracle.limit(_cfg(13, 11, oracle.LIM_ENTTHRESH, entthresh_delta0=0.0), f, oracle.LIM_ENTTHRESH)
    assert np.array_equal(r.f, f)
    r = oracle.limit(_cfg(13, 11, oracle.LIM_ENTTHRESH, entthresh_delta0=0.5, threshold_delta=1e9), f,
                     oracle.LIM_ENTTHRESH)
    assert np.array_equal(r.f, f)
