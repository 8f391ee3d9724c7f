"""Ehrenfests' selection among dense candidates (Sec. 3.2; Sec. 4.3.2).

On lattices of 2^20 sites or more, when a pass records more candidates than
the tail's block holds (2048), the tail runs as a cooperative grid that
preselects them: a radix bound on the k-th largest FP32 dS, FP64 keys for the
candidates near that bound and near delta, the exact count of valid
candidates, and a short list for block 0.  States far from equilibrium
(sites out of equilibrium by 15-20 %) make most sites candidates.  The chosen
set (ties in dS to the lower site), the count of valid candidates and the
populations are checked against the FP64 oracle: the list path (k far below
the count), the path where fewer than k candidates are certainly valid
(every valid candidate listed), the overflow of the list (the one-block
selection over all candidates), exact ties across the threshold, FP64
storage, entropic f*, and D1Q3.
"""
import numpy as np
import pytest

import oracle
from paper_0704_0043_gb300 import lbm

from test_gpu_parity import pair, rand_state

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
UNIT = {lbm.BF16: 2.0 ** -8, lbm.FP16: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_0704_0043_gb300 import build
    build.build()


def check_counts(g, r, k):
    st = g.stats(check=False)
    assert r.stats["n_cand"] > 2048
    assert st["n_cand"] == r.stats["n_cand"], (st["n_cand"], r.stats["n_cand"])
    assert st["n_ehr"] == min(k, r.stats["n_cand"])
    np.testing.assert_array_equal(g.limited_sites(), np.sort(r.selected))
    return st


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.BF16])
def test_dense_candidates_one_step(precision):
    """1024 x 1024 cavity, 15 % population noise: about a million candidates,
    k = 104 (1e-4 of the sites, as the 4096^2 workload)."""
    n, k = 1024, 104
    g, oc = pair(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_WALLS, beta=0.99, u_lid=0.05,
                 precision=precision, limiters=lbm.LIM_MEDIAN | lbm.LIM_EHRENFEST, delta_median=1e-3,
                 delta_ehrenfest=1e-3, k_max=k)
    g.set_populations(rand_state(9, n, n, 1201, eps=0.15, heavy=2000))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    st = check_counts(g, r, k)
    assert r.stats["n_cand"] > n * n // 4
    got = g.get_populations()
    if precision == lbm.FP32:
        err = np.abs(got - r.f)
        assert np.all(err <= 2e-5 * np.abs(r.f) + 2e-7), float(err.max())
    else:
        dev = r.f - W9[:, None, None]
        e = 2e-6 * np.abs(dev).max()
        excess = np.abs(got - r.f) - (UNIT[precision] * (np.abs(dev) + e) + e)
        assert excess.max() <= 0, float(excess.max())
    assert abs(st["mass"] - r.stats["mass"]) <= 1e-8 * r.stats["mass"]


def test_dense_candidates_entropic_fp32():
    """Entropic f* and the exact dS of Eq. DelS as the key."""
    n, k = 1024, 300
    g = lbm.Lattice(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_WALLS, beta=0.99, u_lid=0.05,
                    precision=lbm.FP32, limiters=lbm.LIM_EHRENFEST, delta_ehrenfest=1e-3, k_max=k,
                    equilibrium=lbm.EQ_ENTROPIC)
    c = g.config
    oc = oracle.Config(lattice=c.lattice, nx=c.nx, ny=c.ny, boundary=c.boundary, beta=c.beta, u_lid=c.u_lid,
                       rho_wall=c.rho_wall, limiters=c.limiters, delta_ehrenfest=c.delta_ehrenfest, k_max=c.k_max,
                       equilibrium=c.equilibrium)
    g.set_populations(rand_state(9, n, n, 1202, eps=0.15))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    check_counts(g, r, k)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)


def test_fewer_certain_candidates_than_k_lists_every_valid_one():
    """1024 x 1024 sites near equilibrium but for 48 rows 15 % out of it,
    k = 60000: fewer than k candidates are certainly valid from their FP32 dS,
    so every valid candidate is keyed and listed."""
    n, k = 1024, 60000
    g, oc = pair(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_WALLS, beta=0.99, u_lid=0.05,
                 precision=lbm.FP32, limiters=lbm.LIM_EHRENFEST, delta_ehrenfest=1e-3, k_max=k)
    f = rand_state(9, n, n, 1203, eps=0.002)
    f[:, 100:148, :] = rand_state(9, 48, n, 1213, eps=0.15)
    g.set_populations(f)
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    check_counts(g, r, k)
    assert r.stats["n_cand"] < min(k, 65536)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)


def test_list_overflow_falls_back_to_the_one_block_selection():
    """1024 x 1024 sites, k = 200000: more than 65536 listed candidates, so
    block 0 selects among all of them as without the preselection."""
    n, k = 1024, 200000
    g, oc = pair(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_WALLS, beta=0.99, u_lid=0.05,
                 precision=lbm.FP32, limiters=lbm.LIM_EHRENFEST, delta_ehrenfest=1e-3, k_max=k)
    g.set_populations(rand_state(9, n, n, 1204, eps=0.2))
    f = g.get_populations()
    g.step(1)
    r = oracle.step(oc, f)
    assert r.stats["n_cand"] > 65536
    check_counts(g, r, k)
    np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_dense_ties_across_the_threshold(precision):
    """Limiter pass on a stored state whose rows 40..47 repeat row 40, with
    row 40 pushed far from equilibrium: the largest keys come in groups of
    eight equal ones (one per column), and k = 8 * 50 + 3 cuts a group, which
    the lower sites win."""
    nx, ny, k = 1024, 1024, 403
    g, oc = pair(lattice=lbm.D2Q9, nx=nx, ny=ny, boundary=lbm.BC_PERIODIC, beta=1.0, precision=precision,
                 limiters=lbm.LIM_EHRENFEST, delta_ehrenfest=1e-4, k_max=k)
    f = rand_state(9, ny, nx, 1205, eps=0.2)
    f[1:, 40, :] = W9[1:, None] * (1.0 + 0.6 * np.cos(np.arange(nx) * 0.37)[None, :] * np.array(
        [1, -1, 1, -1, 0.5, -0.5, 0.5, -0.5])[:, None])
    f[:, 40:48, :] = f[:, 40:41, :]
    g.set_populations(f)
    fs = g.get_populations()
    g.limit(lbm.LIM_EHRENFEST)
    r = oracle.limit(oc, fs, lbm.LIM_EHRENFEST)
    check_counts(g, r, k)
    sel = np.sort(r.selected)
    assert np.all((sel // nx >= 40) & (sel // nx < 48))
    if precision == lbm.FP64:
        np.testing.assert_array_equal(g.get_populations(), r.f)
    else:
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)


def test_dense_candidates_fp64_bitwise():
    n, k = 1024, 26
    g, oc = pair(lattice=lbm.D2Q9, nx=n, ny=n, boundary=lbm.BC_WALLS, beta=0.99, u_lid=0.05,
                 precision=lbm.FP64, limiters=lbm.LIM_MEDIAN | lbm.LIM_EHRENFEST | lbm.LIM_POSITIVITY,
                 delta_median=1e-3, delta_ehrenfest=1e-3, k_max=k)
    f = rand_state(9, n, n, 1206, eps=0.15, heavy=500)
    g.set_populations(f)
    g.step(1)
    r = oracle.step(oc, f)
    check_counts(g, r, k)
    np.testing.assert_array_equal(g.get_populations(), r.f)


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_dense_candidates_d1q3(precision):
    """A tube of 2^20 + 3 sites, every site out of equilibrium: the tube
    kernel's candidates through the preselection."""
    nx, k = (1 << 20) + 3, 50
    g, oc = pair(lattice=lbm.D1Q3, nx=nx, ny=1, boundary=lbm.BC_WALLS, beta=0.99, precision=precision,
                 limiters=lbm.LIM_EHRENFEST, delta_ehrenfest=1e-4, k_max=k)
    f = rand_state(3, 1, nx, 1207, eps=0.2)
    g.set_populations(f)
    fs = g.get_populations()
    g.step(1)
    r = oracle.step(oc, fs)
    check_counts(g, r, k)
    if precision == lbm.FP64:
        np.testing.assert_array_equal(g.get_populations(), r.f)
    else:
        np.testing.assert_allclose(g.get_populations(), r.f, rtol=2e-5, atol=2e-7)
