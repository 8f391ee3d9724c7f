"""Pins of the oracle's boundary nodes on the walls (Sec. 4.4).

The paper's cavity has its outer ring of nodes on the walls: boundary nodes are
not collided and not filtered (Sec. 4.4), and after free flight they receive the
populations they lack from the wall rule: bounce-back with a constant lid
profile (Sec. 4.4.1) or the diffusive Maxwell wall (Sec. 4.4.2), which returns
the mass that reaches it in proportion to f*(u_wall) and coincides with
bounce-back in the corners.  The velocity table and the opposite map below come
from the trigonometric definition of Sec. 4.1, not from the oracle.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import PAPER_W9, moments_np, opposite, paper_velocities_d2q9

V9 = paper_velocities_d2q9()
OPP9 = opposite(V9)
ALL = oracle.LIM_POSITIVITY | oracle.LIM_EHRENFEST | oracle.LIM_MEDIAN
WALLS = [oracle.BC_NODE_WALLS, oracle.BC_DIFFUSIVE]


def _cfg(bc, nx=12, ny=10, **kw):
    base = dict(lattice=oracle.D2Q9, nx=nx, ny=ny, boundary=bc, beta=0.95, u_lid=0.1, rho_wall=1.0)
    base.update(kw)
    return oracle.Config(**base)


def _noisy(nx, ny, seed, eps=0.05, rho0=1.0):
    rng = np.random.default_rng(seed)
    f = rho0 * PAPER_W9.reshape(9, 1, 1) * np.ones((9, ny, nx))
    return f * (1 + eps * rng.uniform(-1, 1, f.shape))


def _missing(nx, ny, i, j):
    """Directions whose source x - v_k lies outside the lattice."""
    out = []
    for k in range(9):
        si, sj = i - V9[k, 0], j - V9[k, 1]
        if not (0 <= si < nx and 0 <= sj < ny):
            out.append(k)
    return out


def _arrived(f, i, j, k):
    """Population k that free flight brings to (i, j) from the pre-step field f."""
    return f[k, j - V9[k, 1], i - V9[k, 0]]


def _ring(nx, ny):
    return [(i, j) for j in range(ny) for i in range(nx) if i in (0, nx - 1) or j in (0, ny - 1)]


def _corner(nx, ny, i, j):
    return i in (0, nx - 1) and j in (0, ny - 1)


@pytest.mark.parametrize("bc", WALLS)
def test_rest_state_is_kept_with_the_lid_at_rest(bc):
    nx, ny, rho0 = 11, 9, 2.7
    cfg = _cfg(bc, nx, ny, u_lid=0.0, rho_wall=rho0, limiters=ALL, delta_median=1e-8, delta_ehrenfest=1e-8,
               k_max=3)
    f0 = rho0 * PAPER_W9.reshape(9, 1, 1) * np.ones((9, ny, nx))
    f, st, rc = oracle.run(cfg, f0, 20)
    assert rc == 0
    np.testing.assert_allclose(f, f0, rtol=1e-14, atol=0)  # rounding of 20 collisions only


def test_bounce_back_node_returns_the_arrived_population_plus_the_lid_momentum():
    nx, ny = 9, 8
    f0 = _noisy(nx, ny, 3)
    for u_lid in (0.0, 0.1):
        cfg = _cfg(oracle.BC_NODE_WALLS, nx, ny, beta=0.0, u_lid=u_lid, rho_wall=1.3)
        f1 = oracle.step(cfg, f0).f
        for i, j in _ring(nx, ny):
            miss = _missing(nx, ny, i, j)
            lid = j == ny - 1 and not _corner(nx, ny, i, j)
            for k in range(9):
                if k not in miss:  # arrived by free flight, untouched (no collision)
                    assert f1[k, j, i] == _arrived(f0, i, j, k)
                    continue
                o = OPP9[k]
                if o in miss:  # a corner's link pointing off the lattice: stored value kept
                    assert f1[k, j, i] == f0[k, j, i]
                    continue
                want = _arrived(f0, i, j, o)
                if lid:  # momentum of the moving lid: 6 W_k rho_w (v_k . u_lid)
                    want = want + 6 * PAPER_W9[k] * 1.3 * V9[k, 0] * u_lid
                np.testing.assert_allclose(f1[k, j, i], want, rtol=1e-15, atol=1e-17)


def test_diffusive_wall_returns_the_arrived_mass_in_proportion_to_the_wall_equilibrium():
    nx, ny = 10, 9
    f0 = _noisy(nx, ny, 4, eps=0.2)
    for eq in (oracle.EQ_POLYNOMIAL, oracle.EQ_ENTROPIC):
        cfg = _cfg(oracle.BC_DIFFUSIVE, nx, ny, beta=0.9, u_lid=0.1, equilibrium=eq)
        bb = _cfg(oracle.BC_NODE_WALLS, nx, ny, beta=0.9, u_lid=0.1, equilibrium=eq)
        f1 = oracle.step(cfg, f0).f
        f1_bb = oracle.step(bb, f0).f
        feq = oracle.feq if eq == oracle.EQ_POLYNOMIAL else oracle.feq_entropic
        for i, j in _ring(nx, ny):
            miss = _missing(nx, ny, i, j)
            if _corner(nx, ny, i, j):  # the corners bounce back
                np.testing.assert_array_equal(f1[:, j, i], f1_bb[:, j, i])
                continue
            assert len(miss) == 3
            arrived = sum(_arrived(f0, i, j, OPP9[k]) for k in miss)
            returned = np.array([f1[k, j, i] for k in miss])
            # mass balance at the wall: what arrives is what is returned
            np.testing.assert_allclose(returned.sum(), arrived, rtol=1e-15)
            # the returned populations are proportional to f*(1, u_wall)
            uw = 0.1 if j == ny - 1 else 0.0
            fw = feq(oracle.D2Q9, 1.0, uw, 0.0)[miss]
            np.testing.assert_allclose(returned / returned.sum(), fw / fw.sum(), rtol=1e-14)
            if uw == 0.0:  # a still wall returns W_k-weighted mass (Sec. 4.1 weights)
                np.testing.assert_allclose(returned / returned.sum(), PAPER_W9[miss] / PAPER_W9[miss].sum(),
                                           rtol=1e-14)


@pytest.mark.parametrize("bc", WALLS)
def test_boundary_nodes_are_neither_collided_nor_limited(bc):
    nx, ny = 12, 10
    f0 = _noisy(nx, ny, 5, eps=0.3)
    cfg = _cfg(bc, nx, ny, beta=0.97, limiters=ALL, delta_median=0.0, delta_ehrenfest=1e-6, k_max=5)
    r = oracle.step(cfg, f0)
    assert r.rc == 0
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    assert (r.dS[ring] == 0).all() and (r.phi[ring] == 1).all()
    assert (r.dS[~ring] > 0).all() and r.stats["n_med"] > 0
    for s in r.selected:
        assert not ring.flat[s]
    # the populations a boundary node keeps from free flight are the arrived ones
    for i, j in _ring(nx, ny):
        for k in range(9):
            if k not in _missing(nx, ny, i, j):
                assert r.f[k, j, i] == _arrived(f0, i, j, k)


@pytest.mark.parametrize("bc", WALLS)
def test_node_walls_conserve_mass_with_moving_lid_and_all_limiters(bc):
    """Boundary nodes return every population that reaches them (bounce-back: one
    for one, the two diagonal lid terms cancel; diffusive: gamma balances the
    mass), so the mass the lattice carries forward is constant up to rounding."""
    nx, ny = 14, 11
    cfg = _cfg(bc, nx, ny, beta=0.95, limiters=ALL, delta_median=1e-6, delta_ehrenfest=1e-4, k_max=3)
    f = _noisy(nx, ny, 6)
    m0 = None
    acted = 0
    for _ in range(300):
        r = oracle.step(cfg, f)
        f = r.f
        acted += r.stats["n_med"] + r.stats["n_ehr"]
        if m0 is None:
            m0 = r.stats["mass"]
    assert acted > 0
    assert abs(r.stats["mass"] - m0) <= 1e-13 * m0


@pytest.mark.parametrize("bc", WALLS)
def test_node_walls_keep_mirror_symmetry_without_lid(bc):
    nx, ny = 11, 9
    rng = np.random.default_rng(8)
    rho = 1 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    rho = 0.5 * (rho + rho[:, ::-1])
    ux = 0.03 * rng.uniform(-1, 1, (ny, nx))
    ux = 0.5 * (ux - ux[:, ::-1])
    uy = 0.03 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.5 * (uy + uy[:, ::-1])
    cfg = _cfg(bc, nx, ny, u_lid=0.0, limiters=oracle.LIM_POSITIVITY | oracle.LIM_MEDIAN, delta_median=1e-7)
    f = oracle.init(cfg, rho, ux, uy)
    f, _, rc = oracle.run(cfg, f, 100)
    assert rc == 0
    r, a, b = moments_np(f[:, 1:-1, 1:-1], V9)
    np.testing.assert_allclose(r, r[:, ::-1], rtol=1e-13)
    np.testing.assert_allclose(a, -a[:, ::-1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b, b[:, ::-1], rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", WALLS)
def test_node_walls_step_is_homogeneous_of_degree_one_bitwise(bc):
    nx, ny = 10, 9
    base = dict(beta=0.97, u_lid=0.1, limiters=ALL, k_max=4)
    c1 = _cfg(bc, nx, ny, rho_wall=1.0, delta_median=1e-5, delta_ehrenfest=1e-4, **base)
    c2 = _cfg(bc, nx, ny, rho_wall=2.0, delta_median=2e-5, delta_ehrenfest=2e-4, **base)
    f = _noisy(nx, ny, 11)
    f[3, 4, 4] *= 6.0
    f1, f2 = f.copy(), 2 * f
    for _ in range(20):
        r1, r2 = oracle.step(c1, f1), oracle.step(c2, f2)
        f1, f2 = r1.f, r2.f
        np.testing.assert_array_equal(f2, 2 * f1)
        np.testing.assert_array_equal(r2.selected, r1.selected)


def _stencil_nodes(dS, i, j):
    """Sec. 4.4's stencils with boundary nodes on the walls: a node next to one
    wall uses itself and its two neighbours along that wall, a node next to two
    walls itself and its inward x and y neighbours, other nodes the 3 x 3 block."""
    ny, nx = dS.shape
    nearx, neary = i in (1, nx - 2), j in (1, ny - 2)
    if nearx and neary:
        return np.array([dS[j, i], dS[j, 2 if i == 1 else nx - 3], dS[2 if j == 1 else ny - 3, i]])
    if neary:
        return dS[j, i - 1:i + 2]
    if nearx:
        return dS[j - 1:j + 2, i]
    return dS[j - 1:j + 2, i - 1:i + 2].ravel()


@pytest.mark.parametrize("delta", [0.0, 3e-4])
def test_node_wall_median_stencils_match_numpy_median(delta):
    nx, ny = 11, 9
    cfg = _cfg(oracle.BC_NODE_WALLS, nx, ny, delta_median=delta)
    f = _noisy(nx, ny, 9, eps=0.05)
    r = oracle.limit(cfg, f, oracle.LIM_MEDIAN)
    want = np.ones_like(r.dS)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            med = float(np.median(_stencil_nodes(r.dS, i, j)))
            t = max(med, delta)
            if r.dS[j, i] > t:
                want[j, i] = np.sqrt(t / r.dS[j, i])
    np.testing.assert_allclose(r.phi, want, rtol=1e-15)
    assert 0 < r.stats["n_med"] == (want < 1).sum()
