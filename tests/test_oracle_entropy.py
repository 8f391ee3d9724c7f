"""Pins of the oracle's nonequilibrium entropy dS.

Expected values come from properties the paper states, checked with
independent arithmetic: dS >= 0 with its minimum 0 at f* (Sec. 3.6, Kullback
entropy has its maximum 0 at f = f*), the quadratic scaling
dS(f* + x (f - f*)) = x^2 dS(f) (Sec. 3.8), the LBGK production factor
[1 - (2 beta - 1)^2] of Sec. 3.4, and agreement of the quadratic form with
the exact Kullback form sum f ln(f/f*) (Eq. DelS) computed with numpy's log.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import PAPER_V3, PAPER_W3, PAPER_W9, moments_np, paper_velocities_d2q9

V9 = paper_velocities_d2q9()


def _cfg(lattice, nx, ny, beta=0.8, **kw):
    return oracle.Config(lattice=lattice, nx=nx, ny=ny, boundary=oracle.BC_PERIODIC, beta=beta,
                         **kw)


def _random_field(lattice, nx, ny, eps, seed):
    rng = np.random.default_rng(seed)
    w = PAPER_W9 if lattice == oracle.D2Q9 else PAPER_W3
    q = len(w)
    return w.reshape(q, 1, 1) * (1 + eps * rng.uniform(-1, 1, (q, ny, nx)))


def _feq_field(lattice, f):
    v = V9 if lattice == oracle.D2Q9 else PAPER_V3
    m = moments_np(f, v)
    q, ny, nx = f.shape
    out = np.empty_like(f)
    for j in range(ny):
        for i in range(nx):
            out[:, j, i] = oracle.feq(lattice, m[0][j, i], m[1][j, i],
                                      m[2][j, i] if lattice == oracle.D2Q9 else 0.0)
    return out


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_dS_nonnegative_and_zero_at_equilibrium(lattice):
    nx, ny = (16, 1) if lattice == oracle.D1Q3 else (6, 5)
    cfg = _cfg(lattice, nx, ny)
    f = _random_field(lattice, nx, ny, 0.2, 1)
    ds = oracle.limit(cfg, f, 0).dS
    assert (ds > 0).all()
    fs = _feq_field(lattice, f)
    ds0 = oracle.limit(cfg, fs, 0).dS
    # f* re-derived from its own rounded moments: zero up to rounding squared.
    assert np.abs(ds0).max() < 1e-28


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_dS_scales_quadratically_along_the_nonequilibrium_direction(lattice):
    """dS(f* + x (f - f*)) = x^2 dS(f), Sec. 3.8."""
    nx, ny = (12, 1) if lattice == oracle.D1Q3 else (4, 3)
    cfg = _cfg(lattice, nx, ny)
    f = _random_field(lattice, nx, ny, 0.1, 2)
    fs = _feq_field(lattice, f)
    ds1 = oracle.limit(cfg, f, 0).dS
    for x in (0.25, 0.5, 2.0, 3.0):
        dsx = oracle.limit(cfg, fs + x * (f - fs), 0).dS
        np.testing.assert_allclose(dsx, x * x * ds1, rtol=1e-11)


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_quadratic_form_is_twice_the_kullback_entropy_to_leading_order(lattice):
    """Eq. DelS: dS = sum f ln(f/f*).  Its Taylor expansion at f* is
    (1/2) sum (f - f*)^2 / f*; the paper's quadratic form omits the 1/2, so the
    oracle's dS / exact Kullback -> 2 as the deviation shrinks."""
    nx, ny = (8, 1) if lattice == oracle.D1Q3 else (3, 3)
    cfg = _cfg(lattice, nx, ny)
    base = _random_field(lattice, nx, ny, 0.1, 3)
    fs = _feq_field(lattice, base)
    prev = None
    for eps in (1e-1, 1e-2, 1e-3):
        f = fs + eps * (base - fs)
        ds = oracle.limit(cfg, f, 0).dS
        kull = (f * np.log(f / fs)).sum(axis=0)
        err = np.abs(ds / kull - 2.0).max()
        if prev is not None:
            assert err < prev * 0.2  # converges linearly in eps
        prev = err
    assert prev < 1e-2


@pytest.mark.parametrize("lattice", [oracle.D1Q3, oracle.D2Q9])
def test_post_collision_dS_and_lbgk_entropy_production(lattice):
    """dS(f') = (2 beta - 1)^2 dS(f_in) for the same f* (Eq. collLBGK), and the
    step's LBGK entropy production is [1 - (2 beta - 1)^2] sum dS(f_in)
    (Sec. 3.4).  On a 1-site periodic lattice f_in is the stored field."""
    for seed, beta in enumerate((0.55, 0.8, 0.97, 1.0)):
        cfg = _cfg(lattice, 1, 1, beta=beta)
        f = _random_field(lattice, 1, 1, 0.3, 10 + seed)
        ds_in = oracle.limit(cfg, f, 0).dS[0, 0]
        r = oracle.step(cfg, f)
        a = 2 * beta - 1
        assert abs(r.dS[0, 0] - a * a * ds_in) <= 1e-13 * ds_in
        assert abs(r.stats["dS_lbgk"] - (1 - a * a) * ds_in) <= 1e-13 * ds_in + 1e-300
        assert abs(r.stats["sum_dS"] - r.dS[0, 0]) == 0
        # the next-collision dS field of the stored state agrees with the step
        assert oracle.delta_s(cfg, f)[0, 0] == r.dS[0, 0]


def test_oracle_struct_layouts_match_its_header(tmp_path):
    """The oracle's ctypes mirrors (orc_config, orc_stats) have the C header's
    size and field offsets (a C program built against oracle/lbm_oracle.h prints them)."""
    import ctypes
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    structs = {"orc_config": oracle._Config, "orc_stats": oracle.Stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm_oracle.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.dirname(os.path.abspath(oracle.__file__))
    subprocess.run([gcc, "-std=c11", "-I", inc, "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            cname, what, val = line.split()
            got[(cname, what)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
