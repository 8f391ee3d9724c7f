"""CPU checks of the C ABI: the library builds, loads, exports every function
include/lbm.h declares, and validates configurations (no GPU call)."""
import ctypes
import os
import re

import pytest

from paper_0704_0043_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = lbm_build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_function(lib):
    names = _declared("lbm.h") + _declared("lbm_batch.h")
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_config_validation_without_gpu(lib):
    from paper_0704_0043_gb300 import lbm
    base = dict(lattice=lbm.D2Q9, nx=100, ny=100, precision=lbm.FP32, boundary=lbm.BC_WALLS)
    assert lbm.footprint_bytes(**base) > 2 * 9 * 100 * 100 * 4
    bad = [dict(nx=1), dict(lattice=3), dict(beta=1.5), dict(limiters=64), dict(k_max=-1),
           dict(lattice=lbm.D1Q3, ny=2), dict(lattice=lbm.D1Q3, ny=1, boundary=lbm.BC_CHANNEL),
           dict(precision=7), dict(delta_median=-1.0), dict(median_mode=5),
           dict(kernel=lbm.KERNEL_FUSED, precision=lbm.FP64),
           dict(equilibrium=2), dict(equilibrium=lbm.EQ_ENTROPIC, collision=lbm.COLL_ELBM),
           dict(equilibrium=lbm.EQ_ENTROPIC, precision=lbm.BF16, phi_rule=lbm.PHI_ENTROPY),
           dict(collision=lbm.COLL_ELBM, precision=lbm.FP64), dict(collision=2), dict(limiters=128),
           dict(smooth_k=0.0), dict(smooth_delta=-1.0), dict(threshold_c=float("nan")),
           dict(threshold_delta=-1e-3), dict(limiters=lbm.LIM_SMOOTH, kernel=lbm.KERNEL_FUSED, precision=lbm.FP64),
           dict(kernel=lbm.KERNEL_TUBE), dict(kernel=4),
           dict(lattice=lbm.D1Q3, ny=1, kernel=lbm.KERNEL_TUBE, precision=lbm.BF16),
           dict(lattice=lbm.D1Q3, ny=1, kernel=lbm.KERNEL_TUBE, limiters=lbm.LIM_THRESHOLD)]
    for b in bad:
        cfg = dict(base)
        cfg.update(b)
        with pytest.raises(lbm.LBMError) as e:
            lbm.footprint_bytes(**cfg)
        assert e.value.status == lbm.ERR_INVALID_ARG
    assert lbm.footprint_bytes(**dict(base, precision=lbm.FP64, equilibrium=lbm.EQ_ENTROPIC)) > 0
    tube = dict(lattice=lbm.D1Q3, nx=1000, ny=1, boundary=lbm.BC_WALLS, kernel=lbm.KERNEL_TUBE)
    assert lbm.footprint_bytes(**dict(tube, precision=lbm.FP64)) > 0
    assert lbm.footprint_bytes(**dict(tube, precision=lbm.FP32, boundary=lbm.BC_PERIODIC)) > 0
    # FP64 doubles the population storage
    f32 = lbm.footprint_bytes(**base)
    f64 = lbm.footprint_bytes(**dict(base, precision=lbm.FP64))
    assert f64 > f32


def test_abi_version_and_status_names(lib):
    lib.lbm_abi_version.restype = ctypes.c_int32
    assert lib.lbm_abi_version() == 3
    lib.lbm_status_string.restype = ctypes.c_char_p
    assert lib.lbm_status_string(4) == b"LBM_ERR_NONFINITE"


def test_no_cpu_fallback_in_the_binding():
    """The binding only marshals arguments: it never imports the oracle."""
    src = open(os.path.join(ROOT, "paper_0704_0043_gb300", "lbm.py")).read()
    assert "oracle" not in src.replace("oracle layout", "")


def test_python_struct_layouts_match_the_c_header(tmp_path):
    """The ctypes mirrors of lbm_config and lbm_step_stats have the header's
    size and every field's offset (a C program built against include/lbm.h
    prints them)."""
    import shutil
    import subprocess
    from paper_0704_0043_gb300 import lbm
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    structs = {"lbm_config": lbm.Config, "lbm_step_stats": lbm.StepStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, what, val = line.split()
            got[(cname, what)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
