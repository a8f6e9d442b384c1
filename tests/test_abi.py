"""The C-ABI library builds, loads and exports every symbol include/sf.h
declares; host-side validation works without a GPU (no compute calls)."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

from paper_2406_18031_b300 import build, sf

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sf.lib()


def declared_functions():
    text = (ROOT / "include" / "sf.h").read_text()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sf_create", "sf_reset", "sf_step", "sf_destroy", "sf_status", "sf_params_default",
                     "sf_get_state", "sf_set_state", "sf_strerror", "sf_propagate", "sf_update", "sf_reconstruct",
                     "sf_step_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(sf.EXPORTS) <= set(declared_functions())


def test_struct_layout_matches_header(lib, tmp_path):
    # sf_params: 4 floats, 4 ints, float, 4 ints, 5 floats, float, int, int, int, int
    assert ctypes.sizeof(sf.CParams) == 4 * (4 + 4 + 1 + 4 + 5 + 1 + 1 + 1 + 1 + 1)
    assert ctypes.sizeof(sf.CGrid) == 24
    # the C compiler's view of the header: sizes and every field's offset
    fields = [f for f, _ in sf.CParams._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "sf.h"\nint main(void) {\n'
                   '  printf("%zu %zu\\n", sizeof(sf_params), sizeof(sf_grid));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(sf_params, {f}));\n' for f in fields) + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(sf.CParams) and int(out[1]) == ctypes.sizeof(sf.CGrid)
    assert [int(x) for x in out[2:]] == [getattr(sf.CParams, f).offset for f in fields]


def test_params_default(lib):
    p = sf.CParams()
    assert lib.sf_params_default(ctypes.byref(p), 480, 640, 2) == sf.OK
    assert p.fx == 320 and p.fy == 320 and p.cx == 320 and p.cy == 240
    assert list(p.smooth_iters) == [2, 4, 4, 4]
    assert [round(g, 6) for g in p.gamma] == [1.0, 1.0, 0.01, 1.0, 1.0]
    assert p.lambda_ref == 1.0 and p.flags == sf.CHECK_CFL
    assert lib.sf_params_default(None, 4, 4, 1) == sf.EINVAL
    assert lib.sf_params_default(ctypes.byref(p), 4, 4, 5) == sf.EINVAL


@pytest.mark.parametrize("H,W,L", [(30, 30, 3), (64, 64, 0), (64, 64, 5), (0, 64, 1), (24, 24, 3), (64, 60, 4),
                                   (32768, 32776, 1), (65536, 65536, 2)])
def test_create_rejects_bad_shapes_without_touching_the_device(lib, H, W, L):
    p = sf.CParams()
    lib.sf_params_default(ctypes.byref(p), 64, 64, 1)
    out = ctypes.c_void_p(123)
    assert lib.sf_create(H, W, L, ctypes.byref(p), ctypes.byref(out)) == sf.EINVAL
    assert out.value is None


@pytest.mark.parametrize("field,value", [("fx", 0.0), ("lambda_ref", -1.0), ("gamma2", 0.0), ("gamma0", -1.0),
                                         ("gamma4", 0.0), ("iters0", 5000), ("smooth0", 17), ("nf_max", 9),
                                         ("nf_max", -1), ("update_mode", 3), ("solve_tile", 8),
                                         ("solve_tile", 24), ("solve_tile", 64)])
def test_create_rejects_bad_parameters(lib, field, value):
    p = sf.CParams()
    lib.sf_params_default(ctypes.byref(p), 64, 64, 1)
    if field.startswith("gamma"):
        p.gamma[int(field[-1])] = value
    elif field.startswith("iters"):
        p.iters[0] = value
    elif field.startswith("smooth"):
        p.smooth_iters[0] = value
    else:
        setattr(p, field, value)
    out = ctypes.c_void_p()
    assert lib.sf_create(64, 64, 1, ctypes.byref(p), ctypes.byref(out)) == sf.EINVAL


def test_calls_on_null_context_fail_cleanly(lib):
    assert lib.sf_reset(None) == sf.EINVAL
    assert lib.sf_step(None, None, None, ctypes.c_float(0.01), None, None, None) == sf.EINVAL
    assert lib.sf_status(None) == sf.EINVAL
    t = ctypes.c_longlong(7)
    assert lib.sf_submit_host(None, None, None, ctypes.c_float(0.01), None, None, None, ctypes.byref(t)) == sf.EINVAL
    assert t.value == -1
    assert lib.sf_wait_host(None, -1) == sf.EINVAL
    lib.sf_destroy(None)


def test_strerror(lib):
    for code in (sf.OK, sf.EINVAL, sf.ENOMEM, sf.ECUDA, sf.ETIMEOUT, sf.ENONFINITE, sf.WARN_CFL, 99):
        assert len(sf.strerror(code)) > 0


def test_stage_entry_points_validate_arguments(lib):
    g = sf.grid(16, 16, 8.0, 8.0, 8.0, 8.0)
    assert lib.sf_propagate(ctypes.byref(g), 0, 0, ctypes.c_float(1.0), None, None, None, None, None, None) == sf.EINVAL
    gm = (ctypes.c_float * 5)(1, 1, 1, 1, 1)
    assert lib.sf_update(ctypes.byref(g), 5, 1, 2, 0, gm, ctypes.c_float(1.0), None, None, 16, 16, None, None, None,
                         None, None, None, None, None) == sf.EINVAL
    grids = (sf.CGrid * 1)(g)
    assert lib.sf_reconstruct(0, grids, None, None, ctypes.c_float(1.0), None, None, 0, None, None) == sf.EINVAL


def test_remap_rejects_bad_arguments_without_touching_the_device(lib):
    g = sf.grid(16, 16, 8.0, 8.0, 8.0, 8.0)
    x = ctypes.c_void_p(256)                       # never dereferenced: rejected first
    eye = (ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    bad = (ctypes.c_float * 9)(1, 0, 0, 0, float("nan"), 0, 0, 0, 1)
    cam = (ctypes.c_float * 4)(8.0, 8.0, 8.0, 8.0)
    nocam = (ctypes.c_float * 4)(0.0, 8.0, 8.0, 8.0)
    assert lib.sf_remap_pinhole(ctypes.byref(g), bad, 16, 16, cam, x, None, x, None, None) == sf.EINVAL
    assert lib.sf_remap_pinhole(ctypes.byref(g), eye, 16, 16, nocam, x, None, x, None, None) == sf.EINVAL
    assert lib.sf_remap_pinhole(ctypes.byref(g), eye, 0, 16, cam, x, None, x, None, None) == sf.EINVAL
    assert lib.sf_remap_pinhole(ctypes.byref(g), eye, 16, 16, cam, x, x, x, None, None) == sf.EINVAL
    assert lib.sf_remap_equirect(ctypes.byref(g), eye, 16, -2, x, None, x, None, None) == sf.EINVAL
    assert lib.sf_remap_equirect(None, eye, 16, 32, x, None, x, None, None) == sf.EINVAL
