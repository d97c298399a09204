"""Host-side checks of the C ABI: the library loads, exports every function that
include/dts.h declares, sizes workspaces and rejects bad arguments before any
device work (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1805_04590_gb300 import dts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(dts_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = dts.load()
    names = declared_functions()
    assert "dts_solve" in names and "dts_filter" in names and "dts_solve_backward" in names
    assert "dts_domain_transform" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(dts.EXPORTS) <= set(names)


def test_version_and_status_strings():
    lib = dts.load()
    assert b"sm_103a" in lib.dts_version()
    assert lib.dts_status_string(0) == b"DTS_OK"
    assert lib.dts_status_string(5) == b"DTS_ERR_TIMEOUT"


def _guide(C=3, H=40, W=50, dtype=dts.F32):
    return dts.CGuide(C, H, W, dtype, 0x1000, 0, 0)


def test_workspace_size_layout():
    lib = dts.load()
    p = dts.Params(iterations=5).c()
    g = _guide(H=40, W=50)
    n0 = lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p), 0)
    pitch = 64
    plane = 40 * pitch * 4
    # chained vertical passes: 32 + 2 S control words (S = 2 strips of 32 columns) and the paired
    # tall kernel's 4 x 64 flags, then per strip and 64-row chunk 32 columns of up to 10 floats of
    # chunk records, each region 256-byte aligned
    split = ((32 + 2 * 2 + 4 * 64) * 4 + 255) // 256 * 256 + 2 * 1 * 32 * 10 * 4
    # dY tiled by 8-column strips for the strip kernel: 7 strips of 4 * 2 warps * 9 rows + 1 rows
    # of 8 values (segments of 9 rows, 2 warps for 40 rows), 256-byte aligned
    tiled = (7 * 73 * 8 * 4 + 255) // 256 * 256
    assert n0 == 4 * plane + split + tiled  # dX, dY, working buffer, iterate
    n1 = lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p), 1)
    assert n1 == (3 + 5 + 2 * 3 + 5) * plane + split + tiled  # + K checkpoints, 2N pass inputs, adjoint buffers
    p16 = dts.Params(iterations=5, dist_dtype=dts.F16).c()
    tiled16 = (7 * 73 * 8 * 2 + 255) // 256 * 256
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p16), 0) == \
        2 * (40 * pitch * 2) + 2 * plane + split + tiled16
    bad = dts.Params(sigma_s=-1.0).c()
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(bad), 0) == 0
    # save_checkpoints = 2: K x 2N planes of kept pass inputs in the forward part, no recompute
    # planes in the backward part
    p2 = dts.Params(iterations=5, save_checkpoints=2).c()
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p2), 1) == n1 + (5 * 6 - 6) * plane
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p2), 0) == n0 + (5 - 1 + 5 * 6) * plane
    p3 = dts.Params(save_checkpoints=3).c()
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(p3), 0) == 0


@pytest.mark.parametrize("field,value", [("sigma_s", 0.0), ("sigma_r", -1.0), ("lam", -0.5), ("step", 0.0),
                                         ("iterations", -1), ("passes", 0), ("passes", 17), ("norm", 2),
                                         ("update", 3), ("update", -1), ("conf_mode", 2),
                                         ("charbonnier_eps", -1.0), ("charbonnier_eps", float("nan")), ("dist_dtype", 1)])
def test_invalid_params_rejected_synchronously(field, value):
    lib = dts.load()
    prm = dts.Params()
    setattr(prm, field, value)
    p = prm.c()
    g = _guide()
    rc = lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 1 << 30, None)
    assert rc == 1


def test_invalid_guide_and_pointers_rejected():
    lib = dts.load()
    p = dts.Params().c()
    for g in (_guide(C=0), _guide(H=0), _guide(W=0), _guide(dtype=7), dts.CGuide(3, 4, 5, 0, 0, 0, 0),
              dts.CGuide(3, 4, 5, 0, 0x1000, 0, 4), dts.CGuide(3, 4, 5, 0, 0x1000, 10, 5)):
        assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000,
                             1 << 30, None) == 1
        assert lib.dts_filter(ctypes.byref(g), ctypes.byref(p), 0x2000, 0x3000, 0x5000, 1 << 30, None) == 1
    g = _guide()
    assert lib.dts_solve(ctypes.byref(g), None, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 1 << 30,
                         None) == 1
    assert lib.dts_solve(ctypes.byref(g), 0x2000, 9, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 1 << 30,
                         None) == 1
    assert lib.dts_domain_transform(ctypes.byref(g), ctypes.byref(p), None, 0x10, None) == 1


def test_workspace_errors_and_size_limits():
    lib = dts.load()
    p = dts.Params(iterations=2).c()
    g = _guide()
    # too small, misaligned, missing
    assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 16, None) == 3
    assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5010, 1 << 30,
                         None) == 3
    assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, None, 1 << 30,
                         None) == 3
    # rows longer than the horizontal kernels hold, columns taller than a cluster holds
    for gg in (_guide(H=4, W=20000), _guide(H=20000, W=4)):
        assert lib.dts_solve(ctypes.byref(gg), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000,
                             1 << 40, None) == 2


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1805_04590_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), fn
                assert "dts_oracle" not in src and "liborc" not in src, fn


def test_autotune_table_roundtrip_without_gpu():
    lib = dts.load()
    # cluster shapes "col H items warps cluster"; cluster 0 is the strip kernel (one CTA of
    # `warps` warps per 8 columns, 4 * warps segments of `items` rows per column)
    text = "row 2880 8\nrow 300 16\ncol 1988 16 16 8\ncol 500 32 8 2\ncol 1080 9 30 0\n"
    assert dts.autotune_import(text) is None
    out = dts.autotune_export()
    for line in ("row 2880 8", "row 300 16", "col 1988 16 16 8", "col 500 32 8 2", "col 1080 9 30 0"):
        assert line in out
    # a strip shape that does not cover the column is not a candidate
    dts.autotune_import("col 1500 16 17 0\n")
    assert "col 1500 " not in dts.autotune_export()
    # a shape that is not a candidate for its height is ignored, malformed text rejected
    dts.autotune_import("col 64 40 16 16\n")
    assert "col 64 " not in dts.autotune_export()
    assert lib.dts_autotune_import(b"bogus 1 2\n") == 1


def test_confidence_rejects_bad_arguments():
    lib = dts.load()
    p = dts.Params().c()
    g = _guide()
    for sc in (0.0, -1.0, float("inf"), float("nan")):
        assert lib.dts_confidence(ctypes.byref(g), 0x2000, 0, ctypes.byref(p), sc, 0x3000, 0x5000, 1 << 30, None) == 1
    assert lib.dts_confidence(ctypes.byref(g), None, 0, ctypes.byref(p), 0.1, 0x3000, 0x5000, 1 << 30, None) == 1
    assert lib.dts_confidence(ctypes.byref(g), 0x2000, 9, ctypes.byref(p), 0.1, 0x3000, 0x5000, 1 << 30, None) == 1
    assert lib.dts_confidence(ctypes.byref(g), 0x2000, 0, ctypes.byref(p), 0.1, 0x3000, 0x5000, 16, None) == 3


def test_conjugate_gradient_workspace_and_limits():
    lib = dts.load()
    g = _guide(H=40, W=50)
    base = dts.Params(iterations=5).c()
    cg = dts.Params(iterations=5, update=dts.UPDATE_CG).c()
    n0 = lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(base), 0)
    plane = 40 * 64 * 4
    # planes r, p, q and the FP64 block: 8 scalars and the ticket (128 bytes), 2048 partial sums
    assert lib.dts_workspace_size(ctypes.byref(g), ctypes.byref(cg), 0) == \
        n0 + 3 * plane + (128 + 2048 * 8 + 255) // 256 * 256
    # the objective's weights are c as given; no checkpoints (no backward), no box kernel
    for field, value in (("conf_mode", dts.CONF_SUPPORT), ("save_checkpoints", 1), ("filter_kernel", dts.KERNEL_BOX),
                         ("charbonnier_eps", 1e-3)):
        prm = dts.Params(iterations=5, update=dts.UPDATE_CG)
        setattr(prm, field, value)
        p = prm.c()
        assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 1 << 30,
                             None) == 2, field


def test_charbonnier_is_not_taken_with_conjugate_gradients():
    """The Charbonnier loss goes with the gradient step and the fixed point of Eq. 4; conjugate
    gradients keep the square (DTS_ERR_UNSUPPORTED before any device work)."""
    lib = dts.load()
    g = _guide()
    p = dts.Params(update=dts.UPDATE_CG, charbonnier_eps=1e-3).c()
    assert lib.dts_solve(ctypes.byref(g), 0x2000, 0, 0x3000, None, ctypes.byref(p), 0x4000, 0x5000, 1 << 30,
                         None) == 2


def test_binding_structs_match_the_c_layout(tmp_path):
    """The ctypes mirrors of dts_guide and dts_params in the binding have the C compiler's field
    offsets and sizes (a mismatch would pass every parameter to the library shifted)."""
    from paper_1805_04590_gb300 import dts

    fields = {"dts_guide": (dts.CGuide, ["C", "H", "W", "dtype", "data", "ch_stride", "row_stride"]),
              "dts_params": (dts.CParams, ["lambda", "sigma_s", "sigma_r", "step", "iterations", "passes", "norm",
                                           "update", "conf_mode", "dist_dtype", "save_checkpoints", "filter_kernel",
                                           "charbonnier_eps"])}
    lines = ['#include <stdio.h>', '#include "dts.h"', "int main(void) {"]
    for st, (_, names) in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            lines.append(f'printf("{st} {n} %zu %zu\\n", offsetof({st}, {n}), sizeof((({st}*)0)->{n}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {}
    for line in filter(None, out):
        parts = line.split()
        c_layout[(parts[0], parts[1])] = tuple(int(v) for v in parts[2:])
    for st, (cls, names) in fields.items():
        assert ctypes.sizeof(cls) == c_layout[(st, "size")][0], st
        py_names = [f[0] for f in cls._fields_]
        assert len(py_names) == len(names), st
        for py, n in zip(py_names, names):
            f = getattr(cls, py)
            assert (f.offset, f.size) == c_layout[(st, n)], (st, n)
