"""The C ABI library: it builds, loads, exports every function include/grid.h
declares, and its host-only planner (grid metadata M) matches the oracle bit
for bit.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import _pins
import oracle
from paper_2403_10647_gb300 import _lib
from paper_2403_10647_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grid.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(grid_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build_library()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.SIGNATURES) == names


def test_strerror_and_version(lib):
    assert lib.grid_strerror(0) == b"ok"
    assert b"INT32_MAX" in lib.grid_strerror(_lib.GRID_EOVERFLOW)
    assert lib.grid_version().startswith(b"gb300-grid")


def _plan_c(lib, lo, hi, n, lam):
    info = _lib.GridInfo()
    clo = (ctypes.c_float * 3)(*map(float, lo))
    chi = (ctypes.c_float * 3)(*map(float, hi))
    rc = lib.grid_plan(clo, chi, int(n), float(lam), ctypes.byref(info))
    return rc, info


def test_plan_matches_oracle_bit_for_bit(lib):
    g = np.random.Generator(np.random.Philox(21))
    for k in range(3000):
        lo = (g.standard_normal(3) * 10.0 ** g.uniform(-3, 4)).astype(np.float32)
        ext = (10.0 ** g.uniform(-4, 4, 3)).astype(np.float32)
        if k % 7 == 0:
            ext[g.integers(0, 3)] = 0.0          # flat axis
        if k % 31 == 0:
            ext[:] = 0.0                         # a point
        hi = (lo + ext).astype(np.float32)
        n = int(10 ** g.uniform(0, 8))
        lam = float(np.float32(g.uniform(0.1, 16.0)))
        rc, info = _plan_c(lib, lo, hi, n, lam)
        try:
            p = oracle.plan(lo, hi, n, lam)
            orc = 0
        except oracle.OracleError as e:
            orc = e.code
        assert rc == orc, (k, rc, orc)
        if rc == 0:
            assert tuple(info.res) == tuple(p.res), (k, tuple(info.res), p.res)
            assert np.array_equal(np.array(info.scale[:], np.float32), p.scale), k
            assert info.ncells == p.ncells
            assert info.key_bits == (p.ncells - 1).bit_length()


def test_plan_golden_cases(lib):
    """The library's host plan on the hand-worked resolution cases (closed
    forms, FP64 volumes that FP32 would round)."""
    for row in _pins.read_plan_cases():
        lo, hi, n, lam = row[0:3], row[3:6], int(row[6]), row[7]
        rc, info = _plan_c(lib, lo, hi, n, lam)
        assert rc == 0, row
        assert tuple(info.res) == tuple(int(r) for r in row[8:11]), (row, tuple(info.res))
        assert np.array_equal(np.array(info.scale[:], np.float32), np.array(row[11:14], np.float32)), row
        assert info.ncells == int(row[14]), row


def test_plan_errors(lib):
    rc, _ = _plan_c(lib, (0, 0, 0), (1, 1, 1), 10, 0.0)
    assert rc == _lib.GRID_EINVAL
    rc, _ = _plan_c(lib, (0, 0, 0), (1, 1, 1), 10, float("nan"))
    assert rc == _lib.GRID_EINVAL
    rc, _ = _plan_c(lib, (0, 0, 0), (1, 1, 1), 2 ** 31 - 2, 3.0e38)
    assert rc == _lib.GRID_EOVERFLOW
    rc, info = _plan_c(lib, (0, 0, 0), (0, 0, 0), 0, 1.0)
    assert rc == 0 and tuple(info.res) == (1, 1, 1) and info.ncells == 1 and info.key_bits == 0


def test_null_arguments_rejected(lib):
    assert lib.grid_plan(None, None, 1, 1.0, None) == _lib.GRID_EINVAL
    assert lib.grid_build(None, None, 0, None, 0, 1.0, None, None, None) == _lib.GRID_EINVAL
    assert lib.grid_ctx_create(0, None, None) == _lib.GRID_EINVAL


def test_null_arguments_rejected_serving(lib):
    tk = ctypes.c_uint64()
    assert lib.grid_serve_create(0, None, None) == _lib.GRID_EINVAL
    assert lib.grid_serve_submit(None, 0, None, 0.0, 0, ctypes.byref(tk)) == _lib.GRID_EINVAL
    assert lib.grid_serve_poll(None, 1, None, None, None) == _lib.GRID_EINVAL
    assert lib.grid_serve_wait(None, 1, 0, None, None, None) == _lib.GRID_EINVAL
    assert lib.grid_serve_release(None, 1) == _lib.GRID_EINVAL
    assert lib.grid_serve_get_stats(None, None, 0) == _lib.GRID_EINVAL
    mid = ctypes.c_int32()
    assert lib.grid_serve_register(None, None, 0, None, 0, 1.0, ctypes.byref(mid)) == _lib.GRID_EINVAL
    assert lib.grid_jitter(None, None, None, 0, 0.01, 0) == _lib.GRID_EINVAL
    lib.grid_serve_destroy(None)


# (ctypes mirror, C type name, fields) of every struct the ABI passes by pointer
_STRUCTS = [
    (_lib.GridInfo, "grid_info"), (_lib.GridBuf, "grid_buf"), (_lib.GridOpts, "grid_opts"),
    (_lib.GridMesh, "grid_mesh"), (_lib.GridKernelStat, "grid_kernel_stat"),
    (_lib.GridServeOpts, "grid_serve_opts"), (_lib.GridServeStats, "grid_serve_stats"),
]
# ctypes field names that differ from the header's
_RENAMED = {("grid_mesh", "lam"): "lambda"}


def test_struct_layouts_match_header(tmp_path):
    """sizeof and every field offset of the ctypes mirrors equal what a C
    compiler makes of include/grid.h."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "grid.h"', 'int main(void) {']
    want = []
    for cls, cname in _STRUCTS:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            cf = _RENAMED.get((cname, fname), fname)
            lines.append(f'printf("%zu\\n", offsetof({cname}, {cf}));')
            want.append(getattr(cls, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == want
