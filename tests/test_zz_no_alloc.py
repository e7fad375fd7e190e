"""grid_extract_ranges_noalloc: range extraction for callers that cannot
allocate device memory when they call it (code under another runtime's memory
manager, loops where an allocation would synchronise the device, paths that
must not run out of memory once initialised).

It is checked through the C ABI against grid_extract_ranges (the entry point
that allocates its scratch from a context) and against the CPU oracle's
ranges, bit for bit, on two calls in a row that reuse its fixed scratch
array; a rejected call (a key outside the grid) must not spoil the next one,
which shares the same error word.  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _sorted_keys(seed, count, ncells, clustered):
    g = np.random.Generator(np.random.Philox(seed))
    if clustered:   # dense runs of equal cells with long empty gaps between them
        base = g.integers(0, ncells // 64, count) * 64
        keys = np.minimum(base + g.integers(0, 3, count), ncells - 1)
    else:
        keys = g.integers(0, ncells, count)
    return np.sort(keys).astype(np.int32)


def _noalloc(lib, C, ncells):
    cells = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.grid_extract_ranges_noalloc(ctypes.c_void_p(C.data_ptr()), C.numel(), ncells,
                                         ctypes.c_void_p(cells.data_ptr()), ctypes.c_void_p(stream))
    return rc, cells


def test_noalloc_matches_allocating_entry_point_twice(ctx):
    from paper_2403_10647_gb300 import _lib
    lib = _lib.load()
    cases = [(1, 3_000_000, 1_200_000, True),     # large first: fills much of the scratch table
             (2, 40_000, 90_000, False)]          # then smaller: stale entries must not leak in
    for seed, count, ncells, clustered in cases:
        C = torch.from_numpy(_sorted_keys(seed, count, ncells, clustered)).cuda()
        rc, got = _noalloc(lib, C, ncells)
        assert rc == _lib.GRID_OK, lib.grid_strerror(rc)
        want = ctx.extract_ranges(C, ncells)
        assert torch.equal(got, want), f"case {seed}: ranges differ from grid_extract_ranges"
        assert np.array_equal(got.cpu().numpy(), oracle.ranges(C.cpu().numpy(), ncells)), \
            f"case {seed}: ranges differ from the oracle"
        assert int(got[-1]) == count and int(got[0]) == 0


def test_noalloc_error_does_not_leak_into_the_next_call(ctx):
    """A key equal to ncells is rejected (GRID_EINVAL); the error word it set
    is shared by every call, so the valid call right after must still return
    GRID_OK with the right ranges."""
    from paper_2403_10647_gb300 import _lib
    lib = _lib.load()
    ncells = 50_000
    keys = _sorted_keys(3, 200_000, ncells, False)
    bad = keys.copy()
    bad[-1] = ncells
    rc, _ = _noalloc(lib, torch.from_numpy(bad).cuda(), ncells)
    assert rc == _lib.GRID_EINVAL, lib.grid_strerror(rc)
    C = torch.from_numpy(keys).cuda()
    rc, got = _noalloc(lib, C, ncells)
    assert rc == _lib.GRID_OK, lib.grid_strerror(rc)
    assert torch.equal(got, ctx.extract_ranges(C, ncells))
    assert np.array_equal(got.cpu().numpy(), oracle.ranges(keys, ncells))


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    from paper_2403_10647_gb300 import _lib
    lib = _lib.load()
    C = torch.zeros(16, dtype=torch.int32, device="cuda")
    cells = torch.zeros(1, dtype=torch.int32, device="cuda")
    # ncells far beyond the fixed split table: rejected on the host, nothing launched
    rc = lib.grid_extract_ranges_noalloc(ctypes.c_void_p(C.data_ptr()), 16, 0x7FFF0000,
                                         ctypes.c_void_p(cells.data_ptr()), None)
    assert rc == _lib.GRID_ELIMIT
    assert b"fixed scratch" in lib.grid_strerror(rc)
