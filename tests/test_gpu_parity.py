"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Every comparison is exact: the outputs are integer index arrays, and the one
floating-point decision (world -> cell) is taken in FP32 with the same
operation order on both sides, so the grids must match bit for bit.
"""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.cpu().numpy()


def assert_grid_equal(g, o, what=""):
    info = g.info
    assert tuple(info.res) == tuple(o.plan.res), (what, info.res, o.plan.res)
    assert np.array_equal(np.array(info.scale, np.float32), o.plan.scale), what
    # bit patterns: a -0.0 bound against +0.0 must not pass
    assert np.array_equal(np.array(info.lo, np.float32).view(np.uint32), o.plan.lo.view(np.uint32)), what
    assert np.array_equal(np.array(info.hi, np.float32).view(np.uint32), o.plan.hi.view(np.uint32)), what
    assert info.ncells == o.plan.ncells and info.nrefs == o.NO, (what, info.ncells, info.nrefs, o.NO)
    G, refs = host(g.cells), host(g.refs)
    assert G.shape == o.G.shape and refs.shape == o.refs.shape, what
    bad = np.flatnonzero(G != o.G)
    assert bad.size == 0, (what, "cells differ", bad[:10], G[bad[:10]], o.G[bad[:10]])
    bad = np.flatnonzero(refs != o.refs)
    assert bad.size == 0, (what, "refs differ", bad[:10], refs[bad[:10]], o.refs[bad[:10]])


def build_both(ctx, s, method="alg1"):
    g = ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method=method)
    return g, o


# ---- step by step ----------------------------------------------------------------

STEP_SCENES = [
    ("uniform_20k", lambda: scenes.uniform_soup(20_000, seed=101)),
    ("nonhomog_30k", lambda: scenes.nonhomogeneous_soup(30_000, seed=102, extent=30.0)),
    ("arch_60k", lambda: scenes.architectural(60_000, seed=103, size=(40.0, 10.0, 40.0), nblobs=40)),
]


@pytest.mark.parametrize("name,make", STEP_SCENES, ids=[n for n, _ in STEP_SCENES])
def test_steps_match_oracle(ctx, name, make):
    s = make()
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    # a0 boxes / bounds
    lo, hi = ctx.bounds(v, t)
    olo, ohi = oracle.bounds(s.verts, s.tris)
    assert np.array_equal(np.array(lo, np.float32), olo) and np.array_equal(np.array(hi, np.float32), ohi)
    # a1 metadata
    import paper_2403_10647_gb300 as pg
    info = pg.plan(lo, hi, s.n, s.lam)
    p = oracle.plan(olo, ohi, s.n, s.lam)
    assert tuple(info.res) == tuple(p.res) and np.array_equal(np.array(info.scale, np.float32), p.scale)
    # a2 + a3 CountCells + ExclusiveSum
    recs, nrefs = ctx.count_scan(v, t, info)
    clo, chi, V = oracle.cell_boxes(s.verts, s.tris, p)
    off, NO = oracle.exclusive_sum(V)
    assert nrefs == NO
    r = host(recs).view(np.uint16).reshape(-1, 8).astype(np.int64)
    assert np.array_equal(r[:, 0:3], clo) and np.array_equal(r[:, 3:6], chi)
    assert np.array_equal(host(recs)[:, 3].astype(np.int64) & 0xFFFFFFFF, off)
    # a4 - a7 object-order pairs
    info.nrefs = nrefs
    C, O = ctx.emit_pairs(recs, nrefs, info)
    oC, oO = oracle.object_order_pairs(clo, chi, off, NO, p.res)
    assert np.array_equal(host(O), oO) and np.array_equal(host(C), oC)
    # a8 radix sort
    Cs, Os = ctx.sort_pairs(C, O, info.key_bits)
    sC, sO = oracle.sort_pairs(oC, oO)
    assert np.array_equal(host(Cs), sC) and np.array_equal(host(Os), sO)
    # a9 ranges
    G = ctx.extract_ranges(Cs, info.ncells)
    assert np.array_equal(host(G), oracle.ranges(sC, p.ncells))


def test_hand_example_steps(ctx):
    """The hand-worked Algorithm 1 example, step by step on the GPU."""
    import _pins
    import paper_2403_10647_gb300 as pg
    g = _pins.read_golden("hand_example.txt")
    verts = np.array(g["verts"], np.float32).reshape(-1, 3)
    tris = np.array(g["tris"], np.int32).reshape(-1, 3)
    info = pg.Info(lo=(0.0, 0.0, 0.0), hi=(4.0, 4.0, 1.0), scale=(1.0, 1.0, 1.0), res=(4, 4, 1), key_bits=4,
                   ncells=16, nrefs=0, n=4)
    recs, nrefs = ctx.count_scan(dev(verts, torch.float32), dev(tris, torch.int32), info)
    assert nrefs == int(g["NO"][0])
    C, O = ctx.emit_pairs(recs, nrefs, info)
    assert host(C).tolist() == [int(x) for x in g["C_object_order"]]
    assert host(O).tolist() == [int(x) for x in g["O_object_order"]]
    Cs, Os = ctx.sort_pairs(C, O, 4)
    assert host(Cs).tolist() == [int(x) for x in g["C_sorted"]]
    assert host(Os).tolist() == [int(x) for x in g["O_sorted"]]
    assert host(ctx.extract_ranges(Cs, 16)).tolist() == [int(x) for x in g["G"]]


# ---- the radix sort on its own: sizes spanning tiles and ragged tails ---------------

@pytest.mark.parametrize("count", [1, 2, 31, 4095, 4096, 4097, 3 * 4096 + 17, 250_001, 2_000_003])
@pytest.mark.parametrize("key_bits", [1, 7, 8, 9, 13, 17, 22, 27, 31])
def test_sort_pairs(ctx, count, key_bits):
    g = np.random.Generator(np.random.Philox(count * 64 + key_bits))
    hi = 1 << key_bits
    if key_bits > 12 and count > 4096:   # clustered keys with long runs of equal digits
        C = (g.integers(0, 64, count) * (hi // 64) + g.integers(0, 3, count)).astype(np.int64)
    else:
        C = g.integers(0, hi, count).astype(np.int64)
    C = C.astype(np.int32)
    O = np.arange(count, dtype=np.int32)[::-1].copy()
    Cs, Os = ctx.sort_pairs(dev(C, torch.int32), dev(O, torch.int32), key_bits)
    if count <= 300_000:
        sC, sO = oracle.sort_pairs(C, O)
    else:  # stable argsort is the special case the oracle's sort reduces to
        perm = np.argsort(C, kind="stable")
        sC, sO = C[perm], O[perm]
    assert np.array_equal(host(Cs), sC) and np.array_equal(host(Os), sO)


@pytest.mark.parametrize("n,extent", [(300_000, 63.0), (600_000, 79.4)])
def test_mid_size_upsweep_groups(ctx, n, extent):
    """Sorts of ~6k and ~11k tiles, where the upsweep walks groups of a few
    tiles each (between the one-tile groups of small sorts and the 16-tile
    groups of large ones) and the last group is partial, in both radix
    kernel shapes."""
    import paper_2403_10647_gb300 as pg
    s = scenes.nonhomogeneous_soup(n, seed=431, extent=extent)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    ntiles = (o.NO + 3071) // 3072
    assert 4000 < ntiles < 20000   # groups of 4 and 12 tiles on 152 SMs, the last one partial
    alt = pg.Context(0, tile_shape="384x8")
    try:
        for c in (ctx, alt):
            g = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
            assert_grid_equal(g, o, f"mid-size {n}")
    finally:
        alt.close()


@pytest.mark.parametrize("radix_bits", [8, 9, 10, 11])
def test_radix_widths_agree(radix_bits):
    import paper_2403_10647_gb300 as pg
    c = pg.Context(0, radix_bits=radix_bits)
    try:
        for s in (scenes.uniform_soup(50_000, seed=7), scenes.nonhomogeneous_soup(40_000, seed=8, extent=35.0)):
            g, o = build_both(c, s)
            assert_grid_equal(g, o, f"radix {radix_bits} {s.name}")
    finally:
        c.close()


@pytest.mark.parametrize("ncells,count", [(1, 10), (7, 1), (5000, 0), (5000, 3), (100_000, 300_000),
                                          (3_000_000, 200_000)])
def test_extract_ranges(ctx, ncells, count):
    g = np.random.Generator(np.random.Philox(ncells + count))
    C = np.sort(g.integers(0, ncells, count)).astype(np.int32)
    G = ctx.extract_ranges(dev(C, torch.int32) if count else torch.zeros(0, dtype=torch.int32, device="cuda"),
                           ncells)
    assert np.array_equal(host(G), oracle.ranges(C, ncells))


@pytest.mark.parametrize("pattern", ["one_cell", "ends", "long_runs", "first_and_last_cell", "every_cell"])
def test_extract_ranges_patterns(ctx, pattern):
    """Runs longer than an extraction block (4,096 merged items), gaps of a
    million empty cells, keys only in the first and last cells."""
    g = np.random.Generator(np.random.Philox(4711))
    ncells = 1_000_003
    if pattern == "one_cell":
        C = np.full(50_000, ncells // 2, np.int32)
    elif pattern == "ends":
        C = np.repeat(np.array([0, 1, ncells - 2, ncells - 1], np.int32), [3, 5000, 7, 4100])
    elif pattern == "long_runs":
        C = np.sort(g.choice(ncells, 40, replace=False).astype(np.int32).repeat(g.integers(1, 9000, 40)))
    elif pattern == "first_and_last_cell":
        C = np.array([0] * 3000 + [ncells - 1] * 2, np.int32)
    else:
        C = np.arange(ncells, dtype=np.int32)
    G = ctx.extract_ranges(dev(C, torch.int32), ncells)
    assert np.array_equal(host(G), oracle.ranges(C, ncells)), pattern


def test_extract_ranges_rejects_unsorted_keys(ctx):
    """Keys out of order (a caller's mistake) are reported, not read as a
    grid, and the context stays usable."""
    import paper_2403_10647_gb300 as pg
    g = np.random.Generator(np.random.Philox(4712))
    C = g.integers(0, 1000, 100_000).astype(np.int32)
    with pytest.raises(pg.GridError):
        ctx.extract_ranges(dev(C, torch.int32), 1000)
    C.sort()
    assert np.array_equal(host(ctx.extract_ranges(dev(C, torch.int32), 1000)), oracle.ranges(C, 1000))


@pytest.mark.parametrize("offset", [1, 2, 3, 4])
def test_extract_ranges_unaligned_input(ctx, offset):
    """A caller's sorted keys may start off a 16-byte boundary (a slice of a
    larger array): the range extraction then reads them word by word."""
    g = np.random.Generator(np.random.Philox(77 + offset))
    ncells, count = 300_000, 1_000_003
    C = np.sort(g.integers(0, ncells, count)).astype(np.int32)
    full = dev(np.concatenate([np.zeros(offset, np.int32), C]), torch.int32)
    view = full[offset:]
    assert (view.data_ptr() % 16 == 0) == (offset == 4)
    G = ctx.extract_ranges(view, ncells)
    assert np.array_equal(host(G), oracle.ranges(C, ncells))


# ---- whole builds ---------------------------------------------------------------------

def test_tiny_scenes(ctx):
    g = np.random.Generator(np.random.Philox(99))
    for k in range(60):
        n = int(g.integers(1, 300))
        s = scenes.tiny_scene(g, n, box=float(g.uniform(0.5, 50.0)), max_edge=float(g.uniform(0.01, 20.0)))
        gg, o = build_both(ctx, s)
        assert_grid_equal(gg, o, f"tiny {k}")


@pytest.mark.parametrize("name,make", STEP_SCENES, ids=[n for n, _ in STEP_SCENES])
def test_build_medium(ctx, name, make):
    g, o = build_both(ctx, make())
    assert_grid_equal(g, o, name)


def test_deterministic(ctx):
    s = scenes.nonhomogeneous_soup(100_000, seed=9, extent=46.0)
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    a = ctx.build(v, t, s.lam)
    b = ctx.build(v, t, s.lam)
    assert torch.equal(a.cells, b.cells) and torch.equal(a.refs, b.refs)


def test_build_host_matches_device(ctx):
    s = scenes.uniform_soup(30_000, seed=10)
    g = ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
    cells, refs, info = ctx.build_host(torch.from_numpy(s.verts).pin_memory(),
                                       torch.from_numpy(s.tris).pin_memory(), s.lam)
    assert np.array_equal(cells.numpy(), host(g.cells)) and np.array_equal(refs.numpy(), host(g.refs))
    # pageable memory, caller buffers reused
    cells2, refs2, _ = ctx.build_host(s.verts, s.tris, s.lam, cells_out=cells.clone(), refs_out=refs.clone())
    assert np.array_equal(cells2.numpy(), cells.numpy()) and np.array_equal(refs2.numpy(), refs.numpy())


def test_build_host_culled_errors_and_small_buffers():
    """The host-buffer build in the culling mode equals the oracle's culled
    grid; a refs buffer that is too small is reallocated; a bad index is
    reported with no copy left running, and the context then builds again."""
    import paper_2403_10647_gb300 as pg
    s = scenes.nonhomogeneous_soup(20_000, seed=11, extent=25.0)
    c = pg.Context(0, cull=True)
    try:
        o = oracle.build_grid(s.verts, s.tris, s.lam, cull=True)
        small = torch.empty(3, dtype=torch.int32).pin_memory()
        cells, refs, info = c.build_host(s.verts, s.tris, s.lam,
                                         cells_out=torch.empty(o.G.shape[0], dtype=torch.int32).pin_memory(),
                                         refs_out=small)
        assert info.nrefs == o.NO
        assert np.array_equal(cells.numpy(), o.G) and np.array_equal(refs.numpy(), o.refs)
        bad = s.tris.copy()
        bad[5, 2] = s.verts.shape[0] + 9
        with pytest.raises(pg.GridError):
            c.build_host(s.verts, bad, s.lam, cells_out=cells, refs_out=refs)
        cells2, refs2, _ = c.build_host(s.verts, s.tris, s.lam, cells_out=cells.clone(), refs_out=refs.clone())
        assert np.array_equal(cells2.numpy(), o.G) and np.array_equal(refs2.numpy(), o.refs)
    finally:
        c.close()


# ---- edge cases -----------------------------------------------------------------------

def _scene(verts, tris, lam):
    return scenes.Scene("edge", np.asarray(verts, np.float32).reshape(-1, 3),
                        np.asarray(tris, np.int32).reshape(-1, 3), lam)


def test_empty(ctx):
    g = ctx.build(torch.zeros((0, 3), device="cuda"), torch.zeros((0, 3), dtype=torch.int32, device="cuda"), 4.0)
    assert host(g.cells).tolist() == [0, 0] and g.refs.numel() == 0 and tuple(g.info.res) == (1, 1, 1)


def _signed_zero_scene(g, negative: bool):
    """Random triangles whose min faces (max faces if negative) hold both
    -0.0 and +0.0, in a random order of the two zeros."""
    v = g.random((3000, 3)).astype(np.float32)
    if negative:
        v = -v
    tris = g.integers(0, 3000, (1000, 3))
    for k in range(60):   # 20 zeros per axis on referenced vertices, signs alternating by a coin
        v[tris[k, 0], k % 3] = np.float32(-0.0) if g.random() < 0.5 else np.float32(0.0)
    return _scene(v, tris, 4.0)


@pytest.mark.parametrize("case", ["one_tri", "single_cell", "flat_z", "point", "huge_plus_small", "needle",
                                  "clamped_x", "clamped_xy", "signed_zero_min", "signed_zero_max"])
def test_degenerate_scenes(ctx, case):
    g = np.random.Generator(np.random.Philox(5))
    if case.startswith("signed_zero"):
        s = _signed_zero_scene(g, case.endswith("max"))
    elif case == "one_tri":
        s = _scene([[0, 0, 0], [1, 0.5, 0.2], [0.3, 1, 0.9]], [[0, 1, 2]], 64.0)
    elif case == "single_cell":   # lambda * n / volume < 1: one cell, no sort passes
        s = _scene(g.random((30, 3)), g.integers(0, 30, (10, 3)), 0.05)
    elif case == "flat_z":
        v = g.random((300, 3))
        v[:, 2] = 0.25
        s = _scene(v, g.integers(0, 300, (100, 3)), 4.0)
    elif case == "point":
        s = _scene(np.full((9, 3), 3.5), [[0, 1, 2], [3, 4, 5], [6, 7, 8]], 4.0)
    elif case == "huge_plus_small":   # one triangle spans the whole grid
        v = np.concatenate([[[0, 0, 0], [10, 0, 10], [0, 10, 5]], g.random((3000, 3)) * 10])
        s = _scene(v, np.concatenate([[[0, 1, 2]], 3 + g.integers(0, 3000, (1000, 3))]), 8.0)
    elif case == "needle":  # a long thin diagonal triangle (many false intersections, Sec. 5)
        v = np.concatenate([[[0, 0, 0], [20, 20, 20], [20.01, 20, 20]], g.random((3000, 3)) * 20])
        s = _scene(v, np.concatenate([[[0, 1, 2]], 3 + g.integers(0, 3000, (1000, 3))]), 4.0)
    elif case == "clamped_x":   # a 1-D scene whose resolution rule asks for 160,000 cells: res_x = 65,535
        x = g.random(6000) * 1000.0
        v = np.stack([np.concatenate([x, x + 0.05, x + 0.1]), np.full(18000, 0.5), np.full(18000, 0.25)], axis=1)
        s = _scene(v, np.stack([np.arange(6000), 6000 + np.arange(6000), 12000 + np.arange(6000)], axis=1), 8.0 / 0.3)
    else:   # a 2-D sheet with one long axis: x clamps at 65,535 cells, y does not
        x, y = g.random(4000) * 4000.0, g.random(4000) * 2.0
        v = np.stack([np.concatenate([x, x + 0.2, x]), np.concatenate([y, y, y + 0.1]), np.full(12000, 1.0)], axis=1)
        s = _scene(v, np.stack([np.arange(4000), 4000 + np.arange(4000), 8000 + np.arange(4000)], axis=1), 2000.0)
    gg, o = build_both(ctx, s)
    if case.startswith("signed_zero"):   # the zero bounds are +0.0 on both sides (compared by bits below)
        zb = gg.info.hi if case.endswith("max") else gg.info.lo
        assert all(np.float32(x).view(np.uint32) == 0 for x in zb), zb
    if case.startswith("clamped"):
        assert gg.info.res[0] == 65535, gg.info.res
    assert_grid_equal(gg, o, case)


def test_bad_index_rejected(ctx):
    import paper_2403_10647_gb300 as pg
    s = scenes.uniform_soup(1000, seed=3)
    t = s.tris.copy()
    t[500, 1] = s.verts.shape[0]
    with pytest.raises(pg.GridError) as e:
        ctx.build(dev(s.verts, torch.float32), dev(t, torch.int32), s.lam)
    assert e.value.code == -1
    t[500, 1] = -5
    with pytest.raises(pg.GridError):
        ctx.build(dev(s.verts, torch.float32), dev(t, torch.int32), s.lam)
    # the context stays usable
    g, o = build_both(ctx, s)
    assert_grid_equal(g, o, "after error")


def test_nonfinite_rejected(ctx):
    import paper_2403_10647_gb300 as pg
    s = scenes.uniform_soup(1000, seed=4)
    for bad in (np.nan, np.inf, -np.inf):
        v = s.verts.copy()
        v[s.tris[17, 2], 0] = bad
        with pytest.raises(pg.GridError) as e:
            ctx.build(dev(v, torch.float32), dev(s.tris, torch.int32), s.lam)
        assert e.value.code == -1


def test_bad_lambda_rejected(ctx):
    import paper_2403_10647_gb300 as pg
    s = scenes.uniform_soup(100, seed=4)
    for lam in (0.0, -1.0, float("nan")):
        with pytest.raises(pg.GridError):
            ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), lam)


def test_nrefs_overflow_reported(ctx):
    """Two triangles that each cover all of a 1.7e9-cell grid: NO = 3.5e9
    exceeds INT32_MAX and the build reports it before allocating pairs."""
    import paper_2403_10647_gb300 as pg
    v = [[0, 0, 0], [1, 1, 1], [0, 1, 0], [1, 0, 1], [0, 0, 1], [1, 1, 0]]
    with pytest.raises(pg.GridError) as e:
        ctx.build(dev(np.array(v, np.float32), torch.float32), dev(np.array([[0, 1, 2], [3, 4, 5]]), torch.int32),
                  1200.0 ** 3 / 2)
    assert e.value.code == -3


# ---- the benchmark's workloads at full size ----------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("name", ["uniform_1e5", "nonhomogeneous_1e6", "architectural_1e7"])
def test_full_size_configs(ctx, name):
    s = scenes.CONFIGS[name]()
    g, o = build_both(ctx, s, method="counting")
    assert_grid_equal(g, o, name)


@pytest.mark.parametrize("radix_bits,key_bits", [(10, 20), (10, 30), (11, 11), (11, 22), (11, 31)])
@pytest.mark.parametrize("count", [5_000, 4096 * 37 + 5, 1_500_001])
def test_sort_wide_digits(radix_bits, key_bits, count):
    """The 10- and 11-bit digit kernels (peer masks outside the staging
    buffer when they do not fit) against a stable sort."""
    import paper_2403_10647_gb300 as pg
    g = np.random.Generator(np.random.Philox(radix_bits * 1000 + key_bits + count))
    C = g.integers(0, 1 << key_bits, count).astype(np.int64).astype(np.int32)
    O = np.arange(count, dtype=np.int32)
    c = pg.Context(0, radix_bits=radix_bits)
    try:
        Cs, Os = c.sort_pairs(dev(C, torch.int32), dev(O, torch.int32), key_bits)
    finally:
        c.close()
    perm = np.argsort(C, kind="stable")
    assert np.array_equal(host(Cs), C[perm]) and np.array_equal(host(Os), O[perm])


@pytest.mark.parametrize("radix_bits,lam", [(10, 6.0), (11, 24.0)])
def test_wide_digits_full_build(radix_bits, lam):
    """Whole builds whose keys split into two digits of exactly radix_bits
    bits (20-bit keys at 10, 22-bit keys at 11)."""
    import paper_2403_10647_gb300 as pg
    s = scenes.nonhomogeneous_soup(100_000, seed=31, extent=46.0, lam=lam)
    c = pg.Context(0, radix_bits=radix_bits)
    try:
        g = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
        assert g.info.key_bits == 2 * radix_bits
        o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
        assert_grid_equal(g, o, f"radix {radix_bits}")
    finally:
        c.close()


# ---- batched builds ---------------------------------------------------------------------

def _mixed_batch():
    g = np.random.Generator(np.random.Philox(4242))
    return [
        scenes.uniform_soup(5_000, seed=201),
        scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 4.0),
        _scene([[0, 0, 0], [1, 0.5, 0.2], [0.3, 1, 0.9]], [[0, 1, 2]], 64.0),
        scenes.tiny_scene(g, 37),
        scenes.nonhomogeneous_soup(20_000, seed=202, extent=25.0),
        scenes.architectural(30_000, seed=203, size=(30.0, 8.0, 30.0), nblobs=20),
        scenes.Scene("empty2", np.zeros((5, 3), np.float32), np.zeros((0, 3), np.int32), 2.0),
    ]


def test_batched_matches_oracle_and_plain(ctx):
    batch = _mixed_batch()
    grids = ctx.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch])
    assert len(grids) == len(batch)
    for s, g in zip(batch, grids):
        o = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1" if s.n < 50_000 else "counting")
        assert_grid_equal(g, o, f"batched {s.name}")
        if s.n:
            p = ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
            assert torch.equal(p.cells, g.cells) and torch.equal(p.refs, g.refs), s.name


def test_batched_sort_segments_match_oracle_and_plain():
    """A batch whose global cell ids need a radix pass more than any of its
    meshes is sorted in segments of consecutive meshes (keys counted from
    each segment's first cell): every mesh equals its own build and the
    oracle, with empty meshes and single triangles between segments."""
    import paper_2403_10647_gb300 as pg
    g = np.random.Generator(np.random.Philox(4343))
    batch = []
    for k in range(6):
        batch.append(scenes.uniform_soup(4_000 + 700 * k, seed=210 + k))
        if k == 2:
            batch.append(scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 4.0))
        if k == 4:
            batch.append(scenes.tiny_scene(g, 1))
    batch.append(scenes.nonhomogeneous_soup(6_000, seed=220, extent=12.0))
    lam = 8.0
    c = pg.Context(0, radix_bits=8, local_bits=-1)
    try:
        args = [(dev(s.verts, torch.float32), dev(s.tris, torch.int32), lam) for s in batch]
        c.profile(True)
        grids = c.build_batched(args)
        st = c.kernel_stats()
        c.profile(False)
        ncells = [int(gr.info.ncells) for gr in grids]
        assert max(ncells) <= 1 << 16 < sum(ncells), ncells   # 2 passes each, 3 for the whole batch
        assert "rebase" in st, st.keys()
        for s, gr in zip(batch, grids):
            o = oracle.build_grid(s.verts, s.tris, lam, method="alg1")
            assert_grid_equal(gr, o, f"segmented batch {s.name}")
            if s.n:
                p = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), lam)
                assert torch.equal(p.cells, gr.cells) and torch.equal(p.refs, gr.refs), s.name
    finally:
        c.close()


def test_batched_signed_zero_bounds(ctx):
    """Per-mesh bounds of a batch report zero bounds as +0.0, as plain builds
    and the oracle do (bit patterns compared)."""
    g = np.random.Generator(np.random.Philox(21))
    batch = [_signed_zero_scene(g, False), scenes.uniform_soup(2000, seed=3), _signed_zero_scene(g, True)]
    grids = ctx.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch])
    for s, gr in zip(batch, grids):
        assert_grid_equal(gr, oracle.build_grid(s.verts, s.tris, s.lam, method="alg1"), f"batched {s.name}")


def test_batched_twice_same_result(ctx):
    batch = _mixed_batch()
    args = [(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch]
    a = ctx.build_batched(args)
    b = ctx.build_batched(args)
    for x, y in zip(a, b):
        assert torch.equal(x.cells, y.cells) and torch.equal(x.refs, y.refs)


def test_batched_rejects_bad_mesh(ctx):
    import paper_2403_10647_gb300 as pg
    s = scenes.uniform_soup(1000, seed=5)
    bad = s.tris.copy()
    bad[10, 0] = s.verts.shape[0] + 3
    with pytest.raises(pg.GridError) as e:
        ctx.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam),
                           (dev(s.verts, torch.float32), dev(bad, torch.int32), s.lam)])
    assert e.value.code == -1
    # the context's staging tables are reusable after the failed call
    g = ctx.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)])
    assert_grid_equal(g[0], oracle.build_grid(s.verts, s.tris, s.lam), "after a failed batch")


def test_batched_sequence_views(ctx):
    """The batch result indexes like a list (negative indices, slices) and its
    per-mesh grids are views at cells_offsets / refs_offsets of the two
    shared buffers."""
    batch = _mixed_batch()
    grids = ctx.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch])
    n = len(batch)
    assert grids[-1] is grids[n - 1] and [g.info.n for g in grids[1:3]] == [s.n for s in batch[1:3]]
    with pytest.raises(IndexError):
        grids[n]
    with pytest.raises(IndexError):
        grids[-n - 1]
    assert grids.cells_offsets[0] == 0 and grids.refs_offsets[0] == 0
    for m, g in enumerate(grids):
        c0, r0 = grids.cells_offsets[m], grids.refs_offsets[m]
        assert g.cells.data_ptr() == grids.cells.data_ptr() + 4 * c0
        if g.info.nrefs:
            assert g.refs.data_ptr() == grids.refs.data_ptr() + 4 * r0
        if m + 1 < n:
            assert grids.cells_offsets[m + 1] == c0 + g.info.ncells + 1
            assert grids.refs_offsets[m + 1] == r0 + g.info.nrefs


@pytest.mark.slow
def test_batched_64_meshes_match_plain(ctx):
    """The 64-mesh batch (sizes log-uniform in [1e3, 2e6]) against 64 plain
    builds, mesh by mesh, and against the oracle on a spread of meshes."""
    meshes = scenes.batched_meshes()
    args = [(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in meshes]
    grids = ctx.build_batched(args)
    order = np.argsort([s.n for s in meshes])
    check_oracle = set(order[:3].tolist()) | set(order[len(order) // 2: len(order) // 2 + 2].tolist()) | {int(order[-1])}
    for k, (s, g, a) in enumerate(zip(meshes, grids, args)):
        p = ctx.build(*a)
        assert torch.equal(p.cells, g.cells) and torch.equal(p.refs, g.refs), k
        if k in check_oracle:
            assert_grid_equal(g, oracle.build_grid(s.verts, s.tris, s.lam, method="counting"), f"mesh {k}")
        del p


# ---- failure detection ------------------------------------------------------------------

def test_bounded_wait_times_out_and_context_survives(ctx):
    """The sort's look-back, waiting on a predecessor that never publishes,
    gives up after its poll limit: the call returns GRID_ETIMEOUT within
    seconds, and the same context then builds a grid correctly."""
    import ctypes
    from paper_2403_10647_gb300 import _lib
    lib = _lib.load()
    ms = ctypes.c_double()
    rc = lib.grid_selftest_wait_timeout(ctx._h, ctypes.byref(ms))
    assert rc == _lib.GRID_ETIMEOUT, lib.grid_strerror(rc)
    assert 0.0 < ms.value < 10_000.0, ms.value
    s = scenes.uniform_soup(5_000, seed=99)
    g, o = build_both(ctx, s)
    assert_grid_equal(g, o, "after a timed-out wait")


# ---- grid metadata computed on the device ---------------------------------------------

def _plan_scene(lo, hi, n):
    """n triangles whose union box is exactly [lo, hi]: the first spans it,
    the others are points at lo."""
    lo, hi = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    v = np.stack([lo, hi, np.array([hi[0], lo[1], hi[2]], np.float32)])
    tris = np.zeros((n, 3), np.int32)
    tris[0] = (0, 1, 2)
    return v, tris


def test_device_plan_on_the_closed_form_cases(ctx):
    """The build's grid metadata comes from the device (one host round trip
    fewer) and is checked against the host's; on the hand-worked resolution
    cases it must give exactly their res, scale and ncells."""
    import _pins
    before = ctx.counters()["plan_redos"]
    for row in _pins.read_plan_cases():
        lo, hi, n, lam = row[0:3], row[3:6], int(row[6]), row[7]
        if n > 1_000_000 or row[14] > 10_000_000:
            continue
        v, t = _plan_scene(lo, hi, n)
        g = ctx.build(dev(v, torch.float32), dev(t, torch.int32), lam)
        assert tuple(g.info.res) == tuple(int(r) for r in row[8:11]), (row, tuple(g.info.res))
        assert np.array_equal(np.array(g.info.scale, np.float32), np.array(row[11:14], np.float32)), row
        assert g.info.ncells == int(row[14]), row
    assert ctx.counters()["plan_redos"] == before   # exact cube roots: the device agrees


def test_device_plan_random_bounds_match_oracle(ctx):
    """Random bounds, triangle counts and densities: whatever the device's
    cube root does, the build's metadata equals the oracle's bit for bit
    (a disagreement re-runs CountCells with the host's plan)."""
    g = np.random.Generator(np.random.Philox(23))
    for k in range(200):
        lo = (g.standard_normal(3) * 10.0 ** g.uniform(-2, 3)).astype(np.float32)
        ext = (10.0 ** g.uniform(-2, 2, 3)).astype(np.float32)
        if k % 9 == 0:
            ext[g.integers(0, 3)] = 0.0
        hi = (lo + ext).astype(np.float32)
        n = int(g.integers(1, 64))
        lam = float(np.float32(g.uniform(0.5, 2000.0)))
        v, t = _plan_scene(lo, hi, n)
        try:
            p = oracle.plan(v.min(0), v.max(0), n, lam)
        except oracle.OracleError:
            continue
        if p.ncells > 2_000_000:
            continue
        gr = ctx.build(dev(v, torch.float32), dev(t, torch.int32), lam)
        assert tuple(gr.info.res) == tuple(p.res), (k, tuple(gr.info.res), p.res)
        assert np.array_equal(np.array(gr.info.scale, np.float32).view(np.uint32), p.scale.view(np.uint32)), k
        o = oracle.build_grid(v, t, lam, method="counting")
        assert np.array_equal(host(gr.cells), o.G) and np.array_equal(host(gr.refs), o.refs), k


def _giant_triangle_scene(n_small, seed):
    """One triangle spanning the scene's whole box (so its pairs cover a few
    hundred pair tiles), placed in the middle of the object order, among
    small ones."""
    g = np.random.Generator(np.random.Philox(seed))
    c = g.random((n_small, 3)) * 10.0
    v = np.concatenate([c, c + 0.02, c + [0.02, 0.0, 0.02]]).astype(np.float32)
    tris = np.stack([np.arange(n_small), n_small + np.arange(n_small), 2 * n_small + np.arange(n_small)], 1)
    big_v = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 10.0], [0.0, 10.0, 10.0]], np.float32)
    v = np.concatenate([v, big_v])
    big = np.arange(3 * n_small, 3 * n_small + 3)[None, :]
    tris = np.concatenate([tris[: n_small // 2], big, tris[n_small // 2:]]).astype(np.int32)
    return scenes.Scene("giant", v, tris, 16.0)


def test_pair_tiles_across_builds_of_one_context():
    """A context records the pair tiles' first objects during count/scan once
    its tile buffer is large enough, and falls back to the search otherwise
    (the first build, a larger build, an object over more than 64 tiles):
    every build of a growing and shrinking sequence equals the oracle."""
    import paper_2403_10647_gb300 as pg
    seq = [scenes.uniform_soup(3_000, seed=601), scenes.uniform_soup(30_000, seed=602),
           _giant_triangle_scene(20_000, seed=603), scenes.uniform_soup(3_000, seed=601),
           scenes.nonhomogeneous_soup(40_000, seed=604, extent=20.0), _giant_triangle_scene(20_000, seed=603)]
    c = pg.Context(0)
    try:
        for k, s in enumerate(seq):
            o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
            for rep in range(2):   # the second build of a scene runs with the buffer the first sized
                g = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
                assert_grid_equal(g, o, f"build {k} ({s.name}) rep {rep}")
        giant = seq[2]
        o = oracle.build_grid(giant.verts, giant.tris, giant.lam, method="counting")
        assert int(np.diff(o.G).max()) >= 1 and o.NO > 64 * 3072 + 20_000   # the giant object spans > 64 tiles
    finally:
        c.close()
