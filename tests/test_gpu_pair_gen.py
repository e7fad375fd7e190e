"""The pair-generation modes of grid_build (grid_opts.pair_gen) against the
oracle: the paper's unfused chain (pairs written to device memory, then
sorted), the sorted grid's one-thread-per-object MakePairs (an ablation) and
the first sort pass that regenerates its pairs in both kernels must give the
same object-order pairs and the same grid as the default path, bit for
bit."""
import numpy as np
import pytest

import oracle
import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = ["emit", "per_object", "regen"]


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def mode_ctx():
    import paper_2403_10647_gb300 as pg
    ctxs = {m: pg.Context(0, pair_gen=m) for m in MODES}
    yield ctxs
    for c in ctxs.values():
        c.close()


SCENES = [
    ("uniform_20k", lambda: scenes.uniform_soup(20_000, seed=401)),
    ("nonhomog_30k", lambda: scenes.nonhomogeneous_soup(30_000, seed=402, extent=30.0)),
    ("arch_60k", lambda: scenes.architectural(60_000, seed=403, size=(40.0, 10.0, 40.0), nblobs=40)),
    ("one_triangle", lambda: scenes.Scene("one", np.array([[0, 0, 0], [1, 0.5, 0.2], [0.3, 1, 0.9]], np.float32),
                                          np.array([[0, 1, 2]], np.int32), 64.0)),
    ("empty", lambda: scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 2.0)),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,make", SCENES, ids=[n for n, _ in SCENES])
def test_modes_match_oracle(ctx, mode_ctx, mode, name, make):
    s = make()
    g = mode_ctx[mode].build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
    o = oracle.build_grid(s.verts, s.tris, s.lam)
    assert tuple(g.info.res) == tuple(o.plan.res) and g.info.nrefs == o.NO
    assert np.array_equal(host(g.cells), o.G), (mode, name)
    assert np.array_equal(host(g.refs), o.refs), (mode, name)
    if s.n:
        f = ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
        assert torch.equal(f.cells, g.cells) and torch.equal(f.refs, g.refs)


def test_per_object_pairs_match_oracle(ctx):
    """grid_emit_pairs_per_object writes the object-order lists of Algorithm 1
    (MakeObjectIds .. MakeCellIds), as grid_emit_pairs does."""
    import paper_2403_10647_gb300 as pg
    s = scenes.nonhomogeneous_soup(40_000, seed=404, extent=35.0)
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    lo, hi = ctx.bounds(v, t)
    info = pg.plan(lo, hi, s.n, s.lam)
    recs, nrefs = ctx.count_scan(v, t, info)
    info.nrefs = nrefs
    C, O = ctx.emit_pairs_per_object(recs, nrefs, info)
    p = oracle.plan(*oracle.bounds(s.verts, s.tris), s.n, s.lam)
    clo, chi, V = oracle.cell_boxes(s.verts, s.tris, p)
    off, NO = oracle.exclusive_sum(V)
    oC, oO = oracle.object_order_pairs(clo, chi, off, NO, p.res)
    assert nrefs == NO
    assert np.array_equal(host(C), oC) and np.array_equal(host(O), oO)
    C2, O2 = ctx.emit_pairs(recs, nrefs, info)
    assert torch.equal(C, C2) and torch.equal(O, O2)


@pytest.mark.slow
@pytest.mark.parametrize("mode", MODES)
def test_modes_full_size_nonhomogeneous(ctx, mode_ctx, mode):
    """The 1M-triangle non-homogeneous scene (single triangles covering up to
    ~1e5 cells) in every mode equals the default build."""
    s = scenes.CONFIGS["nonhomogeneous_1e6"]()
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    f = ctx.build(v, t, s.lam)
    g = mode_ctx[mode].build(v, t, s.lam)
    assert torch.equal(f.cells, g.cells) and torch.equal(f.refs, g.refs)


@pytest.mark.parametrize("radix_bits", [8, 9, 10, 11])
def test_alt_tile_shape_matches_oracle(radix_bits):
    """The radix kernels' second block shape (384 threads x 8 pairs per
    3,072-pair tile) gives the oracle's grid at every digit width, in the
    fused and the emit pair generation."""
    import paper_2403_10647_gb300 as pg
    cases = [scenes.uniform_soup(30_000, seed=411), scenes.nonhomogeneous_soup(25_000, seed=412, extent=30.0),
             scenes.architectural(50_000, seed=413, size=(40.0, 10.0, 40.0), nblobs=30)]
    for mode in ("fused", "emit"):
        c = pg.Context(0, radix_bits=radix_bits, pair_gen=mode, tile_shape="384x8")
        try:
            for s in cases:
                g = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
                o = oracle.build_grid(s.verts, s.tris, s.lam)
                assert g.info.nrefs == o.NO, (radix_bits, mode, s.name)
                assert np.array_equal(host(g.cells), o.G) and np.array_equal(host(g.refs), o.refs), \
                    (radix_bits, mode, s.name)
        finally:
            c.close()


def test_alt_tile_shape_batched_and_culled():
    """The second radix-kernel shape in a batched build (each mesh equals
    its own build and the oracle) and in a culled build (equals the
    oracle's culled grid)."""
    import paper_2403_10647_gb300 as pg
    batch = [scenes.uniform_soup(6_000, seed=421), scenes.nonhomogeneous_soup(15_000, seed=422, extent=25.0),
             scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 4.0),
             scenes.architectural(30_000, seed=423, size=(30.0, 8.0, 30.0), nblobs=20)]
    c = pg.Context(0, tile_shape="384x8")
    try:
        grids = c.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch])
        for s, g in zip(batch, grids):
            o = oracle.build_grid(s.verts, s.tris, s.lam)
            assert g.info.nrefs == o.NO, s.name
            assert np.array_equal(host(g.cells), o.G) and np.array_equal(host(g.refs), o.refs), s.name
    finally:
        c.close()
    cc = pg.Context(0, tile_shape="384x8", cull=True)
    try:
        s = batch[1]
        g = cc.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
        o = oracle.build_grid(s.verts, s.tris, s.lam, cull=True)
        assert g.info.nrefs == o.NO
        assert np.array_equal(host(g.cells), o.G) and np.array_equal(host(g.refs), o.refs)
    finally:
        cc.close()


def test_bad_mode_rejected():
    import ctypes
    from paper_2403_10647_gb300 import _lib
    lib = _lib.load()
    o = _lib.GridOpts()
    o.pair_gen = 7
    h = ctypes.c_void_p()
    assert lib.grid_ctx_create(0, ctypes.byref(o), ctypes.byref(h)) == _lib.GRID_EINVAL
    o = _lib.GridOpts()
    o.tile_shape = 2
    assert lib.grid_ctx_create(0, ctypes.byref(o), ctypes.byref(h)) == _lib.GRID_EINVAL


def test_autotune_keeps_a_valid_setting_and_the_same_grid():
    import paper_2403_10647_gb300 as pg
    s = scenes.nonhomogeneous_soup(60_000, seed=407, extent=40.0)
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    c = pg.Context(0)
    try:
        before = c.build(v, t, s.lam)
        r = c.autotune(v, t, s.lam, reps=2)
        assert r["radix_bits"] in (8, 9, 10, 11) and r["pair_gen"] in ("fused", "emit")
        assert r["tile_shape"] in ("256x12", "384x8")
        assert r["local_bits"] in (0, -1, -2)
        tm = r["times_ms"]
        assert len(tm) == 10 and all(ms > 0 for ms in tm.values())
        combos = {k: ms for k, ms in tm.items() if k not in ("other_shape", "other_sort_end")}
        # the winning combination was found with the default shape; the other
        # shape was then tried with it and kept only if faster, then the
        # other sort end with the kept shape
        best = combos[(r["radix_bits"], r["pair_gen"])]
        assert best == min(combos.values())
        if r["tile_shape"] == "384x8":
            assert tm["other_shape"] < best
            best = tm["other_shape"]
        else:
            assert tm["other_shape"] >= best
        assert (tm["other_sort_end"] < best) == (r["local_bits"] != 0)
        after = c.build(v, t, s.lam)
        assert torch.equal(before.cells, after.cells) and torch.equal(before.refs, after.refs)
    finally:
        c.close()


def test_autotune_batched_keeps_the_same_grids():
    """The batch tuner times digit widths, the other block shape and the
    other sort end on a batch, keeps a valid setting, and the batch's grids
    (and each mesh's own build) stay the same."""
    import paper_2403_10647_gb300 as pg
    meshes = scenes.batched_meshes(12, scale=0.02)
    args = [(dev(m.verts, torch.float32), dev(m.tris, torch.int32), m.lam) for m in meshes]
    c = pg.Context(0)
    try:
        before = c.build_batched(args)
        r = c.autotune_batched(args, reps=2)
        assert r["radix_bits"] in (8, 9, 10, 11) and r["tile_shape"] in ("256x12", "384x8")
        assert r["local_bits"] in (0, -1, -2)
        tm = r["times_ms"]
        assert len(tm) == 6 and all(ms > 0 for ms in tm.values())
        widths = {k: ms for k, ms in tm.items() if isinstance(k, int)}
        assert widths[r["radix_bits"]] == min(widths.values())
        after = c.build_batched(args)
        for a, b, m in zip(before, after, meshes):
            assert torch.equal(a.cells, b.cells) and torch.equal(a.refs, b.refs)
            o = oracle.build_grid(m.verts, m.tris, m.lam, method="counting")
            assert np.array_equal(b.cells.cpu().numpy(), o.G) and np.array_equal(b.refs.cpu().numpy(), o.refs)
    finally:
        c.close()
