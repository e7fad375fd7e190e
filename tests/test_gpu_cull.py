"""The culling mode (a triangle/cell separating-axis test ahead of the sort,
Sec. 6's future work) through the C ABI, against the oracle's culling mode,
bit for bit: the kept object-order pairs of grid_cull_pairs, the hand-worked
cases of tests/golden/cull_example.txt, and whole culled builds."""
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


@pytest.fixture(scope="module")
def cull_ctx():
    import paper_2403_10647_gb300 as pg
    c = pg.Context(0, cull=True)
    yield c
    c.close()


SCENES = [
    ("uniform_20k", lambda: scenes.uniform_soup(20_000, seed=501)),
    ("nonhomog_30k", lambda: scenes.nonhomogeneous_soup(30_000, seed=502, extent=30.0)),
    ("arch_60k", lambda: scenes.architectural(60_000, seed=503, size=(40.0, 10.0, 40.0), nblobs=40)),
    ("nonhomog_dense_5k", lambda: scenes.nonhomogeneous_soup(5_000, seed=504, extent=8.0, large_frac=0.05)),
]


@pytest.mark.parametrize("name,make", SCENES, ids=[n for n, _ in SCENES])
def test_cull_pairs_match_oracle(ctx, name, make):
    import paper_2403_10647_gb300 as pg
    s = make()
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    lo, hi = ctx.bounds(v, t)
    info = pg.plan(lo, hi, s.n, s.lam)
    recs, nrefs = ctx.count_scan(v, t, info)
    info.nrefs = nrefs
    C, O = ctx.cull_pairs(v, t, info, recs, nrefs)
    p = oracle.plan(*oracle.bounds(s.verts, s.tris), s.n, s.lam)
    clo, chi, V = oracle.cell_boxes(s.verts, s.tris, p)
    off, NO = oracle.exclusive_sum(V)
    oC, oO, kept = oracle.cull_pairs(s.verts, s.tris, p, clo, chi, NO)
    assert nrefs == NO and C.numel() == oC.shape[0], (C.numel(), oC.shape[0], NO)
    bad = np.flatnonzero((host(C) != oC) | (host(O) != oO))
    assert bad.size == 0, (name, bad[:8], host(C)[bad[:8]], oC[bad[:8]], host(O)[bad[:8]], oO[bad[:8]])
    assert oC.shape[0] < NO   # these scenes all have some false intersections


def test_cull_hand_cases(ctx):
    """The hand-worked cases on a grid with lo = 0 and unit cells, so the
    grid-space vertices are the world ones."""
    import _pins
    import paper_2403_10647_gb300 as pg
    for case in _pins.read_cull_cases():
        q = np.array(case["q"], np.float32).reshape(3, 3)
        b = [int(v) for v in case["box"]]
        info = pg.Info(lo=(0.0, 0.0, 0.0), hi=(6.0, 6.0, 6.0), scale=(1.0, 1.0, 1.0), res=(6, 6, 6), key_bits=8,
                       ncells=216, nrefs=0, n=1)
        v, t = dev(q, torch.float32), dev(np.array([[0, 1, 2]]), torch.int32)
        recs, nrefs = ctx.count_scan(v, t, info)
        assert nrefs == (b[3] - b[0] + 1) * (b[4] - b[1] + 1) * (b[5] - b[2] + 1), case["name"]
        info.nrefs = nrefs
        C, O = ctx.cull_pairs(v, t, info, recs, nrefs)
        C = host(C)
        got = [(int(c % 6), int(c // 6 % 6), int(c // 36)) for c in C]
        want = [tuple(int(x) for x in case["kept"][i:i + 3]) for i in range(0, len(case["kept"]), 3)]
        assert got == want, (case["name"], got, want)


def test_cull_far_face(ctx):
    """A triangle in the grid's far face plane, whose FP32 grid coordinate
    lands 0.0039 cells beyond the last cell: it keeps its cells in the last
    layer, as in the oracle (pin_cull_far_face)."""
    import paper_2403_10647_gb300 as pg
    sc = float(np.float32(61846) / np.float32(804.099365234375))
    info = pg.Info(lo=(0.0, 0.0, 0.0), hi=(804.099365234375, 4.0, 4.0), scale=(sc, 1.0, 1.0), res=(61846, 4, 4),
                   key_bits=20, ncells=61846 * 16, nrefs=0, n=1)
    x = 804.099365234375
    verts = np.array([[x, 0.5, 0.5], [x, 3.5, 0.5], [x, 0.5, 3.5]], np.float32)
    v, t = dev(verts, torch.float32), dev(np.array([[0, 1, 2]]), torch.int32)
    recs, nrefs = ctx.count_scan(v, t, info)
    assert nrefs == 16
    info.nrefs = nrefs
    C, O = ctx.cull_pairs(v, t, info, recs, nrefs)
    C = host(C).astype(np.int64)
    yz = sorted(((int(c) // 61846) % 4, int(c) // (61846 * 4)) for c in C)
    assert (C % 61846 == 61845).all() and yz == sorted((y, z) for z in range(4) for y in range(4) if y + z <= 4)


@pytest.mark.parametrize("name,make", SCENES, ids=[n for n, _ in SCENES])
def test_culled_build_matches_oracle(cull_ctx, name, make):
    s = make()
    g = cull_ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
    o = oracle.build_grid(s.verts, s.tris, s.lam, cull=True)
    assert g.info.nrefs == o.NO and tuple(g.info.res) == tuple(o.plan.res)
    assert np.array_equal(host(g.cells), o.G), name
    assert np.array_equal(host(g.refs), o.refs), name


@pytest.mark.parametrize("case", ["empty", "one", "flat_z", "all_same_cell"])
def test_culled_build_degenerate(cull_ctx, case):
    g = np.random.Generator(np.random.Philox(505))
    if case == "empty":
        v, t = np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32)
    elif case == "one":
        v, t = np.array([[0, 0, 0], [5, 0.5, 0.2], [0.3, 4, 3]], np.float32), np.array([[0, 1, 2]], np.int32)
    elif case == "flat_z":   # every triangle in z = 1: res_z = 1, scale_z = 0
        v = np.concatenate([g.random((300, 2)) * 10.0, np.ones((300, 1))], axis=1).astype(np.float32)
        t = g.integers(0, 300, (100, 3)).astype(np.int32)
    else:                    # a single cell: nothing to sort
        v = (g.random((30, 3)) * 1e-3).astype(np.float32)
        t = g.integers(0, 30, (10, 3)).astype(np.int32)
    res = cull_ctx.build(dev(v, torch.float32), dev(t, torch.int32), 0.1 if case == "all_same_cell" else 4.0)
    o = oracle.build_grid(v, t, 0.1 if case == "all_same_cell" else 4.0, cull=True)
    assert res.info.nrefs == o.NO
    assert np.array_equal(host(res.cells), o.G) and np.array_equal(host(res.refs), o.refs), case


def test_cull_rejects_bad_index(ctx):
    import paper_2403_10647_gb300 as pg
    s = scenes.uniform_soup(2000, seed=506)
    v, t = dev(s.verts, torch.float32), dev(s.tris, torch.int32)
    lo, hi = ctx.bounds(v, t)
    info = pg.plan(lo, hi, s.n, s.lam)
    recs, nrefs = ctx.count_scan(v, t, info)
    info.nrefs = nrefs
    # a triangle whose box has more than two cells: its vertices are read
    i = int(np.flatnonzero(np.diff(np.append(host(recs)[:, 3], nrefs)) > 2)[0])
    bad = t.clone()
    bad[i, 1] = 10**6
    with pytest.raises(pg.GridError):
        ctx.cull_pairs(v, bad, info, recs, nrefs)
    C, O = ctx.cull_pairs(v, t, info, recs, nrefs)   # the context is still usable
    assert C.numel() > 0


@pytest.mark.slow
@pytest.mark.parametrize("name", ["nonhomogeneous_1e6", "architectural_1e7"])
def test_culled_full_size(cull_ctx, name):
    s = scenes.CONFIGS[name]()
    g = cull_ctx.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting", cull=True)
    assert g.info.nrefs == o.NO, (g.info.nrefs, o.NO)
    assert np.array_equal(host(g.cells), o.G), name
    assert np.array_equal(host(g.refs), o.refs), name
