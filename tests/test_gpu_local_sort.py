"""The hybrid end of RadixSort and the range steps (grid_opts.local_bits):
radix passes over the high key bits, then one counting sort per group of
buckets of 2^L cells in shared memory that writes the group's cells and
refs.  Every setting of L, and the all-radix chain (-1), must give the
oracle's grid bit for bit: small and large buckets, short and long cell
runs, groups too large for one block (placed in chunks of whole cells),
cells too crowded for a block (the build then falls back to radix passes
over every key bit and range extraction), a single cell, batched and culled
builds, and the automatic choice between the hybrid and the chain."""
import numpy as np
import pytest

import oracle
import scenes

from test_gpu_parity import assert_grid_equal, dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _build(s, **kw):
    return _build_stats(s, **kw)[0]


def _build_stats(s, **kw):
    """The grid and the kernel families its build launched (plus "plan": the
    context's (local bits, radix passes) for this build)."""
    import paper_2403_10647_gb300 as pg
    c = pg.Context(0, **kw)
    try:
        c.profile(True)
        g = c.build(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam)
        st = c.kernel_stats()
        st["plan"] = c.sort_plan(g.info.key_bits, g.info.nrefs, g.info.ncells)
        return g, st
    finally:
        c.close()


SCENES = {
    "uniform_30k": lambda: scenes.uniform_soup(30_000, seed=401),
    "nonhomog_60k": lambda: scenes.nonhomogeneous_soup(60_000, seed=402, extent=39.0),
    "arch_80k": lambda: scenes.architectural(80_000, seed=403, size=(43.0, 11.0, 43.0), nblobs=50),
}


@pytest.fixture(scope="module")
def oracle_grids():
    out = {}
    for name, make in SCENES.items():
        s = make()
        out[name] = (s, oracle.build_grid(s.verts, s.tris, s.lam, method="counting"))
    return out


@pytest.mark.parametrize("local_bits", [-2, -1, 0, 1, 3, 6, 9, 11])
@pytest.mark.parametrize("name", sorted(SCENES))
def test_local_bits_settings_match_oracle(oracle_grids, name, local_bits):
    s, o = oracle_grids[name]
    g, st = _build_stats(s, local_bits=local_bits)
    assert_grid_equal(g, o, f"{name} local_bits {local_bits}")
    lb, passes = st["plan"]
    if local_bits == -1:
        assert lb == -1 and "local_sort" not in st and "extract" in st
    if local_bits == 0:   # the hybrid at up to 6 pairs per cell, the chain beyond
        assert (lb >= 0) == (o.NO <= 6 * o.plan.ncells), (lb, o.NO / o.plan.ncells)
    if local_bits in (0, -2) and lb >= 0:   # the automatic buckets fit every group in a block: no fallback
        assert "local_sort" in st and "extract" not in st, st.keys()


@pytest.mark.parametrize("radix_bits", [8, 9, 11])
def test_local_sort_with_radix_widths(oracle_grids, radix_bits):
    s, o = oracle_grids["nonhomog_60k"]
    assert_grid_equal(_build(s, radix_bits=radix_bits), o, f"radix {radix_bits}")
    assert_grid_equal(_build(s, radix_bits=radix_bits, tile_shape="384x8"), o, f"radix {radix_bits} 384x8")


def test_buckets_beyond_block_capacity():
    """Buckets of 2^11 cells on a scene with about 40 pairs per cell: most
    buckets hold several times what one block places at once, and each goes
    through the chunked path (a count over the bucket, then chunks of whole
    cells, each gathered in one more pass over the bucket)."""
    s = scenes.nonhomogeneous_soup(300_000, seed=404, extent=40.0)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    per_bucket = o.NO / max(1, (o.plan.ncells + 2047) // 2048)
    assert per_bucket > 3 * 12288, per_bucket
    g, st = _build_stats(s, local_bits=11)
    assert_grid_equal(g, o, "buckets beyond capacity")
    assert "local_sort" in st and "extract" not in st, st.keys()


def _crowded_cell_scene(n_crowd, n_rest, seed, lam=2.0):
    """n_crowd tiny triangles inside one cell-sized region, plus n_rest
    triangles spread over the box: one cell holds a long run of objects."""
    g = np.random.Generator(np.random.Philox(seed))
    rest = g.random((n_rest, 3)) * 10.0
    rest_v = np.concatenate([rest, rest + 0.05, rest + [0.05, 0.0, 0.05]]).astype(np.float32)
    centre, half = np.full(3, 5.0), 0.01
    if n_rest:   # the middle of the cell holding (5, 5, 5), well inside it
        lo, hi = rest_v.min(0), rest_v.max(0)
        p = oracle.plan(lo, hi, n_rest + n_crowd, lam)
        cell = np.floor((centre - lo) * p.scale)
        centre = lo + (cell + 0.5) / p.scale
        half = 0.2 / p.scale.max()
    c = centre + (g.random((n_crowd, 3)) - 0.5) * half
    crowd_v = np.concatenate([c, c + 0.05 * half, c + [0.05 * half, 0.0, 0.05 * half]])
    v = np.concatenate([rest_v, crowd_v]).astype(np.float32)
    nr, nc = n_rest, n_crowd
    tris = np.concatenate([np.stack([np.arange(nr), nr + np.arange(nr), 2 * nr + np.arange(nr)], 1),
                           3 * nr + np.stack([np.arange(nc), nc + np.arange(nc), 2 * nc + np.arange(nc)], 1)])
    perm = g.permutation(tris.shape[0])   # the crowd's objects interleave with the others
    return scenes.Scene("crowded", v, tris[perm].astype(np.int32), lam)


@pytest.mark.parametrize("local_bits", [-2, 4, 11])
def test_crowded_cell_falls_back(local_bits):
    """A cell holding 30,000 objects: beyond what a block sorts in one cell,
    so the build falls back; the grid is still the oracle's."""
    s = _crowded_cell_scene(30_000, 50_000, seed=405)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    assert np.diff(o.G).max() >= 30_000
    g, st = _build_stats(s, local_bits=local_bits)
    assert_grid_equal(g, o, f"crowded cell, local_bits {local_bits}")
    assert "extract" in st


@pytest.mark.parametrize("crowd", [17, 25, 32, 33, 100, 300, 500])
def test_cell_runs_sorted_by_a_warp(crowd):
    """A cell of 17 to 500 objects among ordinary ones: each pair goes to its
    rank by object id inside the long run, with no fallback."""
    s = _crowded_cell_scene(crowd, 60_000, seed=407 + crowd)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    assert np.diff(o.G).max() >= crowd
    g, st = _build_stats(s, local_bits=-2)
    assert_grid_equal(g, o, f"cell of {crowd}")
    assert "local_sort" in st and "extract" not in st, st.keys()


def test_single_cell_beyond_capacity():
    """lambda so small that the grid is one cell: every pair lands in it,
    more pairs than a block places at once."""
    s = _crowded_cell_scene(20_000, 0, seed=406, lam=1e-6)
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    assert o.plan.ncells == 1 and o.NO == 20_000
    assert_grid_equal(_build(s, local_bits=-2), o, "single cell")
    small = _crowded_cell_scene(300, 0, seed=408, lam=1e-6)   # one cell, one group, no fallback
    o = oracle.build_grid(small.verts, small.tris, small.lam, method="counting")
    g, st = _build_stats(small, local_bits=-2)
    assert_grid_equal(g, o, "single cell of 300")
    assert "extract" not in st


@pytest.mark.parametrize("local_bits", [-2, -1, 0, 11])
def test_batched_local_bits(local_bits):
    import paper_2403_10647_gb300 as pg
    from test_gpu_parity import _mixed_batch
    batch = _mixed_batch()
    c = pg.Context(0, local_bits=local_bits)
    try:
        grids = c.build_batched([(dev(s.verts, torch.float32), dev(s.tris, torch.int32), s.lam) for s in batch])
        for s, g in zip(batch, grids):
            o = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1" if s.n < 50_000 else "counting")
            assert_grid_equal(g, o, f"batched {s.name} local_bits {local_bits}")
    finally:
        c.close()


@pytest.mark.parametrize("local_bits", [-2, -1, 0, 11])
def test_culled_local_bits(oracle_grids, local_bits):
    s, _ = oracle_grids["nonhomog_60k"]
    o = oracle.build_grid(s.verts, s.tris, s.lam, cull=True)
    assert_grid_equal(_build(s, cull=True, local_bits=local_bits), o, f"culled local_bits {local_bits}")


def test_bad_local_bits_rejected():
    import paper_2403_10647_gb300 as pg
    for lb in (-3, 12):
        with pytest.raises(pg.GridError):
            pg.Context(0, local_bits=lb)
