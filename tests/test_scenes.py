"""The seeded synthetic workloads: each recipe has the character it claims
(triangle counts, the share of large triangles, the indexed wall quads), and
each workload keeps the grid and pair count that its measurements are quoted
on.  The sizes come from the oracle's plan and CountCells on the generated
scene, so a change to a generator (or to numpy's Philox stream) shows here
before it silently changes a benchmark's workload."""
import numpy as np

import oracle
import scenes


def _grid(s):
    lo, hi = oracle.bounds(s.verts, s.tris)
    p = oracle.plan(lo, hi, s.n, s.lam)
    _, _, V = oracle.cell_boxes(s.verts, s.tris, p)
    return p, V


def _edges(s):
    q = s.verts[s.tris].astype(np.float64)            # [n, 3 vertices, 3]
    return np.stack([np.linalg.norm(q[:, 1] - q[:, 0], axis=1),
                     np.linalg.norm(q[:, 2] - q[:, 1], axis=1),
                     np.linalg.norm(q[:, 0] - q[:, 2], axis=1)], axis=1)


def test_uniform_1e5():
    s = scenes.uniform_soup()
    assert s.n == 100_000 and s.lam == 2.0
    assert s.verts.min() > -0.02 and s.verts.max() < 1.02
    p, V = _grid(s)
    assert tuple(p.res) == (59, 59, 59)
    assert int(V.sum()) == 326_864


def test_nonhomogeneous_1e6():
    s = scenes.nonhomogeneous_soup()
    assert s.n == 1_000_000 and s.lam == 4.0
    # 1% large triangles: their two drawn edges (from vertex 0) are 5 to 40
    # long (up to FP32 rounding); the small ones' LogNormal(ln 0.05, 0.5)
    # edges stay far below 5
    large = _edges(s)[:, [0, 2]].min(axis=1) >= 4.999
    assert int(large.sum()) == 10_000
    p, V = _grid(s)
    assert tuple(p.res) == (157, 158, 163)
    assert int(V.sum()) == 83_011_203
    assert int(V.max()) == 94_752
    # the large triangles hold most of the pairs: the disparity in cells
    # per object that Sec. 5 measures its scenes by
    assert V[large].sum() > 0.5 * V.sum()


def test_architectural_1e7():
    n = 10_000_000
    s = scenes.architectural(n)
    assert s.n == n and s.lam == 8.0
    nquad = int(round(0.05 * n / 2))
    # the wall quads form an indexed mesh: triangle pairs share two vertices
    t = s.tris[:2 * nquad].reshape(nquad, 2, 3)
    assert np.array_equal(t[:, 0, 0], t[:, 1, 0]) and np.array_equal(t[:, 0, 2], t[:, 1, 1])
    assert s.verts.shape[0] == 4 * nquad + 3 * (n - 2 * nquad)
    p, V = _grid(s)
    assert tuple(p.res) == (683, 172, 683)
    assert int(V.sum()) == 200_255_352


def test_profiling_proxy_keeps_the_density():
    """The 2.5M-triangle proxy of the profiles has the 10M scene's pairs per
    triangle within 1%."""
    s = scenes.architectural_scaled(2_500_000)
    p, V = _grid(s)
    assert int(V.sum()) == 49_850_764 and p.ncells == 20_154_100
    assert abs(V.sum() / s.n - 200_255_352 / 1e7) < 0.01 * 20.0


def test_same_seed_same_scene():
    a, b = scenes.nonhomogeneous_soup(5000, seed=3), scenes.nonhomogeneous_soup(5000, seed=3)
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
    c = scenes.nonhomogeneous_soup(5000, seed=4)
    assert not np.array_equal(a.verts, c.verts)
