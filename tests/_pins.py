"""Checks that pin the CPU oracle to facts outside itself.

Each ``pin_*`` function raises AssertionError on a mismatch.  They are
collected twice: by test_oracle_pins.py against the real oracle, and by
test_oracle_mutants.py against copies of oracle.c with planted mistakes, to
show that a plausible mistake anywhere in the oracle fails at least one pin.

What pins what:
  * the hand-worked Algorithm 1 example (tests/golden/hand_example.txt):
    every intermediate array of Sec. 3 / Fig. 4, derived by hand;
  * Fig. 1's 1-cell and 12-cell triangles, a 2-cell straddle and the
    boundary/clamp cases, worked by hand on a 4 x 4 x 4 grid with unit cells,
    and again on a shifted grid with half-unit cells;
  * every vertex lies inside its cell's world extent (exact arithmetic, away
    from cell boundaries);
  * closed forms of the resolution rule (tests/golden/plan_cases.txt);
  * brute force on tiny scenes: the list of every cell is every object whose
    grid box contains it, tested cell by cell (no scans, no sort);
  * library routines for the special cases they reduce to: numpy min/max
    (scene bounds), cumsum (ExclusiveSum), stable argsort (RadixSort),
    searchsorted (G = number of sorted keys below each cell);
  * invariants: NO = sum V, segment lengths, every box cell emitted once,
    G monotone with G[0] = 0 and G[ncells] = NO, ascending ids inside a cell.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def read_plan_cases() -> list:
    rows = []
    with open(os.path.join(GOLDEN, "plan_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def hand_plan(lo=(0, 0, 0), scale=(1, 1, 1), res=(4, 4, 4)) -> oracle.Plan:
    res = np.asarray(res, np.int32)
    return oracle.Plan(np.asarray(lo, np.float32), np.asarray(lo, np.float32) + res.astype(np.float32),
                       res, np.asarray(scale, np.float32), int(np.prod(res.astype(np.int64))))


def pin_hand_example():
    g = read_golden("hand_example.txt")
    verts = np.array(g["verts"], np.float32).reshape(-1, 3)
    tris = np.array(g["tris"], np.int32).reshape(-1, 3)
    p = hand_plan(tuple(map(float, g["lo"])), tuple(map(float, g["scale"])), tuple(map(int, g["res"])))
    ints = lambda k: np.array(g[k], np.int64)  # noqa: E731
    clo, chi, V = oracle.cell_boxes(verts, tris, p)
    assert (clo.ravel() == ints("clo")).all(), ("clo", clo)
    assert (chi.ravel() == ints("chi")).all(), ("chi", chi)
    assert (V == ints("V")).all(), ("V", V)
    off, NO = oracle.exclusive_sum(V)
    assert (off == ints("offsets")).all() and NO == int(g["NO"][0]), ("offsets", off, NO)
    C, O = oracle.object_order_pairs(clo, chi, off, NO, p.res)
    assert (O == ints("O_object_order")).all(), ("O", O)
    assert (C == ints("C_object_order")).all(), ("C", C)
    Cs, Os = oracle.sort_pairs(C, O)
    assert (Cs == ints("C_sorted")).all() and (Os == ints("O_sorted")).all(), ("sorted", Cs, Os)
    G = oracle.ranges(Cs, p.ncells)
    assert (G == ints("G")).all(), ("G", G)
    Gc, refs = oracle.grid_counting(clo, chi, p, NO)
    assert (Gc == ints("G")).all() and (refs == ints("O_sorted")).all(), ("counting", Gc, refs)


def _tri(a, b, c):
    return np.array([a, b, c], np.float32)


def pin_fig1_cells():
    """Fig. 1: one triangle in 1 cell, one spanning 3 x 2 x 2 = 12 cells;
    plus a 2-cell straddle and the boundary / far-face clamp."""
    p = hand_plan()
    cases = [
        # (triangle, expected clo, expected chi, expected V)
        (_tri((0.2, 0.2, 0.2), (0.5, 0.3, 0.2), (0.3, 0.6, 0.7)), (0, 0, 0), (0, 0, 0), 1),
        (_tri((0.5, 0.2, 0.2), (1.5, 0.3, 0.2), (0.7, 0.6, 0.7)), (0, 0, 0), (1, 0, 0), 2),
        (_tri((0.5, 1.2, 2.1), (2.5, 2.5, 2.2), (1.0, 1.5, 3.9)), (0, 1, 2), (2, 2, 3), 12),
        # hi exactly on the plane x = 1 belongs to the next cell
        (_tri((0.5, 0.5, 0.5), (1.0, 0.5, 0.5), (0.7, 0.6, 0.6)), (0, 0, 0), (1, 0, 0), 2),
        # the far face x = 4 clamps into the last cell
        (_tri((3.5, 3.5, 3.5), (4.0, 4.0, 4.0), (3.7, 3.6, 3.6)), (3, 3, 3), (3, 3, 3), 1),
        # a triangle spanning the whole grid
        (_tri((0.0, 0.0, 0.0), (4.0, 0.0, 4.0), (0.0, 4.0, 2.0)), (0, 0, 0), (3, 3, 3), 64),
    ]
    verts = np.concatenate([c[0] for c in cases]).reshape(-1, 3)
    tris = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    clo, chi, V = oracle.cell_boxes(verts, tris, p)
    for i, (_, elo, ehi, ev) in enumerate(cases):
        assert tuple(clo[i]) == elo and tuple(chi[i]) == ehi and V[i] == ev, (i, clo[i], chi[i], V[i])
    # the 12-cell triangle alone: its cells in GlobalCoords order (x fastest)
    off, NO = oracle.exclusive_sum(V[2:3])
    C, O = oracle.object_order_pairs(clo[2:3], chi[2:3], off, NO, p.res)
    want = [x + 4 * (y + 4 * z) for z in (2, 3) for y in (1, 2) for x in (0, 1, 2)]
    assert list(C) == want, (list(C), want)
    assert (O == 0).all()


def pin_shifted_cells():
    """The hand cases again on a grid whose origin is not 0 and whose cells
    are half a unit wide (scale 2): cell = floor(2 * (p - lo))."""
    lo = (-2.0, 6.0, 96.0)
    p = hand_plan(lo=lo, scale=(2, 2, 2), res=(8, 8, 8))
    sh = np.array(lo, np.float32)
    cases = [
        (_tri((0.1, 0.1, 0.1), (0.25, 0.15, 0.1), (0.15, 0.3, 0.35)), (0, 0, 0), (0, 0, 0), 1),
        (_tri((0.25, 0.1, 0.1), (0.75, 0.15, 0.1), (0.35, 0.3, 0.35)), (0, 0, 0), (1, 0, 0), 2),
        (_tri((0.25, 0.6, 1.05), (1.25, 1.25, 1.1), (0.5, 0.75, 1.95)), (0, 1, 2), (2, 2, 3), 12),
        (_tri((3.75, 3.75, 3.75), (4.0, 4.0, 4.0), (3.85, 3.8, 3.8)), (7, 7, 7), (7, 7, 7), 1),
    ]
    verts = (np.concatenate([c[0] for c in cases]).reshape(-1, 3) + sh).astype(np.float32)
    tris = np.arange(verts.shape[0], dtype=np.int32).reshape(-1, 3)
    clo, chi, V = oracle.cell_boxes(verts, tris, p)
    for i, (_, elo, ehi, ev) in enumerate(cases):
        assert tuple(clo[i]) == elo and tuple(chi[i]) == ehi and V[i] == ev, (i, clo[i], chi[i], V[i])


def pin_point_in_cell(seed: int = 14):
    """Every vertex lies inside the world extent of its cell, checked in exact
    (float64) arithmetic for points not within rounding distance of a cell
    boundary: lo + c / scale <= p < lo + (c + 1) / scale."""
    g = np.random.Generator(np.random.Philox(seed))
    for k in range(50):
        n = int(g.integers(5, 200))
        s = scenes.tiny_scene(g, n, box=float(g.uniform(0.1, 100.0)))
        s.verts += np.float32(g.uniform(-50, 50))
        lo, hi = oracle.bounds(s.verts, s.tris)
        p = oracle.plan(lo, hi, n, s.lam)
        pts = np.repeat(np.arange(s.verts.shape[0], dtype=np.int32)[:, None], 3, axis=1)
        used = np.unique(s.tris)
        c, _, _ = oracle.cell_boxes(s.verts, pts[used], p)
        x = s.verts[used].astype(np.float64)
        u = (x - lo.astype(np.float64)) * p.scale.astype(np.float64)   # exact-ish position in cells
        far = np.abs(u - np.round(u)) > 1e-3                             # away from any boundary
        inside = (u >= c) & (u < c + 1)
        at_far_face = (c == p.res - 1) & (u < p.res + 1e-3)
        assert (inside | at_far_face | ~far).all(), k
        assert far.mean() > 0.9, k


def pin_plan_cases():
    for row in read_plan_cases():
        lo, hi, n, lam = row[0:3], row[3:6], int(row[6]), row[7]
        res, scale, ncells = row[8:11], row[11:14], int(row[14])
        p = oracle.plan(np.array(lo, np.float32), np.array(hi, np.float32), n, lam)
        assert tuple(p.res) == tuple(int(r) for r in res), (row, p.res)
        assert np.array_equal(p.scale, np.array(scale, np.float32)), (row, p.scale)
        assert p.ncells == ncells, (row, p.ncells)


def pin_plan_errors():
    lo, hi = np.zeros(3, np.float32), np.ones(3, np.float32)
    for lam in (0.0, -1.0, float("nan"), float("inf")):
        try:
            oracle.plan(lo, hi, 10, lam)
        except oracle.OracleError as e:
            assert e.code == oracle.EINVAL
        else:
            raise AssertionError(f"lambda {lam} accepted")
    try:  # 65535^3 cells clamp per axis but overflow int32 in total
        oracle.plan(lo, hi, 2 ** 31 - 2, 3.0e38)
    except oracle.OracleError as e:
        assert e.code == oracle.EOVERFLOW
    else:
        raise AssertionError("ncells overflow not reported")
    p = oracle.plan(lo, hi, 0, 1.0)
    assert tuple(p.res) == (1, 1, 1) and p.ncells == 1


def pin_bounds():
    g = np.random.Generator(np.random.Philox(7))
    s = scenes.tiny_scene(g, 50, nverts=200)
    lo, hi = oracle.bounds(s.verts, s.tris)
    used = s.verts[np.unique(s.tris)]
    assert np.array_equal(lo, used.min(axis=0)) and np.array_equal(hi, used.max(axis=0))
    bad = s.tris.copy()
    bad[3, 1] = 200
    for t in (bad, np.where(bad == 200, -1, bad).astype(np.int32)):
        try:
            oracle.bounds(s.verts, t)
        except oracle.OracleError as e:
            assert e.code == oracle.EINVAL
        else:
            raise AssertionError("bad index accepted")
    v = s.verts.copy()
    v[s.tris[5, 2], 1] = np.nan
    try:
        oracle.bounds(v, s.tris)
    except oracle.OracleError as e:
        assert e.code == oracle.EINVAL
    else:
        raise AssertionError("NaN accepted")


def pin_bruteforce(nscenes: int = 300, seed: int = 11):
    """Alg. 1 chain == counting placement == brute force on tiny scenes."""
    g = np.random.Generator(np.random.Philox(seed))
    for k in range(nscenes):
        n = int(g.integers(1, 48))
        s = scenes.tiny_scene(g, n, box=float(g.uniform(0.5, 3.0)), max_edge=float(g.uniform(0.05, 1.5)))
        lo, hi = oracle.bounds(s.verts, s.tris)
        p = oracle.plan(lo, hi, n, s.lam)
        if p.ncells > 4096:
            continue
        clo, chi, V = oracle.cell_boxes(s.verts, s.tris, p)
        Gb, rb = oracle.grid_bruteforce(clo, chi, p)
        a = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1")
        assert a.NO == rb.shape[0] == int(V.sum()), (k, a.NO, rb.shape)
        assert np.array_equal(a.G, Gb) and np.array_equal(a.refs, rb), k
        c = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
        assert np.array_equal(c.G, Gb) and np.array_equal(c.refs, rb), k


def pin_brute_boxes(nscenes: int = 200, seed: int = 12):
    """Each object's grid box is the smallest cell box holding its vertices:
    every vertex's own cell (computed per point through the same oracle) lies
    inside [clo, chi], and clo / chi are attained by some vertex."""
    g = np.random.Generator(np.random.Philox(seed))
    for k in range(nscenes):
        n = int(g.integers(1, 30))
        s = scenes.tiny_scene(g, n)
        lo, hi = oracle.bounds(s.verts, s.tris)
        p = oracle.plan(lo, hi, n, s.lam)
        clo, chi, V = oracle.cell_boxes(s.verts, s.tris, p)
        # degenerate triangles (all three corners at one vertex) give each vertex's own cell
        pts = np.repeat(np.arange(s.verts.shape[0], dtype=np.int32)[:, None], 3, axis=1)
        vlo, vhi, vV = oracle.cell_boxes(s.verts, pts, p)
        assert np.array_equal(vlo, vhi) and (vV == 1).all(), k
        cells = vlo[s.tris]                      # [n, 3 corners, 3 axes]
        assert np.array_equal(cells.min(axis=1), clo) and np.array_equal(cells.max(axis=1), chi), k
        assert (V == np.prod(chi.astype(np.int64) - clo + 1, axis=1)).all(), k


def pin_library_routines(seed: int = 13):
    g = np.random.Generator(np.random.Philox(seed))
    V = g.integers(1, 1000, 5000).astype(np.int64)
    off, tot = oracle.exclusive_sum(V)
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(V)[:-1]])) and tot == int(V.sum())
    try:
        oracle.exclusive_sum(np.array([2 ** 30, 2 ** 30, 1], np.int64))
    except oracle.OracleError as e:
        assert e.code == oracle.EOVERFLOW
    else:
        raise AssertionError("NO overflow not reported")
    for nkeys, keyspace in ((1, 1), (777, 3), (20000, 50), (20000, 1 << 20)):
        C = g.integers(0, keyspace, nkeys).astype(np.int32)
        O = np.arange(nkeys, dtype=np.int32)
        Cs, Os = oracle.sort_pairs(C, O)
        perm = np.argsort(C, kind="stable")
        assert np.array_equal(Cs, C[perm]) and np.array_equal(Os, O[perm])
        G = oracle.ranges(Cs, keyspace)
        assert np.array_equal(G, np.searchsorted(Cs, np.arange(keyspace + 1), side="left").astype(np.int32))


def pin_invariants():
    for s in (scenes.uniform_soup(8000, seed=5), scenes.nonhomogeneous_soup(4000, seed=6, extent=20.0)):
        a = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1")
        n = s.n
        assert a.NO == int(a.V.sum())
        assert a.G[0] == 0 and a.G[-1] == a.NO and (np.diff(a.G) >= 0).all()
        C, O = oracle.object_order_pairs(a.clo, a.chi, a.offsets, a.NO, a.plan.res)
        assert np.array_equal(np.bincount(O, minlength=n), a.V)           # segment lengths
        assert (np.diff(O) >= 0).all()                                     # object order
        # each object's emitted cells are exactly its box cells, once each
        res = a.plan.res.astype(np.int64)
        x, y, z = C % res[0], (C // res[0]) % res[1], C // (res[0] * res[1])
        for ax, coord in enumerate((x, y, z)):
            assert (coord >= a.clo[O, ax]).all() and (coord <= a.chi[O, ax]).all()
        assert np.unique(O.astype(np.int64) * a.plan.ncells + C).shape[0] == a.NO
        # sorted pairs: lexicographic (cell, object), so ascending ids inside a cell
        perm = np.lexsort((O, C))
        assert np.array_equal(a.refs, O[perm])
        cells_of_ref = np.repeat(np.arange(a.plan.ncells), np.diff(a.G))
        assert np.array_equal(cells_of_ref, C[perm])


ALL_PINS = [pin_hand_example, pin_fig1_cells, pin_shifted_cells, pin_point_in_cell, pin_plan_cases, pin_plan_errors, pin_bounds,
            pin_bruteforce, pin_brute_boxes, pin_library_routines, pin_invariants]


def run_all():
    """Runs every pin; returns the names of those that failed."""
    failed = []
    for fn in ALL_PINS:
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - a mutant may fail any way
            failed.append(f"{fn.__name__}: {type(e).__name__}")
    return failed
