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
    G monotone with G[0] = 0 and G[ncells] = NO, ascending ids inside a cell;
  * the culling mode: hand-worked cases (tests/golden/cull_example.txt), an
    exact-rational separating-axis test cross-checked against exact polygon
    clipping (the oracle never drops a touching cell and drops every clearly
    separated one), and invariants on scenes (kept pairs are a subsequence of
    the box pairs; vertex and interior-point cells are kept).
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
        # a point below the grid's origin clamps into the first cell (a
        # scene's own bounds never produce one; the clamp still fixes it)
        (_tri((-0.5, 0.5, 0.5), (0.5, -2.0, 0.5), (0.2, 0.6, -0.1)), (0, 0, 0), (0, 0, 0), 1),
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


def pin_bounds_signed_zero():
    """Zero bounds are reported as +0.0, whatever sign of zero the vertices
    carry and in whichever order they come: the minimum over {-0.0, +0.0} is
    a zero, and the reported zero has no sign bit.  Non-zero bounds keep
    their exact values."""
    z, nz = np.float32(0.0), np.float32(-0.0)
    for first, second in ((nz, z), (z, nz), (nz, nz)):
        verts = np.array([[first, first, 1.0], [second, 2.0, second], [3.0, second, first],
                          [1.0, 1.0, 1.0], [2.0, 3.0, 4.0], [1.5, 2.5, 0.5]], np.float32)
        tris = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
        lo, hi = oracle.bounds(verts, tris)
        assert np.array_equal(lo.view(np.uint32), np.zeros(3, np.uint32)), lo.view(np.uint32)
        assert np.array_equal(hi, np.array([3.0, 3.0, 4.0], np.float32))
    # all-negative-zero axis: both bounds are +0.0
    verts = np.array([[nz, 1.0, 1.0], [nz, 2.0, 3.0], [nz, 4.0, 2.0]], np.float32)
    lo, hi = oracle.bounds(verts, np.array([[0, 1, 2]], np.int32))
    assert lo.view(np.uint32)[0] == 0 and hi.view(np.uint32)[0] == 0


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


# ---- false-intersection culling ---------------------------------------------------

def read_cull_cases() -> list:
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "cull_example.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "case":
                cur = {"name": vals[0]}
                cases.append(cur)
            else:
                cur[key] = [float(v) for v in vals]
    return cases


def pin_cull_hand():
    """The hand-worked cases of tests/golden/cull_example.txt: each axis
    family (the normal, u_x x e, u_y x e, u_z x e) separates exactly the
    cells worked out by hand, and touching cells are kept."""
    for case in read_cull_cases():
        q = np.array(case["q"], np.float32).reshape(3, 3)
        b = [int(v) for v in case["box"]]
        kept = [(x, y, z) for z in range(b[2], b[5] + 1) for y in range(b[1], b[4] + 1)
                for x in range(b[0], b[3] + 1) if not oracle.tri_cell_separated(q, x, y, z)]
        want = [tuple(int(v) for v in case["kept"][i:i + 3]) for i in range(0, len(case["kept"]), 3)]
        assert kept == want, (case["name"], kept, want)


def _exact_clip_overlap(tri, cell):
    """Exact (rational) test whether the closed triangle meets the closed
    unit cube at integer corner `cell`: Sutherland-Hodgman clipping of the
    triangle polygon by the cube's six half-spaces; non-empty means they
    touch."""
    from fractions import Fraction as F
    poly = [tuple(F(c) for c in v) for v in tri]
    for a in range(3):
        for lo_side in (True, False):
            bound = F(cell[a]) if lo_side else F(cell[a] + 1)

            def d(pt):
                return pt[a] - bound if lo_side else bound - pt[a]
            out = []
            for i in range(len(poly)):
                P, Q = poly[i - 1], poly[i]
                dp, dq = d(P), d(Q)
                if dq >= 0:
                    if dp < 0:
                        t = dp / (dp - dq)
                        out.append(tuple(P[k] + t * (Q[k] - P[k]) for k in range(3)))
                    out.append(Q)
                elif dp >= 0:
                    t = dp / (dp - dq)
                    out.append(tuple(P[k] + t * (Q[k] - P[k]) for k in range(3)))
            poly = out
            if not poly:
                return False
    return True


def _exact_sat_gap(tri, cell):
    """Exact separating-axis test over all 13 axes of a triangle and a box
    (the three face normals, the triangle normal, the nine edge cross
    products): the largest separation gap divided by the axis' L1 norm
    (<= 0: the two touch or overlap)."""
    from fractions import Fraction as F
    v = [tuple(F(c) for c in p) for p in tri]
    c = tuple(F(cell[a]) + F(1, 2) for a in range(3))
    w = [tuple(p[a] - c[a] for a in range(3)) for p in v]
    e = [tuple(v[(k + 1) % 3][a] - v[k][a] for a in range(3)) for k in range(3)]

    def cross(a, b):
        return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])
    units = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    axes = units + [cross(e[0], e[1])] + [cross(u, ek) for u in units for ek in e]
    best = None
    for ax in axes:
        S = sum(abs(x) for x in ax)
        if S == 0:
            continue
        p = [sum(ax[i] * wk[i] for i in range(3)) for wk in w]
        gap = max(min(p) - S / 2, -S / 2 - max(p)) / S
        best = gap if best is None else max(best, gap)
    return best


def pin_cull_exact(ntri: int = 150, seed: int = 15):
    """Random triangles with dyadic grid coordinates (multiples of 1/32 in
    [0, 6]) against every cell of their cell box, in exact rational
    arithmetic: (1) the 13-axis separating-axis test and polygon clipping
    agree on touch / no touch (pins the axis set); (2) the oracle never drops
    a touching cell (conservative); (3) it drops every cell separated by more
    than 2^-9 cell widths along an axis (tight, above the 2^-10 + W 2^-16
    slack)."""
    g = np.random.Generator(np.random.Philox(seed))
    checked = dropped = 0
    for _ in range(ntri):
        base = g.integers(0, 4 * 32, 3)
        spread = g.integers(1, 2 * 32, (3, 3)) * g.choice([-1, 1], (3, 3))
        tri = np.clip(base[None, :] + spread * (g.random((3, 1)) < 0.8), 0, 6 * 32) / 32.0
        if g.random() < 0.2:          # some flat in one axis, the grid planes included
            tri[:, g.integers(0, 3)] = g.integers(0, 6 * 4) / 4.0
        q = tri.astype(np.float32)
        lo = np.floor(q.min(axis=0)).astype(int)
        hi = np.floor(q.max(axis=0)).astype(int)
        for z in range(lo[2], hi[2] + 1):
            for y in range(lo[1], hi[1] + 1):
                for x in range(lo[0], hi[0] + 1):
                    touch = _exact_clip_overlap(q.tolist(), (x, y, z))
                    gap = _exact_sat_gap(q.tolist(), (x, y, z))
                    assert touch == (gap <= 0), (q.tolist(), (x, y, z), touch, gap)
                    sep = oracle.tri_cell_separated(q, x, y, z)
                    assert not (sep and touch), ("dropped a touching cell", q.tolist(), (x, y, z))
                    if gap > 2.0 ** -9:
                        assert sep, ("kept a separated cell", q.tolist(), (x, y, z), float(gap))
                    checked += 1
                    dropped += sep
    assert checked > 1000 and dropped > 100, (checked, dropped)


def pin_cull_far_face():
    """A triangle lying in the grid's far face plane keeps its cells.  With
    res_x = 61846 over an extent of 804.099365 the FP32 scale puts that plane
    at grid x = 61846.0039, 0.0039 cells beyond the last cell (more than the
    test's slack): the clamp of the grid coordinate to res, like the cell
    mapping's clamp, keeps the triangle in the last cell layer.  In the y-z
    plane it is the right triangle of the hand case right_x, whose 13 kept
    cells were worked out by hand."""
    sc = np.float32(61846) / np.float32(804.099365234375)
    assert float(np.float32(np.float32(804.099365234375) * sc)) - 61846 > 2.0 ** -9
    p = hand_plan(lo=(0, 0, 0), scale=(sc, 1, 1), res=(61846, 4, 4))
    x = np.float32(804.099365234375)
    verts = np.array([[x, 0.5, 0.5], [x, 3.5, 0.5], [x, 0.5, 3.5]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    clo, chi, V = oracle.cell_boxes(verts, tris, p)
    assert clo[0, 0] == chi[0, 0] == 61845 and V[0] == 16
    C, O, kept = oracle.cull_pairs(verts, tris, p, clo, chi, int(V[0]))
    yz = sorted(((int(c) // 61846) % 4, int(c) // (61846 * 4)) for c in C)
    want = sorted((y, z) for z in range(4) for y in range(4) if y + z <= 4)
    assert (C % 61846 == 61845).all() and yz == want, (yz, want)


def pin_cull_invariants():
    """On scenes: the kept pairs are a subsequence of the box pairs (object
    order, GlobalCoords order inside an object); the cell of every vertex and
    of sampled interior points of every triangle is kept; the two placements
    of the kept pairs (stable sort + ranges, stable counting placement)
    agree; large diagonal triangles lose most of their box cells."""
    g = np.random.Generator(np.random.Philox(16))
    for s in (scenes.uniform_soup(3000, seed=7), scenes.nonhomogeneous_soup(3000, seed=8, extent=15.0)):
        full = oracle.build_grid(s.verts, s.tris, s.lam)
        a = oracle.build_grid(s.verts, s.tris, s.lam, method="alg1", cull=True)
        b = oracle.build_grid(s.verts, s.tris, s.lam, method="counting", cull=True)
        assert np.array_equal(a.G, b.G) and np.array_equal(a.refs, b.refs) and a.NO == b.NO
        assert a.G[0] == 0 and a.G[-1] == a.NO and (np.diff(a.G) >= 0).all()
        p = a.plan
        C, O = oracle.object_order_pairs(full.clo, full.chi, full.offsets, full.NO, p.res)
        Ck, Ok, kept = oracle.cull_pairs(s.verts, s.tris, p, full.clo, full.chi, full.NO)
        assert np.array_equal(kept, a.V) and kept.sum() == a.NO and (kept <= full.V).all()
        key_full = O.astype(np.int64) * p.ncells + C
        key_kept = Ok.astype(np.int64) * p.ncells + Ck
        pos = np.searchsorted(key_full, key_kept)     # object-order keys are ascending
        assert (np.diff(key_full) > 0).all() and np.array_equal(key_full[pos], key_kept)
        kept_set = set(key_kept.tolist())
        q = oracle.grid_space(s.verts, s.tris, p).astype(np.float64)
        res = p.res.astype(np.int64)
        bary = g.dirichlet((1, 1, 1), 12)
        for i in range(s.n):
            pts = np.concatenate([q[i], bary @ q[i]])
            for pt in pts:
                f = np.floor(pt)
                if ((pt - f) < 1e-6).any() or ((f + 1 - pt) < 1e-6).any():
                    continue      # on a cell face: either neighbour may hold it
                cell = np.clip(f.astype(np.int64), 0, res - 1)
                cid = int(cell[0] + res[0] * (cell[1] + res[1] * cell[2]))
                assert i * p.ncells + cid in kept_set, (i, pt)
        if "nonhomogeneous" in s.name:
            assert a.NO < 0.5 * full.NO, (a.NO, full.NO)


ALL_PINS = [pin_hand_example, pin_fig1_cells, pin_shifted_cells, pin_point_in_cell, pin_plan_cases, pin_plan_errors,
            pin_bounds, pin_bounds_signed_zero, pin_bruteforce, pin_brute_boxes, pin_library_routines, pin_invariants,
            pin_cull_hand, pin_cull_exact, pin_cull_far_face, pin_cull_invariants]


def run_all():
    """Runs every pin; returns the names of those that failed."""
    failed = []
    for fn in ALL_PINS:
        try:
            fn()
        except Exception as e:  # noqa: BLE001 - a mutant may fail any way
            failed.append(f"{fn.__name__}: {type(e).__name__}")
    return failed
