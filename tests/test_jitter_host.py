"""The host side of the serving loop's per-request vertex jitter (the input
generator the oracle's side of the serving tests uses): Philox4x32-10 against
the generator's published known-answer vectors, and the jitter's
distribution against its definition (mean 0, standard deviation sigma,
|d| <= 2 sqrt(3) sigma).  No GPU."""
import os

import numpy as np

import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = scenes.philox4x32_10(*[np.array([x], np.uint32) for x in r[:4]], r[4], r[5])
        assert [int(o[0]) for o in out] == r[6:]


def test_philox_vectorised_equals_elementwise():
    g = np.random.Generator(np.random.Philox(5))
    c = g.integers(0, 2**32, (4, 50), dtype=np.uint64).astype(np.uint32)
    out = scenes.philox4x32_10(c[0], c[1], c[2], c[3], 0x12345678, 0x9ABCDEF0)
    for j in range(50):
        one = scenes.philox4x32_10(*[c[k][j:j + 1] for k in range(4)], 0x12345678, 0x9ABCDEF0)
        assert [int(o[0]) for o in one] == [int(o[j]) for o in out]


def test_jitter_distribution():
    nv = 400_000
    v = np.zeros((nv, 3), np.float32)
    sigma = 0.01
    d = scenes.jitter_vertices(v, sigma, seed=7).astype(np.float64)
    flat = d.reshape(-1)
    assert abs(flat.mean()) < 5 * sigma / np.sqrt(flat.size)
    assert abs(flat.std() / sigma - 1.0) < 0.01
    assert np.abs(flat).max() <= 2 * np.sqrt(3) * sigma * (1 + 1e-6)
    # coordinates of a vertex are independent draws
    assert abs(np.corrcoef(d[:, 0], d[:, 1])[0, 1]) < 0.01
    assert abs(np.corrcoef(d[:-1, 0], d[1:, 0])[0, 1]) < 0.01


def test_jitter_seeds_and_identity():
    s = scenes.nonhomogeneous_soup(2000, seed=3)
    a = scenes.jitter_vertices(s.verts, 0.01, seed=1)
    b = scenes.jitter_vertices(s.verts, 0.01, seed=1)
    c = scenes.jitter_vertices(s.verts, 0.01, seed=2)
    hi = scenes.jitter_vertices(s.verts, 0.01, seed=(1 << 40) + 1)
    assert a.dtype == np.float32 and a.shape == s.verts.shape
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert not np.array_equal(a, c)
    assert not np.array_equal(a, hi)       # the key's high word matters
    z = scenes.jitter_vertices(s.verts, 0.0, seed=1)
    assert np.array_equal(z, s.verts)      # sigma 0: d = n * 0 = 0 exactly, v + 0 = v


def test_jitter_counter_layout():
    """Coordinate a of vertex i draws counter (i, a, 0, 0): the jitter of a
    prefix of the vertex array does not depend on the vertices after it."""
    s = scenes.uniform_soup(1000, seed=4)
    full = scenes.jitter_vertices(s.verts, 0.05, seed=9)
    part = scenes.jitter_vertices(s.verts[:123], 0.05, seed=9)
    assert np.array_equal(full[:123], part)
    i, a = 57, 2
    x = scenes.philox4x32_10(np.array([i], np.uint32), np.array([a], np.uint32), np.zeros(1, np.uint32),
                             np.zeros(1, np.uint32), 9, 0)
    u = [np.float32(int(xk[0]) >> 8) * np.float32(2.0 ** -24) for xk in x]
    n = np.float32(np.float32(np.float32(u[0] + u[1]) + np.float32(u[2] + u[3])) - np.float32(2.0))
    want = np.float32(s.verts[i, a] + np.float32(n * scenes.jitter_scale(0.05)))
    assert full[i, a] == want
