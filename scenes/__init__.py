"""Seeded synthetic triangle scenes that stand in for the paper's benchmark scenes.

The paper (Sec. 4, Table 1) measures grid construction on non-homogeneous and
architectural scenes (Fairy Forest, Crytek Sponza, San Miguel, ...).  Those
meshes are not available, so the workloads below are generated from seeds with
the same character: uniform soups, soups with a heavy tail of large triangles,
and an architectural scene of large axis-aligned wall quads plus clustered
small clutter.

This module only draws inputs.  It holds none of the grid-construction
arithmetic, and both the CUDA path and the CPU oracle consume what it returns.
Every generator is deterministic for a given seed (numpy's counter-based Philox
bit generator) and returns float32 vertices ``[nv, 3]`` and int32 triangles
``[n, 3]``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 0xC0FFEE


@dataclasses.dataclass
class Scene:
    name: str
    verts: np.ndarray  # float32 [nv, 3]
    tris: np.ndarray   # int32 [n, 3]
    lam: float         # grid density: target cells per triangle

    @property
    def n(self) -> int:
        return int(self.tris.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _unit_vectors(g: np.random.Generator, n: int) -> np.ndarray:
    """Directions uniform on the unit sphere (normalised Gaussians)."""
    d = g.standard_normal((n, 3))
    nrm = np.sqrt((d * d).sum(axis=1, keepdims=True))
    nrm[nrm == 0.0] = 1.0
    return d / nrm


def _soup(c: np.ndarray, e1: np.ndarray, e2: np.ndarray):
    """Triangle soup with centroid c and edge vectors e1, e2 from v0."""
    v0 = c - (e1 + e2) / 3.0
    v1 = v0 + e1
    v2 = v0 + e2
    n = c.shape[0]
    verts = np.empty((n, 3, 3), dtype=np.float32)
    verts[:, 0] = v0
    verts[:, 1] = v1
    verts[:, 2] = v2
    tris = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return verts.reshape(3 * n, 3), tris


def uniform_soup(n: int = 100_000, seed: int = SEED_BASE + 1, lam: float = 2.0) -> Scene:
    """Uniform soup: centroids U[0,1]^3, edge vectors U[-0.01,0.01]^3."""
    g = rng(seed)
    c = g.random((n, 3))
    e1 = g.uniform(-0.01, 0.01, (n, 3))
    e2 = g.uniform(-0.01, 0.01, (n, 3))
    v, t = _soup(c, e1, e2)
    return Scene(f"uniform_soup_{n}", v, t, lam)


def nonhomogeneous_soup(n: int = 1_000_000, seed: int = SEED_BASE + 2, lam: float = 4.0,
                        extent: float = 100.0, large_frac: float = 0.01) -> Scene:
    """Non-homogeneous soup: centroids U[0,extent]^3; 99% small triangles with
    edge lengths LogNormal(ln 0.05, 0.5), 1% large with lengths U[5,40], all
    with directions uniform on the sphere.  The large ones are picked by a
    seeded permutation, so a single triangle can span 1 to ~1e4+ cells."""
    g = rng(seed)
    c = g.random((n, 3)) * extent
    nlarge = int(round(large_frac * n))
    is_large = np.zeros(n, dtype=bool)
    is_large[g.permutation(n)[:nlarge]] = True
    l1 = g.lognormal(math.log(0.05), 0.5, n)
    l2 = g.lognormal(math.log(0.05), 0.5, n)
    big1 = g.uniform(5.0, 40.0, n)
    big2 = g.uniform(5.0, 40.0, n)
    l1 = np.where(is_large, big1, l1)
    l2 = np.where(is_large, big2, l2)
    e1 = _unit_vectors(g, n) * l1[:, None]
    e2 = _unit_vectors(g, n) * l2[:, None]
    v, t = _soup(c, e1, e2)
    return Scene(f"nonhomogeneous_soup_{n}", v, t, lam)


def architectural(n: int = 10_000_000, seed: int = SEED_BASE + 3, lam: float = 8.0,
                  size=(200.0, 50.0, 200.0), nblobs: int = 2000,
                  quad_frac: float = 0.05) -> Scene:
    """Architectural-style scene: a ``size`` building of axis-aligned wall and
    floor quads (side lengths log-uniform in [0.5, 20], clipped to the
    building, each split into 2 triangles sharing 2 of its 4 vertices: about
    ``quad_frac`` of the triangles), plus clutter of small randomly oriented
    triangles (edges log-uniform in [0.01, 0.3]) clustered in ``nblobs``
    Gaussian blobs of sigma 1.5 whose centres are uniform in the building.
    The quads form an indexed mesh, so this scene exercises the vertex
    gather through ``tris``."""
    g = rng(seed)
    size = np.asarray(size, dtype=np.float64)
    nquad = int(round(quad_frac * n / 2))
    nclut = n - 2 * nquad

    # --- wall / floor quads ---------------------------------------------------
    axis = g.integers(0, 3, nquad)                     # normal axis
    lo_side, hi_side = math.log(0.5), math.log(20.0)
    sa = np.exp(g.uniform(lo_side, hi_side, nquad))
    sb = np.exp(g.uniform(lo_side, hi_side, nquad))
    u_ax = (axis + 1) % 3                              # first in-plane axis
    w_ax = (axis + 2) % 3                              # second in-plane axis
    sa = np.minimum(sa, size[u_ax])
    sb = np.minimum(sb, size[w_ax])
    cu = g.random(nquad) * (size[u_ax] - sa)
    cw = g.random(nquad) * (size[w_ax] - sb)
    plane = g.random(nquad) * size[axis]
    corners = np.zeros((nquad, 4, 3), dtype=np.float64)
    rows = np.arange(nquad)
    for k, (du, dw) in enumerate(((0, 0), (1, 0), (1, 1), (0, 1))):
        corners[rows, k, axis] = plane
        corners[rows, k, u_ax] = cu + du * sa
        corners[rows, k, w_ax] = cw + dw * sb
    qverts = corners.reshape(4 * nquad, 3)
    base = 4 * np.arange(nquad, dtype=np.int64)
    qtris = np.empty((nquad, 2, 3), dtype=np.int64)
    qtris[:, 0] = np.stack([base, base + 1, base + 2], axis=1)
    qtris[:, 1] = np.stack([base, base + 2, base + 3], axis=1)
    qtris = qtris.reshape(2 * nquad, 3)

    # --- clutter ----------------------------------------------------------------
    centres = g.random((nblobs, 3)) * size
    blob = g.integers(0, nblobs, nclut)
    c = centres[blob] + g.normal(0.0, 1.5, (nclut, 3))
    c = np.clip(c, 0.0, size)
    lo_e, hi_e = math.log(0.01), math.log(0.3)
    l1 = np.exp(g.uniform(lo_e, hi_e, nclut))
    l2 = np.exp(g.uniform(lo_e, hi_e, nclut))
    e1 = _unit_vectors(g, nclut) * l1[:, None]
    e2 = _unit_vectors(g, nclut) * l2[:, None]
    cverts, ctris = _soup(c, e1, e2)

    verts = np.concatenate([qverts.astype(np.float32), cverts], axis=0)
    tris = np.concatenate([qtris, ctris.astype(np.int64) + 4 * nquad], axis=0).astype(np.int32)
    return Scene(f"architectural_{n}", verts, tris, lam)


def architectural_scaled(n: int, seed: int = SEED_BASE + 3, lam: float = 8.0) -> Scene:
    """The architectural scene with n triangles at the 10M scene's density:
    building 200 x 50 x 200 scaled by cbrt(n / 1e7), 2000 * n / 1e7 clutter
    blobs (at least 4)."""
    f = (n / 1e7) ** (1.0 / 3.0)
    s = architectural(n, seed=seed, lam=lam, size=(200.0 * f, 50.0 * f, 200.0 * f),
                      nblobs=max(4, int(round(2000 * n / 1e7))))
    s.name = f"architectural_scaled_{n}"
    return s


def batch_sizes(nmeshes: int = 64, seed: int = SEED_BASE + 4, lo: float = 1e3, hi: float = 2e6):
    """Triangle counts log-uniform in [lo, hi] for a batch of meshes."""
    g = rng(seed)
    return np.exp(g.uniform(math.log(lo), math.log(hi), nmeshes)).astype(np.int64)


def batched_meshes(nmeshes: int = 64, seed: int = SEED_BASE + 4, lam: float = 4.0,
                   lo: float = 1e3, hi: float = 2e6, scale: float = 1.0):
    """Independent non-homogeneous soups of uneven sizes; mesh k has N_k
    triangles in a box of side 100 * cbrt(N_k / 1e6) so the triangle density
    matches the 1M-triangle soup.  ``scale`` multiplies every N_k (small
    variants for tests)."""
    sizes = batch_sizes(nmeshes, seed, lo, hi)
    out = []
    for k, nk in enumerate(sizes):
        nk = max(1, int(round(nk * scale)))
        ext = 100.0 * (nk / 1e6) ** (1.0 / 3.0)
        out.append(nonhomogeneous_soup(nk, seed=seed * 1000 + k, lam=lam, extent=ext))
    return out


def serving_pool(nmeshes: int = 12, seed: int = SEED_BASE + 5, lo: float = 1e4, hi: float = 1e7):
    """Meshes a rebuild server keeps registered: N_k log-uniform in [lo, hi];
    by a seeded coin flip either a non-homogeneous soup (box side
    100 * cbrt(N_k / 1e6), the 1M soup's density, lambda 4) or an
    architectural scene (building 200 x 50 x 200 scaled by cbrt(N_k / 1e7),
    2000 * N_k / 1e7 clutter blobs, at least 4, lambda 8)."""
    g = rng(seed)
    sizes = np.exp(g.uniform(math.log(lo), math.log(hi), nmeshes)).astype(np.int64)
    arch = g.random(nmeshes) < 0.5
    out = []
    for k, (nk, is_arch) in enumerate(zip(sizes, arch)):
        nk = int(nk)
        if is_arch:
            out.append(architectural_scaled(nk, seed=seed * 1000 + k))
        else:
            out.append(nonhomogeneous_soup(nk, seed=seed * 1000 + k, extent=100.0 * (nk / 1e6) ** (1.0 / 3.0)))
    return out


def poisson_requests(rate: float = 200.0, duration: float = 30.0, nmeshes: int = 12,
                     seed: int = SEED_BASE + 6):
    """A rebuild request stream: Poisson arrivals at `rate` per second for
    `duration` seconds (exponential gaps); each request names a mesh of the
    pool uniformly and carries its own 63-bit jitter seed.  Returns
    (arrival times in s, mesh ids, seeds) as numpy arrays."""
    g = rng(seed)
    m = int(rate * duration * 1.5) + 64
    t = np.cumsum(g.exponential(1.0 / rate, m))
    mesh = g.integers(0, nmeshes, m)
    seeds = g.integers(0, 2**63, m, dtype=np.int64)
    keep = t < duration
    return t[keep], mesh[keep], seeds[keep]


def tiny_scene(g: np.random.Generator, n: int, nverts: int | None = None,
               box: float = 1.0, max_edge: float = 0.5) -> Scene:
    """A small random indexed mesh for exhaustive checks: ``nverts`` vertices
    (default 3n) and ``n`` triangles drawing random vertex indices."""
    if nverts is None:
        nverts = max(3, 3 * n)
    centers = g.random((nverts, 3)) * box
    jitter = (g.random((nverts, 3)) - 0.5) * max_edge
    verts = (centers + jitter).astype(np.float32)
    tris = g.integers(0, nverts, (n, 3)).astype(np.int32)
    return Scene(f"tiny_{n}", verts, tris, float(g.uniform(0.5, 8.0)))


CONFIGS = {
    "uniform_1e5": lambda: uniform_soup(),
    "nonhomogeneous_1e6": lambda: nonhomogeneous_soup(),
    "architectural_1e7": lambda: architectural(),
}


# ---- per-request vertex jitter ------------------------------------------------------
#
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
# as 1, 2, 3", SC'11): a counter-based generator, written here from its
# published definition so the CUDA side (its own implementation) can draw the
# same numbers.  A vertex coordinate's jitter is an Irwin-Hall sum of four
# uniforms, rescaled to unit variance: n = ((u0 + u1) + (u2 + u3)) - 2 with
# u_k = (x_k >> 8) * 2^-24, then delta = n * s where s = sigma * sqrt(3) is
# rounded to float32 once; every operation is a single float32 add or
# multiply, so host and device agree bit for bit.

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint32 arrays (counters) and keys."""
    M = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = (np.asarray(x, np.uint64) & M for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & M
    k1 = np.uint64(k1) & M
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & M
        hi1, lo1 = p1 >> np.uint64(32), p1 & M
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & M, lo1, (hi0 ^ c3 ^ k1) & M, lo0
        k0 = (k0 + np.uint64(PHILOX_W0)) & M
        k1 = (k1 + np.uint64(PHILOX_W1)) & M
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def jitter_scale(sigma: float) -> np.float32:
    """The float32 factor s = sigma * sqrt(3) both sides use."""
    return np.float32(np.float32(sigma) * np.float32(1.7320508075688772))


def jitter_vertices(verts: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """verts + per-coordinate jitter of standard deviation sigma for request
    `seed`: coordinate a of vertex i uses counter (i, a, 0, 0) and key
    (seed & 0xffffffff, seed >> 32)."""
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    nv = v.shape[0]
    i = np.repeat(np.arange(nv, dtype=np.uint64), 3)
    a = np.tile(np.arange(3, dtype=np.uint64), nv)
    zero = np.zeros_like(i)
    x = philox4x32_10(i, a, zero, zero, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    two24 = np.float32(1.0 / 16777216.0)
    u = [((xk >> np.uint32(8)).astype(np.float32) * two24).astype(np.float32) for xk in x]
    n = ((u[0] + u[1]).astype(np.float32) + (u[2] + u[3]).astype(np.float32)).astype(np.float32) - np.float32(2.0)
    d = (n.astype(np.float32) * jitter_scale(sigma)).astype(np.float32)
    return (v.reshape(-1) + d).astype(np.float32).reshape(-1, 3)
