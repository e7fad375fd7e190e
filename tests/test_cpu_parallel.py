"""The multi-core CPU baseline (oracle/cpu_parallel.c, OpenMP) that bench.py
times as a reference point: it must give the oracle's grid bit for bit, at
any thread count.  No GPU."""
import numpy as np
import pytest

import oracle
import scenes


@pytest.mark.parametrize("make", [
    lambda: scenes.uniform_soup(20_000, seed=601),
    lambda: scenes.nonhomogeneous_soup(30_000, seed=602, extent=30.0),
    lambda: scenes.architectural(60_000, seed=603, size=(40.0, 10.0, 40.0), nblobs=40),
    lambda: scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), 2.0),
], ids=["uniform", "nonhomogeneous", "architectural", "empty"])
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_parallel_baseline_equals_oracle(make, threads):
    s = make()
    o = oracle.build_grid(s.verts, s.tris, s.lam, method="counting")
    G, refs, NO = oracle.grid_parallel(s.verts, s.tris, s.lam, nthreads=threads)
    assert NO == o.NO
    assert np.array_equal(G, o.G) and np.array_equal(refs, o.refs)


def test_parallel_baseline_reports_threads():
    assert oracle.parallel_threads(2) == 2
    assert oracle.parallel_threads(0) >= 1
