"""The rebuild-serving loop (grid_serve_*) and its device jitter, through the
C ABI: the device jitter equals the host generator bit for bit, every served
result equals the oracle's grid of the jittered mesh, a request's result is
the same whether it is built alone or in a mix (other requests, batches,
workers, streams), admission refuses past the memory budget, and one failing
request does not fail the others of its batch."""
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


def assert_same_as_oracle(res, o, what=""):
    info = res.info
    assert tuple(info.res) == tuple(o.plan.res), what
    assert np.array_equal(np.array(info.lo, np.float32), o.plan.lo), what
    assert np.array_equal(np.array(info.hi, np.float32), o.plan.hi), what
    assert info.ncells == o.plan.ncells and info.nrefs == o.NO, what
    assert np.array_equal(host(res.cells), o.G), (what, "cells")
    assert np.array_equal(host(res.refs), o.refs), (what, "refs")


# ---- device jitter ---------------------------------------------------------------

@pytest.mark.parametrize("nverts,sigma,seed", [
    (1, 0.01, 0), (7, 0.01, 1), (100_003, 0.01, 12345), (100_003, 0.5, (1 << 40) + 17),
    (5_000, 0.0, 3), (2_000_000, 0.01, 2**64 - 1),
])
def test_device_jitter_matches_host(ctx, nverts, sigma, seed):
    g = np.random.Generator(np.random.Philox(nverts))
    v = (g.random((nverts, 3)) * 100.0 - 20.0).astype(np.float32)
    got = host(ctx.jitter(dev(v, torch.float32), sigma, seed))
    want = scenes.jitter_vertices(v, sigma, seed)
    bad = np.flatnonzero(got.view(np.uint32).ravel() != want.view(np.uint32).ravel())
    assert bad.size == 0, (bad[:8], got.ravel()[bad[:8]], want.ravel()[bad[:8]])


def test_device_jitter_in_place(ctx):
    v = scenes.uniform_soup(3000, seed=8).verts
    t = dev(v, torch.float32)
    want = host(ctx.jitter(t, 0.02, 99))
    ctx.jitter(t, 0.02, 99)   # out == verts is allowed
    assert np.array_equal(host(ctx.jitter(dev(v, torch.float32), 0.02, 99)), want)


def test_context_work_is_ordered_with_torch_default_stream(ctx):
    """Calls made on torch's default stream (the legacy default stream) run in
    its order: the jitter reads an input torch is still writing and torch's
    copy back reads the jitter's output, with no synchronisation between
    them (a context bound to its own non-blocking stream would race both)."""
    nv = 3_000_000
    torch.cuda.synchronize()
    base = torch.arange(3 * nv, device="cuda", dtype=torch.float32).reshape(nv, 3)
    v = base
    for _ in range(20):   # a queue of torch work ahead of the jitter
        v = v * 1.0 + 0.0
    got = ctx.jitter(v, 0.01, 4242).cpu().numpy()
    want = scenes.jitter_vertices(np.arange(3 * nv, dtype=np.float32).reshape(nv, 3), 0.01, 4242)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ---- serving -----------------------------------------------------------------------

def _pool():
    g = np.random.Generator(np.random.Philox(777))
    return [
        scenes.uniform_soup(4_000, seed=301),
        scenes.nonhomogeneous_soup(12_000, seed=302, extent=20.0),
        scenes.architectural(20_000, seed=303, size=(25.0, 6.0, 25.0), nblobs=15),
        scenes.tiny_scene(g, 23),
        scenes.nonhomogeneous_soup(250_000, seed=304, extent=60.0),
    ]


def _requests(nreq, nmesh, seed=55):
    g = np.random.Generator(np.random.Philox(seed))
    mesh = g.integers(0, nmesh, nreq)
    sig = np.where(g.random(nreq) < 0.15, 0.0, 0.01)
    seeds = g.integers(0, 2**63, nreq)
    return [(int(m), float(s), int(sd)) for m, s, sd in zip(mesh, sig, seeds)]


def _serve_all(srv, ids, reqs, serial):
    """Results of every request as host arrays.  serial: submit, wait and
    release one at a time; else submit all first, then collect."""
    out = []
    if serial:
        for m, s, sd in reqs:
            tk = srv.submit(ids[m], s, sd)
            assert tk is not None
            r = srv.wait(tk, timeout=120)
            out.append((host(r.cells), host(r.refs), r.info))
            r.release()
        return out
    tickets = []
    for m, s, sd in reqs:
        tk = srv.submit(ids[m], s, sd)
        assert tk is not None
        tickets.append(tk)
    for tk in tickets:
        r = srv.wait(tk, timeout=120)
        out.append((host(r.cells), host(r.refs), r.info))
        r.release()
    return out


@pytest.fixture(scope="module")
def pool():
    return _pool()


def test_served_results_match_oracle(ctx, pool):
    import paper_2403_10647_gb300 as pg
    srv = pg.Server(0, nworkers=2, max_batch=4)
    try:
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool]
        reqs = [(0, 0.01, 11), (1, 0.01, 12), (2, 0.01, 13), (3, 0.01, 14), (1, 0.0, 0), (4, 0.01, 2**40 + 3)]
        tickets = [srv.submit(ids[m], s, sd) for m, s, sd in reqs]
        for (m, s, sd), tk in zip(reqs, tickets):
            r = srv.wait(tk, timeout=120)
            sc = pool[m]
            v = scenes.jitter_vertices(sc.verts, s, sd)
            o = oracle.build_grid(v, sc.tris, sc.lam, method="alg1" if sc.n < 50_000 else "counting")
            assert_same_as_oracle(r, o, f"mesh {m} sigma {s} seed {sd}")
            r.release()
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["reserved_bytes"] == 0
    finally:
        srv.close()


def test_alone_equals_in_mix(ctx, pool):
    """Each request's result is bit-identical built alone (one worker, batches
    of one, one request in flight) and in a mix (four workers on four
    streams, batches of up to eight, everything queued at once)."""
    import paper_2403_10647_gb300 as pg
    reqs = _requests(48, len(pool))
    alone_srv = pg.Server(0, nworkers=1, max_batch=1)
    try:
        ids = [alone_srv.register(s.verts, s.tris, s.lam) for s in pool]
        alone = _serve_all(alone_srv, ids, reqs, serial=True)
        assert alone_srv.stats()["batched_requests"] == 0
    finally:
        alone_srv.close()
    mix_srv = pg.Server(0, nworkers=4, max_batch=8)
    try:
        ids = [mix_srv.register(s.verts, s.tris, s.lam) for s in pool]
        mixed = _serve_all(mix_srv, ids, reqs, serial=False)
        st = mix_srv.stats()
    finally:
        mix_srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for k, ((ca, ra, ia), (cb, rb, ib)) in enumerate(zip(alone, mixed)):
        assert ia == ib, k
        assert np.array_equal(ca, cb) and np.array_equal(ra, rb), f"request {k} differs in the mix"


def test_batches_form_behind_a_busy_worker(ctx, pool):
    """One worker busy with a large rebuild: the requests queued meanwhile
    are taken together as one batch, and still match the oracle."""
    import paper_2403_10647_gb300 as pg
    big = scenes.nonhomogeneous_soup(1_000_000, seed=305)
    srv = pg.Server(0, nworkers=1, max_batch=16)
    try:
        bid = srv.register(big.verts, big.tris, big.lam)
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool[:4]]
        t0 = srv.submit(bid, 0.01, 1)
        small = [(i % 4, 0.01, 1000 + i) for i in range(12)]
        tks = [srv.submit(ids[m], s, sd) for m, s, sd in small]
        srv.wait(t0, timeout=120).release()
        for (m, s, sd), tk in zip(small, tks):
            r = srv.wait(tk, timeout=120)
            sc = pool[m]
            o = oracle.build_grid(scenes.jitter_vertices(sc.verts, s, sd), sc.tris, sc.lam)
            assert_same_as_oracle(r, o, f"queued request mesh {m}")
            r.release()
        st = srv.stats()
        assert st["batched_requests"] >= 2, st
        assert st["batches"] < 1 + len(small)
    finally:
        srv.close()


def test_small_request_passes_large_ones(ctx, pool):
    """Two workers, three rebuilds too large to batch and a small request
    queued behind them: with the default small lane the small request runs
    before the third large one, which is still unfinished when the small one
    is done.  (In strict arrival order the third large one starts first; how
    the two then finish depends on timing, so only the results are checked.)
    Every result matches the oracle."""
    import paper_2403_10647_gb300 as pg
    big = scenes.nonhomogeneous_soup(1_000_000, seed=306)
    for small_lane in (True, False):
        srv = pg.Server(0, nworkers=2, small_lane=small_lane)
        try:
            bid = srv.register(big.verts, big.tris, big.lam)
            sid = srv.register(pool[0].verts, pool[0].tris, pool[0].lam)
            large = [srv.submit(bid, 0.01, 10 + k) for k in range(3)]
            tk = srv.submit(sid, 0.01, 99)
            r = srv.wait(tk, timeout=120)
            p2 = srv.poll(large[2])   # keep the result: dropping it releases the ticket
            third_done = p2 is not None
            o = oracle.build_grid(scenes.jitter_vertices(pool[0].verts, 0.01, 99), pool[0].tris, pool[0].lam)
            assert_same_as_oracle(r, o, "small request")
            r.release()
            if small_lane:
                assert not third_done, "the small request waited for the third large one"
            for k, t in enumerate(large):
                rl = p2 if k == 2 and p2 is not None else srv.wait(t, timeout=120)
                assert rl.info.nrefs > (1 << 24), rl.info.nrefs
                if k == 2:
                    ob = oracle.build_grid(scenes.jitter_vertices(big.verts, 0.01, 12), big.tris, big.lam,
                                           method="counting")
                    assert_same_as_oracle(rl, ob, "third large request")
                rl.release()
        finally:
            srv.close()


def test_admission_refuses_beyond_budget(ctx, pool):
    import paper_2403_10647_gb300 as pg
    sc = pool[4]
    probe = pg.Server(0, nworkers=1)
    try:
        mid = probe.register(sc.verts, sc.tris, sc.lam)
        tk = probe.submit(mid, 0.01, 1)
        est = probe.stats()["reserved_bytes"]
        probe.wait(tk, timeout=120).release()
    finally:
        probe.close()
    assert est > 0
    srv = pg.Server(0, nworkers=1, hbm_budget=int(est * 1.5))
    try:
        mid = srv.register(sc.verts, sc.tris, sc.lam)
        t1 = srv.submit(mid, 0.01, 1)
        assert t1 is not None
        assert srv.submit(mid, 0.01, 2) is None          # a second would pass the budget
        r = srv.wait(t1, timeout=120)
        assert srv.submit(mid, 0.01, 3) is None          # an unreleased result still holds its share
        r.release()
        t3 = srv.submit(mid, 0.01, 3)
        assert t3 is not None
        srv.wait(t3, timeout=120).release()
        st = srv.stats()
        assert st["refused"] == 2 and st["completed"] == 2 and st["peak_reserved_bytes"] <= int(est * 1.5)
    finally:
        srv.close()


def test_failing_request_does_not_fail_its_batch(ctx, pool):
    """sigma = 3e38 overflows the jitter to non-finite coordinates: that
    request fails with GRID_EINVAL, the rest of its batch still succeeds."""
    import paper_2403_10647_gb300 as pg
    from paper_2403_10647_gb300 import _lib
    big = scenes.nonhomogeneous_soup(1_000_000, seed=306)
    srv = pg.Server(0, nworkers=1, max_batch=8)
    try:
        bid = srv.register(big.verts, big.tris, big.lam)
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool[:3]]
        t0 = srv.submit(bid, 0.0, 0)                     # keeps the worker busy so the rest batch up
        reqs = [(0, 0.01, 5), (1, 3e38, 6), (2, 0.01, 7)]
        tks = [srv.submit(ids[m], s, sd) for m, s, sd in reqs]
        srv.wait(t0, timeout=120).release()
        for (m, s, sd), tk in zip(reqs, tks):
            if s > 1.0:
                with pytest.raises(pg.GridError) as e:
                    srv.wait(tk, timeout=120)
                assert e.value.code == _lib.GRID_EINVAL
                assert srv.release(tk) == 0
                continue
            r = srv.wait(tk, timeout=120)
            sc = pool[m]
            assert_same_as_oracle(r, oracle.build_grid(scenes.jitter_vertices(sc.verts, s, sd), sc.tris, sc.lam))
            r.release()
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 4
    finally:
        srv.close()


def test_bad_tickets_and_arguments(ctx, pool):
    import paper_2403_10647_gb300 as pg
    from paper_2403_10647_gb300 import _lib
    srv = pg.Server(0, nworkers=1)
    try:
        sc = pool[0]
        mid = srv.register(sc.verts, sc.tris, sc.lam)
        with pytest.raises(pg.GridError):
            srv.wait(987654, timeout=1)
        with pytest.raises(pg.GridError):
            srv.submit(mid + 5, 0.01, 1)
        with pytest.raises(pg.GridError):
            srv.submit(mid, -1.0, 1)
        with pytest.raises(pg.GridError):
            srv.submit(mid, float("nan"), 1)
        with pytest.raises(pg.GridError):   # a bad vertex index fails registration
            srv.register(sc.verts, np.array([[0, 1, 10**6]], np.int32), 2.0)
        tk = srv.submit(mid, 0.01, 1)
        r = srv.wait(tk, timeout=120)
        assert srv.poll(tk) is not None
        r.release()
        assert srv.release(tk) == _lib.GRID_EINVAL    # already released
        with pytest.raises(pg.GridError):
            srv.poll(tk)
    finally:
        srv.close()


def test_empty_mesh_is_served(ctx):
    import paper_2403_10647_gb300 as pg
    srv = pg.Server(0, nworkers=2)
    try:
        mid = srv.register(np.zeros((4, 3), np.float32), np.zeros((0, 3), np.int32), 2.0)
        r = srv.wait(srv.submit(mid, 0.01, 1), timeout=60)
        assert host(r.cells).tolist() == [0, 0] and r.refs.numel() == 0 and tuple(r.info.res) == (1, 1, 1)
        r.release()
    finally:
        srv.close()


def test_request_larger_than_the_budget_is_rejected_for_good(ctx, pool):
    """A request whose estimate alone exceeds the budget can never be
    admitted: GRID_ELIMIT, not the retry-later GRID_EAGAIN."""
    import paper_2403_10647_gb300 as pg
    from paper_2403_10647_gb300 import _lib
    srv = pg.Server(0, nworkers=1, hbm_budget=1 << 20)   # below any request's estimate
    try:
        mid = srv.register(pool[0].verts, pool[0].tris, pool[0].lam)
        with pytest.raises(pg.GridError) as e:
            srv.submit(mid, 0.01, 1)
        assert e.value.code == _lib.GRID_ELIMIT
        st = srv.stats()
        assert st["submitted"] == 0 and st["reserved_bytes"] == 0
    finally:
        srv.close()


def test_latency_statistics(ctx, pool):
    import paper_2403_10647_gb300 as pg
    srv = pg.Server(0, nworkers=2, max_batch=4)
    try:
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool[:3]]
        for k in range(30):
            srv.wait(srv.submit(ids[k % 3], 0.01, k), timeout=120).release()
        st = srv.stats(reset=True)
        assert st["completed"] == 30
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"] * 1.0 + 1e-9
        assert st["mean_us"] <= st["max_us"] and st["p50_service_us"] > 0
        assert srv.stats()["completed"] == 0   # reset cleared the counters
    finally:
        srv.close()


# ---- caller-supplied vertex updates -------------------------------------------------

def _deformed(sc, k):
    """New vertex positions for mesh sc, the k-th frame of a deformation: a
    shear and a swell that move the bounds and the cells of the triangles."""
    v = sc.verts.astype(np.float64)
    c = v.mean(axis=0)
    out = v + (0.02 + 0.01 * k) * np.stack([v[:, 1] - c[1], np.sin(v[:, 0]), 0.5 * (v[:, 2] - c[2])], axis=1)
    return np.ascontiguousarray(out.astype(np.float32))


def _update_oracle(sc, verts, sigma, seed):
    v = scenes.jitter_vertices(verts, sigma, seed) if sigma > 0 else verts
    return oracle.build_grid(v, sc.tris, sc.lam, method="alg1" if sc.n < 50_000 else "counting")


def test_vertex_updates_match_oracle(ctx, pool):
    """Requests carrying new vertex positions (from host memory and from
    device memory, with and without jitter on top) are built from those
    positions; the registered vertices stay as they were."""
    import paper_2403_10647_gb300 as pg
    srv = pg.Server(0, nworkers=2, max_batch=4)
    try:
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool]
        cases = []   # (mesh, update or None, where, sigma, seed)
        for m, sc in enumerate(pool):
            cases.append((m, _deformed(sc, 1), "host", 0.0, 0))
            cases.append((m, _deformed(sc, 2), "cuda", 0.0, 0))
            cases.append((m, _deformed(sc, 3), "host", 0.01, 1000 + m))
            cases.append((m, None, "", 0.0, 0))
        tickets = []
        for m, upd, where, s, sd in cases:
            verts = None if upd is None else (dev(upd, torch.float32) if where == "cuda" else upd)
            tickets.append(srv.submit(ids[m], s, sd, verts=verts))
        for (m, upd, where, s, sd), tk in zip(cases, tickets):
            r = srv.wait(tk, timeout=120)
            sc = pool[m]
            assert_same_as_oracle(r, _update_oracle(sc, sc.verts if upd is None else upd, s, sd),
                                  f"mesh {m} update {where or 'none'} sigma {s}")
            r.release()
        st = srv.stats()
        assert st["completed"] == len(cases) and st["failed"] == 0 and st["reserved_bytes"] == 0
    finally:
        srv.close()


def test_vertex_update_buffer_is_copied_at_submission(ctx, pool):
    """The caller may overwrite its buffer as soon as submit returns: the
    request keeps the positions it was submitted with."""
    import paper_2403_10647_gb300 as pg
    sc = pool[1]
    srv = pg.Server(0, nworkers=1)
    try:
        mid = srv.register(sc.verts, sc.tris, sc.lam)
        frames = [_deformed(sc, k) for k in range(4)]
        host_buf = frames[0].copy()
        dev_buf = dev(frames[0], torch.float32)
        tks = []
        for k in range(4):   # one reused host buffer and one reused device buffer, overwritten each frame
            host_buf[:] = frames[k]
            tks.append(srv.submit(mid, 0.0, 0, verts=host_buf))
            dev_buf.copy_(torch.from_numpy(frames[(k + 1) % 4]).cuda())
            tks.append(srv.submit(mid, 0.0, 0, verts=dev_buf))
        host_buf[:] = 0.0
        dev_buf.zero_()
        for k in range(4):
            for j, f in enumerate((frames[k], frames[(k + 1) % 4])):
                r = srv.wait(tks[2 * k + j], timeout=120)
                assert_same_as_oracle(r, _update_oracle(sc, f, 0.0, 0), f"frame {k} buffer {j}")
                r.release()
    finally:
        srv.close()


def test_vertex_updates_alone_equals_in_mix(ctx, pool):
    """Requests with vertex updates give the same result alone (one worker,
    batches of one) and in a mix (four workers, batches of eight, all queued
    at once, mixed with requests on the registered vertices)."""
    import paper_2403_10647_gb300 as pg
    reqs = _requests(32, len(pool), seed=91)
    upd = [(_deformed(pool[m], k % 3) if k % 3 else None) for k, (m, _, _) in enumerate(reqs)]

    def serve(srv, serial):
        ids = [srv.register(s.verts, s.tris, s.lam) for s in pool]
        out, tks = [], []
        for (m, s, sd), u in zip(reqs, upd):
            tk = srv.submit(ids[m], s, sd, verts=u)
            if serial:
                r = srv.wait(tk, timeout=120)
                out.append((host(r.cells), host(r.refs), r.info))
                r.release()
            else:
                tks.append(tk)
        for tk in tks:
            r = srv.wait(tk, timeout=120)
            out.append((host(r.cells), host(r.refs), r.info))
            r.release()
        return out, srv.stats()

    a_srv = pg.Server(0, nworkers=1, max_batch=1)
    try:
        alone, _ = serve(a_srv, True)
    finally:
        a_srv.close()
    m_srv = pg.Server(0, nworkers=4, max_batch=8)
    try:
        mixed, st = serve(m_srv, False)
    finally:
        m_srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for k, ((ca, ra, ia), (cb, rb, ib)) in enumerate(zip(alone, mixed)):
        assert ia == ib, k
        assert np.array_equal(ca, cb) and np.array_equal(ra, rb), f"request {k} differs in the mix"
    # and both equal the oracle on a sample
    for k in (0, 1, 2, 5):
        m, s, sd = reqs[k]
        sc = pool[m]
        o = _update_oracle(sc, sc.verts if upd[k] is None else upd[k], s, sd)
        assert np.array_equal(alone[k][0], o.G) and np.array_equal(alone[k][1], o.refs), k


def test_bad_vertex_updates(ctx, pool):
    """A non-finite update fails its request alone (GRID_EINVAL); a wrong
    vertex count is refused by the binding before the C call."""
    import paper_2403_10647_gb300 as pg
    from paper_2403_10647_gb300 import _lib
    sc = pool[0]
    srv = pg.Server(0, nworkers=1, max_batch=4)
    try:
        mid = srv.register(sc.verts, sc.tris, sc.lam)
        bad = _deformed(sc, 1)
        bad[int(sc.tris[7, 1]), 2] = np.inf
        t_bad = srv.submit(mid, 0.0, 0, verts=bad)
        t_ok = srv.submit(mid, 0.0, 0, verts=_deformed(sc, 2))
        with pytest.raises(pg.GridError) as e:
            srv.wait(t_bad, timeout=120)
        assert e.value.code == _lib.GRID_EINVAL
        assert srv.release(t_bad) == 0
        r = srv.wait(t_ok, timeout=120)
        assert_same_as_oracle(r, _update_oracle(sc, _deformed(sc, 2), 0.0, 0), "good update after a bad one")
        r.release()
        with pytest.raises(ValueError):
            srv.submit(mid, 0.0, 0, verts=_deformed(sc, 1)[:-1])
        assert srv.stats()["reserved_bytes"] == 0
    finally:
        srv.close()


def test_reserved_worker_serves_small_requests_during_large_ones(ctx, pool):
    """A worker reserved for requests that fit a batch (small_workers, on a
    high-priority stream) builds a small request while the only general
    worker is still on a large rebuild queued ahead of it; results match the
    oracle, and without the reserved worker the small request waits."""
    import paper_2403_10647_gb300 as pg
    big = scenes.nonhomogeneous_soup(1_000_000, seed=308)
    for reserved in (1, -1):
        srv = pg.Server(0, nworkers=1, small_workers=reserved, small_lane=False)
        try:
            bid = srv.register(big.verts, big.tris, big.lam)
            sid = srv.register(pool[0].verts, pool[0].tris, pool[0].lam)
            srv.wait(srv.submit(bid, 0.0, 0), timeout=120).release()   # warm both paths
            srv.wait(srv.submit(sid, 0.0, 0), timeout=120).release()
            large = [srv.submit(bid, 0.01, 20 + k) for k in range(2)]
            tk = srv.submit(sid, 0.01, 77)
            r = srv.wait(tk, timeout=120)
            first_done = srv.poll(large[0])
            o = oracle.build_grid(scenes.jitter_vertices(pool[0].verts, 0.01, 77), pool[0].tris, pool[0].lam)
            assert_same_as_oracle(r, o, f"small request, reserved {reserved}")
            r.release()
            if reserved == 1:
                assert first_done is None, "the small request waited for the large rebuild ahead of it"
            else:
                assert first_done is not None, "without a reserved worker the small request ran early"
            if first_done is not None:
                first_done.release()
            for t in large[1:] if first_done is not None else large:
                srv.wait(t, timeout=120).release()
        finally:
            srv.close()


def test_tuned_meshes_give_the_same_grids(ctx, pool):
    """Rebuilds of a mesh alone run with the setting the autotuner chose for
    it at registration (tune_meshes); every setting gives the same grid, so
    a tuned and an untuned server return identical results, equal to the
    oracle's."""
    import paper_2403_10647_gb300 as pg
    reqs = [(m, 0.01, 900 + m) for m in range(len(pool))] + [(4, 0.0, 0), (2, 0.02, 5)]
    res = {}
    for tune in (True, False):
        srv = pg.Server(0, nworkers=1, max_batch=1, small_workers=-1, tune_meshes=tune)
        try:
            ids = [srv.register(s.verts, s.tris, s.lam) for s in pool]
            res[tune] = _serve_all(srv, ids, reqs, serial=True)
            assert srv.stats()["failed"] == 0
        finally:
            srv.close()
    for k, (m, s, sd) in enumerate(reqs):
        (ca, ra, ia), (cb, rb, ib) = res[True][k], res[False][k]
        assert ia == ib and np.array_equal(ca, cb) and np.array_equal(ra, rb), f"request {k}"
        sc = pool[m]
        o = oracle.build_grid(scenes.jitter_vertices(sc.verts, s, sd), sc.tris, sc.lam,
                              method="alg1" if sc.n < 50_000 else "counting")
        assert np.array_equal(ca, o.G) and np.array_equal(ra, o.refs), f"request {k} vs oracle"
