"""GB300-native parallel uniform-grid construction (Costa, Pereira, Jorge,
"Building An Efficient Grid On GPU", Algorithm 1).

A thin Python binding over the C ABI of ``include/grid.h``: every step of the
build runs in the library's CUDA kernels; this module only passes pointers,
sizes and the current CUDA stream.  PyTorch supplies device memory and streams.
Importing the package does not load the library; the first call does, and it
raises if the library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _lib
from ._lib import GridError, GridInfo, GridBuf, GridOpts, GridServeOpts, GridServeStats, check

__all__ = ["Context", "Server", "Info", "Grid", "BatchedGrids", "plan", "GridError"]


@dataclasses.dataclass
class Info:
    lo: tuple
    hi: tuple
    scale: tuple
    res: tuple
    key_bits: int
    ncells: int
    nrefs: int
    n: int

    @classmethod
    def from_c(cls, i: GridInfo) -> "Info":
        return cls(tuple(i.lo), tuple(i.hi), tuple(i.scale), tuple(i.res), int(i.key_bits),
                   int(i.ncells), int(i.nrefs), int(i.n))

    def to_c(self) -> GridInfo:
        c = GridInfo()
        for a in range(3):
            c.lo[a], c.hi[a], c.scale[a], c.res[a] = self.lo[a], self.hi[a], self.scale[a], self.res[a]
        c.key_bits, c.ncells, c.nrefs, c.n = self.key_bits, self.ncells, self.nrefs, self.n
        return c


@dataclasses.dataclass
class Grid:
    cells: "object"   # torch int32 [ncells + 1], CUDA
    refs: "object"    # torch int32 [nrefs], CUDA
    info: Info


class BatchedGrids:
    """The grids of a batched build: len(), indexing and iteration give one
    Grid per mesh.  `cells` and `refs` are the two library buffers holding
    every mesh's arrays back to back; `cells_offsets` / `refs_offsets` say
    where each mesh's arrays start."""

    def __init__(self, cells, refs, infos, cells_offsets, refs_offsets):
        self.cells, self.refs = cells, refs
        self._infos = infos
        self.cells_offsets = [int(x) for x in cells_offsets]
        self.refs_offsets = [int(x) for x in refs_offsets]
        self._grids = [None] * len(self.cells_offsets)

    def __len__(self):
        return len(self._grids)

    def __getitem__(self, m):
        if isinstance(m, slice):
            return [self[k] for k in range(*m.indices(len(self)))]
        m = int(m)
        if m < 0:
            m += len(self)
        if not 0 <= m < len(self):
            raise IndexError("mesh index out of range")
        if self._grids[m] is None:
            info = Info.from_c(self._infos[m])
            c0, r0 = self.cells_offsets[m], self.refs_offsets[m]
            self._grids[m] = Grid(self.cells[c0:c0 + info.ncells + 1], self.refs[r0:r0 + info.nrefs], info)
        return self._grids[m]

    def __iter__(self):
        return (self[m] for m in range(len(self)))


def plan(lo, hi, n: int, lam: float) -> Info:
    """Grid metadata M (resolution, scale, ncells) from scene bounds (host only)."""
    lib = _lib.load()
    clo = (ctypes.c_float * 3)(*[float(x) for x in lo])
    chi = (ctypes.c_float * 3)(*[float(x) for x in hi])
    info = GridInfo()
    check(lib.grid_plan(clo, chi, int(n), float(lam), ctypes.byref(info)), "grid_plan")
    return Info.from_c(info)


class _LibBuffer:
    """Owns one library-allocated device buffer; exposed to torch through the
    CUDA array interface and released with grid_buf_free when torch drops it."""

    def __init__(self, ctx: "Context", buf: GridBuf):
        self._ctx = ctx
        self._buf = buf
        self.__cuda_array_interface__ = {
            "shape": (int(buf.count),), "typestr": "<i4", "data": (int(buf.ptr), False),
            "version": 3, "strides": None, "stream": None,
        }

    def __del__(self):
        try:
            if self._buf.ptr:
                _lib.load().grid_buf_free(self._ctx._h, ctypes.byref(self._buf))
        except Exception:
            pass


class Context:
    """A grid-builder context on one CUDA device (C: grid_ctx)."""

    PAIR_GEN = {"fused": _lib.GRID_PAIRS_FUSED, "emit": _lib.GRID_PAIRS_EMIT,
                "per_object": _lib.GRID_PAIRS_PER_OBJECT, "regen": _lib.GRID_PAIRS_REGEN}

    TILE_SHAPE = {"256x12": 0, "384x8": 1}

    def __init__(self, device: int = 0, radix_bits: int = 0, pair_gen: str = "fused", cull: bool = False,
                 tile_shape: str = "256x12", local_bits: int = 0):
        """local_bits: how builds finish the sort and the range steps (see
        grid_opts.local_bits): 0 (default) = the hybrid (radix passes over the
        high key bits, then a per-bucket counting sort that also writes the
        cell ranges) at up to 6 pairs per cell, else radix passes over every
        key bit and range extraction; -2 = the hybrid always; 1..11 = the
        hybrid with that many cell bits per bucket; -1 = never."""
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        self._lib = _lib.load()
        opts = GridOpts()
        opts.radix_bits = int(radix_bits)
        opts.pair_gen = self.PAIR_GEN[pair_gen]
        opts.cull = 1 if cull else 0
        opts.tile_shape = self.TILE_SHAPE[tile_shape]
        opts.local_bits = int(local_bits)
        h = ctypes.c_void_p()
        check(self._lib.grid_ctx_create(int(device), ctypes.byref(opts), ctypes.byref(h)), "grid_ctx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.grid_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -------------------------------------------------------------
    def _bind_stream(self):
        # torch's default stream is the legacy default stream (handle 0); it is
        # bound as cudaStreamLegacy, as NULL would select the context's own
        # non-blocking stream, which does not order with torch's work
        s = self._torch.cuda.current_stream(self.device)
        h = s.cuda_stream or _lib.CUDA_STREAM_LEGACY
        check(self._lib.grid_ctx_set_stream(self._h, ctypes.c_void_p(h)), "grid_ctx_set_stream")

    def _dev(self, t, dtype, cols=None):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.device == self.device and t.dtype == dtype
                and t.is_contiguous()):
            t = torch.as_tensor(t).to(device=self.device, dtype=dtype).contiguous()
        if cols is not None and not (t.dim() == 2 and t.shape[1] == cols):
            t = t.reshape(-1, cols)
        return t

    def _wrap(self, buf: GridBuf):
        torch = self._torch
        if not buf.ptr:
            return torch.zeros(int(buf.count), dtype=torch.int32, device=self.device)
        return torch.as_tensor(_LibBuffer(self, buf), device=self.device)

    def autotune(self, verts, tris, lam: float, reps: int = 3) -> dict:
        """Times every radix width (8..11) x pair generation (fused, emit) on
        this mesh, then the other radix-kernel block shape with the best of
        them, then the other end of the sort (per-bucket counting sort or all
        radix passes), and keeps the fastest for later builds (same grid
        either way).  Returns {"radix_bits", "pair_gen", "tile_shape",
        "local_bits", "times_ms": {(bits, mode): ms, "other_shape": ms,
        "other_sort_end": ms}}."""
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        t = self._dev(tris, torch.int32, 3)
        self._bind_stream()
        chosen = GridOpts()
        times = (ctypes.c_double * 10)()
        check(self._lib.grid_ctx_autotune(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], float(lam),
                                          int(reps), ctypes.byref(chosen), times), "grid_ctx_autotune")
        names = {v: k for k, v in self.PAIR_GEN.items()}
        tt = {}
        k = 0
        for rb in range(8, 12):
            for mode in ("fused", "emit"):
                tt[(rb, mode)] = float(times[k])
                k += 1
        tt["other_shape"] = float(times[8])
        tt["other_sort_end"] = float(times[9])
        shapes = {v: k for k, v in self.TILE_SHAPE.items()}
        return {"radix_bits": int(chosen.radix_bits), "pair_gen": names[int(chosen.pair_gen)],
                "tile_shape": shapes[int(chosen.tile_shape)], "local_bits": int(chosen.local_bits),
                "times_ms": tt}

    def _mesh_array(self, meshes):
        torch = self._torch
        keep = []
        arr = (_lib.GridMesh * len(meshes))()
        for m, (verts, tris, lam) in enumerate(meshes):
            v = self._dev(verts, torch.float32, 3)
            t = self._dev(tris, torch.int32, 3)
            keep += [v, t]
            arr[m].verts, arr[m].nverts = v.data_ptr(), v.shape[0]
            arr[m].tris, arr[m].n, arr[m].lam = t.data_ptr(), t.shape[0], float(lam)
        return arr, keep

    def autotune_batched(self, meshes, reps: int = 3) -> dict:
        """Times the batch `meshes` ((verts, tris, lam) each) built as one with
        every radix width (8..11), then the other block shape, then the other
        end of the sort, and keeps the fastest for later builds.  Returns
        {"radix_bits", "tile_shape", "local_bits", "times_ms": {bits: ms,
        "other_shape": ms, "other_sort_end": ms}}."""
        arr, keep = self._mesh_array(meshes)
        self._bind_stream()
        chosen = GridOpts()
        times = (ctypes.c_double * 6)()
        check(self._lib.grid_ctx_autotune_batched(self._h, arr, len(meshes), int(reps), ctypes.byref(chosen), times),
              "grid_ctx_autotune_batched")
        del keep
        tt = {rb: float(times[rb - 8]) for rb in range(8, 12)}
        tt["other_shape"] = float(times[4])
        tt["other_sort_end"] = float(times[5])
        shapes = {v: k for k, v in self.TILE_SHAPE.items()}
        return {"radix_bits": int(chosen.radix_bits), "tile_shape": shapes[int(chosen.tile_shape)],
                "local_bits": int(chosen.local_bits), "times_ms": tt}

    def sort_plan(self, key_bits: int, count: int, ncells: int) -> tuple:
        """(local bits L, radix passes) this context's builds use for
        `count` pairs over `ncells` cells with key_bits-bit keys; L = -1
        when every key bit goes through radix passes."""
        lb, p = ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.grid_ctx_sort_plan(self._h, int(key_bits), int(count), int(ncells), ctypes.byref(lb),
                                           ctypes.byref(p)), "grid_ctx_sort_plan")
        return int(lb.value), int(p.value)

    def counters(self) -> dict:
        """{"fallbacks", "plan_redos"}: builds that took a slower way to the
        same grid (see grid_ctx_counters)."""
        fb, pr = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.grid_ctx_counters(self._h, ctypes.byref(fb), ctypes.byref(pr)), "grid_ctx_counters")
        return {"fallbacks": int(fb.value), "plan_redos": int(pr.value)}

    def profile(self, enable: bool = True) -> None:
        """Per-kernel CUDA-event timing on (clears the statistics)."""
        check(self._lib.grid_ctx_profile(self._h, 1 if enable else 0), "grid_ctx_profile")

    def kernel_stats(self) -> dict:
        """{kernel family: {"launches", "ms", "bytes"}} since the last profile() call."""
        arr = (_lib.GridKernelStat * 32)()
        n = ctypes.c_int()
        check(self._lib.grid_ctx_kernel_stats(self._h, arr, 32, ctypes.byref(n)), "grid_ctx_kernel_stats")
        return {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].total_ms),
                                       "bytes": float(arr[i].bytes)} for i in range(n.value)}

    def mem_in_use(self) -> int:
        v = ctypes.c_int64()
        check(self._lib.grid_ctx_mem_in_use(self._h, ctypes.byref(v)))
        return int(v.value)

    # -- whole build -----------------------------------------------------------
    def build(self, verts, tris, lam: float) -> Grid:
        """BuildParallelGrid on device tensors: verts float32 [nv, 3], tris int32 [n, 3]."""
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        t = self._dev(tris, torch.int32, 3)
        self._bind_stream()
        cb, rb, info = GridBuf(), GridBuf(), GridInfo()
        check(self._lib.grid_build(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], float(lam),
                                   ctypes.byref(cb), ctypes.byref(rb), ctypes.byref(info)), "grid_build")
        return Grid(self._wrap(cb), self._wrap(rb), Info.from_c(info))

    def build_batched(self, meshes) -> "BatchedGrids":
        """BuildParallelGrid of every (verts, tris, lam) in `meshes` at once.
        Returns a sequence with one Grid per mesh whose cells / refs are views
        into two library buffers (bit-identical to building each mesh
        alone); a mesh's views are made when it is first accessed."""
        arr, keep = self._mesh_array(meshes)
        nm = len(meshes)
        infos = (GridInfo * nm)()
        coff = (ctypes.c_int64 * nm)()
        roff = (ctypes.c_int64 * nm)()
        cb, rb = GridBuf(), GridBuf()
        self._bind_stream()
        check(self._lib.grid_build_batched(self._h, arr, nm, ctypes.byref(cb), ctypes.byref(rb), infos, coff, roff),
              "grid_build_batched")
        return BatchedGrids(self._wrap(cb), self._wrap(rb), infos, coff, roff)

    def build_host(self, verts, tris, lam: float, cells_out=None, refs_out=None):
        """The same build from/to host memory (numpy arrays or CPU tensors,
        pinned for asynchronous copies).  Returns (cells, refs, info); the
        output buffers are (re)allocated when missing or too small."""
        torch = self._torch
        v = torch.as_tensor(verts).reshape(-1, 3)
        t = torch.as_tensor(tris).reshape(-1, 3)
        assert v.dtype == torch.float32 and t.dtype == torch.int32 and v.device.type == "cpu"
        v, t = v.contiguous(), t.contiguous()
        info = GridInfo()
        self._bind_stream()

        def call(co, ro):
            cp = co.data_ptr() if co is not None else None
            rp = ro.data_ptr() if ro is not None else None
            return self._lib.grid_build_host(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0],
                                             float(lam), cp, co.numel() if co is not None else 0, rp,
                                             ro.numel() if ro is not None else 0, ctypes.byref(info))

        rc = call(cells_out, refs_out)
        if rc == _lib.GRID_ENOSPC:
            cells_out = torch.empty(int(info.ncells) + 1, dtype=torch.int32)
            refs_out = torch.empty(max(int(info.nrefs), 1), dtype=torch.int32)
            rc = call(cells_out, refs_out)
        check(rc, "grid_build_host")
        nc, nr = int(info.ncells) + 1, int(info.nrefs)
        return cells_out[:nc], refs_out[:nr], Info.from_c(info)

    def jitter(self, verts, sigma: float, seed: int):
        """Per-request vertex jitter of the serving loop (grid_jitter): a new
        float32 [nv, 3] device tensor, verts + sigma-scaled Philox4x32-10
        Irwin-Hall noise for request `seed`."""
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        out = torch.empty_like(v)
        self._bind_stream()
        check(self._lib.grid_jitter(self._h, v.data_ptr(), out.data_ptr(), v.shape[0], float(sigma),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF), "grid_jitter")
        return out

    # -- steps -------------------------------------------------------------------
    def bounds(self, verts, tris):
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        t = self._dev(tris, torch.int32, 3)
        self._bind_stream()
        lo, hi = (ctypes.c_float * 3)(), (ctypes.c_float * 3)()
        check(self._lib.grid_bounds(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], lo, hi),
              "grid_bounds")
        return tuple(lo), tuple(hi)

    def count_scan(self, verts, tris, info: Info):
        """CountCells + ExclusiveSum -> (recs int32 [n, 4] (grid_objrec), nrefs)."""
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        t = self._dev(tris, torch.int32, 3)
        recs = torch.empty((t.shape[0], 4), dtype=torch.int32, device=self.device)
        self._bind_stream()
        nr = ctypes.c_int64()
        ci = info.to_c()
        check(self._lib.grid_count_scan(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0],
                                        ctypes.byref(ci), recs.data_ptr(), ctypes.byref(nr)), "grid_count_scan")
        return recs, int(nr.value)

    def emit_pairs(self, recs, nrefs: int, info: Info):
        """MakeObjectIds .. MakeCellIds -> object-order (C, O)."""
        torch = self._torch
        C = torch.empty(nrefs, dtype=torch.int32, device=self.device)
        O = torch.empty(nrefs, dtype=torch.int32, device=self.device)
        self._bind_stream()
        ci = info.to_c()
        check(self._lib.grid_emit_pairs(self._h, recs.data_ptr(), recs.shape[0], int(nrefs), ctypes.byref(ci),
                                        C.data_ptr(), O.data_ptr()), "grid_emit_pairs")
        return C, O

    def cull_pairs(self, verts, tris, info: Info, recs, nrefs: int):
        """False-intersection culling of the box pairs -> the kept (C, O) in
        object order (int32 device tensors of the kept length)."""
        torch = self._torch
        v = self._dev(verts, torch.float32, 3)
        t = self._dev(tris, torch.int32, 3)
        C = torch.empty(max(nrefs, 1), dtype=torch.int32, device=self.device)
        O = torch.empty(max(nrefs, 1), dtype=torch.int32, device=self.device)
        self._bind_stream()
        ci = info.to_c()
        nk = ctypes.c_int64()
        check(self._lib.grid_cull_pairs(self._h, v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(ci),
                                        recs.data_ptr(), int(nrefs), C.data_ptr(), O.data_ptr(), ctypes.byref(nk)),
              "grid_cull_pairs")
        k = int(nk.value)
        return C[:k], O[:k]

    def emit_pairs_per_object(self, recs, nrefs: int, info: Info):
        """The same object-order (C, O), one thread per object (the sorted
        grid's MakePairs; an ablation)."""
        torch = self._torch
        C = torch.empty(nrefs, dtype=torch.int32, device=self.device)
        O = torch.empty(nrefs, dtype=torch.int32, device=self.device)
        self._bind_stream()
        ci = info.to_c()
        check(self._lib.grid_emit_pairs_per_object(self._h, recs.data_ptr(), recs.shape[0], int(nrefs),
                                                   ctypes.byref(ci), C.data_ptr(), O.data_ptr()),
              "grid_emit_pairs_per_object")
        return C, O

    def sort_pairs(self, C, O, key_bits: int):
        """RadixSort(C, O): stable sort by the low key_bits bits of C."""
        torch = self._torch
        C = self._dev(C, torch.int32)
        O = self._dev(O, torch.int32)
        Co = torch.empty_like(C)
        Oo = torch.empty_like(O)
        self._bind_stream()
        check(self._lib.grid_sort_pairs(self._h, C.data_ptr(), O.data_ptr(), C.numel(), int(key_bits),
                                        Co.data_ptr(), Oo.data_ptr()), "grid_sort_pairs")
        return Co, Oo

    def extract_ranges(self, C_sorted, ncells: int):
        """RunLengthEncode + NonEmptyCells + ExclusiveSum -> cells [ncells + 1]."""
        torch = self._torch
        C = self._dev(C_sorted, torch.int32)
        G = torch.empty(int(ncells) + 1, dtype=torch.int32, device=self.device)
        self._bind_stream()
        check(self._lib.grid_extract_ranges(self._h, C.data_ptr(), C.numel(), int(ncells), G.data_ptr()),
              "grid_extract_ranges")
        return G


class _Lease:
    """Keeps one served result alive: the cells / refs views point into
    server-owned memory, which grid_serve_release frees once the last view is
    dropped (or release() is called)."""

    def __init__(self, server: "Server", ticket: int):
        self._server = server
        self.ticket = ticket
        self.released = False

    def release(self):
        if not self.released:
            self.released = True
            h = getattr(self._server, "_h", None)
            if h:
                self._server._lib.grid_serve_release(h, self.ticket)

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class _View:
    """A non-owning CUDA-array-interface view into a served result."""

    def __init__(self, lease: _Lease, buf: GridBuf):
        self._lease = lease
        self.__cuda_array_interface__ = {
            "shape": (int(buf.count),), "typestr": "<i4", "data": (int(buf.ptr or 0), False),
            "version": 3, "strides": None, "stream": None,
        }


@dataclasses.dataclass
class ServedGrid:
    ticket: int
    cells: "object"   # torch int32 [ncells + 1], CUDA, view into server memory
    refs: "object"    # torch int32 [nrefs], CUDA, view into server memory
    info: Info
    lease: _Lease

    def release(self):
        """Frees the result now; the cells / refs views must not be used after."""
        self.lease.release()


class Server:
    """Rebuild-serving loop (C: grid_server): registered meshes stay resident
    on the device; each request rebuilds one with its own vertex jitter.
    Worker threads with their own streams batch whatever is queued when they
    become free; admission is by a device-memory budget."""

    def __init__(self, device: int = 0, nworkers: int = 0, max_batch: int = 0, batch_pairs: int = 0,
                 hbm_budget: int = 0, radix_bits: int = 0, small_lane: bool = True, small_workers: int = 0,
                 tune_meshes: bool = True):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        self._lib = _lib.load()
        o = GridServeOpts()
        o.nworkers, o.max_batch, o.batch_pairs = int(nworkers), int(max_batch), int(batch_pairs)
        o.hbm_budget, o.radix_bits = int(hbm_budget), int(radix_bits)
        o.arrival_order = 0 if small_lane else 1   # small lane: small requests pass large ones
        o.small_workers = int(small_workers)       # 0: one reserved worker for small requests, -1: none
        o.tune_meshes = 0 if tune_meshes else -1   # autotune each registered mesh for its rebuilds alone
        h = ctypes.c_void_p()
        check(self._lib.grid_serve_create(int(device), ctypes.byref(o), ctypes.byref(h)), "grid_serve_create")
        self._h = h
        self._nverts = {}   # mesh id -> registered vertex count (the size a vertex update must have)

    def close(self):
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            self._lib.grid_serve_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, verts, tris, lam: float) -> int:
        """Copies a mesh (numpy arrays or tensors, host or device) into server
        memory; returns its mesh id."""
        torch = self._torch
        v = torch.as_tensor(verts, dtype=torch.float32).reshape(-1, 3).contiguous()
        t = torch.as_tensor(tris, dtype=torch.int32).reshape(-1, 3).contiguous()
        mid = ctypes.c_int32()
        check(self._lib.grid_serve_register(self._h, v.data_ptr() if v.numel() else None, v.shape[0],
                                            t.data_ptr() if t.numel() else None, t.shape[0], float(lam),
                                            ctypes.byref(mid)), "grid_serve_register")
        self._nverts[int(mid.value)] = int(v.shape[0])
        return int(mid.value)

    def submit(self, mesh_id: int, sigma: float = 0.0, seed: int = 0, verts=None):
        """Queues a rebuild; returns its ticket, or None when admission refuses.
        verts: the mesh's new vertex positions for this request (float32
        [nverts, 3]; a numpy array or a host or CUDA tensor), copied before
        the call returns; None rebuilds the registered vertices.  sigma and
        seed jitter the request's vertices on the device (sigma 0: none)."""
        tk = ctypes.c_uint64()
        keep = None
        ptr = None
        if verts is not None:
            torch = self._torch
            keep = verts if isinstance(verts, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(verts))
            if keep.dtype != torch.float32 or not keep.is_contiguous() or keep.dim() != 2 or keep.shape[1] != 3:
                raise ValueError("verts must be a contiguous float32 [nverts, 3] array")
            nv = self._nverts.get(int(mesh_id))   # unknown ids are left to the C call (GRID_EINVAL)
            if nv is not None and keep.shape[0] != nv:
                raise ValueError("verts must have the registered mesh's vertex count")
            if keep.is_cuda:   # the server's copy does not wait on torch's streams
                torch.cuda.current_stream(keep.device).synchronize()
            ptr = keep.data_ptr() if keep.numel() else None
        rc = self._lib.grid_serve_submit(self._h, int(mesh_id), ptr, float(sigma), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                         ctypes.byref(tk))
        del keep
        if rc == _lib.GRID_EAGAIN:
            return None
        check(rc, "grid_serve_submit")
        return int(tk.value)

    def _result(self, ticket, cb, rb, info) -> ServedGrid:
        torch = self._torch
        lease = _Lease(self, ticket)

        def view(b):
            if not b.ptr or b.count == 0:
                return torch.zeros(int(b.count), dtype=torch.int32, device=self.device)
            return torch.as_tensor(_View(lease, b), device=self.device)
        return ServedGrid(ticket, view(cb), view(rb), Info.from_c(info), lease)

    def poll(self, ticket: int):
        """The finished result, or None while the request is queued or running."""
        cb, rb, info = GridBuf(), GridBuf(), GridInfo()
        rc = self._lib.grid_serve_poll(self._h, int(ticket), ctypes.byref(cb), ctypes.byref(rb),
                                       ctypes.byref(info))
        if rc == _lib.GRID_ENOTREADY:
            return None
        check(rc, "grid_serve_poll")
        return self._result(int(ticket), cb, rb, info)

    def wait(self, ticket: int, timeout: float | None = None) -> ServedGrid:
        """Waits for a request (timeout in seconds; None = no limit)."""
        cb, rb, info = GridBuf(), GridBuf(), GridInfo()
        us = -1 if timeout is None else int(timeout * 1e6)
        check(self._lib.grid_serve_wait(self._h, int(ticket), us, ctypes.byref(cb), ctypes.byref(rb),
                                        ctypes.byref(info)), "grid_serve_wait")
        return self._result(int(ticket), cb, rb, info)

    def release(self, ticket: int) -> int:
        """Frees a finished request without waiting for its views (returns the C status)."""
        return int(self._lib.grid_serve_release(self._h, int(ticket)))

    def stats(self, reset: bool = False) -> dict:
        st = GridServeStats()
        check(self._lib.grid_serve_get_stats(self._h, ctypes.byref(st), 1 if reset else 0), "grid_serve_get_stats")
        return {name: getattr(st, name) for name, _ in GridServeStats._fields_}
