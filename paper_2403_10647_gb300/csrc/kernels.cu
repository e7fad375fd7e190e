// CUDA kernels (sm_103a) of the parallel uniform-grid construction
// (Costa, Pereira, Jorge, "Building An Efficient Grid On GPU", Algorithm 1).
//
//   bounds_kernel        boxes of Algorithm 1: per-triangle AABB, block-reduced
//                        scene bounds, index / finiteness checks.
//   count_scan_kernel    CountCells + ExclusiveSum: per-object cell box and cell
//                        count V, single-pass decoupled look-back scan -> start
//                        offsets and NO.
//   tile_search_kernel   first object of every pair tile (binary search).
//   emit_kernel          MakeObjectIds + InclusiveSum (as a max-scan of object
//                        start marks) + SegmentedExclusiveSum (rid = j - start)
//                        + MakeCellIds (GlobalCoords): the object-order lists.
//   upsweep_kernel       per-tile digit counts of one RadixSort pass, prefixed
//                        across groups of tiles by a decoupled look-back; the
//                        last group turns its prefixes into the pass's digit
//                        starts.  The first pass generates its pairs (the emit
//                        steps above) instead of reading them and stores them
//                        once for its downsweep.
//   downsweep_kernel     one stable LSD radix-sort pass (RadixSort of Algorithm
//                        1): warp multisplit ranking, shared-memory staged,
//                        coalesced scatter.
//   extract_split_kernel, extract_kernel
//                        RunLengthEncode + NonEmptyCells + ExclusiveSum fused as
//                        a merge path of the sorted keys against the cell ids.
//   cull_emit_kernel     culling mode (the triangle/cell test Sec. 6 leaves as
//                        future work): regenerates each tile's box pairs,
//                        tests them, compacts the kept ones in object order.
//   bounds_batched_kernel, localize_kernel
//                        the same method over a batch of meshes flattened into
//                        one problem.
//   wait_selftest_kernel the radix sort's bounded look-back run against a
//                        predecessor that never publishes (failure detection).
// The radix kernels are built for two block shapes (256 x 12 and 384 x 8
// pairs per 3,072-pair tile) and for digits of 8 to 11 bits.
#include <atomic>
#include <cstdint>
#include <cstdio>

#include "device.cuh"
#include "kernels.h"

namespace gg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ unsigned warp_incl_max(unsigned v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = max(v, u);
    }
    return v;
}

// Exclusive block-wide sum of one value per thread; s_tmp holds BLOCK/32
// entries.  Returns the exclusive prefix, writes the block total to *total.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_excl_sum(T v, T *s_tmp, T *total)
{
    constexpr int W = BLOCK / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_sum(v);
    if (lane == 31) s_tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        T x = lane < W ? s_tmp[lane] : T(0);
        x = warp_incl_sum(x);
        if (lane < W) s_tmp[lane] = x;
    }
    __syncthreads();
    T wex = w ? s_tmp[w - 1] : T(0);
    *total = s_tmp[W - 1];
    __syncthreads();
    return wex + inc - v;
}

// Shared-memory index with one pad word per 32: rows written in blocked
// arrangement (thread t at t * ITEMS + i) and read warp-striped both hit 32
// distinct banks.
__device__ __forceinline__ unsigned pad32(unsigned e) { return e + (e >> 5); }

template <int T>
__host__ __device__ constexpr int padded() { return T + T / 32; }

// MakeObjectIds + InclusiveSum for one pair tile, in shared memory: marks
// each object whose pair segment starts inside [j0, j0 + cnt) at its start
// position with its tile-local index, then an inclusive max-scan carries the
// owning object forward.  Afterwards om[i] + (returned first object) is the
// object of the thread's pair j0 + tid * ITEMS + i.  mark holds padded<T>()
// entries and must be zero on entry (zero_marks, once per block); every
// thread clears the entries it reads, so it is zero again on return and the
// next tile needs no clearing pass.  s_tmp holds BLOCK / 32 entries.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ void zero_marks(unsigned *mark)
{
    for (int p = threadIdx.x; p < padded<BLOCK * ITEMS>(); p += BLOCK) mark[p] = 0u;
}

template <int BLOCK, int ITEMS>
__device__ __forceinline__ unsigned tile_objects(const ObjRec *__restrict__ recs,
                                                 const unsigned *__restrict__ tile_obj, unsigned t,
                                                 unsigned j0, unsigned cnt, unsigned *mark,
                                                 unsigned *s_tmp, unsigned (&om)[ITEMS])
{
    constexpr int W = BLOCK / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned of = tile_obj[t], ol = tile_obj[t + 1];
    for (unsigned o = of + 1u + tid; o <= ol; o += BLOCK) {
        const unsigned s = __ldg(&recs[o].start);
        const unsigned p = s - j0;
        if (s >= j0 && p < cnt) mark[pad32(p)] = o - of;
    }
    __syncthreads();
    unsigned m = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = pad32(tid * ITEMS + i);
        m = max(m, mark[e]);
        mark[e] = 0u;
        om[i] = m;
    }
    const unsigned inc = warp_incl_max(m);
    if (lane == 31) s_tmp[w] = inc;
    __syncthreads();
    unsigned prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) prev = 0u;
#pragma unroll
    for (int ww = 0; ww < W - 1; ++ww)
        if (ww < w) prev = max(prev, s_tmp[ww]);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) om[i] = max(om[i], prev);
    return of;
}

// Batched builds: the mesh owning object o (largest m with obj_base[m] <= o;
// empty meshes own no object).
__device__ __forceinline__ int mesh_of(const MeshTab &mt, long long o)
{
    int lo = 0, hi = mt.nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(mt.obj_base + mid) <= o)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// SegmentedExclusiveSum + MakeCellIds (GlobalCoords, Sec. 3) for the ITEMS
// consecutive pairs e = tid * ITEMS + i of a tile (blocked arrangement).  The
// relative offset rid = j - start is decomposed with divisions only for the
// thread's first pair: inside a thread's run the pairs of one object are
// consecutive, and a pair whose object differs from its predecessor's is that
// object's first pair (rid = 0), so every other pair advances (x, y, z) by one
// step, x fastest.
// In a batched build (mt.md set) each object's mesh supplies the grid
// strides, the key offset cell_base and the object-id offset.
template <int ITEMS>
__device__ __forceinline__ void gen_blocked(const ObjRec *__restrict__ recs, unsigned of, const unsigned (&om)[ITEMS],
                                            unsigned j0, unsigned cnt, unsigned res_x, unsigned res_y,
                                            const MeshTab &mt, unsigned (&keys)[ITEMS], unsigned (&objs)[ITEMS])
{
    const unsigned e0 = threadIdx.x * ITEMS;
    unsigned o = 0u, x = 0u, y = 0u, z = 0u, mx = 1u, my = 1u, lox = 0u, loy = 0u, loz = 0u;
    unsigned rx = res_x, ry = res_y, kbase = 0u, obase = 0u;
    unsigned key = 0u, dy = 0u, dz = 0u;   // the current key and its steps to the next row and slab
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = e0 + i;
        keys[i] = 0u;
        objs[i] = 0u;
        if (e < cnt) {
            const unsigned oe = of + om[i];
            if (i == 0 || oe != o) {
                o = oe;
                const uint4 r = __ldg(reinterpret_cast<const uint4 *>(recs) + o);
                lox = r.x & 0xFFFFu;
                loy = r.x >> 16;
                loz = r.y & 0xFFFFu;
                mx = (r.y >> 16) - lox + 1u;
                my = (r.z & 0xFFFFu) - loy + 1u;
                if (mt.md) {
                    const int m = mesh_of(mt, o);
                    rx = (unsigned)__ldg(&mt.md[m].res[0]);
                    ry = (unsigned)__ldg(&mt.md[m].res[1]);
                    kbase = __ldg(&mt.md[m].cell_base);
                    obase = (unsigned)__ldg(mt.obj_base + m);
                }
                if (i == 0) {
                    const unsigned rid = j0 + e - r.w;
                    const unsigned mxy = mx * my;
                    z = rid / mxy;
                    const unsigned rem = rid - z * mxy;
                    y = rem / mx;
                    x = rem - y * mx;
                } else {
                    x = y = z = 0u;
                }
                key = kbase + (lox + x) + rx * ((loy + y) + ry * (loz + z));
                dy = rx - (mx - 1u);                    // from a row's last cell to the next row's first
                dz = rx * ry - (my - 1u) * rx - (mx - 1u);   // from a slab's last cell to the next slab's first
            } else if (++x == mx) {
                x = 0u;
                if (++y == my) {
                    y = 0u;
                    key += dz;
                } else {
                    key += dy;
                }
            } else {
                ++key;
            }
            keys[i] = key;
            objs[i] = o - obase;
        }
    }
}

// ---------------------------------------------------------------------------
// a0: boxes + scene bounds
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) bounds_kernel(const float *__restrict__ verts, long long nverts,
                                                     const int *__restrict__ tris, long long n,
                                                     Ctl *ctl)
{
    float lo[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
    float hi[3] = {-lo[0], -lo[1], -lo[2]};
    unsigned err = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int vi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) vi[k] = __ldg(tris + 3 * i + k);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (vi[k] < 0 || (long long)vi[k] >= nverts) {
                err |= ERR_BADINDEX;
                continue;
            }
            const float *p = verts + 3ll * vi[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float x = __ldg(p + a);
                if (!isfinite(x)) {
                    err |= ERR_NONFINITE;
                } else {
                    lo[a] = fminf(lo[a], x);
                    hi[a] = fmaxf(hi[a], x);
                }
            }
        }
    }
    __shared__ unsigned s_lo[3], s_hi[3], s_err;
    if (threadIdx.x < 3) {
        s_lo[threadIdx.x] = 0u;
        s_hi[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) s_err = 0u;
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMax(&s_lo[a], ~float_to_ordered(lo[a]));
            atomicMax(&s_hi[a], float_to_ordered(hi[a]));
        }
        if (err) atomicOr(&s_err, err);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMax(&ctl->lo_inv[threadIdx.x], s_lo[threadIdx.x]);
        atomicMax(&ctl->hi_ord[threadIdx.x], s_hi[threadIdx.x]);
    }
    if (threadIdx.x == 0 && s_err) atomicOr(&ctl->err, s_err);
}

// ---------------------------------------------------------------------------
// a2 + a3: CountCells + ExclusiveSum (single pass, decoupled look-back)
// ---------------------------------------------------------------------------

constexpr unsigned long long LB64_AGG = 1ull << 62;
constexpr unsigned long long LB64_PREFIX = 2ull << 62;
constexpr unsigned long long LB64_VALUE = (1ull << 62) - 1ull;

// Decoupled look-back of tile t over 64-bit status words (flag | value), run
// by one whole warp: publishes t's aggregate, reads 32 predecessors per round
// trip (lane q reads tile k - q), adds every aggregate up to the nearest
// inclusive prefix, then publishes t's own inclusive prefix.  A word not yet
// published ahead of that prefix means polling the window again, at most
// SPIN_LIMIT times (then ERR_TIMEOUT and the partial sum).  Returns the
// exclusive prefix in every lane.
__device__ __forceinline__ unsigned long long warp_lookback64(unsigned long long *st, unsigned t,
                                                              unsigned long long total, Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    unsigned long long excl = 0;
    if (t == 0) {
        if (lane == 0) st_relaxed_u64(&st[0], LB64_PREFIX | total);
        return 0ull;
    }
    if (lane == 0) st_relaxed_u64(&st[t], LB64_AGG | total);
    long long k = (long long)t - 1;
    unsigned spins = 0;
    while (true) {
        const long long idx = k - lane;
        const unsigned long long v = idx >= 0 ? ld_relaxed_u64(&st[idx]) : LB64_PREFIX;
        const unsigned pre = __ballot_sync(0xffffffffu, (v & LB64_PREFIX) != 0ull);
        const unsigned zero = __ballot_sync(0xffffffffu, v == 0ull);
        const int p = pre ? __ffs(pre) - 1 : 32;                // nearest prefix in the window
        const unsigned upto = p < 31 ? (2u << p) - 1u : 0xffffffffu;
        if (zero & upto) {                                       // a nearer tile has not published
            if (++spins > SPIN_LIMIT) {
                if (lane == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
                break;
            }
            if (spins > 8) __nanosleep(64);
            continue;
        }
        unsigned long long part = lane <= p ? (v & LB64_VALUE) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        excl += part;
        if (p < 32) break;
        k -= 32;
    }
    if (lane == 0) st_relaxed_u64(&st[t], LB64_PREFIX | ((excl + total) & LB64_VALUE));
    return excl;
}

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK, COUNT_MIN_BLOCKS) count_scan_kernel(CountArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    __shared__ unsigned long long s_pref[T];
    __shared__ unsigned long long s_tmp[BLOCK / 32];
    __shared__ unsigned s_tile;
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(&a.ctl->tickets[0], 1u);
    if (a.device_plan) {   // the plan kernel's M, in place of the host's
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            a.lo[ax] = a.ctl->plan_lo[ax];
            a.scale[ax] = a.ctl->plan_scale[ax];
            a.res[ax] = a.ctl->plan_res[ax];
        }
    }
    __syncthreads();
    const unsigned tile = s_tile;
    const long long base = (long long)tile * T;

#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const long long o = base + i * BLOCK + tid;
        unsigned V = 0u;
        if (o < a.n) {
            // the triangle and the grid it maps into: the single mesh's, or
            // in a batched build the owning mesh's
            const int *tris = a.tris;
            const float *verts = a.verts;
            long long nverts = a.nverts, lo_obj = o;
            float glo[3] = {a.lo[0], a.lo[1], a.lo[2]}, gsc[3] = {a.scale[0], a.scale[1], a.scale[2]};
            int gres[3] = {a.res[0], a.res[1], a.res[2]};
            if (a.mt.md) {
                const int m = mesh_of(a.mt, o);
                const MeshDesc &md = a.mt.md[m];
                tris = md.tris;
                verts = md.verts;
                nverts = md.nverts;
                lo_obj = o - __ldg(a.mt.obj_base + m);
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    glo[ax] = md.lo[ax];
                    gsc[ax] = md.scale[ax];
                    gres[ax] = md.res[ax];
                }
            }
            int vi[3];
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vi[k] = __ldg(tris + 3 * lo_obj + k);
                ok = ok && vi[k] >= 0 && (long long)vi[k] < nverts;
            }
            if (!ok) {  // never read outside verts: flag and use vertex 0
                atomicOr(&a.ctl->err, ERR_BADINDEX);
                vi[0] = vi[1] = vi[2] = 0;
            }
            unsigned clo[3], chi[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float p0 = __ldg(verts + 3ll * vi[0] + ax);
                const float p1 = __ldg(verts + 3ll * vi[1] + ax);
                const float p2 = __ldg(verts + 3ll * vi[2] + ax);
                const float bl = fminf(fminf(p0, p1), p2);
                const float bh = fmaxf(fmaxf(p0, p1), p2);
                clo[ax] = (unsigned)cell_coord(bl, glo[ax], gsc[ax], gres[ax]);
                chi[ax] = (unsigned)cell_coord(bh, glo[ax], gsc[ax], gres[ax]);
            }
            unsigned long long cnt = (unsigned long long)(chi[0] - clo[0] + 1u) *
                                     (unsigned long long)(chi[1] - clo[1] + 1u) *
                                     (unsigned long long)(chi[2] - clo[2] + 1u);
            V = cnt > 0x80000000ull ? 0x80000000u : (unsigned)cnt;
            // the box now, the pair offset once the scan has it: nothing
            // of the record stays live across the scan
            reinterpret_cast<uint4 *>(a.recs)[o] =
                make_uint4(clo[0] | (clo[1] << 16), clo[2] | (chi[0] << 16), chi[1] | (chi[2] << 16), 0u);
        }
        s_pref[i * BLOCK + tid] = V;
    }
    __syncthreads();
    unsigned long long run = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned long long v = s_pref[tid * ITEMS + i];
        s_pref[tid * ITEMS + i] = run;
        run += v;
    }
    unsigned long long total;
    const unsigned long long texcl = block_excl_sum<BLOCK>(run, s_tmp, &total);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) s_pref[tid * ITEMS + i] += texcl;

    if (tid < 32) {
        const unsigned long long excl = warp_lookback64(a.status, tile, total, a.ctl);
        if (tid == 0) {
            s_excl = excl;
            if (excl + total > 0x7FFFFFFFull) atomicOr(&a.ctl->err, ERR_OVERFLOW);
            if (base + T >= a.n) a.ctl->nrefs = excl + total;
        }
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
    bool tile_redo = false;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int p = i * BLOCK + tid;
        const long long o = base + p;
        if (o < a.n) {
            const unsigned start = (unsigned)(excl + s_pref[p]);
            a.recs[o].start = start;
            if (a.mt.md) {
                const int m = mesh_of(a.mt, o);
                if (__ldg(a.mt.obj_base + m) == o) a.pair_base[m] = start;
            }
            if (a.tile_obj && excl + total <= 0x7FFFFFFFull) {
                // the pair tiles whose first pair is one of this object's
                // [start, end): tile_search's answer, recorded here
                const unsigned end = (unsigned)(excl + (p + 1 < T ? s_pref[p + 1] : total));
                const unsigned t0 = (start + (unsigned)PAIR_TILE - 1u) / (unsigned)PAIR_TILE;
                const unsigned tl = (end - 1u) / (unsigned)PAIR_TILE + 1u;   // tiles t0 .. tl - 1 (end > start)
                if (tl <= a.tile_cap && tl - t0 <= 64u) {
                    for (unsigned t = t0; t < tl; ++t) a.tile_obj[t] = (unsigned)o;
                } else if (tl > t0) {
                    tile_redo = true;
                }
                if (o == a.n - 1) {   // the entry after the last tile
                    const unsigned nt = (end + (unsigned)PAIR_TILE - 1u) / (unsigned)PAIR_TILE;
                    if (nt < a.tile_cap) a.tile_obj[nt] = (unsigned)o; else tile_redo = true;
                }
            }
        }
    }
    if (tile_redo) atomicOr(&a.ctl->err, ERR_TILE_REDO);
}

// ---------------------------------------------------------------------------
// a1 on the device: grid metadata M from the bounds
// ---------------------------------------------------------------------------

__global__ void plan_kernel(Ctl *ctl, long long n, float lambda)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3], e[3];
    int res[3] = {1, 1, 1};
    float scale[3] = {0.0f, 0.0f, 0.0f};
    const bool ok = ctl->err == 0u && n > 0;
    int d = 0;
    double vol = 1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // the bounds as the host reads them: a zero bound is +0.0
        lo[a] = ok ? __fadd_rn(ordered_to_float(~ctl->lo_inv[a]), 0.0f) : 0.0f;
        const float hi = ok ? __fadd_rn(ordered_to_float(ctl->hi_ord[a]), 0.0f) : 0.0f;
        e[a] = __fsub_rn(hi, lo[a]);
        if (ok && e[a] > 0.0f) {
            ++d;
            vol = __dmul_rn(vol, (double)e[a]);
        }
    }
    if (d > 0) {
        const double q = __ddiv_rn(__dmul_rn((double)lambda, (double)n), vol);
        const double k = d == 3 ? cbrt(q) : (d == 2 ? __dsqrt_rn(q) : q);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!(e[a] > 0.0f)) continue;
            double r = ceil(__dmul_rn((double)e[a], k));
            if (!(r >= 1.0)) r = 1.0;
            if (r > 65535.0) r = 65535.0;
            res[a] = (int)r;
            scale[a] = __fdiv_rn((float)res[a], e[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ctl->plan_lo[a] = lo[a];
        ctl->plan_scale[a] = scale[a];
        ctl->plan_res[a] = res[a];
    }
}

cudaError_t launch_plan(Ctl *ctl, long long n, float lambda, cudaStream_t s)
{
    plan_kernel<<<1, 32, 0, s>>>(ctl, n, lambda);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pair tiles: first object of each tile
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) tile_search_kernel(const ObjRec *__restrict__ recs, long long n,
                                                          unsigned tile, unsigned ntiles,
                                                          unsigned *__restrict__ tile_obj)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    if (t == ntiles) {
        tile_obj[t] = (unsigned)(n - 1);
        return;
    }
    const unsigned j = t * tile;
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (__ldg(&recs[mid].start) <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    tile_obj[t] = (unsigned)lo;
}

// ---------------------------------------------------------------------------
// a4 - a7: object-order pairs (C, O), one thread per pair
// ---------------------------------------------------------------------------

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) emit_kernel(EmitArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_mark = smem;                 // [padded T]
    unsigned *s_obj = smem + padded<T>();    // [padded T]
    __shared__ unsigned s_tmp[BLOCK / 32];
    const unsigned t = blockIdx.x;
    const unsigned j0 = t * (unsigned)T;
    const unsigned cnt = min((unsigned)T, a.count - j0);
    zero_marks<BLOCK, ITEMS>(s_mark);
    __syncthreads();
    unsigned om[ITEMS];
    const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, t, j0, cnt, s_mark, s_tmp, om);
    unsigned keys[ITEMS], objs[ITEMS];
    gen_blocked<ITEMS>(a.recs, of, om, j0, cnt, a.res_x, a.res_y, a.mt, keys, objs);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = threadIdx.x * ITEMS + i;
        s_mark[pad32(e)] = keys[i];
        s_obj[pad32(e)] = objs[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = i * BLOCK + threadIdx.x;
        if (e < cnt) {
            a.C[j0 + e] = s_mark[pad32(e)];
            a.O[j0 + e] = s_obj[pad32(e)];
        }
    }
}

// ---------------------------------------------------------------------------
// False-intersection culling (the overlap test ahead of the sort that Sec. 6
// leaves as future work): each box pair is tested, the kept ones are written
// compacted, in object order.
// ---------------------------------------------------------------------------

// A triangle in grid space: vertices q (q[3k + a]), edges e_0 = q_1 - q_0,
// e_1 = q_2 - q_1, e_2 = q_0 - q_2 and the normal n = e_0 x e_1.
struct GridTri {
    float q[9];
    float e[9];
    float n[3];
};

// Grid coordinates q = min((v - lo) * scale, res): the cell mapping's two
// FP32 operations and its clamp to the grid's far face (the FP32 scale can put
// the far face's vertices a rounding error beyond res).
__device__ __forceinline__ void grid_tri(const float *__restrict__ verts, long long nverts,
                                         const int *__restrict__ tris, unsigned o, const float (&lo)[3],
                                         const float (&scale)[3], const float (&resf)[3], GridTri &t, Ctl *ctl)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int vi = __ldg(tris + 3ll * o + k);
        if (vi < 0 || (long long)vi >= nverts) {   // never read outside verts: flag and use vertex 0
            atomicOr(&ctl->err, ERR_BADINDEX);
            vi = 0;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            t.q[3 * k + a] = fminf(__fmul_rn(__fsub_rn(__ldg(verts + 3ll * vi + a), lo[a]), scale[a]), resf[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t.e[a] = __fsub_rn(t.q[3 + a], t.q[a]);
        t.e[3 + a] = __fsub_rn(t.q[6 + a], t.q[3 + a]);
        t.e[6 + a] = __fsub_rn(t.q[a], t.q[6 + a]);
    }
    t.n[0] = __fsub_rn(__fmul_rn(t.e[1], t.e[5]), __fmul_rn(t.e[2], t.e[4]));
    t.n[1] = __fsub_rn(__fmul_rn(t.e[2], t.e[3]), __fmul_rn(t.e[0], t.e[5]));
    t.n[2] = __fsub_rn(__fmul_rn(t.e[0], t.e[4]), __fmul_rn(t.e[1], t.e[3]));
}

// One separating axis a against the cell: projections of the local vertices
// w, box radius S / 2 widened by the slack S t.  Each product and sum is one
// round-to-nearest FP32 operation in a fixed order, so the decision is the
// same on every IEEE machine.
__device__ __forceinline__ bool axis_separates(float a0, float a1, float a2, const float (&w)[9], float t)
{
    float pmin = 0.0f, pmax = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float p = __fadd_rn(__fmul_rn(a0, w[3 * k]), __fmul_rn(a1, w[3 * k + 1]));
        p = __fadd_rn(p, __fmul_rn(a2, w[3 * k + 2]));
        pmin = k == 0 ? p : fminf(pmin, p);
        pmax = k == 0 ? p : fmaxf(pmax, p);
    }
    const float S = __fadd_rn(__fadd_rn(fabsf(a0), fabsf(a1)), fabsf(a2));
    const float R = __fadd_rn(__fmul_rn(0.5f, S), __fmul_rn(S, t));
    return pmin > R || pmax < -R;
}

// Axes that can separate a cell of the triangle's cell box: bit 0 the
// normal, bit 1 + 3 j + f the f-th cross product with edge j.  An axis with
// at most one non-zero component is parallel to a coordinate axis; along it
// the triangle's extent meets the cell's (the cell lies in the box), so the
// vertex projections nearest the cell stay within S / 2 of its centre
// (rounding included) while the test needs them beyond S / 2 + S t: such an
// axis never separates and is skipped without changing any decision.
__device__ __forceinline__ unsigned live_axes(const GridTri &t)
{
    auto two = [](float a, float b, float c) {
        return (a != 0.0f ? 1 : 0) + (b != 0.0f ? 1 : 0) + (c != 0.0f ? 1 : 0) >= 2;
    };
    unsigned m = two(t.n[0], t.n[1], t.n[2]) ? 1u : 0u;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ex = t.e[3 * j], ey = t.e[3 * j + 1], ez = t.e[3 * j + 2];
        if (ez != 0.0f && ey != 0.0f) m |= 2u << (3 * j);
        if (ez != 0.0f && ex != 0.0f) m |= 4u << (3 * j);
        if (ey != 0.0f && ex != 0.0f) m |= 8u << (3 * j);
    }
    return m;
}

// The culling test: is triangle t separated from cell (x, y, z), the closed
// unit cube centred at (x, y, z) + 1/2?  Axes: the normal, then unit x e for
// every edge (those of `live` only); slack t = max|w| 2^-16 + 2^-10 (bounds
// the rounding error of the projections from above by a wide margin: a
// touching cell is never rejected).
__device__ __forceinline__ bool tri_cell_separated(const GridTri &t, unsigned live, unsigned x, unsigned y,
                                                   unsigned z)
{
    const float c[3] = {__fadd_rn(__uint2float_rn(x), 0.5f), __fadd_rn(__uint2float_rn(y), 0.5f),
                        __fadd_rn(__uint2float_rn(z), 0.5f)};
    float w[9];
    float W = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            w[3 * k + a] = __fsub_rn(t.q[3 * k + a], c[a]);
            W = fmaxf(W, fabsf(w[3 * k + a]));
        }
    const float slack = __fadd_rn(__fmul_rn(W, 1.52587890625e-05f), 9.765625e-04f);   // 2^-16, 2^-10
    if ((live & 1u) && axis_separates(t.n[0], t.n[1], t.n[2], w, slack)) return true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float ex = t.e[3 * j], ey = t.e[3 * j + 1], ez = t.e[3 * j + 2];
        if (((live >> (3 * j)) & 2u) && axis_separates(0.0f, -ez, ey, w, slack)) return true;
        if (((live >> (3 * j)) & 4u) && axis_separates(ez, 0.0f, -ex, w, slack)) return true;
        if (((live >> (3 * j)) & 8u) && axis_separates(-ey, ex, 0.0f, w, slack)) return true;
    }
    return false;
}

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) cull_emit_kernel(CullArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_mark = smem;                     // [padded T]: object marks, then the tile's keys
    unsigned *s_obj = smem + padded<T>();        // [padded T]: the tile's objects
    unsigned *s_okey = smem + 2 * padded<T>();   // [padded T]: kept keys, compacted
    unsigned *s_oobj = smem + 3 * padded<T>();   // [padded T]: kept objects, compacted
    __shared__ unsigned s_tmp[BLOCK / 32];
    __shared__ unsigned s_tile;
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x;
    // tiles in ticket order, so every tile a look-back waits for has started
    if (tid == 0) s_tile = atomicAdd(&a.ctl->tickets[7], 1u);
    __syncthreads();
    const unsigned t = s_tile;
    const unsigned ntiles = (a.count + T - 1) / T;
    const unsigned j0 = t * (unsigned)T;
    const unsigned cnt = min((unsigned)T, a.count - j0);
    zero_marks<BLOCK, ITEMS>(s_mark);
    __syncthreads();
    {
        unsigned om[ITEMS], keys[ITEMS], objs[ITEMS];
        const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, t, j0, cnt, s_mark, s_tmp, om);
        gen_blocked<ITEMS>(a.recs, of, om, j0, cnt, a.res_x, a.res_y, MeshTab{}, keys, objs);
        __syncthreads();   // every thread is done with the object marks
        // the thread's own items go to shared memory: the test loop below is
        // not unrolled (one copy of the test) and no item stays in registers
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            s_mark[pad32(tid * ITEMS + i)] = keys[i];
            s_obj[pad32(tid * ITEMS + i)] = objs[i];
        }
    }
    const float lo[3] = {a.lo[0], a.lo[1], a.lo[2]}, scale[3] = {a.scale[0], a.scale[1], a.scale[2]};
    const float resf[3] = {a.res_f[0], a.res_f[1], a.res_f[2]};
    // The thread's items are consecutive pairs: inside one object the cell
    // steps through the box, x fastest (GlobalCoords), so coordinates are
    // stepped, not divided out of the key.  Two exact shortcuts skip the
    // test: a cell holding a vertex of the triangle is always kept (each
    // vertex projection nearest the cell lies within S / 2 of its centre),
    // and so is every cell of a box of at most two cells (each holds a vertex).
    GridTri tri;
    unsigned cur = 0xFFFFFFFFu, mask = 0u, live = 0u;
    unsigned x = 0, y = 0, z = 0, lox = 0, loy = 0, hix = 0, hiy = 0;
    unsigned long long vc[3] = {0ull, 0ull, 0ull};   // the vertices' cells, x | y << 16 | z << 32
    bool small = true;
#pragma unroll 1
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = tid * ITEMS + i;
        if (e >= cnt) break;
        const unsigned o = s_obj[pad32(e)];
        if (o != cur) {
            cur = o;
            const uint4 r = __ldg(reinterpret_cast<const uint4 *>(a.recs) + o);
            lox = r.x & 0xFFFFu;
            loy = r.x >> 16;
            const unsigned loz = r.y & 0xFFFFu;
            hix = r.y >> 16;
            hiy = r.z & 0xFFFFu;
            const unsigned hiz = r.z >> 16;
            const unsigned mx = hix - lox + 1u, my = hiy - loy + 1u, mz = hiz - loz + 1u;
            if (i > 0) {   // an object that starts inside the thread's run starts at its first cell
                x = lox;
                y = loy;
                z = loz;
            } else {       // the thread's first pair may lie anywhere inside its object
                const unsigned rid = j0 + e - r.w;
                const unsigned mxy = mx * my;
                const unsigned zz = rid / mxy, rem = rid - zz * mxy;
                const unsigned yy = rem / mx;
                x = lox + (rem - yy * mx);
                y = loy + yy;
                z = loz + zz;
            }
            small = (unsigned long long)mx * my * mz <= 2ull;
            if (!small) {
                grid_tri(a.verts, a.nverts, a.tris, o, lo, scale, resf, tri, a.ctl);
                live = live_axes(tri);
                const unsigned bl[3] = {lox, loy, loz}, bh[3] = {hix, hiy, hiz};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    unsigned long long key = 0ull;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        // the vertex's cell: floor of its (clamped) grid
                        // coordinate, into the box as the cell mapping
                        // clamps it; the vertex lies in that closed cell
                        const float f = floorf(tri.q[3 * k + ax]);
                        const unsigned cc = f <= (float)bl[ax] ? bl[ax] : (f >= (float)bh[ax] ? bh[ax] : (unsigned)f);
                        key |= (unsigned long long)cc << (16 * ax);
                    }
                    vc[k] = key;
                }
            }
        } else if (++x > hix) {
            x = lox;
            if (++y > hiy) {
                y = loy;
                ++z;
            }
        }
        bool keep = small;
        if (!keep) {
            const unsigned long long rc =
                (unsigned long long)x | ((unsigned long long)y << 16) | ((unsigned long long)z << 32);
            keep = rc == vc[0] || rc == vc[1] || rc == vc[2];
        }
        if (!keep) keep = !tri_cell_separated(tri, live, x, y, z);
        if (keep) mask |= 1u << i;
    }
    unsigned total;
    unsigned pos = block_excl_sum<BLOCK>((unsigned)__popc(mask), s_tmp, &total);
#pragma unroll 1
    for (int i = 0; i < ITEMS; ++i) {
        if ((mask >> i) & 1u) {
            const unsigned e = pad32(tid * ITEMS + i);
            s_okey[pad32(pos)] = s_mark[e];
            s_oobj[pad32(pos)] = s_obj[e];
            ++pos;
        }
    }
    if (tid < 32) {
        const unsigned long long excl = warp_lookback64(a.status, t, total, a.ctl);
        if (tid == 0) {
            s_excl = excl;
            if (t == ntiles - 1) a.ctl->nkept = excl + total;
        }
    }
    __syncthreads();
    const unsigned long long base = s_excl;
    for (unsigned e = tid; e < total; e += BLOCK) {
        const unsigned long long d = base + e;
        if (d < a.count) {   // always true for consistent records; never write past the buffers
            a.C[d] = s_okey[pad32(e)];
            a.O[d] = s_oobj[pad32(e)];
        } else {
            atomicOr(&a.ctl->err, ERR_RANGE);
        }
    }
}

// ---------------------------------------------------------------------------
// a8: RadixSort(C, O) - stable LSD passes, each an upsweep and a downsweep
// ---------------------------------------------------------------------------
//
// Upsweep of pass p: per tile of PAIR_TILE pairs, the count of each digit;
// per group of gtiles consecutive tiles, one block walks its tiles in order
// and writes each tile's digit offsets inside the group, then a decoupled
// look-back across groups yields each group's offsets.  Groups start gtiles
// times less often than tiles, so look-back chains stay short at GB300's
// tile rate; small passes use fewer tiles per group (down to one) so that
// their groups still fill the GPU.  The last group's inclusive prefixes are the
// pass's digit totals; its block scans them into the digit starts.  The
// first pass's upsweep generates the pairs (no pair array exists yet) and
// stores them for the first downsweep.
//
// Downsweep of pass p: every tile independently ranks its elements stably
// by digit and scatters them to dbase[d] + group offset + tile offset +
// rank; no tile waits for another.

constexpr unsigned LB_PREFIX = 0x80000000u;   // status word: value = inclusive prefix;
                                              // else value - 1 = aggregate; 0 = not ready

// Decoupled look-back of group g for one digit over row-major status words
// (st + h * R is group h's row), four predecessors per round trip.  Bounded:
// past SPIN_LIMIT polls of an unpublished word it records ERR_TIMEOUT and
// returns what it has.
__device__ __forceinline__ unsigned group_lookback(const unsigned *col, unsigned R, unsigned g, Ctl *ctl)
{
    unsigned excl = 0;
    long long k = (long long)g - 1;
    unsigned spins = 0;
    while (k >= 0) {
        unsigned v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = k - q >= 0 ? ld_relaxed_u32(col + (size_t)(k - q) * R) : LB_PREFIX;
        int used = 0;
        bool done = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (done || used < q || v[q] == 0u) continue;   // stop at the first word not published yet
            if (v[q] & LB_PREFIX) {
                excl += v[q] & ~LB_PREFIX;
                done = true;
            } else {
                excl += v[q] - 1u;
            }
            used = q + 1;
        }
        if (done) break;
        k -= used;
        if (used == 0) {
            if (++spins > SPIN_LIMIT) {
                atomicOr(&ctl->err, ERR_TIMEOUT);
                break;
            }
            if (spins > 4) __nanosleep(64);
        }
    }
    return excl;
}

// Failure-detection self-test: the sort's look-back run as group 1 of a
// column whose group-0 word nothing ever publishes.  The wait gives up after
// SPIN_LIMIT polls and records ERR_TIMEOUT, as a real look-back would if a
// predecessor never arrived.
__global__ void wait_selftest_kernel(const unsigned *col, Ctl *ctl, unsigned *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = group_lookback(col, 1u, 1u, ctl);
}

// Resident blocks per SM each radix-kernel shape is compiled for.
template <int BLOCK>
__host__ __device__ constexpr int pass_min_blocks()
{
    return BLOCK == ALT_BLOCK ? ALT_PASS_MIN_BLOCKS : PASS_MIN_BLOCKS;
}

template <int BLOCK>
__host__ __device__ constexpr int gen_min_blocks()
{
    return BLOCK == ALT_BLOCK ? ALT_GEN_MIN_BLOCKS : GEN_MIN_BLOCKS;
}

template <int BLOCK, int ITEMS, int RBITS, int SRC>
__global__ void __launch_bounds__(BLOCK, SRC == SRC_GEN ? gen_min_blocks<BLOCK>() : 2048 / BLOCK)
    upsweep_kernel(UpArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    constexpr int R = 1 << RBITS;
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_cnt2 = smem;                         // [2][R] digit counts of even / odd tiles
    unsigned *s_run = s_cnt2 + 2 * R;                // [R] counts of the group's tiles so far
    unsigned *s_mark = s_run + R;                    // [padded T] object marks (generated pairs)
    __shared__ unsigned s_tmp[BLOCK / 32];
    const int tid = threadIdx.x;
    const unsigned g = blockIdx.x;
    const unsigned t0 = g * a.gtiles, t1 = min(t0 + a.gtiles, a.ntiles);
    const unsigned sh = a.shift, mk = (1u << a.bits) - 1u;
    for (int i = tid; i < 3 * R; i += BLOCK) smem[i] = 0u;
    if (SRC == SRC_GEN) zero_marks<BLOCK, ITEMS>(s_mark);
    __syncthreads();

    // a tile's keys, 16 bytes per load where the whole run is in range and
    // the array is 16-byte aligned (a batch's later sort segments start
    // anywhere in the output arrays)
    const bool kvec = (reinterpret_cast<unsigned long long>(a.keys_in) & 15ull) == 0ull;
    const bool gvec = (reinterpret_cast<unsigned long long>(a.gen_keys) & 15ull) == 0ull &&
                      (reinterpret_cast<unsigned long long>(a.gen_vals) & 15ull) == 0ull;
    auto load_keys = [&](unsigned t, unsigned (&k)[ITEMS]) {
        const unsigned j0 = t * (unsigned)T;
        const unsigned cnt = min((unsigned)T, a.count - j0);
#pragma unroll
        for (int i = 0; i < ITEMS; i += 4) {
            const unsigned e = tid * ITEMS + i;
            if (kvec && e + 3 < cnt) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(a.keys_in + j0 + e));
                k[i] = v.x;
                k[i + 1] = v.y;
                k[i + 2] = v.z;
                k[i + 3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) k[i + q] = e + q < cnt ? a.keys_in[j0 + e + q] : 0u;
            }
        }
    };
    unsigned keys[ITEMS];

    for (unsigned t = t0; t < t1; ++t) {
        const unsigned j0 = t * (unsigned)T;
        const unsigned cnt = min((unsigned)T, a.count - j0);
        unsigned *s_cnt = s_cnt2 + ((t - t0) & 1u) * R;
        if (SRC == SRC_GEN) {
            unsigned om[ITEMS], objs[ITEMS];
            const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, t, j0, cnt, s_mark, s_tmp, om);
            gen_blocked<ITEMS>(a.recs, of, om, j0, cnt, a.res_x, a.res_y, a.mt, keys, objs);
            if (a.gen_keys) {
                // store the object-order pairs once, for the first downsweep
                // to read instead of generating them a second time
                static_assert(ITEMS % 4 == 0, "16-byte stores of a thread's run");
#pragma unroll
                for (int i = 0; i < ITEMS; i += 4) {
                    const unsigned e = tid * ITEMS + i;
                    if (gvec && e + 3 < cnt) {
                        __stcg(reinterpret_cast<uint4 *>(a.gen_keys + j0 + e),
                               make_uint4(keys[i], keys[i + 1], keys[i + 2], keys[i + 3]));
                        __stcg(reinterpret_cast<uint4 *>(a.gen_vals + j0 + e),
                               make_uint4(objs[i], objs[i + 1], objs[i + 2], objs[i + 3]));
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (e + q < cnt) {
                                a.gen_keys[j0 + e + q] = keys[i + q];
                                a.gen_vals[j0 + e + q] = objs[i + q];
                            }
                        }
                    }
                }
            }
        } else {
            load_keys(t, keys);
        }
        const unsigned nv = cnt > (unsigned)(tid * ITEMS) ? min((unsigned)ITEMS, cnt - tid * ITEMS) : 0u;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if ((unsigned)i < nv) atomicAdd(&s_cnt[(keys[i] >> sh) & mk], 1u);
        __syncthreads();
        // one barrier per tile: the next tile counts into the other buffer,
        // and this one is next counted into two tiles on, after the next
        // barrier (each thread clears the digits it reads)
        for (int d = tid; d < R; d += BLOCK) {
            a.intra[(size_t)t * R + d] = (unsigned short)s_run[d];
            s_run[d] += s_cnt[d];
            s_cnt[d] = 0u;
        }
    }
    unsigned *s_cnt = s_cnt2;

    // the group's offsets: decoupled look-back across groups, per digit
    for (int d = tid; d < R; d += BLOCK) {
        const unsigned tot = s_run[d];
        unsigned *col = a.status + d;
        unsigned excl = 0;
        if (g == 0) {
            st_relaxed_u32(col, LB_PREFIX | tot);
        } else {
            st_relaxed_u32(col + (size_t)g * R, tot + 1u);
            excl = group_lookback(col, R, g, a.ctl);
            st_relaxed_u32(col + (size_t)g * R, LB_PREFIX | (excl + tot));
        }
        a.gpref[(size_t)g * R + d] = excl;
        s_cnt[d] = excl + tot;
    }
    // the last group's inclusive prefixes are the pass's digit totals: its
    // block turns them into the digit starts the downsweep adds
    if (g != gridDim.x - 1) return;
    __syncthreads();
    const int nd = 1 << a.bits;
    unsigned carry = 0;
    for (int c0 = 0; c0 < nd; c0 += BLOCK) {
        const int d = c0 + tid;
        const unsigned v = d < nd ? s_cnt[d] : 0u;
        unsigned tot;
        const unsigned ex = block_excl_sum<BLOCK>(v, s_tmp, &tot);
        if (d < nd) a.dbase[d] = carry + ex;
        carry += tot;
    }
}

// Shared-memory index for 64-bit elements: one pad element per 16, so blocked
// writes (thread t at t * ITEMS + i) and warp-striped reads are conflict-free.
__device__ __forceinline__ unsigned pad16(unsigned e) { return e + (e >> 4); }

template <int T>
__host__ __device__ constexpr int padded16() { return T + T / 16; }

// Peer masks of the ranking step: one word per (warp, digit) per item of a
// batch.  When a batch of them fits in the staging buffer, which is idle
// while a tile is being ranked, they live there and items go through the
// ranking steps in batches of 4, 2 or 1 (the largest that fits); otherwise
// they get shared memory of their own and items go one at a time.
template <int BLOCK, int ITEMS, int RBITS>
__host__ __device__ constexpr bool masks_alias()
{
    return (BLOCK / 32) * (1 << RBITS) * 4 <= padded16<BLOCK * ITEMS>() * 8;
}

template <int BLOCK, int ITEMS, int RBITS>
__host__ __device__ constexpr int mask_batch()
{
    return (4 * (BLOCK / 32) * (1 << RBITS) * 4 <= padded16<BLOCK * ITEMS>() * 8)   ? 4
           : (2 * (BLOCK / 32) * (1 << RBITS) * 4 <= padded16<BLOCK * ITEMS>() * 8) ? 2
                                                                                     : 1;
}

// Shared memory of one downsweep block: staging (64-bit elements; the object
// marks and, when they fit, the peer masks alias it), input values, peer
// masks when they do not fit, 16-bit warp digit counts, digit starts, global
// bases.
template <int BLOCK, int ITEMS, int RBITS>
__host__ __device__ constexpr size_t down_smem_bytes()
{
    return sizeof(unsigned long long) * padded16<BLOCK * ITEMS>() + sizeof(unsigned) * BLOCK * ITEMS +
           (masks_alias<BLOCK, ITEMS, RBITS>() ? 0 : sizeof(unsigned) * (BLOCK / 32) * (1 << RBITS)) +
           sizeof(unsigned short) * (BLOCK / 32) * (1 << RBITS) + sizeof(unsigned) * (2 * (1 << RBITS) + BLOCK / 32);
}

__device__ __forceinline__ unsigned long long pack_kv(unsigned k, unsigned v)
{
    return ((unsigned long long)k << 32) | v;
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One-dimensional bulk copy global -> shared by the TMA engine, completing
// on a shared-memory mbarrier (transaction bytes).  dst, src and bytes must
// be multiples of 16.
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst), b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// Waits for phase 0 of the mbarrier, at most SPIN_LIMIT polls; false if the
// wait gave up (the caller records ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_phase0(unsigned long long *bar)
{
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    for (unsigned spins = 0; spins < SPIN_LIMIT; ++spins) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(b)
                     : "memory");
        if (done) return true;
        if (spins > 8) __nanosleep(32);
    }
    return false;
}

// STABLE: rank equal digits in element order (every pass of a plain LSD
// sort).  Otherwise equal digits of one warp may be ranked in any order: the
// first pass of the hybrid placement, whose only job is to order the pairs by
// its digit (the later passes need that order, not the order inside a
// digit, and the per-bucket counting sort puts each cell's objects in
// ascending order at the end).
template <int BLOCK, int ITEMS, int RBITS, int IN, bool STABLE>
__global__ void __launch_bounds__(BLOCK, pass_min_blocks<BLOCK>()) downsweep_kernel(DownArgs a, unsigned gtiles)
{
    constexpr int W = BLOCK / 32;
    constexpr int T = BLOCK * ITEMS;
    constexpr int R = 1 << RBITS;
    constexpr bool ALIAS = masks_alias<BLOCK, ITEMS, RBITS>();
    constexpr int BATCH = ALIAS ? mask_batch<BLOCK, ITEMS, RBITS>() : 1;
    static_assert(ITEMS % 2 == 0 && ITEMS % BATCH == 0 && T < 65536, "16-bit ranks and counts");
    static_assert(!ALIAS || BATCH * W * R * 4 <= padded16<T>() * 8, "aliased peer masks fit in the staging buffer");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *s_elem = reinterpret_cast<unsigned long long *>(smem_raw);   // [padded16 T] staging
    unsigned *s_mark = reinterpret_cast<unsigned *>(smem_raw);       // object marks while generating
    unsigned *s_vin = reinterpret_cast<unsigned *>(s_elem + padded16<T>());   // [T] values, element order
    unsigned *s_wmask = ALIAS ? reinterpret_cast<unsigned *>(smem_raw) : s_vin + T;   // [BATCH][W][R] peer masks
    unsigned short *s_wh = reinterpret_cast<unsigned short *>(s_vin + T + (ALIAS ? 0 : W * R));   // [W][R] warp counts
    unsigned *s_wh32 = reinterpret_cast<unsigned *>(s_wh);                    // the same, as words
    unsigned *s_dstart = reinterpret_cast<unsigned *>(s_wh + W * R);          // [R]
    unsigned *s_gbase = s_dstart + R;           // [R]
    unsigned *s_tmp = s_gbase + R;              // [W]
    __shared__ __align__(8) unsigned long long s_vbar;   // the value tile's bulk copy

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned nd = 1u << a.bits;
    const unsigned sh = a.shift, mk = nd - 1u;
    const unsigned ltmask = lanemask_lt();
    const unsigned bit = 1u << lane;
    const unsigned tile = blockIdx.x;
    const unsigned group = tile / gtiles;   // the upsweep group holding this tile
    const unsigned j0 = tile * (unsigned)T;
    const unsigned cnt = min((unsigned)T, a.count - j0);
    for (int i = tid; i < W * R / 2; i += BLOCK) s_wh32[i] = 0u;
    for (int d = tid; d < R; d += BLOCK)
        s_gbase[d] = d < (int)nd ? __ldg(a.dbase + d) + __ldg(a.gpref + (size_t)group * R + d) +
                                       __ldg(a.intra + (size_t)tile * R + d)
                                 : 0u;

    // keys of this lane's items in registers, values in shared memory;
    // item i of this lane is element e = w * 32 * ITEMS + i * 32 + lane
    unsigned keys[ITEMS];
    bool bulk = false;   // values arriving by a bulk copy
    if (IN == IN_GEN) {
        unsigned om[ITEMS], objs[ITEMS];
        zero_marks<BLOCK, ITEMS>(s_mark);
        __syncthreads();
        const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, tile, j0, cnt, s_mark, s_tmp, om);
        gen_blocked<ITEMS>(a.recs, of, om, j0, cnt, a.res_x, a.res_y, a.mt, keys, objs);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) s_elem[pad16(tid * ITEMS + i)] = pack_kv(keys[i], objs[i]);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            const unsigned long long v = s_elem[pad16(e)];
            keys[i] = (unsigned)(v >> 32);
            s_vin[e] = (unsigned)v;
        }
        __syncthreads();   // the staging buffer is read out; the masks take it
    } else {
        // the tile's values are one contiguous run: the TMA engine copies
        // its 16-byte part in one bulk transfer (when the caller's array is
        // 16-byte aligned), the last few words go by cp.async
        bulk = (reinterpret_cast<unsigned long long>(a.vals_in) & 15ull) == 0ull && cnt >= 4u;
        const unsigned nbulk = bulk ? (cnt & ~3u) : 0u;
        if (bulk && tid == 0) {
            mbar_init(&s_vbar, 1u);
            bulk_copy_g2s(s_vin, a.vals_in + j0, nbulk * 4u, &s_vbar);
        }
        for (unsigned e = nbulk + tid; e < cnt; e += BLOCK) cp_async4(&s_vin[e], a.vals_in + j0 + e);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            keys[i] = e < cnt ? __ldcs(a.keys_in + j0 + e) : 0u;
        }
    }
    // IN_PAIR_KEEP: the input is ordered by key bits [keep_lo, shift), so a
    // tile whose first and last elements share them holds one value of them
    // and its equal digits may take any order; other tiles rank stably
    bool stable = STABLE;
    if (IN == IN_PAIR_KEEP && cnt > 0u) {
        const unsigned k0 = __ldg(a.keys_in + j0), k1 = __ldg(a.keys_in + j0 + cnt - 1u);
        const unsigned span = (unsigned)(sh - a.keep_lo);
        const unsigned km = span >= 32u ? 0xFFFFFFFFu : (1u << span) - 1u;
        stable = (((k0 ^ k1) >> a.keep_lo) & km) != 0u;
    }
    if (stable)
        for (int i = tid; i < BATCH * W * R; i += BLOCK) s_wmask[i] = 0u;
    __syncthreads();

    // warp-level multisplit, stable in element order (items in order,
    // lanes in order): the lanes holding digit d find each other by
    // OR-ing their lane bit into a shared mask word for d; the lowest of
    // them reserves the group's slots in the warp's 16-bit digit count
    // with one shared atomic, clears the mask word, and the old count is
    // broadcast.  BATCH items go through each step together so their
    // shared-memory round trips overlap; the reservations are issued in
    // item order, which keeps the ranks stable.
    unsigned ranks[ITEMS / 2];   // 16-bit ranks, two per register
    if (!stable) {
        // runs of equal digits in consecutive lanes (pairs of one object often
        // share the high digits): the run's first lane reserves the run's
        // slots with one shared atomic and the others count from it
        const unsigned lemask = ltmask | bit;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            const bool ok = e < cnt;
            const unsigned d = ok ? (keys[i] >> sh) & mk : 0xFFFFFFFFu;   // the tail forms a run of its own
            const unsigned dprev = __shfl_up_sync(0xffffffffu, d, 1);
            const bool head = lane == 0 || d != dprev;
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            const unsigned start = 31u - __clz(hm & lemask);
            const unsigned above = hm & ~lemask;
            const unsigned end = above ? (unsigned)__ffs(above) - 1u : 32u;
            unsigned old = 0u;
            if (head && ok) {
                const unsigned hs = (d & 1u) * 16u;
                old = (atomicAdd(&s_wh32[(w * R + d) >> 1], (end - start) << hs) >> hs) & 0xFFFFu;
            }
            const unsigned r = __shfl_sync(0xffffffffu, old, start) + (lane - start);
            if (i % 2 == 0)
                ranks[i / 2] = r;
            else
                ranks[i / 2] |= r << 16;
        }
    }
#pragma unroll
    for (int ib = 0; ib < (STABLE ? ITEMS : 0); ib += BATCH) {
        if (!stable) break;
        unsigned d[BATCH], peers[BATCH], old[BATCH];
        bool ok[BATCH];
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            const unsigned e = w * 32 * ITEMS + (ib + q) * 32 + lane;
            ok[q] = e < cnt;
            d[q] = (keys[ib + q] >> sh) & mk;
            if (ok[q]) atomicOr(&s_wmask[(q * W + w) * R + d[q]], bit);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < BATCH; ++q) peers[q] = ok[q] ? s_wmask[(q * W + w) * R + d[q]] : 0u;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            old[q] = 0u;
            if (ok[q] && (peers[q] & ltmask) == 0u) {
                const unsigned hs = (d[q] & 1u) * 16u;
                old[q] = (atomicAdd(&s_wh32[(w * R + d[q]) >> 1], (unsigned)__popc(peers[q]) << hs) >> hs) &
                         0xFFFFu;
                s_wmask[(q * W + w) * R + d[q]] = 0u;
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < BATCH; ++q) {
            const unsigned r = __shfl_sync(0xffffffffu, old[q], ok[q] ? __ffs(peers[q]) - 1 : lane) +
                               __popc(peers[q] & ltmask);
            const int i = ib + q;
            if (i % 2 == 0)
                ranks[i / 2] = r;
            else
                ranks[i / 2] |= r << 16;
        }
    }
    __syncthreads();

    // per digit: exclusive offsets across warps and the tile's count
    for (int d = tid; d < R; d += BLOCK) {
        unsigned sum = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) {
            const unsigned c = s_wh[ww * R + d];
            s_wh[ww * R + d] = (unsigned short)sum;
            sum += c;
        }
        s_dstart[d] = sum;
    }
    __syncthreads();
    // exclusive scan of the tile's digit counts -> local digit starts
    {
        constexpr int C = (R + BLOCK - 1) / BLOCK;   // digits per thread
        unsigned loc[C];
        unsigned s = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            loc[k] = tid * C + k < R ? s_dstart[tid * C + k] : 0u;
            s += loc[k];
        }
        unsigned tot;
        unsigned ex = block_excl_sum<BLOCK>(s, s_tmp, &tot);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            if (tid * C + k < R) {
                s_dstart[tid * C + k] = ex;
                s_gbase[tid * C + k] -= ex;   // global start of the digit's run minus its local start
            }
            ex += loc[k];
        }
    }
    if (IN != IN_GEN) {
        cp_async_wait_all();
        if (bulk && !mbar_wait_phase0(&s_vbar)) atomicOr(&a.ctl->err, ERR_TIMEOUT);
    }
    __syncthreads();
    // stage the tile in shared memory in locally sorted order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = w * 32 * ITEMS + i * 32 + lane;
        if (e < cnt) {
            const unsigned d = (keys[i] >> sh) & mk;
            const unsigned rk = (ranks[i / 2] >> (16 * (i % 2))) & 0xFFFFu;
            const unsigned pos = s_dstart[d] + s_wh[w * R + d] + rk;
            if (pos < cnt)
                s_elem[pos] = pack_kv(keys[i], s_vin[e]);
            else
                atomicOr(&a.ctl->err, ERR_RANGE);   // never with consistent counts
        }
    }
    __syncthreads();
    // scatter: consecutive threads write consecutive positions of a digit run
    bool bad = false;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned pos = i * BLOCK + tid;
        if (pos < cnt) {
            const unsigned long long v = s_elem[pos];
            const unsigned k = (unsigned)(v >> 32);
            const unsigned dst = s_gbase[(k >> sh) & mk] + pos;
            if (dst < a.count) {
                __stcg(a.keys_out + dst, k);
                __stcg(a.vals_out + dst, (unsigned)v);
            } else {
                bad = true;
            }
        }
    }
    if (bad) atomicOr(&a.ctl->err, ERR_RANGE);
}

// ---------------------------------------------------------------------------
// a9: RunLengthEncode + NonEmptyCells + ExclusiveSum via a merge path
// ---------------------------------------------------------------------------

// Merge order: cell c precedes key k iff c <= k, so G[c] = number of keys
// before cell c in the merged sequence = number of keys < c.  Returns the
// number of keys among the first d merged items.
__device__ __forceinline__ unsigned long long merge_split(const unsigned *keys, unsigned long long nA,
                                                          unsigned long long nB, unsigned long long d)
{
    unsigned long long lo = d > nB ? d - nB : 0ull;
    unsigned long long hi = d < nA ? d : nA;
    while (lo < hi) {
        const unsigned long long mid = (lo + hi) >> 1;
        // key[mid] precedes cell (d - mid - 1)?
        if ((unsigned long long)__ldg(keys + mid) < d - mid - 1ull)
            lo = mid + 1ull;
        else
            hi = mid;
    }
    return lo;
}

// The split of every extraction block's first diagonal, all in parallel.
__global__ void __launch_bounds__(256) extract_split_kernel(ExtractArgs a, unsigned long long nblocks)
{
    const unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblocks) return;
    const unsigned long long nA = a.count, nB = a.ncells + 1ull;
    const unsigned long long d = min(b * (unsigned long long)EXTRACT_TILE, nA + nB);
    a.splits[b] = (unsigned)merge_split(a.keys, nA, nB, d);
    // the keys are sorted: the last one bounds them all
    if (b == 0 && nA > 0 && (unsigned long long)__ldg(a.keys + nA - 1) >= a.ncells) atomicOr(&a.ctl->err, ERR_RANGE);
}

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) extract_kernel(ExtractArgs a)
{
    constexpr int D = BLOCK * ITEMS;
    static_assert((D & (D - 1)) == 0, "the lower-bound steps halve from D");
    __shared__ unsigned s_keys[D];
    const int tid = threadIdx.x;
    const unsigned long long nA = a.count, nB = a.ncells + 1ull;
    const unsigned long long M = nA + nB;
    const unsigned long long d0 = (unsigned long long)blockIdx.x * D;
    const unsigned long long d1 = min(d0 + D, M);
    const unsigned long long i0 = a.splits[blockIdx.x], i1 = a.splits[blockIdx.x + 1];
    // splits out of order, or more keys than merged items, come only from
    // keys that are not sorted: report them and touch nothing (the sizes
    // below would wrap)
    if (i1 < i0 || i1 - i0 > d1 - d0) {
        if (threadIdx.x == 0) atomicOr(&a.ctl->err, ERR_RANGE);
        return;
    }
    // every key before i0 is below c0 and every key from i1 on is at least
    // c1, so G[c] = i0 + (keys of this block below c); cell ids fit 32 bits
    const unsigned c0 = (unsigned)(d0 - i0), c1 = (unsigned)(d1 - i1);
    const unsigned na = (unsigned)(i1 - i0), nc = c1 - c0;
    // the block's keys: 16-byte loads over the aligned middle (many bytes in
    // flight per thread), single words at the ragged ends; nothing outside
    // [i0, i1) is read
    {
        // (a caller's array may start off a 16-byte boundary: then words only)
        const bool vec = (reinterpret_cast<unsigned long long>(a.keys) & 15ull) == 0ull;
        const unsigned long long a_lo = (i0 + 3ull) & ~3ull, a_hi = i1 & ~3ull;
        if (vec && a_lo < a_hi) {
            const unsigned head = (unsigned)(a_lo - i0), nv = (unsigned)((a_hi - a_lo) >> 2);
            const uint4 *src = reinterpret_cast<const uint4 *>(a.keys + a_lo);
            for (unsigned v = tid; v < nv; v += BLOCK) {
                const uint4 q = __ldcs(src + v);
                const unsigned k = head + 4u * v;
                s_keys[k] = q.x;
                s_keys[k + 1] = q.y;
                s_keys[k + 2] = q.z;
                s_keys[k + 3] = q.w;
            }
            if (tid < (int)head) s_keys[tid] = __ldcs(a.keys + i0 + tid);
            const unsigned tail0 = (unsigned)(a_hi - i0);
            if (tid < (int)(na - tail0)) s_keys[tail0 + tid] = __ldcs(a.keys + a_hi + tid);
        } else {
            for (unsigned k = tid; k < na; k += BLOCK) s_keys[k] = __ldcs(a.keys + i0 + k);
        }
    }
    __syncthreads();
    // each thread takes a run of consecutive cells: the first cell's lower
    // bound is a full branch-free search over the block's keys, each later
    // one starts from its predecessor's and usually lies within the next
    // 8 keys (3 steps), else a full search from there
    const unsigned cpt = (nc + BLOCK - 1) / BLOCK;
    const unsigned k0 = min(tid * cpt, nc), k1 = min(k0 + cpt, nc);
    unsigned pos = 0;
    for (unsigned k = k0; k < k1; ++k) {
        const unsigned c = c0 + k;
        if (k != k0 && pos + 8u <= na && s_keys[pos + 7u] >= c) {
#pragma unroll
            for (unsigned step = 4u; step >= 1u; step >>= 1) {
                const unsigned q = pos + step;
                pos = s_keys[q - 1u] < c ? q : pos;
            }
        } else {
#pragma unroll
            for (unsigned step = (unsigned)D; step >= 1u; step >>= 1) {   // D, a power of two, bounds na
                const unsigned q = pos + step;
                pos = (q <= na && s_keys[q - 1u] < c) ? q : pos;
            }
        }
        // written straight from the thread's run: the runs of neighbouring
        // lanes are a few cells apart, so a warp's stores share sectors
        a.G[(unsigned long long)c0 + k] = (unsigned)i0 + pos;
    }
}

// ---------------------------------------------------------------------------
// a8 (low digits) + a9 per bucket: counting sort by cell, cell ranges
// ---------------------------------------------------------------------------
//
// The radix passes have ordered the pairs by key >> lbits, so each bucket of
// 2^lbits consecutive cells is one contiguous run of pairs.  Consecutive
// buckets are grouped (a group closes where the running pair count crosses
// a multiple of group_pairs, or at 2^LOCAL_LMAX cells), and one block per
// group counts the group's pairs per cell with shared-memory atomics (the
// value an atomic returns is the pair's slot inside its cell), scans the
// counts into the cells' offsets (G of the group's cells, less the group's
// first pair), and puts every pair at its cell's offset plus its slot.  The
// slots of a cell come out in no fixed order; the pairs of one cell belong to
// distinct objects, and the stable sort of object-order pairs leaves them in
// ascending object order, so each cell's run is put in ascending order
// afterwards.  The result is the stable sort's, bit for bit.

// Does bucket b open a group?  sp, sb, sn: starts of buckets b - 1, b and
// b + 1.  A group closes where the running pair count crosses a multiple of
// group_pairs, at every bmax-th bucket (2^LOCAL_LMAX cells at most), and
// around every bucket of more than LOCAL_CAP - group_pairs pairs, which
// forms a group of its own; so no group holds more than LOCAL_CAP pairs
// unless one bucket alone does.
__device__ __forceinline__ bool opens_group(unsigned b, unsigned sp, unsigned sb, unsigned sn,
                                            unsigned group_pairs, unsigned bmax)
{
    const unsigned big = (unsigned)LOCAL_CAP - group_pairs;
    return b == 0u || b % bmax == 0u || sp / group_pairs != sb / group_pairs || sb - sp > big || sn - sb > big;
}

// First pair of bucket b (b <= nbuckets): the number of keys whose bucket is
// below b.
__device__ __forceinline__ unsigned bucket_start(const LocalArgs &a, unsigned b)
{
    if (b >= a.nbuckets) return a.count;
    unsigned lo = 0, hi = a.count;
    while (lo < hi) {
        const unsigned mid = lo + ((hi - lo) >> 1);
        if ((__ldg(a.keys + mid) >> a.lbits) < b)
            lo = mid + 1u;
        else
            hi = mid;
    }
    return lo;
}

// Each block searches the starts of its 256 buckets and of the two next to
// them once, shares them in shared memory, and opens the groups.
__global__ void __launch_bounds__(256) bucket_split_kernel(LocalArgs a)
{
    __shared__ unsigned s_st[256 + 2];   // starts of buckets b0 - 1 .. b0 + 256
    const unsigned b0 = blockIdx.x * 256u, b = b0 + threadIdx.x;
    if (b <= a.nbuckets) s_st[threadIdx.x + 1] = bucket_start(a, b);
    if (threadIdx.x == 0) s_st[0] = b0 ? bucket_start(a, b0 - 1u) : 0u;
    if (threadIdx.x == 255 && b + 1u <= a.nbuckets) s_st[257] = bucket_start(a, b + 1u);
    __syncthreads();
    if (b > a.nbuckets) return;
    const unsigned sb = s_st[threadIdx.x + 1];
    a.starts[b] = sb;
    if (b == a.nbuckets) {
        a.G[a.ncells] = a.count;
        return;
    }
    const unsigned bmax = (1u << LOCAL_LMAX) >> a.lbits;
    const unsigned sp = b ? s_st[threadIdx.x] : 0u, sn = s_st[threadIdx.x + 2];
    if (opens_group(b, sp, sb, sn, a.group_pairs, bmax)) {
        const unsigned g = atomicAdd(&a.ctl->tickets[2], 1u);
        if (g < a.max_groups)
            a.groups[g] = b;
        else
            atomicOr(&a.ctl->err, ERR_RANGE);   // never: max_groups bounds the groups
    }
}

// In place: h[0 .. n) becomes its exclusive prefix sums and h[n] their total.
// Ends with a barrier.
template <int BLOCK>
__device__ __forceinline__ void scan_counts(unsigned *h, unsigned n, unsigned *s_tmp)
{
    const unsigned per = (n + BLOCK - 1) / BLOCK;
    const unsigned c0 = min(threadIdx.x * per, n), c1 = min(c0 + per, n);
    unsigned sum = 0;
    for (unsigned c = c0; c < c1; ++c) sum += h[c];
    unsigned tot;
    unsigned ex = block_excl_sum<BLOCK>(sum, s_tmp, &tot);
    for (unsigned c = c0; c < c1; ++c) {
        const unsigned v = h[c];
        h[c] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) h[n] = tot;
    __syncthreads();
}

// Position of the set bit of `bits` (one bit per position) at or before j,
// and of the first one after j (n if none before n): the run of the cell
// whose bit marks its start.
__device__ __forceinline__ unsigned run_start(const unsigned *bits, unsigned j)
{
    unsigned w = j >> 5;
    unsigned x = bits[w] & (0xFFFFFFFFu >> (31u - (j & 31u)));   // bits <= j
    while (x == 0u) x = bits[--w];   // position 0 always opens a run
    return (w << 5) + 31u - __clz(x);
}

__device__ __forceinline__ unsigned run_end(const unsigned *bits, unsigned j, unsigned n)
{
    unsigned w = j >> 5;
    unsigned x = (j & 31u) == 31u ? 0u : bits[w] & (0xFFFFFFFEu << (j & 31u));   // bits > j
    const unsigned last = (n - 1u) >> 5;
    while (x == 0u && w < last) x = bits[++w];
    return x ? min((w << 5) + (unsigned)__ffs(x) - 1u, n) : n;
}

// The run [lo, hi) of s_o holding position j: its ends are found in j's bit
// word or its two neighbours (a run longer than 32 searches on).
__device__ __forceinline__ void run_bounds(const unsigned *bits, unsigned j, unsigned n, unsigned nw, unsigned &lo,
                                           unsigned &hi)
{
    const unsigned w = j >> 5, bp = j & 31u;
    const unsigned x0 = bits[w];
    const unsigned xm = w > 0u ? bits[w - 1u] : 0u;
    const unsigned xp = w + 1u < nw ? bits[w + 1u] : 0u;
    const unsigned below = x0 & (0xFFFFFFFFu >> (31u - bp));
    const unsigned above = bp == 31u ? 0u : x0 & (0xFFFFFFFEu << bp);
    if (below)
        lo = (w << 5) + 31u - __clz(below);
    else if (xm)
        lo = ((w - 1u) << 5) + 31u - __clz(xm);
    else
        lo = run_start(bits, j);
    if (above)
        hi = (w << 5) + (unsigned)__ffs(above) - 1u;
    else if (xp)
        hi = ((w + 1u) << 5) + (unsigned)__ffs(xp) - 1u;
    else
        hi = run_end(bits, j, n);
    hi = min(hi, n);
}

// Members of the run [lo, hi) below v: up to 8 with independent loads, then
// one at a time.
__device__ __forceinline__ unsigned rank_in_run(const unsigned *s_o, unsigned lo, unsigned hi, unsigned v)
{
    unsigned r = 0;
#pragma unroll
    for (unsigned q = 0; q < 8u; ++q) {
        const unsigned i = lo + q;
        if (i < hi) r += s_o[i] < v ? 1u : 0u;
    }
    for (unsigned i = lo + 8u; i < hi; ++i) r += s_o[i] < v ? 1u : 0u;
    return r;
}

// A hint that brings [p, p + count) of a 32-bit array into L2 ahead of its
// reads (one bulk prefetch; the range is shrunk to 16-byte boundaries inside
// it, so no byte outside the array is named).
__device__ __forceinline__ void l2_prefetch_u32(const unsigned *p, unsigned count)
{
    const unsigned long long b = (unsigned long long)p;
    const unsigned long long lo = (b + 15ull) & ~15ull, hi = (b + 4ull * count) & ~15ull;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// One block per group of buckets, in passes over the group's pairs: count
// them per cell (shared atomics), scan the counts into the cells' offsets
// (written out as G), then place the pairs cell by cell in shared memory
// (atomics on per-cell cursors hand out slots inside a cell in no fixed
// order) and write each pair to its cell's offset plus its rank among the
// cell's pairs by object id: the order a stable sort of object-order pairs
// leaves them in.  While a group runs, the block's next group's keys and
// values are prefetched into L2.  A group of more than LOCAL_CAP pairs is
// placed in chunks of whole cells (each chunk gathers its pairs in one more
// pass over the group).  A group with a cell of more than LOCAL_RUN_MAX pairs
// is left alone and flagged ERR_LOCAL_FALLBACK: the host then places the
// whole build by radix passes over every key bit and range extraction instead.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, LOCAL_MIN_BLOCKS) local_sort_kernel(LocalArgs a)
{
    constexpr int HN = 1 << LOCAL_LMAX;
    constexpr int PER = HN / BLOCK;   // cells per thread in the scan
    static_assert(HN % BLOCK == 0 && PER >= 1, "cells per thread");
    constexpr unsigned Q = (unsigned)LOCAL_CAP - LOCAL_RUN_MAX;   // chunk k: cells with offsets in [k Q, (k + 1) Q)
    constexpr unsigned NBW = (unsigned)LOCAL_CAP / 32u;
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *h = smem;                 // [HN + 1] per-cell counts, then offsets
    unsigned *hc = h + HN + 1;          // [HN] per-cell cursors of the current chunk
    unsigned *s_o = hc + HN;            // [LOCAL_CAP] the chunk's values, by cell
    __shared__ unsigned s_bits[NBW];    // one bit per position of s_o: a cell's run starts
    __shared__ unsigned s_tmp[BLOCK / 32];
    __shared__ unsigned s_end, s_clo, s_chi;
    const int tid = threadIdx.x;
    const unsigned ngroups = min(ld_relaxed_u32(&a.ctl->tickets[2]), a.max_groups);
    const unsigned bmax = (1u << LOCAL_LMAX) >> a.lbits;
    // the pairs of group gg lie in [starts[b0], starts[min(b0 + bmax, nbuckets)])
    auto prefetch = [&](unsigned gg) {
        if (gg >= ngroups) return;
        const unsigned b0 = a.groups[gg], e = min(b0 + bmax, a.nbuckets);
        const unsigned s0 = a.starts[b0], s1 = a.starts[e];
        if (s1 > s0) {
            l2_prefetch_u32(a.keys + s0, s1 - s0);
            l2_prefetch_u32(a.vals + s0, s1 - s0);
        }
    };
    if (tid == 0) prefetch(blockIdx.x);
    // blocks take groups in turn: a fixed grid, no block without a group
    for (unsigned g = blockIdx.x; g < ngroups; g += gridDim.x) {
    __syncthreads();   // the previous group's last reads of shared memory are done
    if (tid == 0) prefetch(g + gridDim.x);
    const unsigned b0 = a.groups[g];
    // the group's end: the next bucket that opens a group, at most bmax on
    unsigned b1 = min(b0 + bmax, a.nbuckets);
    if (bmax > 1u) {
        if (tid == 0) s_end = b1;
        __syncthreads();
        for (unsigned b = b0 + 1u + tid; b < b1; b += BLOCK) {
            const unsigned sn = b + 1u < a.nbuckets ? a.starts[b + 1u] : a.count;
            if (opens_group(b, a.starts[b - 1u], a.starts[b], sn, a.group_pairs, bmax)) atomicMin(&s_end, b);
        }
        __syncthreads();
        b1 = s_end;
    }
    const unsigned long long cbase64 = (unsigned long long)b0 << a.lbits;
    const unsigned cbase = (unsigned)cbase64;
    const unsigned nh = (b1 - b0) << a.lbits;   // cells of the whole buckets, <= HN
    const unsigned nc = (unsigned)min((unsigned long long)nh, a.ncells - cbase64);   // cells inside the grid
    const unsigned s = a.starts[b0], m = a.starts[b1] - s;
    if (a.starts[b1] < s || nh > (unsigned)HN) {   // starts of sorted keys never decrease
        if (tid == 0) atomicOr(&a.ctl->err, ERR_RANGE);
        continue;
    }
    const unsigned *keys = a.keys + s, *vals = a.vals + s;
    unsigned *refs = a.refs + s;
    const bool one_chunk = m <= (unsigned)LOCAL_CAP;
    bool bad = false;
    // count the pairs per cell.  The loops over the group's pairs take U
    // pairs per thread at a time, every load issued before any is used.
    constexpr int U = 8;
    for (unsigned c = tid; c < (unsigned)HN; c += BLOCK) h[c] = 0u;
    if (one_chunk)
        for (unsigned w = tid; w < NBW; w += BLOCK) s_bits[w] = 0u;
    __syncthreads();
    for (unsigned j0 = tid; j0 < m; j0 += U * BLOCK) {
        unsigned kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) kk[u] = j0 + u * BLOCK < m ? __ldg(keys + j0 + u * BLOCK) : cbase + nc;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned c = kk[u] - cbase;   // wraps below the group
            if (c < nc)
                atomicAdd(&h[c], 1u);
            else
                bad |= j0 + u * BLOCK < m;   // a key outside the group: the keys were not ordered by bucket
        }
    }
    __syncthreads();
    // scan the counts: thread t owns cells [t PER, (t + 1) PER); a cell
    // of more than LOCAL_RUN_MAX pairs sends the build to the fallback.
    // With one chunk the same pass also sets the placement cursors, marks
    // each non-empty cell's run start and writes G.
    {
        const unsigned c0 = (unsigned)tid * PER;
        unsigned cnt[PER];
        if constexpr (PER == 4) {
            const uint4 q = *reinterpret_cast<const uint4 *>(h + c0);
            cnt[0] = q.x; cnt[1] = q.y; cnt[2] = q.z; cnt[3] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < PER; ++i) cnt[i] = h[c0 + i];
        }
        unsigned sum = 0;
        bool long_run = false;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            sum += cnt[i];
            long_run |= cnt[i] > (unsigned)LOCAL_RUN_MAX;
        }
        unsigned tot;
        unsigned ex = block_excl_sum<BLOCK>(sum, s_tmp, &tot);
        unsigned off[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            off[i] = ex;
            ex += cnt[i];
        }
        if constexpr (PER == 4) {
            *reinterpret_cast<uint4 *>(h + c0) = make_uint4(off[0], off[1], off[2], off[3]);
        } else {
#pragma unroll
            for (int i = 0; i < PER; ++i) h[c0 + i] = off[i];
        }
        if (tid == 0) h[HN] = tot;
        if (one_chunk) {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                hc[c0 + i] = off[i];
                if (cnt[i]) atomicOr(&s_bits[off[i] >> 5], 1u << (off[i] & 31u));
            }
        }
        unsigned *gp = a.G + cbase64 + c0;
        if (PER == 4 && c0 + 4u <= nc && ((unsigned long long)gp & 15ull) == 0ull) {
            *reinterpret_cast<uint4 *>(gp) = make_uint4(s + off[0], s + off[1 % PER], s + off[2 % PER], s + off[3 % PER]);
        } else {
#pragma unroll
            for (int i = 0; i < PER; ++i)
                if (c0 + i < nc) gp[i] = s + off[i];
        }
        if (__syncthreads_or(long_run)) {
            if (tid == 0) atomicOr(&a.ctl->err, ERR_LOCAL_FALLBACK);
            continue;
        }
    }
    const unsigned nchunks = one_chunk ? 1u : (m + Q - 1u) / Q;
    for (unsigned k = 0; k < nchunks; ++k) {
        unsigned clo = 0, chi = nc;
        if (!one_chunk) {   // the chunk's cells: binary searches over the offsets
            if (tid == 0) {
                unsigned lo = 0, hi = nc;
                while (lo < hi) {
                    const unsigned mid = (lo + hi) >> 1;
                    if (h[mid] < k * Q) lo = mid + 1u; else hi = mid;
                }
                s_clo = lo;
                hi = nc;
                while (lo < hi) {
                    const unsigned mid = (lo + hi) >> 1;
                    if (h[mid] < (k + 1u) * Q) lo = mid + 1u; else hi = mid;
                }
                s_chi = lo;
            }
            __syncthreads();
            clo = s_clo;
            chi = s_chi;
        }
        const unsigned base = h[clo], cm = (one_chunk ? m : h[chi]) - base;   // the chunk's pairs: [base, base + cm)
        if (!one_chunk) {
            for (unsigned w = tid; w < (cm + 31u) / 32u; w += BLOCK) s_bits[w] = 0u;
            for (unsigned c = clo + tid; c < chi; c += BLOCK) hc[c] = h[c] - base;
            __syncthreads();
            for (unsigned c = clo + tid; c < chi; c += BLOCK) {
                const unsigned p = h[c] - base;   // not hc[c]: placement below moves the cursors
                if (h[c + 1] > h[c]) atomicOr(&s_bits[p >> 5], 1u << (p & 31u));
            }
        }
        // place the chunk's pairs by cell (slots inside a cell in no fixed order)
        for (unsigned j0 = tid; j0 < m; j0 += U * BLOCK) {
            unsigned kk[U], vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) kk[u] = j0 + u * BLOCK < m ? __ldg(keys + j0 + u * BLOCK) : cbase + nc;
#pragma unroll
            for (int u = 0; u < U; ++u) vv[u] = j0 + u * BLOCK < m ? __ldg(vals + j0 + u * BLOCK) : 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned c = kk[u] - cbase;
                if (c >= clo && c < chi) s_o[atomicAdd(&hc[c], 1u)] = vv[u];
            }
        }
        __syncthreads();
        // each pair to its cell's start plus its rank by object id inside the cell
        const unsigned nw = (cm + 31u) >> 5;
        for (unsigned j = tid; j < cm; j += BLOCK) {
            const unsigned v = s_o[j];
            unsigned lo, hi;
            run_bounds(s_bits, j, cm, nw, lo, hi);
            __stcs(refs + base + lo + rank_in_run(s_o, lo, hi, v), v);
        }
        __syncthreads();
    }
    if (bad) atomicOr(&a.ctl->err, ERR_RANGE);
    }
}

// ---------------------------------------------------------------------------
// batched builds: per-mesh bounds, per-mesh cell arrays
// ---------------------------------------------------------------------------

// Each thread takes BOUNDS_ITEMS consecutive triangles of the flattened batch;
// a warp whose triangles all belong to one mesh reduces in registers, other
// warps update per lane.  bstate[m * 6 + a] holds ~ordered(min) for a < 3 and
// ordered(max) for a >= 3 (both atomicMax).
constexpr int BOUNDS_ITEMS = 8;

__global__ void __launch_bounds__(256) bounds_batched_kernel(MeshTab mt, long long ntot, unsigned *bstate, Ctl *ctl)
{
    const long long t0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * BOUNDS_ITEMS;
    const float inf = __int_as_float(0x7f800000);
    float lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
    unsigned err = 0;
    int m0 = -1;
    auto flush = [&](int m) {
        if (m < 0) return;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (lo[a] <= hi[a]) {
                atomicMax(&bstate[m * 6 + a], ~float_to_ordered(lo[a]));
                atomicMax(&bstate[m * 6 + 3 + a], float_to_ordered(hi[a]));
            }
            lo[a] = inf;
            hi[a] = -inf;
        }
    };
    for (int k = 0; k < BOUNDS_ITEMS; ++k) {
        const long long o = t0 + k;
        if (o >= ntot) break;
        const int m = mesh_of(mt, o);
        if (m != m0) {
            flush(m0);
            m0 = m;
        }
        const MeshDesc &md = mt.md[m];
        const long long li = o - __ldg(mt.obj_base + m);
        for (int v = 0; v < 3; ++v) {
            const int vi = __ldg(md.tris + 3 * li + v);
            if (vi < 0 || (long long)vi >= md.nverts) {
                err |= ERR_BADINDEX;
                continue;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float x = __ldg(md.verts + 3ll * vi + a);
                if (!isfinite(x)) {
                    err |= ERR_NONFINITE;
                } else {
                    lo[a] = fminf(lo[a], x);
                    hi[a] = fmaxf(hi[a], x);
                }
            }
        }
    }
    // one mesh for the whole warp: reduce in registers, one lane updates
    const bool same = __all_sync(0xffffffffu, m0 == __shfl_sync(0xffffffffu, m0, 0));
    if (same) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
            }
        }
        if ((threadIdx.x & 31) == 0) flush(m0);
    } else {
        flush(m0);
    }
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0 && err) atomicOr(&ctl->err, err);
}

__global__ void __launch_bounds__(256) localize_kernel(const unsigned *__restrict__ G,
                                                       const long long *__restrict__ cells_off,
                                                       const unsigned *__restrict__ pair_base, int nm,
                                                       long long total, unsigned *__restrict__ out)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= total) return;
    int lo = 0, hi = nm - 1;   // mesh m: largest with cells_off[m] <= q (every slice is non-empty)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cells_off + mid) <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    // mesh m's cell k is global cell cell_base[m] + k = q - m (each earlier mesh has one extra entry)
    out[q] = __ldg(G + (q - lo)) - __ldg(pair_base + lo);
}

// A batch sorted in segments: each object's pair offset made relative to its
// segment's first pair (segment s holds objects from seg_obj0[s]).
__global__ void __launch_bounds__(256) rebase_recs_kernel(ObjRec *__restrict__ recs, long long n,
                                                          const long long *__restrict__ seg_obj0,
                                                          const unsigned *__restrict__ seg_p0, int nseg)
{
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    int lo = 0, hi = nseg - 1;   // largest s with seg_obj0[s] <= o
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seg_obj0 + mid) <= o)
            lo = mid;
        else
            hi = mid - 1;
    }
    recs[o].start -= __ldg(seg_p0 + lo);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_bounds(const float *verts, long long nverts, const int *tris, long long n, Ctl *ctl,
                          int nsm, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)nsm * 8;
    if (blocks > cap) blocks = cap;
    bounds_kernel<<<(unsigned)blocks, 256, 0, s>>>(verts, nverts, tris, n, ctl);
    return cudaGetLastError();
}

cudaError_t launch_bounds_batched(const MeshTab &mt, long long ntot, unsigned *bstate, Ctl *ctl, cudaStream_t s)
{
    if (ntot <= 0) return cudaSuccess;
    const long long per_block = 256ll * BOUNDS_ITEMS;
    bounds_batched_kernel<<<(unsigned)((ntot + per_block - 1) / per_block), 256, 0, s>>>(mt, ntot, bstate, ctl);
    return cudaGetLastError();
}

cudaError_t launch_localize(const unsigned *G, const long long *cells_off, const unsigned *pair_base, int nm,
                            long long total, unsigned *out, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    localize_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(G, cells_off, pair_base, nm, total, out);
    return cudaGetLastError();
}

cudaError_t launch_rebase_recs(ObjRec *recs, long long n, const long long *seg_obj0, const unsigned *seg_p0, int nseg,
                               cudaStream_t s)
{
    if (n <= 0 || nseg < 1) return cudaSuccess;
    rebase_recs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(recs, n, seg_obj0, seg_p0, nseg);
    return cudaGetLastError();
}

cudaError_t launch_count_scan(const CountArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const long long tiles = (a.n + COUNT_TILE - 1) / COUNT_TILE;
    count_scan_kernel<COUNT_BLOCK, COUNT_TILE / COUNT_BLOCK><<<(unsigned)tiles, COUNT_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// Raises a kernel's dynamic shared-memory limit once per device.  Launchers
// run concurrently from several host threads (one per serving worker), so the
// per-device "done" bits are atomic; a repeated call is harmless.
template <typename K>
cudaError_t allow_dynamic_smem(K k, size_t smem, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

cudaError_t launch_tile_search(const ObjRec *recs, long long n, unsigned tile, unsigned ntiles,
                               unsigned *tile_obj, cudaStream_t s)
{
    const unsigned blocks = (ntiles + 1 + 255) / 256;
    tile_search_kernel<<<blocks, 256, 0, s>>>(recs, n, tile, ntiles, tile_obj);
    return cudaGetLastError();
}

cudaError_t launch_emit(const EmitArgs &a, cudaStream_t s)
{
    if (a.count == 0) return cudaSuccess;
    const unsigned tiles = (a.count + PAIR_TILE - 1) / PAIR_TILE;
    auto k = emit_kernel<PAIR_BLOCK, PAIR_TILE / PAIR_BLOCK>;
    const size_t smem = 2 * sizeof(unsigned) * padded<PAIR_TILE>();
    static std::atomic<unsigned long long> configured{0};
    if (cudaError_t e = allow_dynamic_smem(k, smem, configured)) return e;
    k<<<tiles, PAIR_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(const unsigned *col, Ctl *ctl, unsigned *out, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(col, ctl, out);
    return cudaGetLastError();
}

cudaError_t launch_cull_emit(const CullArgs &a, cudaStream_t s)
{
    if (a.count == 0) return cudaSuccess;
    const unsigned tiles = (a.count + PAIR_TILE - 1) / PAIR_TILE;
    auto k = cull_emit_kernel<PAIR_BLOCK, PAIR_TILE / PAIR_BLOCK>;
    const size_t smem = 4 * sizeof(unsigned) * padded<PAIR_TILE>();
    static std::atomic<unsigned long long> configured{0};
    if (cudaError_t e = allow_dynamic_smem(k, smem, configured)) return e;
    k<<<tiles, PAIR_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RBITS, int SRC, int BLOCK>
static cudaError_t launch_up_t(const UpArgs &a, cudaStream_t s)
{
    constexpr int ITEMS = PAIR_TILE / BLOCK;
    auto k = upsweep_kernel<BLOCK, ITEMS, RBITS, SRC>;
    const size_t smem = sizeof(unsigned) * (3 * (1 << RBITS) + (SRC == SRC_GEN ? padded<PAIR_TILE>() : 0));
    static std::atomic<unsigned long long> configured{0};
    if (cudaError_t e = allow_dynamic_smem(k, smem, configured)) return e;
    if (a.gtiles < 1 || a.gtiles > (unsigned)GROUP_TILES) return cudaErrorInvalidValue;
    const unsigned groups = (a.ntiles + a.gtiles - 1) / a.gtiles;
    k<<<groups, BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RBITS, int IN, int BLOCK, bool STABLE = true>
static cudaError_t launch_down_t(const DownArgs &a, unsigned ntiles, unsigned gtiles, cudaStream_t s)
{
    constexpr int ITEMS = PAIR_TILE / BLOCK;
    auto k = downsweep_kernel<BLOCK, ITEMS, RBITS, IN, STABLE>;
    constexpr size_t smem = down_smem_bytes<BLOCK, ITEMS, RBITS>();
    static std::atomic<unsigned long long> configured{0};
    if (cudaError_t e = allow_dynamic_smem(k, smem, configured)) return e;
    k<<<ntiles, BLOCK, smem, s>>>(a, gtiles);
    return cudaGetLastError();
}

unsigned group_tiles(unsigned ntiles, int nsm)
{
    // about 8 blocks per SM before groups grow past one tile
    const unsigned per = ntiles / (unsigned)(8 * (nsm > 0 ? nsm : 1));
    return per < 1u ? 1u : (per > (unsigned)GROUP_TILES ? (unsigned)GROUP_TILES : per);
}

template <int BLOCK>
static cudaError_t launch_up_b(const UpArgs &a, int rbits, int src, cudaStream_t s)
{
#define GG_UP(RB)                                                                                   \
    case RB:                                                                                        \
        return src == SRC_GEN ? launch_up_t<RB, SRC_GEN, BLOCK>(a, s) : launch_up_t<RB, SRC_MEM, BLOCK>(a, s);
    switch (rbits) {
        GG_UP(8)
        GG_UP(9)
        GG_UP(10)
        GG_UP(11)
    default:
        return cudaErrorInvalidValue;
    }
#undef GG_UP
}

template <int BLOCK>
static cudaError_t launch_down_b(const DownArgs &a, int rbits, int in, unsigned ntiles, unsigned gtiles,
                                 cudaStream_t s)
{
#define GG_DOWN(RB)                                                                                     \
    case RB:                                                                                            \
        return in == IN_GEN         ? launch_down_t<RB, IN_GEN, BLOCK>(a, ntiles, gtiles, s)            \
               : in == IN_PAIR      ? launch_down_t<RB, IN_PAIR, BLOCK>(a, ntiles, gtiles, s)           \
               : in == IN_PAIR_KEEP ? launch_down_t<RB, IN_PAIR_KEEP, BLOCK>(a, ntiles, gtiles, s)      \
                                    : launch_down_t<RB, IN_PAIR, BLOCK, false>(a, ntiles, gtiles, s);
    switch (rbits) {
        GG_DOWN(8)
        GG_DOWN(9)
        GG_DOWN(10)
        GG_DOWN(11)
    default:
        return cudaErrorInvalidValue;
    }
#undef GG_DOWN
}

cudaError_t launch_upsweep(const UpArgs &a, int rbits, int src, int shape, cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
    if (shape == SHAPE_MAIN) return launch_up_b<PAIR_BLOCK>(a, rbits, src, s);
    if (shape == SHAPE_ALT) return launch_up_b<ALT_BLOCK>(a, rbits, src, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_downsweep(const DownArgs &a, int rbits, int in, unsigned ntiles, unsigned gtiles, int shape,
                             cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    if (gtiles < 1 || gtiles > (unsigned)GROUP_TILES) return cudaErrorInvalidValue;
    if (shape == SHAPE_MAIN) return launch_down_b<PAIR_BLOCK>(a, rbits, in, ntiles, gtiles, s);
    if (shape == SHAPE_ALT) return launch_down_b<ALT_BLOCK>(a, rbits, in, ntiles, gtiles, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bucket_split(const LocalArgs &a, cudaStream_t s)
{
    bucket_split_kernel<<<(a.nbuckets + 1 + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_local_sort(const LocalArgs &a, cudaStream_t s)
{
    if (a.nbuckets == 0) return cudaSuccess;
    if (a.lbits < 0 || a.lbits > LOCAL_LMAX) return cudaErrorInvalidValue;
    auto k = local_sort_kernel<LOCAL_BLOCK>;
    const size_t smem = sizeof(unsigned) * (2 * (1 << LOCAL_LMAX) + 1 + LOCAL_CAP);
    static std::atomic<unsigned long long> configured{0};
    if (cudaError_t e = allow_dynamic_smem(k, smem, configured)) return e;
    if (a.max_groups == 0) return cudaSuccess;
    // a grid of a few rounds of resident blocks; each block loops over groups
    int dev = 0, nsm = 0;
    if (cudaError_t e = cudaGetDevice(&dev)) return e;
    if (cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) return e;
    const unsigned grid = min(a.max_groups, (unsigned)(nsm * LOCAL_MIN_BLOCKS * 4));
    k<<<grid, LOCAL_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

unsigned long long extract_blocks(unsigned long long count, unsigned long long ncells)
{
    return (count + ncells + 1ull + EXTRACT_TILE - 1) / EXTRACT_TILE;
}

cudaError_t launch_extract_split(const ExtractArgs &a, cudaStream_t s)
{
    const unsigned long long nb = extract_blocks(a.count, a.ncells);
    extract_split_kernel<<<(unsigned)((nb + 1 + 255) / 256), 256, 0, s>>>(a, nb);
    return cudaGetLastError();
}

cudaError_t launch_extract(const ExtractArgs &a, cudaStream_t s)
{
    const unsigned long long nb = extract_blocks(a.count, a.ncells);
    extract_kernel<EXTRACT_BLOCK, EXTRACT_TILE / EXTRACT_BLOCK><<<(unsigned)nb, EXTRACT_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gg
