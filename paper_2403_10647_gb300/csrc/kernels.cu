// CUDA kernels (sm_103a) of the parallel uniform-grid construction
// (Costa, Pereira, Jorge, "Building An Efficient Grid On GPU", Algorithm 1).
//
//   bounds_kernel      boxes of Algorithm 1: per-triangle AABB, block-reduced
//                      scene bounds, index / finiteness checks.
//   count_scan_kernel  CountCells + ExclusiveSum: per-object cell box and cell
//                      count V, single-pass decoupled look-back scan -> start
//                      offsets and NO.
//   tile_search_kernel first object of every pair tile (binary search).
//   emit_kernel        MakeObjectIds + InclusiveSum (as a max-scan of object
//                      start marks) + SegmentedExclusiveSum (rid = j - start)
//                      + MakeCellIds (GlobalCoords): one thread per pair.
//   hist_kernel        digit histograms of every radix-sort pass in one read
//                      (keys generated on the fly or loaded).
//   pass_kernel        one stable LSD radix-sort pass (RadixSort of Algorithm
//                      1): warp-level multisplit ranking, decoupled look-back
//                      across tiles per digit, shared-memory staged scatter.
//                      The first pass can generate its pairs instead of
//                      reading them, so (C, O) in object order never touch HBM.
//   extract_kernel     RunLengthEncode + NonEmptyCells + ExclusiveSum fused as
//                      a merge path of the sorted keys against the cell ids.
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

// GlobalCoords (Sec. 3) + cell linearisation for pair j of object record r.
__device__ __forceinline__ unsigned pair_cell(uint4 r, unsigned j, unsigned res_x, unsigned res_y)
{
    const unsigned lox = r.x & 0xFFFFu, loy = r.x >> 16, loz = r.y & 0xFFFFu;
    const unsigned hix = r.y >> 16, hiy = r.z & 0xFFFFu;
    const unsigned mx = hix - lox + 1u, my = hiy - loy + 1u;
    const unsigned mxy = mx * my;
    const unsigned rid = j - r.w;
    const unsigned z = rid / mxy;
    const unsigned rem = rid - z * mxy;
    const unsigned y = rem / mx;
    const unsigned x = rem - y * mx;
    return (lox + x) + res_x * ((loy + y) + res_y * (loz + z));
}

// MakeObjectIds + InclusiveSum for one pair tile, in shared memory: marks
// each object whose pair segment starts inside [j0, j0 + cnt) at its start
// position with its tile-local index, then an inclusive max-scan carries the
// owning object forward.  After the call mark[e] + *o_first is the object of
// pair j0 + e.  mark has BLOCK * ITEMS entries; s_tmp BLOCK / 32.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ unsigned tile_objects(const ObjRec *__restrict__ recs,
                                                 const unsigned *__restrict__ tile_obj, unsigned t,
                                                 unsigned j0, unsigned cnt, unsigned *mark,
                                                 unsigned *s_tmp)
{
    constexpr int T = BLOCK * ITEMS;
    constexpr int W = BLOCK / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned of = tile_obj[t], ol = tile_obj[t + 1];
    for (int p = tid; p < T; p += BLOCK) mark[p] = 0u;
    __syncthreads();
    for (unsigned o = of + 1u + tid; o <= ol; o += BLOCK) {
        const unsigned s = __ldg(&recs[o].start);
        const unsigned p = s - j0;
        if (s >= j0 && p < cnt) mark[p] = o - of;
    }
    __syncthreads();
    unsigned v[ITEMS];
    unsigned m = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        m = max(m, mark[tid * ITEMS + i]);
        v[i] = m;
    }
    unsigned inc = warp_incl_max(m);
    if (lane == 31) s_tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned x = lane < W ? s_tmp[lane] : 0u;
        x = warp_incl_max(x);
        if (lane < W) s_tmp[lane] = x;
    }
    __syncthreads();
    unsigned prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) prev = 0u;
    if (w > 0) prev = max(prev, s_tmp[w - 1]);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) mark[tid * ITEMS + i] = max(v[i], prev);
    __syncthreads();
    return of;
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

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) count_scan_kernel(CountArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    __shared__ unsigned long long s_pref[T];
    __shared__ unsigned long long s_tmp[BLOCK / 32];
    __shared__ unsigned s_tile;
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(&a.ctl->tickets[0], 1u);
    __syncthreads();
    const unsigned tile = s_tile;
    const long long base = (long long)tile * T;

    uint4 rec[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const long long o = base + i * BLOCK + tid;
        unsigned V = 0u;
        rec[i] = make_uint4(0u, 0u, 0u, 0u);
        if (o < a.n) {
            int vi[3];
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vi[k] = __ldg(a.tris + 3 * o + k);
                ok = ok && vi[k] >= 0 && (long long)vi[k] < a.nverts;
            }
            if (!ok) {  // never read outside verts: flag and use vertex 0
                atomicOr(&a.ctl->err, ERR_BADINDEX);
                vi[0] = vi[1] = vi[2] = 0;
            }
            unsigned clo[3], chi[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float p0 = __ldg(a.verts + 3ll * vi[0] + ax);
                const float p1 = __ldg(a.verts + 3ll * vi[1] + ax);
                const float p2 = __ldg(a.verts + 3ll * vi[2] + ax);
                const float bl = fminf(fminf(p0, p1), p2);
                const float bh = fmaxf(fmaxf(p0, p1), p2);
                clo[ax] = (unsigned)cell_coord(bl, a.lo[ax], a.scale[ax], a.res[ax]);
                chi[ax] = (unsigned)cell_coord(bh, a.lo[ax], a.scale[ax], a.res[ax]);
            }
            unsigned long long cnt = (unsigned long long)(chi[0] - clo[0] + 1u) *
                                     (unsigned long long)(chi[1] - clo[1] + 1u) *
                                     (unsigned long long)(chi[2] - clo[2] + 1u);
            V = cnt > 0x80000000ull ? 0x80000000u : (unsigned)cnt;
            rec[i].x = clo[0] | (clo[1] << 16);
            rec[i].y = clo[2] | (chi[0] << 16);
            rec[i].z = chi[1] | (chi[2] << 16);
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

    if (tid == 0) {
        unsigned long long *st = a.status;
        unsigned long long excl = 0;
        if (tile == 0) {
            st_relaxed_u64(&st[0], LB64_PREFIX | total);
        } else {
            st_relaxed_u64(&st[tile], LB64_AGG | total);
            long long k = (long long)tile - 1;
            unsigned spins = 0;
            while (k >= 0) {
                const unsigned long long v = ld_relaxed_u64(&st[k]);
                if (v == 0ull) {
                    if (++spins > SPIN_LIMIT) {
                        atomicOr(&a.ctl->err, ERR_TIMEOUT);
                        break;
                    }
                    if (spins > 8) __nanosleep(64);
                    continue;
                }
                excl += v & LB64_VALUE;
                if (v & LB64_PREFIX) break;
                --k;
            }
            st_relaxed_u64(&st[tile], LB64_PREFIX | ((excl + total) & LB64_VALUE));
        }
        s_excl = excl;
        if (excl + total > 0x7FFFFFFFull) atomicOr(&a.ctl->err, ERR_OVERFLOW);
        if (base + T >= a.n) a.ctl->nrefs = excl + total;
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const long long o = base + i * BLOCK + tid;
        if (o < a.n) {
            uint4 r = rec[i];
            r.w = (unsigned)(excl + s_pref[i * BLOCK + tid]);
            reinterpret_cast<uint4 *>(a.recs)[o] = r;
        }
    }
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
    __shared__ unsigned s_mark[T];
    __shared__ unsigned s_tmp[BLOCK / 32];
    const unsigned t = blockIdx.x;
    const unsigned j0 = t * (unsigned)T;
    const unsigned cnt = min((unsigned)T, a.count - j0);
    const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, t, j0, cnt, s_mark, s_tmp);
#pragma unroll 4
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = i * BLOCK + threadIdx.x;
        if (e < cnt) {
            const unsigned o = of + s_mark[e];
            const uint4 r = __ldg(reinterpret_cast<const uint4 *>(a.recs) + o);
            a.C[j0 + e] = pair_cell(r, j0 + e, a.res_x, a.res_y);
            a.O[j0 + e] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// a8: radix sort - digit histograms of all passes
// ---------------------------------------------------------------------------

template <int BLOCK, int ITEMS, int RBITS, int SRC>
__global__ void __launch_bounds__(BLOCK) hist_kernel(HistArgs a)
{
    constexpr int T = BLOCK * ITEMS;
    constexpr int R = 1 << RBITS;
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_hist = smem;                          // [npasses][R]
    unsigned *s_mark = s_hist + MAX_PASSES * R;       // [T] (generated keys only)
    __shared__ unsigned s_tmp[BLOCK / 32];
    __shared__ unsigned s_last;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.npasses * R; i += BLOCK) s_hist[i] = 0u;
    __syncthreads();

    for (unsigned t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const unsigned j0 = t * (unsigned)T;
        const unsigned cnt = min((unsigned)T, a.count - j0);
        unsigned keys[ITEMS];
        if (SRC == SRC_GEN) {
            const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, t, j0, cnt, s_mark, s_tmp);
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const unsigned e = tid * ITEMS + i;
                keys[i] = 0u;
                if (e < cnt) {
                    const unsigned o = of + s_mark[e];
                    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(a.recs) + o);
                    keys[i] = pair_cell(r, j0 + e, a.res_x, a.res_y);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const unsigned e = tid * ITEMS + i;
                keys[i] = e < cnt ? __ldg(a.keys_in + j0 + e) : 0u;
            }
        }
        const unsigned nv = cnt > (unsigned)(tid * ITEMS) ? min((unsigned)ITEMS, cnt - tid * ITEMS) : 0u;
#pragma unroll
        for (int p = 0; p < MAX_PASSES; ++p) {
            if (p >= a.npasses) break;
            const unsigned sh = a.shift[p], mk = (1u << a.bits[p]) - 1u;
            unsigned prev = 0xFFFFFFFFu, run = 0u;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if ((unsigned)i < nv) {
                    const unsigned d = (keys[i] >> sh) & mk;
                    if (d == prev) {
                        ++run;
                    } else {
                        if (run) atomicAdd(&s_hist[p * R + prev], run);
                        prev = d;
                        run = 1u;
                    }
                }
            }
            if (run) atomicAdd(&s_hist[p * R + prev], run);
        }
        // this tile's look-back row of the first sort pass starts at zero
        for (int d = tid; d < a.status_row; d += BLOCK) a.status0[(size_t)t * a.status_row + d] = 0u;
        __syncthreads();
    }
    __syncthreads();
    for (int i = tid; i < a.npasses * R; i += BLOCK) {
        const unsigned v = s_hist[i];
        if (v) atomicAdd(&a.hist[(i / R) * MAX_RADIX + (i % R)], v);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&a.ctl->hist_done, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: exclusive scan of every pass's histogram -> digit bases
#pragma unroll
    for (int p = 0; p < MAX_PASSES; ++p) {
        if (p >= a.npasses) break;
        const int nd = 1 << a.bits[p];
        unsigned carry = 0;
        for (int c0 = 0; c0 < nd; c0 += BLOCK) {
            const int d = c0 + tid;
            const unsigned v = d < nd ? __ldcg(&a.hist[p * MAX_RADIX + d]) : 0u;
            unsigned tot;
            const unsigned ex = block_excl_sum<BLOCK>(v, s_tmp, &tot);
            if (d < nd) {
                a.dbase[p * MAX_RADIX + d] = carry + ex;
                a.hist[p * MAX_RADIX + d] = 0u;   // leave the histogram zeroed for the next use
            }
            carry += tot;
        }
    }
    if (tid < MAX_PASSES) a.ctl->tickets[1 + tid] = 0u;
    if (tid == 0) a.ctl->hist_done = 0u;
}

// ---------------------------------------------------------------------------
// a8: radix sort - one onesweep-style LSD pass
// ---------------------------------------------------------------------------

constexpr unsigned LB_PREFIX = 0x80000000u;   // value = inclusive prefix
                                              // else value - 1 = tile aggregate; 0 = not ready

template <int BLOCK, int ITEMS, int RBITS>
constexpr size_t pass_smem_bytes()
{
    return sizeof(unsigned) * (2 * BLOCK * ITEMS + (BLOCK / 32) * ((1 << RBITS) + 1) +
                               ((1 << RBITS) + 1) + (1 << RBITS) + BLOCK / 32 + 4);
}

template <int BLOCK, int ITEMS, int RBITS, int SRC>
__global__ void __launch_bounds__(BLOCK) pass_kernel(PassArgs a)
{
    constexpr int W = BLOCK / 32;
    constexpr int T = BLOCK * ITEMS;
    constexpr int R = 1 << RBITS;
    constexpr int RW = R + 1;                 // one extra bucket for the tail of the last tile
    static_assert(R % BLOCK == 0, "digits per thread");
    extern __shared__ __align__(16) unsigned smem[];
    unsigned *s_keys = smem;                  // [T]  (aliases the object marks while generating)
    unsigned *s_vals = s_keys + T;            // [T]
    unsigned *s_whist = s_vals + T;           // [W][R + 1]
    unsigned *s_dstart = s_whist + W * RW;    // [R + 1]
    unsigned *s_gbase = s_dstart + RW;        // [R]
    unsigned *s_tmp = s_gbase + R;            // [W]
    unsigned *s_misc = s_tmp + W;             // [4]

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_misc[0] = atomicAdd(a.ticket, 1u);
    for (int i = tid; i < W * RW; i += BLOCK) s_whist[i] = 0u;
    __syncthreads();
    const unsigned tile = s_misc[0];
    const unsigned j0 = tile * (unsigned)T;
    const unsigned cnt = min((unsigned)T, a.count - j0);
    const unsigned sh = a.shift, mk = (1u << a.bits) - 1u;

    unsigned keys[ITEMS], vals[ITEMS];
    if (SRC == SRC_GEN) {
        const unsigned of = tile_objects<BLOCK, ITEMS>(a.recs, a.tile_obj, tile, j0, cnt, s_keys, s_tmp);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            keys[i] = 0u;
            vals[i] = 0u;
            if (e < cnt) {
                const unsigned o = of + s_keys[e];
                const uint4 r = __ldg(reinterpret_cast<const uint4 *>(a.recs) + o);
                keys[i] = pair_cell(r, j0 + e, a.res_x, a.res_y);
                vals[i] = o;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            keys[i] = e < cnt ? __ldcs(a.keys_in + j0 + e) : 0u;
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const unsigned e = w * 32 * ITEMS + i * 32 + lane;
            vals[i] = e < cnt ? __ldcs(a.vals_in + j0 + e) : 0u;
        }
    }

    // warp-level multisplit: rank of each element among equal digits, in
    // element order (items in order, lanes in order)
    unsigned ranks[ITEMS];
    unsigned *wh = s_whist + w * RW;
    const unsigned ltmask = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = w * 32 * ITEMS + i * 32 + lane;
        const unsigned d = e < cnt ? (keys[i] >> sh) & mk : (unsigned)R;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned before = wh[d];
        const unsigned lt = __popc(peers & ltmask);
        __syncwarp();
        if (lt == 0) wh[d] = before + __popc(peers);
        __syncwarp();
        ranks[i] = before + lt;
    }
    __syncthreads();

    // per digit: exclusive offsets across warps, tile count, publish aggregate
    for (int d = tid; d < RW; d += BLOCK) {
        unsigned sum = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) {
            const unsigned c = s_whist[ww * RW + d];
            s_whist[ww * RW + d] = sum;
            sum += c;
        }
        s_dstart[d] = sum;
        if (d < R) {
            unsigned *st = a.status + (size_t)tile * R + d;
            st_relaxed_u32(st, tile == 0 ? (LB_PREFIX | sum) : sum + 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the tile's digit counts -> local digit starts
    {
        constexpr int C = R / BLOCK;
        unsigned loc[C];
        unsigned s = 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            loc[k] = s_dstart[tid * C + k];
            s += loc[k];
        }
        unsigned tot;
        unsigned ex = block_excl_sum<BLOCK>(s, s_tmp, &tot);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            s_dstart[tid * C + k] = ex;
            ex += loc[k];
        }
        if (tid == 0) s_dstart[R] = tot;
    }
    __syncthreads();
    // stage the tile in shared memory in locally sorted order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned e = w * 32 * ITEMS + i * 32 + lane;
        const unsigned d = e < cnt ? (keys[i] >> sh) & mk : (unsigned)R;
        const unsigned pos = s_dstart[d] + s_whist[w * RW + d] + ranks[i];
        s_keys[pos] = keys[i];
        s_vals[pos] = vals[i];
    }
    // decoupled look-back per digit
    for (int d = tid; d < R; d += BLOCK) {
        const unsigned cntd = s_dstart[d + 1] - s_dstart[d];
        unsigned excl = 0;
        if (tile > 0) {
            const unsigned *st = a.status + d;
            long long k = (long long)tile - 1;
            unsigned spins = 0;
            while (k >= 0) {
                const unsigned v = ld_relaxed_u32(st + (size_t)k * R);
                if (v == 0u) {
                    if (++spins > SPIN_LIMIT) {
                        atomicOr(&a.ctl->err, ERR_TIMEOUT);
                        break;
                    }
                    if (spins > 8) __nanosleep(32);
                    continue;
                }
                if (v & LB_PREFIX) {
                    excl += v & ~LB_PREFIX;
                    break;
                }
                excl += v - 1u;
                --k;
            }
            st_relaxed_u32(a.status + (size_t)tile * R + d, LB_PREFIX | (excl + cntd));
        }
        s_gbase[d] = a.dbase[d] + excl - s_dstart[d];
        if (a.status_next) a.status_next[(size_t)tile * R + d] = 0u;
    }
    __syncthreads();
    // scatter: consecutive threads write consecutive positions of a digit run
    bool bad = false;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const unsigned pos = i * BLOCK + tid;
        if (pos < cnt) {
            const unsigned k = s_keys[pos];
            const unsigned dst = s_gbase[(k >> sh) & mk] + pos;
            if (dst < a.count) {
                __stcg(a.keys_out + dst, k);
                __stcg(a.vals_out + dst, s_vals[pos]);
            } else {
                bad = true;
            }
        }
    }
    if (bad) atomicOr(&a.ctl->err, ERR_RANGE);
}

// ---------------------------------------------------------------------------
// a9: RunLengthEncode + NonEmptyCells + ExclusiveSum as one merge path
// ---------------------------------------------------------------------------

// Merge order: cell c precedes key k iff c <= k, so G[c] = number of keys
// before cell c in the merged sequence = number of keys < c.
__device__ __forceinline__ unsigned long long merge_split(const unsigned *keys, unsigned long long nA,
                                                          unsigned long long nB, unsigned long long d,
                                                          unsigned long long c_base)
{
    unsigned long long lo = d > nB ? d - nB : 0ull;
    unsigned long long hi = d < nA ? d : nA;
    while (lo < hi) {
        const unsigned long long mid = (lo + hi) >> 1;
        // key[mid] precedes cell (d - mid - 1)?
        if ((unsigned long long)keys[mid] < c_base + (d - mid - 1ull))
            lo = mid + 1ull;
        else
            hi = mid;
    }
    return lo;
}

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) extract_kernel(ExtractArgs a)
{
    constexpr int D = BLOCK * ITEMS;
    __shared__ unsigned s_keys[D];
    __shared__ unsigned s_G[D];
    __shared__ unsigned long long s_split[2];
    const int tid = threadIdx.x;
    const unsigned long long nA = a.count, nB = a.ncells + 1ull;
    const unsigned long long M = nA + nB;
    const unsigned long long d0 = (unsigned long long)blockIdx.x * D;
    const unsigned long long d1 = min(d0 + D, M);
    if (tid < 2) s_split[tid] = merge_split(a.keys, nA, nB, tid == 0 ? d0 : d1, 0ull);
    __syncthreads();
    const unsigned long long i0 = s_split[0], i1 = s_split[1];
    const unsigned long long c0 = d0 - i0, c1 = d1 - i1;
    const unsigned na = (unsigned)(i1 - i0), nb = (unsigned)(c1 - c0);
    for (unsigned k = tid; k < na; k += BLOCK) s_keys[k] = __ldcs(a.keys + i0 + k);
    __syncthreads();
    const unsigned td0 = tid * ITEMS;
    const unsigned nd = (unsigned)(d1 - d0);
    if (td0 < nd) {
        // local split on the diagonal td0 of (s_keys[0..na), cells c0 ..)
        unsigned lo = td0 > nb ? td0 - nb : 0u;
        unsigned hi = min(td0, na);
        while (lo < hi) {
            const unsigned mid = (lo + hi) >> 1;
            if ((unsigned long long)s_keys[mid] < c0 + (td0 - mid - 1u))
                lo = mid + 1u;
            else
                hi = mid;
        }
        unsigned ia = lo, ib = td0 - lo;
        const unsigned steps = min((unsigned)ITEMS, nd - td0);
        unsigned bad = 0;
        for (unsigned s = 0; s < steps; ++s) {
            const bool take_cell = ib < nb && (ia >= na || c0 + ib <= (unsigned long long)s_keys[ia]);
            if (take_cell) {
                s_G[ib] = (unsigned)(i0 + ia);
                ++ib;
            } else {
                if (s_keys[ia] >= a.ncells) bad = 1u;
                ++ia;
            }
        }
        if (bad) atomicOr(&a.ctl->err, ERR_RANGE);
    }
    __syncthreads();
    for (unsigned k = tid; k < nb; k += BLOCK) a.G[c0 + k] = s_G[k];
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

cudaError_t launch_count_scan(const CountArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const long long tiles = (a.n + COUNT_TILE - 1) / COUNT_TILE;
    count_scan_kernel<COUNT_BLOCK, COUNT_TILE / COUNT_BLOCK><<<(unsigned)tiles, COUNT_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
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
    emit_kernel<PAIR_BLOCK, PAIR_TILE / PAIR_BLOCK><<<tiles, PAIR_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <int RBITS, int SRC>
static cudaError_t launch_hist_t(const HistArgs &a, int nsm, cudaStream_t s)
{
    constexpr int ITEMS = PAIR_TILE / PAIR_BLOCK;
    auto k = hist_kernel<PAIR_BLOCK, ITEMS, RBITS, SRC>;
    const size_t smem = sizeof(unsigned) * (MAX_PASSES * (1 << RBITS) + (SRC == SRC_GEN ? PAIR_TILE : 0));
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned blocks = a.ntiles;
    const unsigned cap = (unsigned)nsm * 4u;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k<<<blocks, PAIR_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RBITS, int SRC>
static cudaError_t launch_pass_t(const PassArgs &a, unsigned ntiles, cudaStream_t s)
{
    constexpr int ITEMS = PAIR_TILE / PAIR_BLOCK;
    auto k = pass_kernel<PAIR_BLOCK, ITEMS, RBITS, SRC>;
    constexpr size_t smem = pass_smem_bytes<PAIR_BLOCK, ITEMS, RBITS>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k<<<ntiles, PAIR_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hist(const HistArgs &a, int rbits, int src, int nsm, cudaStream_t s)
{
    if (a.ntiles == 0) return cudaSuccess;
#define GG_HIST(RB)                                                        \
    case RB:                                                               \
        return src == SRC_GEN ? launch_hist_t<RB, SRC_GEN>(a, nsm, s)     \
                              : launch_hist_t<RB, SRC_MEM>(a, nsm, s);
    switch (rbits) {
        GG_HIST(8)
        GG_HIST(9)
        GG_HIST(10)
        GG_HIST(11)
    default:
        return cudaErrorInvalidValue;
    }
#undef GG_HIST
}

cudaError_t launch_pass(const PassArgs &a, int rbits, int src, unsigned ntiles, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
#define GG_PASS(RB)                                                        \
    case RB:                                                               \
        return src == SRC_GEN ? launch_pass_t<RB, SRC_GEN>(a, ntiles, s)  \
                              : launch_pass_t<RB, SRC_MEM>(a, ntiles, s);
    switch (rbits) {
        GG_PASS(8)
        GG_PASS(9)
        GG_PASS(10)
        GG_PASS(11)
    default:
        return cudaErrorInvalidValue;
    }
#undef GG_PASS
}

cudaError_t launch_extract(const ExtractArgs &a, cudaStream_t s)
{
    const unsigned long long M = a.count + a.ncells + 1ull;
    const unsigned long long blocks = (M + EXTRACT_TILE - 1) / EXTRACT_TILE;
    extract_kernel<EXTRACT_BLOCK, EXTRACT_TILE / EXTRACT_BLOCK><<<(unsigned)blocks, EXTRACT_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gg
