// Host runtime of the grid builder: context, stream-ordered memory pool,
// grid planner (metadata M of Algorithm 1), build orchestration and the
// C ABI declared in include/grid.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "grid.h"
#include "kernels.h"

using gg::Ctl;
using gg::ObjRec;

// The hybrid placement's first radix pass may rank equal digits out of order
// (1) or keeps them in order (0, for comparison).
#ifndef GG_FIRST_ANY
#define GG_FIRST_ANY 1
#endif
// Bits the hybrid placement's first radix pass takes beyond an even split
// (its ranking is the cheaper one).
#ifndef GG_FIRST_EXTRA
#define GG_FIRST_EXTRA 0
#endif
#ifndef GG_LOCAL_PAIRS_PER_CELL
#define GG_LOCAL_PAIRS_PER_CELL 6.0
#endif
constexpr double LOCAL_PAIRS_PER_CELL = GG_LOCAL_PAIRS_PER_CELL;

namespace {

constexpr int64_t kInt32Max = 0x7FFFFFFFll;

// Keeps the caller's current device and restores it on exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Grow-only device buffer from the context's pool.
struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

enum KernelId {
    K_BOUNDS, K_COUNT, K_TILES, K_EMIT, K_UP_GEN, K_DOWN_GEN, K_UP, K_DOWN, K_SPLIT, K_EXTRACT, K_LOCALIZE,
    K_PER_OBJECT, K_CULL, K_BSPLIT, K_LOCAL, K_DOWN_ANY, K_PLAN, K_DOWN_KEEP, K_REBASE, K_NUM
};
const char *const kKernelNames[K_NUM] = {"bounds",  "count_scan",    "tile_search",   "emit",
                                         "upsweep_gen", "downsweep_gen", "upsweep", "downsweep",
                                         "extract_split", "extract",   "localize", "make_pairs_per_object",
                                         "cull_emit", "bucket_split", "local_sort", "downsweep_first", "plan",
                                         "downsweep_keep", "rebase"};

struct PendingTiming {
    int kid;
    cudaEvent_t start, stop;
};

}  // namespace

struct grid_ctx {
    int device = 0;
    int nsm = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;   // grid_build_host: the refs' copy overlaps range extraction
    cudaEvent_t copy_ev = nullptr;
    cudaMemPool_t pool = nullptr;
    grid_opts opts{};
    int rbits_max = 9;
    int shape = 0;               // block shape of the radix kernels (gg::SHAPE_*)
    int pair_gen = GRID_PAIRS_FUSED;
    bool cull = false;
    int local_bits = 0;          // grid_opts.local_bits
    int64_t fallbacks = 0;       // hybrid placements redone by radix passes over every key bit
    int64_t plan_redos = 0;      // builds whose device M differed from the host's

    Ctl *d_ctl = nullptr;        // device control block
    Ctl *h_ctl = nullptr;        // pinned host mirror
    unsigned *d_dbase = nullptr; // [MAX_PASSES][MAX_RADIX]

    Scratch recs, k2status, tile_obj, keys_sorted, keys[1], vals[1], intra, gpref, gstatus, splits;
    Scratch vals_sorted, bstarts, bgroups;   // hybrid placement: last radix pass's values, bucket
                                             // starts, bucket groups
    Scratch in_verts, in_tris, out_cells, out_refs;  // host-buffer builds
    Scratch b_desc, b_base, b_state, b_pairbase, b_cellsoff, b_G;   // batched builds
    Scratch b_seg;                  // batched builds sorted in segments: the segments' tables
    Scratch pairs_C, pairs_O;    // object-order pairs of the unfused pair_gen modes and of culling
    void *h_stage = nullptr;     // pinned host tables of batched builds (grow-only)
    size_t h_stage_bytes = 0;
    bool stage_busy = false;     // a copy from h_stage may still be in flight
    Scratch cstatus;             // culling emit look-back words
    std::atomic<int64_t> in_use{0};

    // per-kernel accounting
    bool profile = false;
    int64_t launches[K_NUM] = {};
    double kernel_ms[K_NUM] = {};
    double kernel_bytes[K_NUM] = {};
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> free_events;
};

namespace {

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return GRID_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // not sticky: clear it
        return GRID_ENOMEM;
    }
    return GRID_ECUDA;
}

#define GG_TRY(expr)                       \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != GRID_OK) return _rc;    \
    } while (0)

#define GG_CUDA(expr) GG_TRY(cuda_err(expr))

int pool_alloc(grid_ctx *c, size_t bytes, void **out)
{
    *out = nullptr;
    if (bytes == 0) return GRID_OK;
    cudaError_t e = cudaMallocFromPoolAsync(out, bytes, c->pool, c->stream);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_err(e);
    }
    c->in_use += (int64_t)bytes;
    return GRID_OK;
}

void pool_free(grid_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    cudaFreeAsync(p, c->stream);
    c->in_use -= (int64_t)bytes;
}

int ensure(grid_ctx *c, Scratch &s, size_t bytes)
{
    if (s.bytes >= bytes) return GRID_OK;
    pool_free(c, s.ptr, s.bytes);
    s.ptr = nullptr;
    s.bytes = 0;
    size_t want = bytes + bytes / 8;  // headroom against small growth
    want = (want + 255) & ~size_t(255);
    void *p = nullptr;
    GG_TRY(pool_alloc(c, want, &p));
    s.ptr = p;
    s.bytes = want;
    return GRID_OK;
}

void release(grid_ctx *c, Scratch &s)
{
    pool_free(c, s.ptr, s.bytes);
    s.ptr = nullptr;
    s.bytes = 0;
}

// Pinned host staging of at least `bytes` for a batched build's tables, so
// their copies are asynchronous.  If an earlier call left copies from it in
// flight (it returned before its final synchronisation), wait for them first.
int host_stage(grid_ctx *c, size_t bytes, char **out)
{
    if (c->stage_busy) {
        GG_CUDA(cudaStreamSynchronize(c->stream));
        c->stage_busy = false;
    }
    if (c->h_stage_bytes < bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        const size_t want = (bytes + bytes / 2 + 4095) & ~size_t(4095);
        void *p = nullptr;
        GG_CUDA(cudaMallocHost(&p, want));
        c->h_stage = p;
        c->h_stage_bytes = want;
    }
    *out = (char *)c->h_stage;
    return GRID_OK;
}

cudaEvent_t take_event(grid_ctx *c)
{
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one kernel launch: counts it, adds its algorithmic bytes and, when
// profiling, records events on the launching stream around it.
struct KernelScope {
    grid_ctx *c;
    int kid;
    cudaEvent_t start = nullptr;
    KernelScope(grid_ctx *ctx, int k, double bytes) : c(ctx), kid(k)
    {
        c->launches[kid] += 1;
        c->kernel_bytes[kid] += bytes;
        if (c->profile) {
            start = take_event(c);
            if (start) cudaEventRecord(start, c->stream);
        }
    }
    ~KernelScope()
    {
        if (!start) return;
        cudaEvent_t stop = take_event(c);
        if (!stop) {
            c->free_events.push_back(start);
            return;
        }
        cudaEventRecord(stop, c->stream);
        c->pending.push_back(PendingTiming{kid, start, stop});
    }
};

void resolve_timings(grid_ctx *c)
{
    for (const PendingTiming &t : c->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) c->kernel_ms[t.kid] += ms;
        else cudaGetLastError();
        c->free_events.push_back(t.start);
        c->free_events.push_back(t.stop);
    }
    c->pending.clear();
}

// Error bits raised by the kernels -> GRID_* code.
int ctl_error(unsigned err)
{
    err &= ~(gg::ERR_LOCAL_FALLBACK | gg::ERR_TILE_REDO);   // requests to the host, handled where they arise
    if (err & (gg::ERR_BADINDEX | gg::ERR_NONFINITE | gg::ERR_RANGE)) return GRID_EINVAL;
    if (err & gg::ERR_OVERFLOW) return GRID_EOVERFLOW;
    if (err & gg::ERR_TIMEOUT) return GRID_ETIMEOUT;
    return GRID_OK;
}

// Scene bounds from their ordered-integer reductions.  The reduction ranks
// -0.0 below +0.0; a zero bound is reported as +0.0 (adding +0.0 clears the
// sign of a zero and changes no other value).
float bound_lo(unsigned lo_inv) { return gg::ordered_to_float(~lo_inv) + 0.0f; }
float bound_hi(unsigned hi_ord) { return gg::ordered_to_float(hi_ord) + 0.0f; }

int read_ctl(grid_ctx *c)
{
    GG_CUDA(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    GG_CUDA(cudaStreamSynchronize(c->stream));
    return GRID_OK;
}

int reset_ctl(grid_ctx *c)
{
    GG_CUDA(cudaMemsetAsync(c->d_ctl, 0, sizeof(Ctl), c->stream));
    return GRID_OK;
}

// ---- grid metadata M -------------------------------------------------------
// res_a = clamp(ceil(e_a * k), 1, RES_MAX), k = (lambda n / prod_nonzero e)^(1/d)
// in FP64; scale_a = (float)res_a / e_a in FP32.
int plan(const float lo[3], const float hi[3], int64_t n, float lambda, grid_info *info)
{
    if (n < 0 || !std::isfinite(lambda) || !(lambda > 0.0f)) return GRID_EINVAL;
    std::memset(info, 0, sizeof(*info));
    float e[3];
    int d = 0;
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        info->lo[a] = lo[a];
        info->hi[a] = hi[a];
        e[a] = hi[a] - lo[a];
        info->res[a] = 1;
        info->scale[a] = 0.0f;
        if (n > 0 && e[a] > 0.0f) {
            ++d;
            vol = vol * (double)e[a];
        }
    }
    if (d > 0) {
        const double q = ((double)lambda * (double)n) / vol;
        const double k = d == 3 ? std::cbrt(q) : (d == 2 ? std::sqrt(q) : q);
        for (int a = 0; a < 3; ++a) {
            if (!(e[a] > 0.0f)) continue;
            double r = std::ceil((double)e[a] * k);
            if (!(r >= 1.0)) r = 1.0;
            if (r > (double)GRID_RES_MAX) r = (double)GRID_RES_MAX;
            info->res[a] = (int32_t)r;
            info->scale[a] = (float)info->res[a] / e[a];
        }
    }
    info->n = n;
    info->ncells = (int64_t)info->res[0] * info->res[1] * info->res[2];
    info->key_bits = 0;
    if (info->ncells > 1) {
        uint64_t m = (uint64_t)(info->ncells - 1);
        int b = 0;
        while (m) {
            ++b;
            m >>= 1;
        }
        info->key_bits = b;
    }
    if (info->ncells > kInt32Max) return GRID_EOVERFLOW;
    return GRID_OK;
}

// ---- radix-sort pass layout --------------------------------------------------
struct SortCfg {
    int passes = 0;
    int rbits = 8;  // widest kernel instantiation (sizes the per-tile tables)
    int rb[gg::MAX_PASSES] = {8, 8, 8, 8};   // each pass's kernels: its digit width, at least 8
    int shift[gg::MAX_PASSES] = {0, 0, 0, 0};
    int bits[gg::MAX_PASSES] = {0, 0, 0, 0};
};

// Passes over the key bits [lo_bit, key_bits): as few as digits of at most
// rbits_max bits allow, the bits split as evenly as possible; first_extra
// moves that many bits from the last pass to the first (at most up to
// rbits_max).
SortCfg sort_cfg(int key_bits, int rbits_max, int lo_bit = 0, int first_extra = 0)
{
    SortCfg s;
    const int nbits = key_bits - lo_bit;
    if (nbits <= 0) return s;
    s.passes = (nbits + rbits_max - 1) / rbits_max;
    int sh = lo_bit, widest = 0;
    for (int p = 0; p < s.passes; ++p) {
        int b = nbits / s.passes + (p < nbits % s.passes ? 1 : 0);
        if (s.passes > 1) {
            const int base0 = nbits / s.passes + (nbits % s.passes ? 1 : 0);
            const int e = std::max(0, std::min(std::min(first_extra, rbits_max - base0), nbits / s.passes - 1));
            if (p == 0) b += e;
            if (p == s.passes - 1) b -= e;
        }
        s.shift[p] = sh;
        s.bits[p] = b;
        s.rb[p] = std::max(8, b);
        sh += b;
        widest = std::max(widest, b);
    }
    s.rbits = std::max(8, widest);
    return s;
}

unsigned pair_tiles(int64_t count) { return (unsigned)((count + gg::PAIR_TILE - 1) / gg::PAIR_TILE); }

// Radix sort of (keys, vals) over the configured passes.  If gen is set, the
// first pass generates the object-order pairs from recs/tile_obj; otherwise
// it reads keys_in/vals_in.  The last pass writes keys_last / vals_last;
// pass outputs alternate between those and one scratch pair of arrays so
// the last lands there.  first_any: the first pass need not keep equal
// digits in input order, and the later ones need keep only the order of the
// key bits below their digit down to the first pass's lowest bit (the hybrid
// placement restores the order inside each bucket itself).
int sort_pairs(grid_ctx *c, const SortCfg &sc, unsigned count, bool gen, const ObjRec *recs, int64_t nobj,
               const unsigned *tile_obj, unsigned res_x, unsigned res_y, const gg::MeshTab &mt,
               const unsigned *keys_in, const unsigned *vals_in, unsigned *keys_last, unsigned *vals_last,
               bool first_any = false)
{
    const unsigned ntiles = pair_tiles(count);
    const unsigned gtiles = gg::group_tiles(ntiles, c->nsm);
    const unsigned ngroups = (ntiles + gtiles - 1) / gtiles;
    const int R = 1 << sc.rbits;
    const size_t elem = (size_t)count * sizeof(unsigned);
    // generated pairs are stored once by the first upsweep unless the first
    // pass regenerates them in both of its kernels
    const bool store = gen && c->pair_gen != GRID_PAIRS_REGEN;
    GG_TRY(ensure(c, c->intra, (size_t)ntiles * R * sizeof(unsigned short)));
    GG_TRY(ensure(c, c->gpref, (size_t)ngroups * R * sizeof(unsigned)));
    // every pass gets its own zeroed look-back words: one clear for the sort
    const size_t status_words = (size_t)ngroups * R;
    GG_TRY(ensure(c, c->gstatus, (size_t)std::max(sc.passes, 1) * status_words * sizeof(unsigned)));
    if (sc.passes > 0)
        GG_CUDA(cudaMemsetAsync(c->gstatus.ptr, 0, (size_t)sc.passes * status_words * sizeof(unsigned),
                                c->stream));
    if (sc.passes > 1 || store) {
        GG_TRY(ensure(c, c->keys[0], elem));
        GG_TRY(ensure(c, c->vals[0], elem));
    }
    unsigned *ko[gg::MAX_PASSES], *vo[gg::MAX_PASSES];
    for (int p = 0; p < sc.passes; ++p) {
        const bool to_last = ((sc.passes - 1 - p) % 2) == 0;
        ko[p] = to_last ? keys_last : (unsigned *)c->keys[0].ptr;
        vo[p] = to_last ? vals_last : (unsigned *)c->vals[0].ptr;
    }
    // the stored pairs go to the pair of arrays the first pass does not write
    unsigned *gk = nullptr, *gv = nullptr;
    if (store) {
        const bool first_to_last = ko[0] == keys_last;
        gk = first_to_last ? (unsigned *)c->keys[0].ptr : keys_last;
        gv = first_to_last ? (unsigned *)c->vals[0].ptr : vals_last;
        keys_in = gk;
        vals_in = gv;
    }
    for (int p = 0; p < sc.passes; ++p) {
        const bool first = p == 0;
        const unsigned *kin = first ? keys_in : ko[p - 1];
        const unsigned *vin = first ? vals_in : vo[p - 1];
        gg::UpArgs u{};
        u.keys_in = kin;
        u.recs = recs;
        u.tile_obj = tile_obj;
        u.mt = mt;
        u.res_x = res_x;
        u.res_y = res_y;
        u.gen_keys = first ? gk : nullptr;
        u.gen_vals = first ? gv : nullptr;
        u.count = count;
        u.ntiles = ntiles;
        u.gtiles = gtiles;
        u.shift = sc.shift[p];
        u.bits = sc.bits[p];
        u.intra = (unsigned short *)c->intra.ptr;
        u.gpref = (unsigned *)c->gpref.ptr;
        u.status = (unsigned *)c->gstatus.ptr + (size_t)p * status_words;
        u.dbase = c->d_dbase + p * gg::MAX_RADIX;
        u.ctl = c->d_ctl;
        const bool gen_up = first && gen;
        const bool gen_down = gen_up && !store;
        {
            KernelScope ks(c, gen_up ? K_UP_GEN : K_UP,
                           gen_up ? 16.0 * nobj + (store ? 8.0 * count : 0.0) : 4.0 * count);
            GG_CUDA(gg::launch_upsweep(u, sc.rb[p], gen_up ? gg::SRC_GEN : gg::SRC_MEM, c->shape, c->stream));
        }
        gg::DownArgs a{};
        a.keys_in = kin;
        a.vals_in = vin;
        a.recs = recs;
        a.tile_obj = tile_obj;
        a.mt = mt;
        a.res_x = res_x;
        a.res_y = res_y;
        a.keys_out = ko[p];
        a.vals_out = vo[p];
        a.count = count;
        a.shift = sc.shift[p];
        a.bits = sc.bits[p];
        a.dbase = c->d_dbase + p * gg::MAX_RADIX;
        a.gpref = (const unsigned *)c->gpref.ptr;
        a.intra = (const unsigned short *)c->intra.ptr;
        a.ctl = c->d_ctl;
        const int in = gen_down ? gg::IN_GEN
                       : first_any ? (first ? gg::IN_PAIR_ANY : gg::IN_PAIR_KEEP)
                                   : gg::IN_PAIR;
        a.keep_lo = sc.shift[0];
        KernelScope ks(c, gen_down ? K_DOWN_GEN
                          : in == gg::IN_PAIR_ANY ? K_DOWN_ANY
                          : in == gg::IN_PAIR_KEEP ? K_DOWN_KEEP : K_DOWN,
                       gen_down ? 16.0 * nobj + 8.0 * count : 16.0 * count);
        GG_CUDA(gg::launch_downsweep(a, sc.rb[p], in, ntiles, gtiles, c->shape,
                                     c->stream));
    }
    return GRID_OK;
}

bool valid_lambda(float lambda) { return std::isfinite(lambda) && lambda > 0.0f; }

// RunLengthEncode + NonEmptyCells + ExclusiveSum: merge-path splits, then the
// per-block merge of sorted keys against cell ids.
int extract_ranges(grid_ctx *c, const unsigned *keys, int64_t count, int64_t ncells, unsigned *cells)
{
    const unsigned long long nb = gg::extract_blocks((unsigned long long)count, (unsigned long long)ncells);
    GG_TRY(ensure(c, c->splits, (size_t)(nb + 1) * sizeof(unsigned)));
    gg::ExtractArgs xa{};
    xa.keys = keys;
    xa.count = (unsigned long long)count;
    xa.ncells = (unsigned long long)ncells;
    xa.G = cells;
    xa.splits = (unsigned *)c->splits.ptr;
    xa.ctl = c->d_ctl;
    {
        KernelScope ks(c, K_SPLIT, 4.0 * (nb + 1));
        GG_CUDA(gg::launch_extract_split(xa, c->stream));
    }
    KernelScope ks(c, K_EXTRACT, 4.0 * count + 4.0 * (ncells + 1));
    GG_CUDA(gg::launch_extract(xa, c->stream));
    return GRID_OK;
}

// Does a build of `count` pairs over `ncells` cells use the hybrid placement
// (radix passes over the high key bits, then the per-bucket counting sort)?
// A context's local_bits decides (-1: never; -2 or 1..11: always); by
// default (0) it is used at up to LOCAL_PAIRS_PER_CELL pairs per cell: with
// more, the cells' runs are long and ordering them inside a block costs more
// than the radix passes and range extraction it saves (measured on GB300:
// 2.5 pairs per cell gain, 20 lose).
bool use_hybrid(const grid_ctx *c, int64_t count, int64_t ncells)
{
    if (c->local_bits == -1) return false;
    if (c->local_bits != 0) return true;
    return (double)count <= LOCAL_PAIRS_PER_CELL * (double)std::max<int64_t>(ncells, 1);
}

// Local bits L of the hybrid placement for `count` pairs over `ncells` cells
// with key_bits-bit keys: the radix passes sort the bits from L up and one
// block per bucket of 2^L cells sorts the rest.  L_hi is the largest L whose
// mean bucket (count * 2^L / ncells pairs) stays within half of what one
// block places at once; the passes are the fewest that bring the remaining
// bits down to L_hi with digits of at most rbits_max bits; L is then the
// smallest value those passes reach with 8-bit digits (the fastest radix
// kernels, and the smallest buckets, which matters on skewed scenes), but
// not below L_hi - 3 (smaller buckets only add per-block work), or L_hi if
// 8-bit digits cannot reach it.  One bucket of more pairs than a block holds
// would leave a single block with the whole sort: at least one pass then.
// A context's fixed local_bits (1..11) is used as it is.
int choose_local_bits(const grid_ctx *c, int key_bits, int64_t count, int64_t ncells)
{
    if (key_bits <= 0) return 0;
    if (c->local_bits > 0) return std::min(c->local_bits, key_bits);
    const double per_cell = (double)count / (double)std::max<int64_t>(ncells, 1);
    int l_hi = 0;
    while (l_hi < gg::LOCAL_LMAX && per_cell * (double)(2ll << l_hi) <= 0.5 * gg::LOCAL_CAP) ++l_hi;
    l_hi = std::min(l_hi, key_bits);
    int passes = (key_bits - l_hi + c->rbits_max - 1) / c->rbits_max;
    if (passes == 0 && count > gg::LOCAL_CAP) passes = 1;
    const int l8 = std::max(0, key_bits - 8 * passes);
    return l8 <= l_hi ? std::max(l8, l_hi - 3) : l_hi;
}

// RadixSort + RunLengthEncode / NonEmptyCells / ExclusiveSum, hybrid: the
// radix passes order the pairs by the key bits from L up (the first pass
// generating them when gen is set, else reading keys_in / vals_in), then
// one block per bucket of 2^L cells sorts its pairs by cell in shared memory
// and writes the bucket's part of cells (G) and refs.
int sort_place(grid_ctx *c, int key_bits, int64_t ncells, unsigned count, bool gen, const ObjRec *recs,
               int64_t nobj, const unsigned *tile_obj, unsigned res_x, unsigned res_y, const gg::MeshTab &mt,
               const unsigned *keys_in, const unsigned *vals_in, unsigned *refs, unsigned *cells)
{
    const int L = choose_local_bits(c, key_bits, count, ncells);
    const SortCfg sc = sort_cfg(key_bits, c->rbits_max, L, GG_FIRST_EXTRA);
    const unsigned *K = keys_in, *V = vals_in;
    if (sc.passes > 0 || gen) {
        GG_TRY(ensure(c, c->keys_sorted, (size_t)count * sizeof(unsigned)));
        GG_TRY(ensure(c, c->vals_sorted, (size_t)count * sizeof(unsigned)));
        unsigned *k2 = (unsigned *)c->keys_sorted.ptr, *v2 = (unsigned *)c->vals_sorted.ptr;
        if (sc.passes > 0) {
            GG_TRY(sort_pairs(c, sc, count, gen, recs, nobj, tile_obj, res_x, res_y, mt, keys_in, vals_in, k2, v2,
                              GG_FIRST_ANY != 0));
        } else {   // one bucket holds every cell: the object-order pairs are its input
            gg::EmitArgs ea{};
            ea.recs = recs;
            ea.tile_obj = tile_obj;
            ea.mt = mt;
            ea.res_x = res_x;
            ea.res_y = res_y;
            ea.count = count;
            ea.C = k2;
            ea.O = v2;
            KernelScope ks(c, K_EMIT, 16.0 * nobj + 8.0 * count);
            GG_CUDA(gg::launch_emit(ea, c->stream));
        }
        K = k2;
        V = v2;
    }
    gg::LocalArgs la{};
    la.keys = K;
    la.vals = V;
    la.count = count;
    la.ncells = (unsigned long long)ncells;
    la.lbits = L;
    la.nbuckets = (unsigned)(((unsigned long long)ncells - 1ull) >> L) + 1u;
    // groups open at bucket 0, at every bmax-th bucket, where the pair count
    // crosses a multiple of group_pairs, and around each bucket of more than
    // LOCAL_CAP - group_pairs (>= group_pairs) pairs; each holds a bucket
    const unsigned long long bmax = (1ull << gg::LOCAL_LMAX) >> L;
    const unsigned long long per = gg::LOCAL_GROUP_PAIRS;
    la.max_groups = (unsigned)std::min<unsigned long long>(
        la.nbuckets, 2ull + la.nbuckets / bmax + 3ull * ((unsigned long long)count / per + 1ull));
    la.group_pairs = gg::LOCAL_GROUP_PAIRS;
    GG_TRY(ensure(c, c->bstarts, (size_t)(la.nbuckets + 1) * sizeof(unsigned)));
    GG_TRY(ensure(c, c->bgroups, (size_t)la.max_groups * sizeof(unsigned)));
    la.starts = (unsigned *)c->bstarts.ptr;
    la.groups = (unsigned *)c->bgroups.ptr;
    la.refs = refs;
    la.G = cells;
    la.ctl = c->d_ctl;
    GG_CUDA(cudaMemsetAsync(&c->d_ctl->tickets[2], 0, sizeof(unsigned), c->stream));
    {
        KernelScope ks(c, K_BSPLIT, 4.0 * (la.nbuckets + 1));
        GG_CUDA(gg::launch_bucket_split(la, c->stream));
    }
    KernelScope ks(c, K_LOCAL, 12.0 * count + 4.0 * ncells);
    GG_CUDA(gg::launch_local_sort(la, c->stream));
    return GRID_OK;
}

// RadixSort over every key bit, then RunLengthEncode / NonEmptyCells /
// ExclusiveSum by range extraction (the paper's chain): the placement a
// hybrid build falls back to when a group of buckets is too large for one
// block (ERR_LOCAL_FALLBACK).  Same arguments as sort_place.
int place_lsd(grid_ctx *c, int key_bits, int64_t ncells, unsigned count, bool gen, const ObjRec *recs,
              int64_t nobj, const unsigned *tile_obj, unsigned res_x, unsigned res_y, const gg::MeshTab &mt,
              const unsigned *keys_in, const unsigned *vals_in, unsigned *refs, unsigned *cells)
{
    const SortCfg sc = sort_cfg(key_bits, c->rbits_max);
    GG_TRY(ensure(c, c->keys_sorted, (size_t)count * sizeof(unsigned)));
    unsigned *keys = (unsigned *)c->keys_sorted.ptr;
    if (sc.passes > 0) {
        GG_TRY(sort_pairs(c, sc, count, gen, recs, nobj, tile_obj, res_x, res_y, mt, keys_in, vals_in, keys, refs));
    } else if (gen) {
        gg::EmitArgs ea{};
        ea.recs = recs;
        ea.tile_obj = tile_obj;
        ea.mt = mt;
        ea.res_x = res_x;
        ea.res_y = res_y;
        ea.count = count;
        ea.C = keys;
        ea.O = refs;
        KernelScope ks(c, K_EMIT, 16.0 * nobj + 8.0 * count);
        GG_CUDA(gg::launch_emit(ea, c->stream));
    } else {   // one cell: every key is the same
        GG_CUDA(cudaMemcpyAsync(keys, keys_in, (size_t)count * 4, cudaMemcpyDeviceToDevice, c->stream));
        GG_CUDA(cudaMemcpyAsync(refs, vals_in, (size_t)count * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
    return extract_ranges(c, keys, count, ncells, cells);
}

// After a hybrid placement and read_ctl: if a group asked for it, clears the
// request and places the build again with place_lsd.  *redone tells whether
// it did (the caller then reads the control block again).
int fallback_if_asked(grid_ctx *c, bool *redone, int key_bits, int64_t ncells, unsigned count, bool gen,
                      const ObjRec *recs, int64_t nobj, const unsigned *tile_obj, unsigned res_x, unsigned res_y,
                      const gg::MeshTab &mt, const unsigned *keys_in, const unsigned *vals_in, unsigned *refs,
                      unsigned *cells)
{
    *redone = false;
    if (!(c->h_ctl->err & gg::ERR_LOCAL_FALLBACK)) return GRID_OK;
    c->h_ctl->err &= ~gg::ERR_LOCAL_FALLBACK;
    GG_CUDA(cudaMemcpyAsync(&c->d_ctl->err, &c->h_ctl->err, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
    c->fallbacks += 1;
    *redone = true;
    return place_lsd(c, key_bits, ncells, count, gen, recs, nobj, tile_obj, res_x, res_y, mt, keys_in, vals_in,
                     refs, cells);
}

// Output placement for build_core: returns device pointers for cells
// (ncells + 1) and refs (nrefs).
struct OutAlloc {
    virtual int alloc(grid_ctx *c, int64_t ncells1, int64_t nrefs, unsigned **cells, unsigned **refs) = 0;
    // called once the refs are final (their last kernel is enqueued), before
    // the range steps
    virtual int refs_ready(grid_ctx *, const unsigned *, int64_t) { return GRID_OK; }
    virtual ~OutAlloc() = default;
};

// Culling emit over the box placement's NO pairs: the kept pairs, compacted
// in object order, into C / O; *nkept from the device (synchronises).
int cull_pairs(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, const grid_info &I,
               const ObjRec *recs, int64_t n, int64_t NO, unsigned *C, unsigned *O, int64_t *nkept)
{
    *nkept = 0;
    if (NO == 0) return GRID_OK;
    const unsigned ntiles = pair_tiles(NO);
    GG_TRY(ensure(c, c->tile_obj, (size_t)(ntiles + 1) * sizeof(unsigned)));
    {
        KernelScope ks(c, K_TILES, 4.0 * (ntiles + 1));
        GG_CUDA(gg::launch_tile_search(recs, n, gg::PAIR_TILE, ntiles, (unsigned *)c->tile_obj.ptr, c->stream));
    }
    GG_TRY(ensure(c, c->cstatus, (size_t)ntiles * 8));
    GG_CUDA(cudaMemsetAsync(c->cstatus.ptr, 0, (size_t)ntiles * 8, c->stream));
    GG_CUDA(cudaMemsetAsync(&c->d_ctl->tickets[7], 0, sizeof(unsigned), c->stream));
    gg::CullArgs ca{};
    ca.recs = recs;
    ca.tile_obj = (const unsigned *)c->tile_obj.ptr;
    ca.verts = verts;
    ca.nverts = nverts;
    ca.tris = tris;
    for (int a = 0; a < 3; ++a) {
        ca.lo[a] = I.lo[a];
        ca.scale[a] = I.scale[a];
        ca.res_f[a] = (float)I.res[a];
    }
    ca.res_x = (unsigned)I.res[0];
    ca.res_y = (unsigned)I.res[1];
    ca.count = (unsigned)NO;
    ca.C = C;
    ca.O = O;
    ca.status = (unsigned long long *)c->cstatus.ptr;
    ca.ctl = c->d_ctl;
    {
        // reads the records and the triangles' vertices, writes the kept pairs
        // (counted at the box placement's NO: the bytes it may write)
        KernelScope ks(c, K_CULL, 16.0 * n + 48.0 * n + 8.0 * NO);
        GG_CUDA(gg::launch_cull_emit(ca, c->stream));
    }
    GG_TRY(read_ctl(c));
    GG_TRY(ctl_error(c->h_ctl->err));
    *nkept = (int64_t)c->h_ctl->nkept;
    return GRID_OK;
}

// The object-order pairs (C, O) written to device memory by the emit kernel
// (GRID_PAIRS_EMIT) or one thread per object (GRID_PAIRS_PER_OBJECT).
int pairs_in_memory(grid_ctx *c, const ObjRec *recs, int64_t n, const unsigned *tile_obj, const grid_info &I,
                    unsigned count, unsigned *C, unsigned *O)
{
    if (c->pair_gen == GRID_PAIRS_PER_OBJECT) {
        KernelScope ks(c, K_PER_OBJECT, 16.0 * n + 8.0 * count);
        GG_CUDA(gg::launch_make_pairs_per_object(recs, n, (unsigned)I.res[0], (unsigned)I.res[1], count, C, O,
                                                 c->d_ctl, c->stream));
        return GRID_OK;
    }
    gg::EmitArgs ea{};
    ea.recs = recs;
    ea.tile_obj = tile_obj;
    ea.res_x = (unsigned)I.res[0];
    ea.res_y = (unsigned)I.res[1];
    ea.count = count;
    ea.C = C;
    ea.O = O;
    KernelScope ks(c, K_EMIT, 16.0 * n + 8.0 * count);
    GG_CUDA(gg::launch_emit(ea, c->stream));
    return GRID_OK;
}

// BuildParallelGrid (Algorithm 1) on device-resident inputs.
int build_core(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
               float lambda, grid_info *info, OutAlloc &out)
{
    if (n < 0 || nverts < 0 || n > kInt32Max - 1 || !valid_lambda(lambda)) return GRID_EINVAL;
    if (n > 0 && (!verts || !tris)) return GRID_EINVAL;
    grid_info I;
    unsigned *cells = nullptr, *refs = nullptr;
    if (n == 0) {
        const float z[3] = {0.f, 0.f, 0.f};
        GG_TRY(plan(z, z, 0, lambda, &I));
        GG_TRY(out.alloc(c, 2, 0, &cells, &refs));
        GG_CUDA(cudaMemsetAsync(cells, 0, 2 * sizeof(unsigned), c->stream));
        GG_CUDA(cudaStreamSynchronize(c->stream));
        if (info) *info = I;
        return GRID_OK;
    }
    // a0: boxes + bounds, a1 on the device, a2 + a3 with the device's M: one
    // host synchronisation for bounds, M and NO together
    GG_TRY(reset_ctl(c));
    {
        KernelScope ks(c, K_BOUNDS, 48.0 * n);
        GG_CUDA(gg::launch_bounds(verts, nverts, tris, n, c->d_ctl, c->nsm, c->stream));
    }
    {
        KernelScope ks(c, K_PLAN, 0.0);
        GG_CUDA(gg::launch_plan(c->d_ctl, n, lambda, c->stream));
    }
    const int64_t ctiles = (n + gg::COUNT_TILE - 1) / gg::COUNT_TILE;
    GG_TRY(ensure(c, c->recs, (size_t)n * sizeof(ObjRec)));
    GG_TRY(ensure(c, c->k2status, (size_t)ctiles * 8));
    gg::CountArgs ca{};
    ca.verts = verts;
    ca.nverts = nverts;
    ca.tris = tris;
    ca.n = n;
    ca.recs = (ObjRec *)c->recs.ptr;
    ca.status = (unsigned long long *)c->k2status.ptr;
    ca.ctl = c->d_ctl;
    ca.device_plan = true;
    // the pair tiles' first objects come out of the count when the buffer
    // kept from earlier builds holds them
    ca.tile_obj = (unsigned *)c->tile_obj.ptr;
    ca.tile_cap = (unsigned)std::min<size_t>(c->tile_obj.bytes / sizeof(unsigned), 0xFFFFFFFFull);
    auto count_scan = [&]() -> int {
        GG_CUDA(cudaMemsetAsync(c->k2status.ptr, 0, (size_t)ctiles * 8, c->stream));
        KernelScope ks(c, K_COUNT, 64.0 * n);
        GG_CUDA(gg::launch_count_scan(ca, c->stream));
        return GRID_OK;
    };
    GG_TRY(count_scan());
    GG_TRY(read_ctl(c));
    if (c->h_ctl->err & (gg::ERR_BADINDEX | gg::ERR_NONFINITE)) return GRID_EINVAL;
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = bound_lo(c->h_ctl->lo_inv[a]);
        hi[a] = bound_hi(c->h_ctl->hi_ord[a]);
    }
    // a1 on the host, the reference: the device's M must equal it (the two
    // cube roots can differ by a rounding, which moves a resolution only if
    // e * k lies within that of an integer); otherwise CountCells and
    // ExclusiveSum run again with the host's M
    GG_TRY(plan(lo, hi, n, lambda, &I));
    bool same = true;
    for (int a = 0; a < 3; ++a) {
        unsigned sh, sd, lh, ld;
        std::memcpy(&sh, &I.scale[a], 4);
        std::memcpy(&sd, &c->h_ctl->plan_scale[a], 4);
        std::memcpy(&lh, &I.lo[a], 4);
        std::memcpy(&ld, &c->h_ctl->plan_lo[a], 4);
        same = same && I.res[a] == c->h_ctl->plan_res[a] && sh == sd && lh == ld;
    }
    if (!same) {
        c->plan_redos += 1;
        ca.device_plan = false;
        for (int a = 0; a < 3; ++a) {
            ca.lo[a] = I.lo[a];
            ca.scale[a] = I.scale[a];
            ca.res[a] = I.res[a];
        }
        // the first count's tickets, NO and any overflow bit are stale
        GG_CUDA(cudaMemsetAsync(&c->d_ctl->err, 0, sizeof(unsigned), c->stream));
        GG_CUDA(cudaMemsetAsync(&c->d_ctl->tickets[0], 0, sizeof(unsigned), c->stream));
        GG_TRY(count_scan());
        GG_TRY(read_ctl(c));
    }
    GG_TRY(ctl_error(c->h_ctl->err));
    const int64_t NO = (int64_t)c->h_ctl->nrefs;
    if (NO > kInt32Max) return GRID_EOVERFLOW;
    I.nrefs = NO;

    if (c->cull) {
        // the box pairs minus the culled ones, in object order, then the
        // in-memory sort and the range steps over the kept pairs
        GG_TRY(ensure(c, c->pairs_C, (size_t)std::max<int64_t>(NO, 1) * sizeof(unsigned)));
        GG_TRY(ensure(c, c->pairs_O, (size_t)std::max<int64_t>(NO, 1) * sizeof(unsigned)));
        unsigned *C = (unsigned *)c->pairs_C.ptr, *O = (unsigned *)c->pairs_O.ptr;
        int64_t NK = 0;
        GG_TRY(cull_pairs(c, verts, nverts, tris, I, (const ObjRec *)c->recs.ptr, n, NO, C, O, &NK));
        I.nrefs = NK;
        GG_TRY(out.alloc(c, I.ncells + 1, NK, &cells, &refs));
        if (NK > 0 && use_hybrid(c, NK, I.ncells)) {
            GG_TRY(sort_place(c, I.key_bits, I.ncells, (unsigned)NK, false, nullptr, 0, nullptr, 0, 0, gg::MeshTab{},
                              C, O, refs, cells));
            GG_TRY(out.refs_ready(c, refs, NK));
            GG_TRY(read_ctl(c));
            GG_TRY(ctl_error(c->h_ctl->err));
            bool redone = false;
            GG_TRY(fallback_if_asked(c, &redone, I.key_bits, I.ncells, (unsigned)NK, false, nullptr, 0, nullptr, 0, 0,
                                     gg::MeshTab{}, C, O, refs, cells));
            if (redone) {
                GG_TRY(out.refs_ready(c, refs, NK));
                GG_TRY(read_ctl(c));
            }
            GG_TRY(ctl_error(c->h_ctl->err));
            if (info) *info = I;
            return GRID_OK;
        } else if (NK > 0) {
            const unsigned kc = (unsigned)NK;
            const SortCfg sc = sort_cfg(I.key_bits, c->rbits_max);
            const unsigned *keys = C;
            if (sc.passes == 0) {
                GG_CUDA(cudaMemcpyAsync(refs, O, (size_t)kc * 4, cudaMemcpyDeviceToDevice, c->stream));
            } else {
                GG_TRY(ensure(c, c->keys_sorted, (size_t)kc * sizeof(unsigned)));
                GG_TRY(sort_pairs(c, sc, kc, false, nullptr, 0, nullptr, 0, 0, gg::MeshTab{}, C, O,
                                  (unsigned *)c->keys_sorted.ptr, refs));
                keys = (const unsigned *)c->keys_sorted.ptr;
            }
            GG_TRY(out.refs_ready(c, refs, kc));
            GG_TRY(extract_ranges(c, keys, kc, I.ncells, cells));
        } else {
            GG_CUDA(cudaMemsetAsync(cells, 0, (size_t)(I.ncells + 1) * sizeof(unsigned), c->stream));
        }
        GG_TRY(read_ctl(c));
        GG_TRY(ctl_error(c->h_ctl->err));
        if (info) *info = I;
        return GRID_OK;
    }

    GG_TRY(out.alloc(c, I.ncells + 1, NO, &cells, &refs));
    const unsigned count = (unsigned)NO;
    const SortCfg sc = sort_cfg(I.key_bits, c->rbits_max);
    if (count > 0) {
        const unsigned ntiles = pair_tiles(count);
        const bool tiles_done = ca.tile_obj && (size_t)ntiles + 1 <= ca.tile_cap &&
                                !(c->h_ctl->err & gg::ERR_TILE_REDO);
        GG_TRY(ensure(c, c->tile_obj, (size_t)(ntiles + 1) * sizeof(unsigned)));
        const ObjRec *recs = (const ObjRec *)c->recs.ptr;
        unsigned *tile_obj = (unsigned *)c->tile_obj.ptr;
        if (!tiles_done) {
            KernelScope ks(c, K_TILES, 4.0 * (ntiles + 1));
            GG_CUDA(gg::launch_tile_search(recs, n, gg::PAIR_TILE, ntiles, tile_obj, c->stream));
        }
        const bool in_memory = c->pair_gen == GRID_PAIRS_EMIT || c->pair_gen == GRID_PAIRS_PER_OBJECT;
        if (use_hybrid(c, count, I.ncells)) {
            // hybrid: radix passes over the high key bits, then the per-bucket
            // counting sort writes refs and cells
            unsigned *C = nullptr, *O = nullptr;
            if (in_memory) {
                GG_TRY(ensure(c, c->pairs_C, (size_t)count * sizeof(unsigned)));
                GG_TRY(ensure(c, c->pairs_O, (size_t)count * sizeof(unsigned)));
                C = (unsigned *)c->pairs_C.ptr;
                O = (unsigned *)c->pairs_O.ptr;
                GG_TRY(pairs_in_memory(c, recs, n, tile_obj, I, count, C, O));
            }
            const unsigned rx = (unsigned)I.res[0], ry = (unsigned)I.res[1];
            GG_TRY(sort_place(c, I.key_bits, I.ncells, count, !in_memory, recs, n, tile_obj, rx, ry, gg::MeshTab{}, C,
                              O, refs, cells));
            GG_TRY(out.refs_ready(c, refs, count));
            GG_TRY(read_ctl(c));
            GG_TRY(ctl_error(c->h_ctl->err));
            bool redone = false;
            GG_TRY(fallback_if_asked(c, &redone, I.key_bits, I.ncells, count, !in_memory, recs, n, tile_obj, rx, ry,
                                     gg::MeshTab{}, C, O, refs, cells));
            if (redone) {
                GG_TRY(out.refs_ready(c, refs, count));
                GG_TRY(read_ctl(c));
                GG_TRY(ctl_error(c->h_ctl->err));
            }
            if (info) *info = I;
            return GRID_OK;
        }
        GG_TRY(ensure(c, c->keys_sorted, (size_t)count * sizeof(unsigned)));
        unsigned *keys_sorted = (unsigned *)c->keys_sorted.ptr;
        if (sc.passes == 0 || in_memory) {
            // object-order (C, O) in device memory: straight into the outputs
            // when there is nothing to sort, else into scratch for the sort
            unsigned *C = keys_sorted, *O = refs;
            if (sc.passes > 0) {
                GG_TRY(ensure(c, c->pairs_C, (size_t)count * sizeof(unsigned)));
                GG_TRY(ensure(c, c->pairs_O, (size_t)count * sizeof(unsigned)));
                C = (unsigned *)c->pairs_C.ptr;
                O = (unsigned *)c->pairs_O.ptr;
            }
            GG_TRY(pairs_in_memory(c, recs, n, tile_obj, I, count, C, O));
            if (sc.passes > 0)
                GG_TRY(sort_pairs(c, sc, count, false, nullptr, 0, nullptr, 0, 0, gg::MeshTab{}, C, O, keys_sorted,
                                  refs));
        } else {
            GG_TRY(sort_pairs(c, sc, count, true, recs, n, tile_obj, (unsigned)I.res[0], (unsigned)I.res[1],
                              gg::MeshTab{}, nullptr, nullptr, keys_sorted, refs));
        }
        GG_TRY(out.refs_ready(c, refs, count));
        GG_TRY(extract_ranges(c, keys_sorted, count, I.ncells, cells));
    } else {
        GG_CUDA(cudaMemsetAsync(cells, 0, (size_t)(I.ncells + 1) * sizeof(unsigned), c->stream));
    }
    GG_TRY(read_ctl(c));
    GG_TRY(ctl_error(c->h_ctl->err));
    if (info) *info = I;
    return GRID_OK;
}

struct PoolOut : OutAlloc {
    grid_buf *cells_buf, *refs_buf;
    PoolOut(grid_buf *cb, grid_buf *rb) : cells_buf(cb), refs_buf(rb) {}
    int alloc(grid_ctx *c, int64_t ncells1, int64_t nrefs, unsigned **cells, unsigned **refs) override
    {
        void *pc = nullptr, *pr = nullptr;
        GG_TRY(pool_alloc(c, (size_t)ncells1 * 4, &pc));
        int rc = pool_alloc(c, (size_t)nrefs * 4, &pr);
        if (rc != GRID_OK) {
            pool_free(c, pc, (size_t)ncells1 * 4);
            return rc;
        }
        cells_buf->ptr = pc;
        cells_buf->count = ncells1;
        cells_buf->bytes = (size_t)ncells1 * 4;
        refs_buf->ptr = pr;
        refs_buf->count = nrefs;
        refs_buf->bytes = (size_t)nrefs * 4;
        *cells = (unsigned *)pc;
        *refs = (unsigned *)pr;
        return GRID_OK;
    }
};

struct ScratchOut : OutAlloc {
    int64_t ncells1 = 0, nrefs = 0;
    int alloc(grid_ctx *c, int64_t nc1, int64_t nr, unsigned **cells, unsigned **refs) override
    {
        GG_TRY(ensure(c, c->out_cells, (size_t)nc1 * 4));
        GG_TRY(ensure(c, c->out_refs, (size_t)std::max<int64_t>(nr, 1) * 4));
        ncells1 = nc1;
        nrefs = nr;
        *cells = (unsigned *)c->out_cells.ptr;
        *refs = (unsigned *)c->out_refs.ptr;
        return GRID_OK;
    }
};

// Outputs in the context's scratch, bound for host buffers: once the refs
// are final their device-to-host copy starts on the context's copy stream,
// so it overlaps range extraction on the build stream.
struct HostOut : ScratchOut {
    int32_t *h_refs;
    int64_t refs_cap;
    bool copied = false;
    HostOut(int32_t *hr, int64_t cap) : h_refs(hr), refs_cap(cap) {}
    int refs_ready(grid_ctx *c, const unsigned *refs, int64_t count) override
    {
        if (!h_refs || count <= 0 || count > refs_cap) return GRID_OK;   // copied after the build, or ENOSPC
        if (!c->copy_stream) GG_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->copy_ev) GG_CUDA(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming));
        GG_CUDA(cudaEventRecord(c->copy_ev, c->stream));
        GG_CUDA(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0));
        copied = true;   // from here on the caller waits for the copy stream, whatever happens
        GG_CUDA(cudaMemcpyAsync(h_refs, refs, (size_t)count * 4, cudaMemcpyDeviceToHost, c->copy_stream));
        return GRID_OK;
    }
};

}  // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

const char *grid_version(void) { return "gb300-grid 0.1 (sm_103a)"; }

const char *grid_strerror(int code)
{
    switch (code) {
    case GRID_OK: return "ok";
    case GRID_EINVAL: return "invalid argument or input";
    case GRID_ENOMEM: return "out of memory";
    case GRID_EOVERFLOW: return "grid too large: ncells or nrefs above INT32_MAX";
    case GRID_EAGAIN: return "admission refused, retry later";
    case GRID_ETIMEOUT: return "timed out";
    case GRID_ECUDA: return "CUDA runtime error";
    case GRID_ENOSPC: return "host output buffer too small";
    case GRID_ENOTREADY: return "result not ready";
    case GRID_ELIMIT: return "request exceeds the fixed scratch capacity of the allocation-free entry point";
    default: return "unknown error";
    }
}

int grid_ctx_create(int device, const grid_opts *opts, grid_ctx **out)
{
    if (!out) return GRID_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GRID_EINVAL;
    }
    DeviceGuard g(device);
    grid_ctx *c = new (std::nothrow) grid_ctx();
    if (!c) return GRID_ENOMEM;
    c->device = device;
    if (opts) c->opts = *opts;
    if (c->opts.radix_bits >= 8 && c->opts.radix_bits <= 11) c->rbits_max = c->opts.radix_bits;
    if (c->opts.pair_gen < GRID_PAIRS_FUSED || c->opts.pair_gen > GRID_PAIRS_REGEN) {
        delete c;
        return GRID_EINVAL;
    }
    c->pair_gen = c->opts.pair_gen;
    if (c->opts.cull != 0 && c->opts.cull != 1) {
        delete c;
        return GRID_EINVAL;
    }
    c->cull = c->opts.cull == 1;
    if (c->opts.tile_shape != 0 && c->opts.tile_shape != 1) {
        delete c;
        return GRID_EINVAL;
    }
    c->shape = c->opts.tile_shape;
    if (c->opts.local_bits < -2 || c->opts.local_bits > gg::LOCAL_LMAX) {
        delete c;
        return GRID_EINVAL;
    }
    c->local_bits = c->opts.local_bits;
    int rc = GRID_OK;
    do {
        if ((rc = cuda_err(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device)))) break;
        if ((rc = cuda_err(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking)))) break;
        c->stream = c->own;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if ((rc = cuda_err(cudaMemPoolCreate(&c->pool, &props)))) break;
        uint64_t thr = UINT64_MAX;
        if ((rc = cuda_err(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr)))) break;
        const size_t small = sizeof(Ctl) + sizeof(unsigned) * gg::MAX_PASSES * gg::MAX_RADIX;
        void *p = nullptr;
        if ((rc = cuda_err(cudaMalloc(&p, small)))) break;
        if ((rc = cuda_err(cudaMemset(p, 0, small)))) break;
        c->d_ctl = (Ctl *)p;
        c->d_dbase = (unsigned *)((char *)p + sizeof(Ctl));
        if ((rc = cuda_err(cudaMallocHost(&p, sizeof(Ctl))))) break;
        c->h_ctl = (Ctl *)p;
        std::memset(c->h_ctl, 0, sizeof(Ctl));
    } while (0);
    if (rc != GRID_OK) {
        grid_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return GRID_OK;
}

void grid_ctx_destroy(grid_ctx *c)
{
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        Scratch *all[] = {&c->recs, &c->k2status, &c->tile_obj, &c->splits, &c->keys_sorted, &c->keys[0],
                          &c->vals_sorted, &c->bstarts, &c->bgroups,
                          &c->vals[0], &c->intra, &c->gpref, &c->gstatus, &c->in_verts, &c->in_tris,
                          &c->out_cells, &c->out_refs, &c->b_desc, &c->b_base, &c->b_state, &c->b_pairbase,
                          &c->b_cellsoff, &c->b_G, &c->b_seg, &c->pairs_C, &c->pairs_O, &c->cstatus};
        for (Scratch *s : all) release(c, *s);
        if (c->stream) cudaStreamSynchronize(c->stream);
        resolve_timings(c);
        for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
        c->free_events.clear();
        if (c->d_ctl) cudaFree(c->d_ctl);
        if (c->h_ctl) cudaFreeHost(c->h_ctl);
        if (c->h_stage) cudaFreeHost(c->h_stage);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        if (c->own) cudaStreamDestroy(c->own);
        if (c->copy_stream) {
            cudaStreamSynchronize(c->copy_stream);
            cudaStreamDestroy(c->copy_stream);
        }
        if (c->copy_ev) cudaEventDestroy(c->copy_ev);
    }
    delete c;
}

int grid_ctx_get_opts(grid_ctx *c, grid_opts *out)
{
    if (!c || !out) return GRID_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->radix_bits = c->rbits_max;
    out->pair_gen = c->pair_gen;
    out->cull = c->cull ? 1 : 0;
    out->tile_shape = c->shape;
    out->local_bits = c->local_bits;
    return GRID_OK;
}

int grid_ctx_set_opts(grid_ctx *c, const grid_opts *o)
{
    if (!c || !o) return GRID_EINVAL;
    if ((o->radix_bits != 0 && (o->radix_bits < 8 || o->radix_bits > 11)) || o->pair_gen < GRID_PAIRS_FUSED ||
        o->pair_gen > GRID_PAIRS_REGEN || (o->cull != 0 && o->cull != 1) || (o->tile_shape != 0 && o->tile_shape != 1) ||
        o->local_bits < -2 || o->local_bits > gg::LOCAL_LMAX)
        return GRID_EINVAL;
    if (o->radix_bits) c->rbits_max = o->radix_bits;
    c->pair_gen = o->pair_gen;
    c->cull = o->cull == 1;
    c->shape = o->tile_shape;
    c->local_bits = o->local_bits;
    return GRID_OK;
}

int grid_ctx_set_stream(grid_ctx *c, void *stream)
{
    if (!c) return GRID_EINVAL;
    c->stream = stream ? (cudaStream_t)stream : c->own;
    return GRID_OK;
}

int grid_ctx_mem_in_use(grid_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return GRID_EINVAL;
    *bytes = c->in_use.load();
    return GRID_OK;
}

int grid_ctx_sort_plan(grid_ctx *c, int32_t key_bits, int64_t count, int64_t ncells, int32_t *local_bits,
                       int32_t *passes)
{
    if (!c || !local_bits || key_bits < 0 || key_bits > 31 || count < 0 || ncells < 1) return GRID_EINVAL;
    if (!use_hybrid(c, count, ncells)) {
        *local_bits = -1;
        if (passes) *passes = sort_cfg(key_bits, c->rbits_max).passes;
        return GRID_OK;
    }
    const int L = choose_local_bits(c, key_bits, count, ncells);
    *local_bits = L;
    if (passes) *passes = sort_cfg(key_bits, c->rbits_max, L).passes;
    return GRID_OK;
}

int grid_ctx_counters(grid_ctx *c, int64_t *fallbacks, int64_t *plan_redos)
{
    if (!c) return GRID_EINVAL;
    if (fallbacks) *fallbacks = c->fallbacks;
    if (plan_redos) *plan_redos = c->plan_redos;
    return GRID_OK;
}

int grid_ctx_profile(grid_ctx *c, int enable)
{
    if (!c) return GRID_EINVAL;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    resolve_timings(c);
    c->profile = enable != 0;
    for (int k = 0; k < K_NUM; ++k) {
        c->launches[k] = 0;
        c->kernel_ms[k] = 0.0;
        c->kernel_bytes[k] = 0.0;
    }
    return GRID_OK;
}

int grid_ctx_kernel_stats(grid_ctx *c, grid_kernel_stat *out, int max, int *count)
{
    if (!c || !count || (max > 0 && !out)) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_CUDA(cudaStreamSynchronize(c->stream));
    resolve_timings(c);
    int k2 = 0;
    for (int k = 0; k < K_NUM && k2 < max; ++k) {
        if (!c->launches[k]) continue;
        grid_kernel_stat &o = out[k2++];
        std::memset(&o, 0, sizeof(o));
        std::snprintf(o.name, sizeof(o.name), "%s", kKernelNames[k]);
        o.launches = c->launches[k];
        o.total_ms = c->kernel_ms[k];
        o.bytes = c->kernel_bytes[k];
    }
    *count = k2;
    return GRID_OK;
}

int grid_build(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n, float lambda,
               grid_buf *out_cells, grid_buf *out_refs, grid_info *info)
{
    if (!c || !out_cells || !out_refs) return GRID_EINVAL;
    *out_cells = grid_buf{nullptr, 0, 0};
    *out_refs = grid_buf{nullptr, 0, 0};
    DeviceGuard g(c->device);
    PoolOut po(out_cells, out_refs);
    int rc = build_core(c, verts, nverts, tris, n, lambda, info, po);
    if (rc != GRID_OK) {
        grid_buf_free(c, out_cells);
        grid_buf_free(c, out_refs);
    }
    return rc;
}

int grid_ctx_autotune(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                      float lambda, int32_t reps, grid_opts *chosen, double *times)
{
    if (!c) return GRID_EINVAL;
    if (reps <= 0) reps = 3;
    if (reps > 64) return GRID_EINVAL;
    DeviceGuard g(c->device);
    const int saved_rbits = c->rbits_max, saved_pg = c->pair_gen, saved_shape = c->shape, saved_lb = c->local_bits;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return GRID_ECUDA;
    }
    // median ms of `reps` builds with the context's current setting, after
    // one warm-up build
    auto time_setting = [&](double *med) -> int {
        std::vector<float> ms;
        for (int r = 0; r <= reps; ++r) {
            grid_buf cells{}, refs{};
            cudaEventRecord(e0, c->stream);
            PoolOut po(&cells, &refs);
            int rc = build_core(c, verts, nverts, tris, n, lambda, nullptr, po);
            cudaEventRecord(e1, c->stream);
            grid_buf_free(c, &cells);
            grid_buf_free(c, &refs);
            if (rc != GRID_OK) return rc;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                return GRID_ECUDA;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r > 0) ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        *med = ms[ms.size() / 2];
        return GRID_OK;
    };
    const int modes[2] = {GRID_PAIRS_FUSED, GRID_PAIRS_EMIT};
    double best = -1.0;
    int best_rbits = saved_rbits, best_pg = saved_pg, best_shape = saved_shape, k = 0, rc = GRID_OK;
    // digit width x pair generation, with the context's block shape
    for (int rb = 8; rb <= 11 && rc == GRID_OK; ++rb) {
        for (int mi = 0; mi < 2 && rc == GRID_OK; ++mi, ++k) {
            c->rbits_max = rb;
            c->pair_gen = modes[mi];
            double med = 0.0;
            if ((rc = time_setting(&med)) != GRID_OK) break;
            if (times) times[k] = med;
            if (best < 0.0 || med < best) {
                best = med;
                best_rbits = rb;
                best_pg = modes[mi];
            }
        }
    }
    // then the other block shape with the winner
    if (rc == GRID_OK) {
        c->rbits_max = best_rbits;
        c->pair_gen = best_pg;
        c->shape = saved_shape == gg::SHAPE_MAIN ? gg::SHAPE_ALT : gg::SHAPE_MAIN;
        double med = 0.0;
        rc = time_setting(&med);
        if (rc == GRID_OK) {
            if (times) times[8] = med;
            if (med < best) {
                best = med;
                best_shape = c->shape;
            }
        }
    }
    // then the other way to finish the sort and the range steps: radix
    // passes over every key bit and extraction when the context uses the
    // per-bucket counting sort, and the automatic hybrid otherwise
    int best_lb = saved_lb;
    if (rc == GRID_OK) {
        c->shape = best_shape;
        // the context's own choice for this mesh (its pair and cell counts
        // come from one more build), then the other one: radix passes over
        // every key bit if it chose the hybrid, the hybrid if it did not
        grid_info probe{};
        grid_buf cells{}, refs{};
        PoolOut po(&cells, &refs);
        c->local_bits = saved_lb;
        rc = build_core(c, verts, nverts, tris, n, lambda, &probe, po);
        grid_buf_free(c, &cells);
        grid_buf_free(c, &refs);
        c->local_bits = use_hybrid(c, probe.nrefs, probe.ncells) ? -1 : -2;
        double med = 0.0;
        if (rc == GRID_OK) rc = time_setting(&med);
        if (rc == GRID_OK) {
            if (times) times[9] = med;
            if (med < best) {
                best = med;
                best_lb = c->local_bits;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GRID_OK) {
        c->rbits_max = saved_rbits;
        c->pair_gen = saved_pg;
        c->shape = saved_shape;
        c->local_bits = saved_lb;
        return rc;
    }
    c->rbits_max = best_rbits;
    c->pair_gen = best_pg;
    c->shape = best_shape;
    c->local_bits = best_lb;
    if (chosen) {
        std::memset(chosen, 0, sizeof(*chosen));
        chosen->radix_bits = best_rbits;
        chosen->pair_gen = best_pg;
        chosen->cull = c->cull ? 1 : 0;
        chosen->tile_shape = best_shape;
        chosen->local_bits = best_lb;
    }
    return GRID_OK;
}

int grid_ctx_autotune_batched(grid_ctx *c, const grid_mesh *meshes, int32_t nmeshes, int32_t reps,
                              grid_opts *chosen, double *times)
{
    if (!c || !meshes || nmeshes < 1) return GRID_EINVAL;
    if (reps <= 0) reps = 3;
    if (reps > 64) return GRID_EINVAL;
    DeviceGuard g(c->device);
    const int saved_rbits = c->rbits_max, saved_shape = c->shape, saved_lb = c->local_bits;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return GRID_ECUDA;
    }
    std::vector<grid_info> infos((size_t)nmeshes);
    std::vector<int64_t> coff((size_t)nmeshes), roff((size_t)nmeshes);
    // median ms of `reps` batched builds with the context's current setting,
    // after one warm-up build
    auto time_setting = [&](double *med) -> int {
        std::vector<float> ms;
        for (int r = 0; r <= reps; ++r) {
            grid_buf cells{}, refs{};
            cudaEventRecord(e0, c->stream);
            int rc = grid_build_batched(c, meshes, nmeshes, &cells, &refs, infos.data(), coff.data(), roff.data());
            cudaEventRecord(e1, c->stream);
            grid_buf_free(c, &cells);
            grid_buf_free(c, &refs);
            if (rc != GRID_OK) return rc;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                return GRID_ECUDA;
            }
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r > 0) ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        *med = ms[ms.size() / 2];
        return GRID_OK;
    };
    double best = -1.0;
    int best_rbits = saved_rbits, best_shape = saved_shape, best_lb = saved_lb, rc = GRID_OK;
    grid_buf probe_cells{}, probe_refs{};
    for (int rb = 8; rb <= 11 && rc == GRID_OK; ++rb) {
        c->rbits_max = rb;
        double med = 0.0;
        if ((rc = time_setting(&med)) != GRID_OK) break;
        if (times) times[rb - 8] = med;
        if (best < 0.0 || med < best) {
            best = med;
            best_rbits = rb;
        }
    }
    if (rc == GRID_OK) {   // the other block shape with the winning digit width
        c->rbits_max = best_rbits;
        c->shape = saved_shape == gg::SHAPE_MAIN ? gg::SHAPE_ALT : gg::SHAPE_MAIN;
        double med = 0.0;
        if ((rc = time_setting(&med)) == GRID_OK) {
            if (times) times[4] = med;
            if (med < best) {
                best = med;
                best_shape = c->shape;
            }
        }
    }
    if (rc == GRID_OK) {   // the other way to finish the sort and the range steps (as grid_ctx_autotune)
        c->shape = best_shape;
        c->local_bits = saved_lb;
        rc = grid_build_batched(c, meshes, nmeshes, &probe_cells, &probe_refs, infos.data(), coff.data(),
                                roff.data());
        int64_t np = 0, nc = 0;
        for (int m = 0; m < nmeshes; ++m) {
            np += infos[m].nrefs;
            nc += infos[m].ncells;
        }
        grid_buf_free(c, &probe_cells);
        grid_buf_free(c, &probe_refs);
        c->local_bits = use_hybrid(c, np, nc) ? -1 : -2;
        double med = 0.0;
        if (rc == GRID_OK) rc = time_setting(&med);
        if (rc == GRID_OK) {
            if (times) times[5] = med;
            if (med < best) {
                best = med;
                best_lb = c->local_bits;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GRID_OK) {
        c->rbits_max = saved_rbits;
        c->shape = saved_shape;
        c->local_bits = saved_lb;
        return rc;
    }
    c->rbits_max = best_rbits;
    c->shape = best_shape;
    c->local_bits = best_lb;
    if (chosen) {
        std::memset(chosen, 0, sizeof(*chosen));
        chosen->radix_bits = best_rbits;
        chosen->pair_gen = GRID_PAIRS_FUSED;
        chosen->cull = c->cull ? 1 : 0;
        chosen->tile_shape = best_shape;
        chosen->local_bits = best_lb;
    }
    return GRID_OK;
}

int grid_build_host(grid_ctx *c, const float *h_verts, int64_t nverts, const int32_t *h_tris, int64_t n,
                    float lambda, int32_t *h_cells, int64_t cells_cap, int32_t *h_refs, int64_t refs_cap,
                    grid_info *info)
{
    if (!c || n < 0 || nverts < 0) return GRID_EINVAL;
    if (n > 0 && (!h_verts || !h_tris)) return GRID_EINVAL;
    DeviceGuard g(c->device);
    const size_t vb = (size_t)nverts * 3 * sizeof(float), tb = (size_t)n * 3 * sizeof(int32_t);
    GG_TRY(ensure(c, c->in_verts, std::max<size_t>(vb, 16)));
    GG_TRY(ensure(c, c->in_tris, std::max<size_t>(tb, 16)));
    if (!c->copy_stream) GG_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    if (!c->copy_ev) GG_CUDA(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming));
    HostOut so(h_cells ? h_refs : nullptr, refs_cap);
    grid_info I;
    int rc = [&]() -> int {
        // the vertices come in on the copy stream while the triangles come
        // in on the build stream (once the build stream is done with the
        // input scratch); the build waits for both
        GG_CUDA(cudaEventRecord(c->copy_ev, c->stream));
        GG_CUDA(cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0));
        if (vb) GG_CUDA(cudaMemcpyAsync(c->in_verts.ptr, h_verts, vb, cudaMemcpyHostToDevice, c->copy_stream));
        if (tb) GG_CUDA(cudaMemcpyAsync(c->in_tris.ptr, h_tris, tb, cudaMemcpyHostToDevice, c->stream));
        GG_CUDA(cudaEventRecord(c->copy_ev, c->copy_stream));
        GG_CUDA(cudaStreamWaitEvent(c->stream, c->copy_ev, 0));
        GG_TRY(build_core(c, (const float *)c->in_verts.ptr, nverts, (const int32_t *)c->in_tris.ptr, n, lambda,
                          &I, so));
        if (info) *info = I;
        if (!h_cells || !h_refs || cells_cap < so.ncells1 || refs_cap < so.nrefs) return GRID_ENOSPC;
        GG_CUDA(cudaMemcpyAsync(h_cells, c->out_cells.ptr, (size_t)so.ncells1 * 4, cudaMemcpyDeviceToHost,
                                c->stream));
        if (so.nrefs && !so.copied)
            GG_CUDA(cudaMemcpyAsync(h_refs, c->out_refs.ptr, (size_t)so.nrefs * 4, cudaMemcpyDeviceToHost,
                                    c->stream));
        return GRID_OK;
    }();
    // no copy from or into the caller's memory is left in flight on return
    const int rc1 = cuda_err(cudaStreamSynchronize(c->stream));
    const int rc2 = cuda_err(cudaStreamSynchronize(c->copy_stream));
    if (rc == GRID_OK) rc = rc1 != GRID_OK ? rc1 : rc2;
    return rc;
}

// ---- batches sorted in segments ----------------------------------------------
//
// One sort over a whole batch keys its pairs by the batch's global cell id,
// which can need a radix pass more than any of its meshes alone (64 meshes of
// up to 7.7M cells: 27-bit keys, 4 passes of 8-bit digits, against 23 bits
// and 3 passes for the largest mesh). The batch's pairs are generated mesh
// after mesh, so consecutive meshes whose cells together fit the largest
// mesh's pass count can be sorted, extracted and cut into their cells arrays
// as one segment each, with keys counted from the segment's first cell.

int key_bits_of(long long ncells)
{
    int b = 0;
    for (unsigned long long v = ncells > 1 ? (unsigned long long)(ncells - 1) : 0ull; v; v >>= 1) ++b;
    return b;
}

// The first mesh of every segment, then nm; false when one sort over the
// whole batch takes no more radix passes than its largest mesh.
bool sort_segments(const grid_ctx *c, const grid_info *infos, int nm, long long ncells_all, std::vector<int> &segs)
{
    int kmax = 0;
    for (int m = 0; m < nm; ++m) kmax = std::max(kmax, key_bits_of(infos[m].ncells));
    const int pmax = std::max(sort_cfg(kmax, c->rbits_max).passes, 1);
    if (sort_cfg(key_bits_of(ncells_all), c->rbits_max).passes <= pmax) return false;
    const long long cap = 1ll << std::min(pmax * c->rbits_max, 31);   // cells pmax passes sort
    segs.assign(1, 0);
    long long acc = 0;
    for (int m = 0; m < nm; ++m) {
        if (acc > 0 && acc + infos[m].ncells > cap) {
            segs.push_back(m);
            acc = 0;
        }
        acc += infos[m].ncells;
    }
    segs.push_back(nm);
    return segs.size() > 2;
}

// Sort, range extraction and the cells arrays of a batch, segment by segment
// (segs from sort_segments). desc, obj_base, pair_base (nm + 1 entries, the
// last NO) and cells_off describe the whole batch as its count/scan left it;
// recs hold global pair offsets on entry, segment-relative ones on return.
int build_segments(grid_ctx *c, const std::vector<int> &segs, int nm, const gg::MeshDesc *desc,
                   const long long *obj_base, const unsigned *pair_base, const long long *cells_off,
                   const grid_info *infos, long long ntot, unsigned *refs, unsigned *cells)
{
    const int ns = (int)segs.size() - 1;
    // per mesh a descriptor whose cell base counts from its segment's first
    // cell, and its pair base from the segment's first pair; per segment its
    // object bases and output cell offsets from its first mesh (m1 - m0 + 1
    // entries at m0 + s), its first object and first pair
    std::vector<gg::MeshDesc> d2(desc, desc + nm);
    std::vector<long long> ob2(nm + ns), co2(nm + ns), sobj0(ns);
    std::vector<unsigned> pb2(nm), sp0(ns);
    for (int s = 0; s < ns; ++s) {
        const int m0 = segs[s], m1 = segs[s + 1];
        for (int m = m0; m < m1; ++m) {
            d2[m].cell_base = desc[m].cell_base - desc[m0].cell_base;
            pb2[m] = pair_base[m] - pair_base[m0];
        }
        for (int m = m0; m <= m1; ++m) {
            ob2[m + s] = obj_base[m] - obj_base[m0];
            co2[m + s] = cells_off[m] - cells_off[m0];
        }
        sobj0[s] = obj_base[m0];
        sp0[s] = pair_base[m0];
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t o_d = 0, o_ob = o_d + al(sizeof(gg::MeshDesc) * nm), o_co = o_ob + al(8 * (size_t)(nm + ns)),
                 o_so = o_co + al(8 * (size_t)(nm + ns)), o_pb = o_so + al(8 * (size_t)ns),
                 o_sp = o_pb + al(4 * (size_t)nm), total = o_sp + al(4 * (size_t)ns);
    GG_TRY(ensure(c, c->b_seg, total));
    char *base = (char *)c->b_seg.ptr;
    GG_CUDA(cudaMemcpyAsync(base + o_d, d2.data(), sizeof(gg::MeshDesc) * nm, cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(base + o_ob, ob2.data(), 8 * (size_t)(nm + ns), cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(base + o_co, co2.data(), 8 * (size_t)(nm + ns), cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(base + o_so, sobj0.data(), 8 * (size_t)ns, cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(base + o_pb, pb2.data(), 4 * (size_t)nm, cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(base + o_sp, sp0.data(), 4 * (size_t)ns, cudaMemcpyHostToDevice, c->stream));
    const gg::MeshDesc *d_desc = (const gg::MeshDesc *)(base + o_d);
    const long long *d_ob = (const long long *)(base + o_ob), *d_co = (const long long *)(base + o_co);
    const unsigned *d_pb = (const unsigned *)(base + o_pb);
    ObjRec *recs = (ObjRec *)c->recs.ptr;
    {
        KernelScope ks(c, K_REBASE, 8.0 * ntot);
        GG_CUDA(gg::launch_rebase_recs(recs, ntot, (const long long *)(base + o_so), (const unsigned *)(base + o_sp),
                                       ns, c->stream));
    }
    unsigned *G = (unsigned *)c->b_G.ptr;
    for (int s = 0; s < ns; ++s) {
        const int m0 = segs[s], m1 = segs[s + 1];
        const long long obj0 = obj_base[m0], n_s = obj_base[m1] - obj0;
        const unsigned P0 = pair_base[m0], count = pair_base[m1] - P0;
        const long long ncells_s = (long long)desc[m1 - 1].cell_base + infos[m1 - 1].ncells - desc[m0].cell_base;
        unsigned *Gs = G + desc[m0].cell_base;   // the segment's cells, its own pair offsets
        const gg::MeshTab mt{d_desc + m0, d_ob + m0 + s, m1 - m0};
        if (count > 0) {
            const ObjRec *recs_s = recs + obj0;
            const unsigned ntiles = pair_tiles(count);
            GG_TRY(ensure(c, c->tile_obj, (size_t)(ntiles + 1) * sizeof(unsigned)));
            unsigned *tile_obj = (unsigned *)c->tile_obj.ptr;
            {
                KernelScope ks(c, K_TILES, 4.0 * (ntiles + 1));
                GG_CUDA(gg::launch_tile_search(recs_s, n_s, gg::PAIR_TILE, ntiles, tile_obj, c->stream));
            }
            GG_TRY(ensure(c, c->keys_sorted, (size_t)count * sizeof(unsigned)));
            unsigned *keys_sorted = (unsigned *)c->keys_sorted.ptr;
            const SortCfg sc = sort_cfg(key_bits_of(ncells_s), c->rbits_max);
            if (sc.passes == 0) {
                gg::EmitArgs ea{};
                ea.recs = recs_s;
                ea.tile_obj = tile_obj;
                ea.mt = mt;
                ea.count = count;
                ea.C = keys_sorted;
                ea.O = refs + P0;
                KernelScope ks(c, K_EMIT, 16.0 * n_s + 8.0 * count);
                GG_CUDA(gg::launch_emit(ea, c->stream));
            } else {
                GG_TRY(sort_pairs(c, sc, count, true, recs_s, n_s, tile_obj, 0, 0, mt, nullptr, nullptr, keys_sorted,
                                  refs + P0));
            }
            GG_TRY(extract_ranges(c, keys_sorted, count, ncells_s, Gs));
        } else {
            GG_CUDA(cudaMemsetAsync(Gs, 0, (size_t)(ncells_s + 1) * sizeof(unsigned), c->stream));
        }
        // before the next segment's extraction overwrites this one's last entry
        const long long nq = cells_off[m1] - cells_off[m0];
        KernelScope ks(c, K_LOCALIZE, 8.0 * nq);
        GG_CUDA(gg::launch_localize(Gs, d_co + m0 + s, d_pb + m0, m1 - m0, nq, cells + cells_off[m0], c->stream));
    }
    return read_ctl(c);   // the host tables above stay alive until the copies have run
}

int grid_build_batched(grid_ctx *c, const grid_mesh *meshes, int32_t nmeshes, grid_buf *out_cells,
                       grid_buf *out_refs, grid_info *infos, int64_t *cells_offsets, int64_t *refs_offsets)
{
    if (!c || !meshes || nmeshes < 1 || nmeshes > (1 << 20) || !out_cells || !out_refs || !infos ||
        !cells_offsets || !refs_offsets)
        return GRID_EINVAL;
    *out_cells = grid_buf{nullptr, 0, 0};
    *out_refs = grid_buf{nullptr, 0, 0};
    DeviceGuard g(c->device);
    const int nm = nmeshes;
    // the batch's host tables in pinned memory: descriptors, object bases,
    // bounds state, cell offsets, pair bases (64-byte aligned each)
    auto al = [](size_t b) { return (b + 63) & ~size_t(63); };
    const size_t sz_desc = al(sizeof(gg::MeshDesc) * nm), sz_base = al(sizeof(long long) * (nm + 1)),
                 sz_state = al(sizeof(unsigned) * 6 * nm), sz_coff = al(sizeof(long long) * (nm + 1)),
                 sz_pb = al(sizeof(unsigned) * (nm + 1));
    char *stage = nullptr;
    GG_TRY(host_stage(c, sz_desc + sz_base + sz_state + sz_coff + sz_pb, &stage));
    gg::MeshDesc *desc = (gg::MeshDesc *)stage;
    long long *obj_base = (long long *)(stage + sz_desc);
    unsigned *bstate = (unsigned *)(stage + sz_desc + sz_base);
    long long *cells_off = (long long *)(stage + sz_desc + sz_base + sz_state);
    unsigned *pair_base = (unsigned *)(stage + sz_desc + sz_base + sz_state + sz_coff);
    obj_base[0] = 0;
    for (int m = 0; m < nm; ++m) {
        const grid_mesh &mesh = meshes[m];
        if (mesh.n < 0 || mesh.nverts < 0 || !valid_lambda(mesh.lambda)) return GRID_EINVAL;
        if (mesh.n > 0 && (!mesh.verts || !mesh.tris)) return GRID_EINVAL;
        obj_base[m + 1] = obj_base[m] + mesh.n;
        if (obj_base[m + 1] > kInt32Max - 1) return GRID_EOVERFLOW;
    }
    const long long ntot = obj_base[nm];
    for (int m = 0; m < nm; ++m) {
        desc[m] = gg::MeshDesc{};
        desc[m].verts = meshes[m].verts;
        desc[m].tris = meshes[m].tris;
        desc[m].nverts = meshes[m].nverts;
        desc[m].n = meshes[m].n;
    }
    GG_TRY(ensure(c, c->b_desc, sizeof(gg::MeshDesc) * nm));
    GG_TRY(ensure(c, c->b_base, sizeof(long long) * (nm + 1)));
    GG_TRY(ensure(c, c->b_state, sizeof(unsigned) * 6 * nm));
    GG_TRY(ensure(c, c->b_pairbase, sizeof(unsigned) * nm));
    GG_TRY(ensure(c, c->b_cellsoff, sizeof(long long) * (nm + 1)));
    gg::MeshTab mt{(const gg::MeshDesc *)c->b_desc.ptr, (const long long *)c->b_base.ptr, nm};
    GG_TRY(reset_ctl(c));
    GG_CUDA(cudaMemsetAsync(c->b_state.ptr, 0, sizeof(unsigned) * 6 * nm, c->stream));
    c->stage_busy = true;
    GG_CUDA(cudaMemcpyAsync(c->b_desc.ptr, desc, sizeof(gg::MeshDesc) * nm, cudaMemcpyHostToDevice, c->stream));
    GG_CUDA(cudaMemcpyAsync(c->b_base.ptr, obj_base, sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice,
                            c->stream));

    // a0: every mesh's scene bounds in one pass over the flattened triangles
    {
        KernelScope ks(c, K_BOUNDS, 48.0 * ntot);
        GG_CUDA(gg::launch_bounds_batched(mt, ntot, (unsigned *)c->b_state.ptr, c->d_ctl, c->stream));
    }
    GG_CUDA(cudaMemcpyAsync(bstate, c->b_state.ptr, sizeof(unsigned) * 6 * nm, cudaMemcpyDeviceToHost, c->stream));
    GG_TRY(read_ctl(c));
    GG_TRY(ctl_error(c->h_ctl->err));

    // a1: each mesh's metadata; cell ids of mesh m start at cell_base[m]
    cells_off[0] = 0;
    long long cell_base = 0;
    for (int m = 0; m < nm; ++m) {
        float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
        if (meshes[m].n > 0) {
            for (int a = 0; a < 3; ++a) {
                lo[a] = bound_lo(bstate[6 * m + a]);
                hi[a] = bound_hi(bstate[6 * m + 3 + a]);
            }
        }
        GG_TRY(plan(lo, hi, meshes[m].n, meshes[m].lambda, &infos[m]));
        for (int a = 0; a < 3; ++a) {
            desc[m].lo[a] = infos[m].lo[a];
            desc[m].scale[a] = infos[m].scale[a];
            desc[m].res[a] = infos[m].res[a];
        }
        desc[m].cell_base = (unsigned)cell_base;
        cell_base += infos[m].ncells;
        if (cell_base > kInt32Max) return GRID_EOVERFLOW;
        cells_off[m + 1] = cells_off[m] + infos[m].ncells + 1;
    }
    const long long ncells_all = cell_base;
    GG_CUDA(cudaMemcpyAsync(c->b_desc.ptr, desc, sizeof(gg::MeshDesc) * nm, cudaMemcpyHostToDevice, c->stream));

    // a2 + a3 over all objects: one scan, so each mesh's pairs follow the last
    const int64_t ctiles = (ntot + gg::COUNT_TILE - 1) / gg::COUNT_TILE;
    unsigned *pair_base_d = (unsigned *)c->b_pairbase.ptr;
    GG_CUDA(cudaMemsetAsync(pair_base_d, 0, sizeof(unsigned) * nm, c->stream));
    if (ntot > 0) {
        GG_TRY(ensure(c, c->recs, (size_t)ntot * sizeof(ObjRec)));
        GG_TRY(ensure(c, c->k2status, (size_t)ctiles * 8));
        GG_CUDA(cudaMemsetAsync(c->k2status.ptr, 0, (size_t)ctiles * 8, c->stream));
        gg::CountArgs ca{};
        ca.n = ntot;
        ca.recs = (ObjRec *)c->recs.ptr;
        ca.status = (unsigned long long *)c->k2status.ptr;
        ca.ctl = c->d_ctl;
        ca.mt = mt;
        ca.pair_base = pair_base_d;
        KernelScope ks(c, K_COUNT, 64.0 * ntot);
        GG_CUDA(gg::launch_count_scan(ca, c->stream));
    }
    GG_CUDA(cudaMemcpyAsync(pair_base, pair_base_d, sizeof(unsigned) * nm, cudaMemcpyDeviceToHost, c->stream));
    GG_TRY(read_ctl(c));
    GG_TRY(ctl_error(c->h_ctl->err));
    const int64_t NO = ntot > 0 ? (int64_t)c->h_ctl->nrefs : 0;
    if (NO > kInt32Max) return GRID_EOVERFLOW;
    pair_base[nm] = (unsigned)NO;
    for (int m = nm - 1; m >= 0; --m)   // an empty mesh starts where the next one does
        if (meshes[m].n == 0) pair_base[m] = pair_base[m + 1];
    for (int m = 0; m < nm; ++m) {
        infos[m].nrefs = (int64_t)pair_base[m + 1] - pair_base[m];
        cells_offsets[m] = cells_off[m];
        refs_offsets[m] = pair_base[m];
    }

    // outputs: every mesh's cells array back to back, refs back to back
    const long long ncells_out = cells_off[nm];
    void *pc = nullptr, *pr = nullptr;
    GG_TRY(pool_alloc(c, (size_t)ncells_out * 4, &pc));
    int rc = pool_alloc(c, (size_t)NO * 4, &pr);
    if (rc != GRID_OK) {
        pool_free(c, pc, (size_t)ncells_out * 4);
        return rc;
    }
    *out_cells = grid_buf{pc, ncells_out, (size_t)ncells_out * 4};
    *out_refs = grid_buf{pr, NO, (size_t)NO * 4};
    rc = [&]() -> int {
        GG_TRY(ensure(c, c->b_G, (size_t)(ncells_all + 1) * sizeof(unsigned)));
        unsigned *G = (unsigned *)c->b_G.ptr;
        std::vector<int> segs;
        if (NO > 0 && !use_hybrid(c, (unsigned)NO, ncells_all) && sort_segments(c, infos, nm, ncells_all, segs)) {
            GG_TRY(build_segments(c, segs, nm, desc, obj_base, pair_base, cells_off, infos, ntot, (unsigned *)pr,
                                  (unsigned *)pc));
            c->stage_busy = false;
            return ctl_error(c->h_ctl->err);
        }
        if (NO > 0) {
            const unsigned count = (unsigned)NO;
            const unsigned ntiles = pair_tiles(count);
            GG_TRY(ensure(c, c->tile_obj, (size_t)(ntiles + 1) * sizeof(unsigned)));
            const ObjRec *recs = (const ObjRec *)c->recs.ptr;
            unsigned *tile_obj = (unsigned *)c->tile_obj.ptr;
            {
                KernelScope ks(c, K_TILES, 4.0 * (ntiles + 1));
                GG_CUDA(gg::launch_tile_search(recs, ntot, gg::PAIR_TILE, ntiles, tile_obj, c->stream));
            }
            GG_TRY(ensure(c, c->keys_sorted, (size_t)count * sizeof(unsigned)));
            unsigned *keys_sorted = (unsigned *)c->keys_sorted.ptr;
            int key_bits = 0;
            for (unsigned long long v = (unsigned long long)(ncells_all - 1); v; v >>= 1) ++key_bits;
            const SortCfg sc = sort_cfg(key_bits, c->rbits_max);
            if (use_hybrid(c, count, ncells_all)) {
                GG_TRY(sort_place(c, key_bits, ncells_all, count, true, recs, ntot, tile_obj, 0, 0, mt, nullptr, nullptr,
                                  (unsigned *)pr, G));
            } else if (sc.passes == 0) {
                gg::EmitArgs ea{};
                ea.recs = recs;
                ea.tile_obj = tile_obj;
                ea.mt = mt;
                ea.count = count;
                ea.C = keys_sorted;
                ea.O = (unsigned *)pr;
                KernelScope ks(c, K_EMIT, 16.0 * ntot + 8.0 * count);
                GG_CUDA(gg::launch_emit(ea, c->stream));
            } else {
                GG_TRY(sort_pairs(c, sc, count, true, recs, ntot, tile_obj, 0, 0, mt, nullptr, nullptr, keys_sorted,
                                  (unsigned *)pr));
            }
            if (!use_hybrid(c, count, ncells_all)) GG_TRY(extract_ranges(c, keys_sorted, count, ncells_all, G));
        } else {
            GG_CUDA(cudaMemsetAsync(G, 0, (size_t)(ncells_all + 1) * sizeof(unsigned), c->stream));
        }
        GG_CUDA(cudaMemcpyAsync(c->b_cellsoff.ptr, cells_off, sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice,
                                c->stream));
        GG_CUDA(cudaMemcpyAsync(pair_base_d, pair_base, sizeof(unsigned) * nm, cudaMemcpyHostToDevice, c->stream));
        auto localize = [&]() -> int {
            KernelScope ks(c, K_LOCALIZE, 8.0 * ncells_out);
            GG_CUDA(gg::launch_localize(G, (const long long *)c->b_cellsoff.ptr, pair_base_d, nm, ncells_out,
                                        (unsigned *)pc, c->stream));
            return GRID_OK;
        };
        GG_TRY(localize());
        GG_TRY(read_ctl(c));
        c->stage_busy = false;
        GG_TRY(ctl_error(c->h_ctl->err));
        if (NO > 0 && use_hybrid(c, NO, ncells_all)) {
            int key_bits = 0;
            for (unsigned long long v = (unsigned long long)(ncells_all - 1); v; v >>= 1) ++key_bits;
            bool redone = false;
            GG_TRY(fallback_if_asked(c, &redone, key_bits, ncells_all, (unsigned)NO, true, (const ObjRec *)c->recs.ptr,
                                     ntot, (const unsigned *)c->tile_obj.ptr, 0, 0, mt, nullptr, nullptr,
                                     (unsigned *)pr, G));
            if (redone) {
                GG_TRY(localize());
                GG_TRY(read_ctl(c));
                GG_TRY(ctl_error(c->h_ctl->err));
            }
        }
        return GRID_OK;
    }();
    if (rc != GRID_OK) {
        grid_buf_free(c, out_cells);
        grid_buf_free(c, out_refs);
    }
    return rc;
}

void grid_buf_free(grid_ctx *c, grid_buf *b)
{
    if (!c || !b || !b->ptr) return;
    DeviceGuard g(c->device);
    pool_free(c, b->ptr, b->bytes);
    *b = grid_buf{nullptr, 0, 0};
}

int grid_selftest_wait_timeout(grid_ctx *c, double *elapsed_ms)
{
    if (!c) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_TRY(reset_ctl(c));
    GG_TRY(ensure(c, c->splits, 16));   // word 0: the column nothing publishes, word 1: the result
    unsigned *w = (unsigned *)c->splits.ptr;
    GG_CUDA(cudaMemsetAsync(w, 0, 16, c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return GRID_ECUDA;
    }
    cudaEventRecord(e0, c->stream);
    int rc = cuda_err(gg::launch_wait_selftest(w, c->d_ctl, w + 1, c->stream));
    cudaEventRecord(e1, c->stream);
    if (rc == GRID_OK) rc = read_ctl(c);
    if (rc == GRID_OK) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (elapsed_ms) *elapsed_ms = ms;
        rc = ctl_error(c->h_ctl->err);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int grid_jitter(grid_ctx *c, const float *verts, float *out, int64_t nverts, float sigma, uint64_t seed)
{
    if (!c || nverts < 0 || !std::isfinite(sigma) || sigma < 0.0f) return GRID_EINVAL;
    if (nverts > 0 && (!verts || !out)) return GRID_EINVAL;
    if (nverts == 0) return GRID_OK;
    DeviceGuard g(c->device);
    gg::JitterDesc one{};
    one.src = verts;
    one.dst = out;
    one.seed = seed;
    one.s = sigma * 1.7320508075688772f;
    GG_CUDA(gg::launch_jitter(one, nullptr, nullptr, 1, 3 * nverts, c->stream));
    return GRID_OK;
}

// ---- steps ------------------------------------------------------------------

int grid_bounds(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n, float lo[3],
                float hi[3])
{
    if (!c || !lo || !hi || n < 0 || nverts < 0) return GRID_EINVAL;
    if (n > 0 && (!verts || !tris)) return GRID_EINVAL;
    DeviceGuard g(c->device);
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 0.0f;
    if (n == 0) return GRID_OK;
    GG_TRY(reset_ctl(c));
    {
        KernelScope ks(c, K_BOUNDS, 48.0 * n);
        GG_CUDA(gg::launch_bounds(verts, nverts, tris, n, c->d_ctl, c->nsm, c->stream));
    }
    GG_TRY(read_ctl(c));
    GG_TRY(ctl_error(c->h_ctl->err));
    for (int a = 0; a < 3; ++a) {
        lo[a] = bound_lo(c->h_ctl->lo_inv[a]);
        hi[a] = bound_hi(c->h_ctl->hi_ord[a]);
    }
    return GRID_OK;
}

int grid_plan(const float lo[3], const float hi[3], int64_t n, float lambda, grid_info *info)
{
    if (!lo || !hi || !info) return GRID_EINVAL;
    return plan(lo, hi, n, lambda, info);
}

int grid_count_scan(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                    const grid_info *info, grid_objrec *recs, int64_t *nrefs)
{
    if (!c || !info || !nrefs || n < 0 || n > kInt32Max - 1 || nverts < 0) return GRID_EINVAL;
    if (n > 0 && (!verts || !tris || !recs)) return GRID_EINVAL;
    DeviceGuard g(c->device);
    *nrefs = 0;
    if (n == 0) return GRID_OK;
    const int64_t ctiles = (n + gg::COUNT_TILE - 1) / gg::COUNT_TILE;
    GG_TRY(reset_ctl(c));
    GG_TRY(ensure(c, c->k2status, (size_t)ctiles * 8));
    GG_CUDA(cudaMemsetAsync(c->k2status.ptr, 0, (size_t)ctiles * 8, c->stream));
    gg::CountArgs ca{};
    ca.verts = verts;
    ca.nverts = nverts;
    ca.tris = tris;
    ca.n = n;
    for (int a = 0; a < 3; ++a) {
        ca.lo[a] = info->lo[a];
        ca.scale[a] = info->scale[a];
        ca.res[a] = info->res[a];
    }
    ca.recs = (ObjRec *)recs;
    ca.status = (unsigned long long *)c->k2status.ptr;
    ca.ctl = c->d_ctl;
    {
        KernelScope ks(c, K_COUNT, 64.0 * n);
        GG_CUDA(gg::launch_count_scan(ca, c->stream));
    }
    GG_TRY(read_ctl(c));
    *nrefs = (int64_t)c->h_ctl->nrefs;
    GG_TRY(ctl_error(c->h_ctl->err));
    if (*nrefs > kInt32Max) return GRID_EOVERFLOW;
    return GRID_OK;
}

int grid_emit_pairs(grid_ctx *c, const grid_objrec *recs, int64_t n, int64_t nrefs, const grid_info *info,
                    int32_t *C, int32_t *O)
{
    if (!c || !info || n < 0 || nrefs < 0 || nrefs > kInt32Max) return GRID_EINVAL;
    if (nrefs == 0) return GRID_OK;
    if (n == 0 || !recs || !C || !O) return GRID_EINVAL;
    DeviceGuard g(c->device);
    const unsigned ntiles = pair_tiles(nrefs);
    GG_TRY(reset_ctl(c));
    GG_TRY(ensure(c, c->tile_obj, (size_t)(ntiles + 1) * sizeof(unsigned)));
    {
        KernelScope ks(c, K_TILES, 4.0 * (ntiles + 1));
        GG_CUDA(gg::launch_tile_search((const ObjRec *)recs, n, gg::PAIR_TILE, ntiles,
                                       (unsigned *)c->tile_obj.ptr, c->stream));
    }
    gg::EmitArgs ea{};
    ea.recs = (const ObjRec *)recs;
    ea.tile_obj = (const unsigned *)c->tile_obj.ptr;
    ea.res_x = (unsigned)info->res[0];
    ea.res_y = (unsigned)info->res[1];
    ea.count = (unsigned)nrefs;
    ea.C = (unsigned *)C;
    ea.O = (unsigned *)O;
    {
        KernelScope ks(c, K_EMIT, 16.0 * n + 8.0 * nrefs);
        GG_CUDA(gg::launch_emit(ea, c->stream));
    }
    GG_TRY(read_ctl(c));
    return ctl_error(c->h_ctl->err);
}

int grid_emit_pairs_per_object(grid_ctx *c, const grid_objrec *recs, int64_t n, int64_t nrefs,
                               const grid_info *info, int32_t *C, int32_t *O)
{
    if (!c || !info || n < 0 || nrefs < 0 || nrefs > kInt32Max) return GRID_EINVAL;
    if (nrefs == 0) return GRID_OK;
    if (n == 0 || !recs || !C || !O) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_TRY(reset_ctl(c));
    {
        KernelScope ks(c, K_PER_OBJECT, 16.0 * n + 8.0 * nrefs);
        GG_CUDA(gg::launch_make_pairs_per_object((const ObjRec *)recs, n, (unsigned)info->res[0],
                                                 (unsigned)info->res[1], (unsigned)nrefs, (unsigned *)C,
                                                 (unsigned *)O, c->d_ctl, c->stream));
    }
    GG_TRY(read_ctl(c));
    return ctl_error(c->h_ctl->err);
}

int grid_cull_pairs(grid_ctx *c, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                    const grid_info *info, const grid_objrec *recs, int64_t nrefs, int32_t *C, int32_t *O,
                    int64_t *nkept)
{
    if (!c || !info || !nkept || n < 0 || nverts < 0 || nrefs < 0 || nrefs > kInt32Max) return GRID_EINVAL;
    *nkept = 0;
    if (nrefs == 0) return GRID_OK;
    if (n == 0 || !verts || !tris || !recs || !C || !O) return GRID_EINVAL;
    if (info->res[0] < 1 || info->res[1] < 1 || info->res[2] < 1) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_TRY(reset_ctl(c));
    return cull_pairs(c, verts, nverts, tris, *info, (const ObjRec *)recs, n, nrefs, (unsigned *)C,
                      (unsigned *)O, nkept);
}

int grid_sort_pairs(grid_ctx *c, const int32_t *C, const int32_t *O, int64_t count, int32_t key_bits,
                    int32_t *C_out, int32_t *O_out)
{
    if (!c || count < 0 || count > kInt32Max || key_bits < 0 || key_bits > 31) return GRID_EINVAL;
    if (count == 0) return GRID_OK;
    if (!C || !O || !C_out || !O_out || C == C_out || O == O_out) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_TRY(reset_ctl(c));
    const SortCfg sc = sort_cfg(key_bits, c->rbits_max);
    if (sc.passes == 0) {
        GG_CUDA(cudaMemcpyAsync(C_out, C, (size_t)count * 4, cudaMemcpyDeviceToDevice, c->stream));
        GG_CUDA(cudaMemcpyAsync(O_out, O, (size_t)count * 4, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        GG_TRY(sort_pairs(c, sc, (unsigned)count, false, nullptr, 0, nullptr, 0, 0, gg::MeshTab{}, (const unsigned *)C,
                          (const unsigned *)O, (unsigned *)C_out, (unsigned *)O_out));
    }
    GG_TRY(read_ctl(c));
    return ctl_error(c->h_ctl->err);
}

int grid_extract_ranges(grid_ctx *c, const int32_t *C_sorted, int64_t count, int64_t ncells, int32_t *cells)
{
    if (!c || count < 0 || count > kInt32Max || ncells < 1 || ncells > kInt32Max || !cells) return GRID_EINVAL;
    if (count > 0 && !C_sorted) return GRID_EINVAL;
    DeviceGuard g(c->device);
    GG_TRY(reset_ctl(c));
    GG_TRY(extract_ranges(c, (const unsigned *)C_sorted, count, ncells, (unsigned *)cells));
    GG_TRY(read_ctl(c));
    return ctl_error(c->h_ctl->err);
}

}  // extern "C"
