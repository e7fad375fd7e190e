// Rebuild-serving loop: registered meshes stay resident on the device and are
// rebuilt on request, each request with its own vertex jitter (a moving
// scene).  Not a step of the paper's method, which builds one grid per call;
// this is the deployment layer around it.
//
// Design:
//   * one worker thread per stream, each with its own grid_ctx (pool,
//     scratch, control block), so builds on different workers overlap on the
//     GPU, including their host synchronisations (bounds, pair count);
//   * continuous batching: a worker that becomes free takes every queued
//     request (in arrival order, up to max_batch and batch_pairs estimated
//     pairs) and builds them as one flattened problem with
//     grid_build_batched, so many small rebuilds share one launch per step;
//   * jitter on the device (jitter_kernel below, also behind grid_jitter):
//     one launch per batch writes each request's perturbed vertices into the
//     worker's vertex buffer;
//   * admission by device memory: each admitted request reserves an estimate
//     of its bytes until its result is released; submissions beyond the
//     budget are refused (GRID_EAGAIN) rather than queued without bound;
//   * results are views into the batch's output buffers, kept alive by a
//     reference count until every request of the batch is released.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "grid.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Mesh {
    float *verts = nullptr;   // device, server-owned
    int32_t *tris = nullptr;  // device, server-owned
    int64_t nverts = 0, n = 0;
    float lambda = 1.0f;
    int64_t est_pairs = 0;    // with headroom
    int64_t est_bytes = 0;    // admission estimate of one rebuild
    bool tuned = false;       // opts holds the autotuner's setting for rebuilds of this mesh alone
    grid_opts opts{};
};

// Output buffers of one build; freed when the last request viewing them is
// released.
struct BatchOut {
    grid_ctx *ctx = nullptr;
    grid_buf cells{}, refs{};
    ~BatchOut()
    {
        grid_buf_free(ctx, &cells);
        grid_buf_free(ctx, &refs);
    }
};

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE };

struct Request {
    uint64_t ticket = 0;
    int32_t mesh = 0;
    float sigma = 0.0f;
    uint64_t seed = 0;
    float *uverts = nullptr;    // the caller's vertex update (server-owned device copy), or null
    size_t ubytes = 0;
    int64_t est_bytes = 0;
    Clock::time_point t_submit{};
    ReqState state = Q_QUEUED;
    int rc = GRID_OK;
    grid_info info{};
    grid_buf cells{}, refs{};   // views into out
    std::shared_ptr<BatchOut> out;
};

struct Worker {
    grid_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool small_only = false;    // takes only requests that fit a batch, on a high-priority stream
    float *jverts = nullptr;    // jittered vertices of the current batch
    size_t jbytes = 0;
    gg::JitterDesc *h_desc = nullptr, *d_desc = nullptr;   // [max_batch]
    long long *h_ebase = nullptr, *d_ebase = nullptr;      // [max_batch + 1]
    std::thread th;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Latency statistics in bounded memory: counts in geometric buckets of 1%
// width from 1 us up (values below 1 us share bucket 0), plus the exact
// count, sum and maximum.  A percentile is reported as its bucket's upper
// edge, within 1% above the exact nearest-rank value.
struct LatencyHist {
    static constexpr int NB = 2400;          // 1.01^2400 us, about 2.2e10 us: beyond any wait
    std::vector<uint64_t> counts = std::vector<uint64_t>(NB, 0);
    uint64_t n = 0;
    double sum = 0.0, max = 0.0;
    static int bucket(double us)
    {
        if (!(us > 1.0)) return 0;
        const int b = 1 + (int)(std::log(us) / std::log(1.01));
        return b < NB ? b : NB - 1;
    }
    void add(double us)
    {
        counts[bucket(us)] += 1;
        n += 1;
        sum += us;
        max = std::max(max, us);
    }
    double percentile(double q) const
    {
        if (n == 0) return 0.0;
        uint64_t k = (uint64_t)std::ceil(q * (double)n), acc = 0;   // nearest rank
        if (k < 1) k = 1;
        for (int b = 0; b < NB; ++b) {
            acc += counts[b];
            if (acc >= k) return std::min(b == 0 ? 1.0 : std::pow(1.01, (double)b), max);
        }
        return max;
    }
    void clear()
    {
        std::fill(counts.begin(), counts.end(), 0);
        n = 0;
        sum = max = 0.0;
    }
};

}  // namespace

namespace gg {

// ---------------------------------------------------------------------------
// per-request vertex jitter (serving loop)
// ---------------------------------------------------------------------------

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
// round constants 0xD2511F53 / 0xCD9E8D57, the key bumped by the Weyl
// increments 0x9E3779B9 / 0xBB67AE85 after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Unit-variance normal as an Irwin-Hall sum of four 24-bit uniforms, minus
// its mean 2 (variance 4/12, so the caller's factor is sigma * sqrt(3)).
// Every step is one float add in round-to-nearest: the host generator of the
// tests performs the same operations in the same order.
__device__ __forceinline__ float irwin_hall4(uint4 x)
{
    const float q = 5.9604644775390625e-8f;   // 2^-24
    const float u0 = __fmul_rn(__uint2float_rn(x.x >> 8), q);
    const float u1 = __fmul_rn(__uint2float_rn(x.y >> 8), q);
    const float u2 = __fmul_rn(__uint2float_rn(x.z >> 8), q);
    const float u3 = __fmul_rn(__uint2float_rn(x.w >> 8), q);
    return __fsub_rn(__fadd_rn(__fadd_rn(u0, u1), __fadd_rn(u2, u3)), 2.0f);
}

__global__ void __launch_bounds__(256) jitter_kernel(JitterDesc one, const JitterDesc *__restrict__ d,
                                                     const long long *__restrict__ ebase, int nm, long long total)
{
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < total; e += (long long)gridDim.x * 256) {
        JitterDesc jd = one;
        long long local = e;
        if (d) {   // owner: the last mesh whose first element is <= e
            int lo = 0, hi = nm - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ebase[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            jd = d[lo];
            local = e - ebase[lo];
        }
        const unsigned long long i = (unsigned long long)local / 3ull;
        const unsigned a = (unsigned)(local - 3ll * (long long)i);
        const uint4 x = philox4x32_10(make_uint4((unsigned)i, a, 0u, 0u), (unsigned)jd.seed,
                                      (unsigned)(jd.seed >> 32));
        jd.dst[local] = __fadd_rn(jd.src[local], __fmul_rn(irwin_hall4(x), jd.s));
    }
}

cudaError_t launch_jitter(const JitterDesc &one, const JitterDesc *d, const long long *ebase, int nm,
                          long long total, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    const long long want = (total + 255) / 256;
    const unsigned blocks = (unsigned)(want < 4864 ? want : 4864);   // 152 SMs x 32 blocks, grid-stride beyond
    jitter_kernel<<<blocks, 256, 0, s>>>(one, d, ebase, nm, total);
    return cudaGetLastError();
}

}  // namespace gg

struct grid_server {
    int device = 0;
    grid_serve_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Mesh> meshes;    // deque: references stay valid as meshes are added
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int64_t budget = 0, reserved = 0, peak_reserved = 0;
    bool stop = false;
    std::vector<std::unique_ptr<Worker>> workers;
    int busy_large = 0;         // workers running a request above batch_pairs
    int n_small_workers = 0;    // workers reserved for requests that fit a batch
    std::mutex register_mu;
    // vertex updates: copied at submission into blocks of a server-owned
    // pool on a stream of their own, freed once their request is built
    std::mutex upload_mu;
    cudaStream_t upload = nullptr;
    cudaMemPool_t upool = nullptr;

    // statistics since the last reset
    int64_t submitted = 0, completed = 0, failed = 0, refused = 0, batches = 0, batched_requests = 0;
    LatencyHist lat_us, service_us;
    bool have_first = false;
    Clock::time_point t_first{}, t_last{};
};

namespace {

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return GRID_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GRID_ENOMEM : GRID_ECUDA;
}

// Bytes one rebuild may hold: outputs (cells, refs), the build's scratch
// (pair keys and values double-buffered, sorted keys, per-object records,
// per-cell ranges of a batch) and the jittered vertices.
int64_t estimate_bytes(int64_t pairs, int64_t ncells, int64_t n, int64_t nverts)
{
    return 4 * (ncells + 1) + 4 * pairs       // outputs
         + 28 * pairs + 4 * (ncells + 1)      // keys + values x2, sorted keys and values, object-order
                                              // pairs of the unfused modes, batch ranges
         + 16 * n + 12 * nverts + (1 << 20);  // records, jittered vertices, small tables
}

int grow(Worker *w, size_t bytes)
{
    if (w->jbytes >= bytes) return GRID_OK;
    if (w->jverts) cudaFreeAsync(w->jverts, w->stream);
    w->jverts = nullptr;
    w->jbytes = 0;
    const size_t want = align256(bytes + bytes / 4);
    void *p = nullptr;
    if (cudaError_t e = cudaMallocAsync(&p, want, w->stream)) return cuda_rc(e);
    w->jverts = (float *)p;
    w->jbytes = want;
    return GRID_OK;
}

// Builds one batch of requests on worker w.  On return each request holds its
// result or error code.
void run_batch(Worker *w, const std::vector<Request *> &rs, const std::vector<Mesh> &ms)
{
    const int nb = (int)rs.size();
    // jitter: each perturbed request gets its own slice of the vertex buffer
    std::vector<const float *> vsrc(nb);
    size_t need = 0;
    for (int k = 0; k < nb; ++k) {
        // the caller's update if the request carries one, else the
        // registered vertices; jitter (sigma > 0) perturbs that source
        vsrc[k] = rs[k]->uverts ? rs[k]->uverts : ms[k].verts;
        if (rs[k]->sigma > 0.0f && ms[k].nverts > 0) need += align256((size_t)ms[k].nverts * 12);
    }
    int rc = GRID_OK;
    if (need > 0) {
        rc = grow(w, need);
        if (rc == GRID_OK) {
            size_t off = 0;
            int nj = 0;
            long long e = 0;
            for (int k = 0; k < nb; ++k) {
                if (!(rs[k]->sigma > 0.0f && ms[k].nverts > 0)) continue;
                float *dst = (float *)((char *)w->jverts + off);
                off += align256((size_t)ms[k].nverts * 12);
                gg::JitterDesc &d = w->h_desc[nj];
                d = gg::JitterDesc{};
                d.src = vsrc[k];
                d.dst = dst;
                d.seed = rs[k]->seed;
                d.s = rs[k]->sigma * 1.7320508075688772f;
                w->h_ebase[nj] = e;
                e += 3 * ms[k].nverts;
                vsrc[k] = dst;
                ++nj;
            }
            w->h_ebase[nj] = e;
            rc = cuda_rc(cudaMemcpyAsync(w->d_desc, w->h_desc, sizeof(gg::JitterDesc) * nj,
                                         cudaMemcpyHostToDevice, w->stream));
            if (rc == GRID_OK)
                rc = cuda_rc(cudaMemcpyAsync(w->d_ebase, w->h_ebase, sizeof(long long) * (nj + 1),
                                             cudaMemcpyHostToDevice, w->stream));
            if (rc == GRID_OK)
                rc = cuda_rc(gg::launch_jitter(w->h_desc[0], w->d_desc, w->d_ebase, nj, e, w->stream));
        }
    }
    if (rc != GRID_OK) {
        for (Request *r : rs) r->rc = rc;
        return;
    }
    if (nb == 1) {
        auto out = std::make_shared<BatchOut>();
        out->ctx = w->ctx;
        Request *r = rs[0];
        grid_opts keep{};
        const bool tuned = ms[0].tuned && grid_ctx_get_opts(w->ctx, &keep) == GRID_OK &&
                           grid_ctx_set_opts(w->ctx, &ms[0].opts) == GRID_OK;   // the mesh's own setting
        r->rc = grid_build(w->ctx, vsrc[0], ms[0].nverts, ms[0].tris, ms[0].n, ms[0].lambda, &out->cells,
                           &out->refs, &r->info);
        if (tuned) grid_ctx_set_opts(w->ctx, &keep);
        if (r->rc == GRID_OK) {
            r->cells = out->cells;
            r->refs = out->refs;
            r->out = std::move(out);
        }
        return;
    }
    std::vector<grid_mesh> meshes(nb);
    for (int k = 0; k < nb; ++k) {
        meshes[k] = grid_mesh{};
        meshes[k].verts = vsrc[k];
        meshes[k].nverts = ms[k].nverts;
        meshes[k].tris = ms[k].tris;
        meshes[k].n = ms[k].n;
        meshes[k].lambda = ms[k].lambda;
    }
    std::vector<grid_info> infos(nb);
    std::vector<int64_t> coff(nb), roff(nb);
    auto out = std::make_shared<BatchOut>();
    out->ctx = w->ctx;
    rc = grid_build_batched(w->ctx, meshes.data(), nb, &out->cells, &out->refs, infos.data(), coff.data(),
                            roff.data());
    if (rc == GRID_OK) {
        for (int k = 0; k < nb; ++k) {
            Request *r = rs[k];
            r->rc = GRID_OK;
            r->info = infos[k];
            const int64_t nc1 = infos[k].ncells + 1, nr = infos[k].nrefs;
            r->cells = grid_buf{(char *)out->cells.ptr + 4 * coff[k], nc1, (size_t)nc1 * 4};
            r->refs = grid_buf{nr ? (void *)((char *)out->refs.ptr + 4 * roff[k]) : nullptr, nr, (size_t)nr * 4};
            r->out = out;
        }
        return;
    }
    // A batch fails as a whole (one bad mesh, or too large together): build
    // each request alone so the others still get their results.
    out.reset();
    for (int k = 0; k < nb; ++k) {
        auto one = std::make_shared<BatchOut>();
        one->ctx = w->ctx;
        Request *r = rs[k];
        r->rc = grid_build(w->ctx, vsrc[k], ms[k].nverts, ms[k].tris, ms[k].n, ms[k].lambda, &one->cells,
                           &one->refs, &r->info);
        if (r->rc == GRID_OK) {
            r->cells = one->cells;
            r->refs = one->refs;
            r->out = std::move(one);
        }
    }
}

void worker_main(grid_server *S, Worker *w)
{
    cudaSetDevice(S->device);
    std::vector<Request *> rs;
    std::vector<Mesh> ms;
    for (;;) {
        rs.clear();
        ms.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto is_large = [&](uint64_t t) {
                auto it = S->reqs.find(t);
                return it != S->reqs.end() && S->meshes[it->second->mesh].est_pairs > S->opts.batch_pairs;
            };
            auto has_work = [&] {
                if (!w->small_only) return !S->queue.empty();
                for (uint64_t t : S->queue)
                    if (!is_large(t)) return true;
                return false;
            };
            S->cv_work.wait(lk, [&] { return S->stop || has_work(); });
            if (S->stop) return;
            // a reserved worker passes over large requests; without reserved
            // workers, unless strict arrival order is asked for, the last
            // worker not busy with a large request passes over large ones
            // while a smaller one waits
            bool skip_large = w->small_only;
            if (!skip_large && S->n_small_workers == 0 && !S->opts.arrival_order &&
                S->busy_large >= (int)S->workers.size() - 1 && S->workers.size() > 1) {
                for (uint64_t t : S->queue)
                    if (!is_large(t)) {
                        skip_large = true;
                        break;
                    }
            }
            int64_t pairs = 0;
            for (auto qi = S->queue.begin(); qi != S->queue.end() && (int)rs.size() < S->opts.max_batch;) {
                auto it = S->reqs.find(*qi);
                if (it == S->reqs.end()) {   // cannot happen: queued requests are never released
                    qi = S->queue.erase(qi);
                    continue;
                }
                Request *r = it->second.get();
                const Mesh &m = S->meshes[r->mesh];
                if (skip_large && m.est_pairs > S->opts.batch_pairs) {
                    ++qi;
                    continue;
                }
                if (!rs.empty() && pairs + m.est_pairs > S->opts.batch_pairs) break;
                qi = S->queue.erase(qi);
                r->state = Q_RUNNING;
                rs.push_back(r);
                ms.push_back(m);
                pairs += m.est_pairs;
            }
            if (pairs > S->opts.batch_pairs) S->busy_large += 1;   // a single large request
        }
        if (rs.empty()) continue;
        int64_t batch_est = 0;
        for (const Mesh &m : ms) batch_est += m.est_pairs;
        const Clock::time_point t0 = Clock::now();
        run_batch(w, rs, ms);
        // a build that failed before its first synchronisation may leave the
        // jitter table copies in flight: drain the stream before the pinned
        // tables are reused
        if (cudaStreamSynchronize(w->stream) != cudaSuccess) {
            cudaGetLastError();
            for (Request *r : rs)
                if (r->rc == GRID_OK) r->rc = GRID_ECUDA;
        }
        // the builds that read the vertex updates have finished
        for (Request *r : rs) {
            if (r->uverts) cudaFreeAsync(r->uverts, w->stream);
            r->uverts = nullptr;
        }
        const Clock::time_point t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double service = std::chrono::duration<double, std::micro>(t1 - t0).count();
            for (Request *r : rs) {
                r->state = Q_DONE;
                S->completed += 1;
                if (r->rc != GRID_OK) S->failed += 1;
                S->lat_us.add(std::chrono::duration<double, std::micro>(t1 - r->t_submit).count());
                S->service_us.add(service);
            }
            S->batches += 1;
            if (rs.size() > 1) S->batched_requests += (int64_t)rs.size();
            if (batch_est > S->opts.batch_pairs) S->busy_large -= 1;
            S->t_last = t1;
        }
        S->cv_done.notify_all();
    }
}

void fill_result(const Request &r, grid_buf *cells, grid_buf *refs, grid_info *info)
{
    if (cells) *cells = r.cells;
    if (refs) *refs = r.refs;
    if (info) *info = r.info;
}

void destroy_worker(Worker *w)
{
    if (w->stream) cudaStreamSynchronize(w->stream);
    if (w->jverts) cudaFreeAsync(w->jverts, w->stream);
    if (w->stream) cudaStreamSynchronize(w->stream);
    if (w->ctx) grid_ctx_destroy(w->ctx);
    if (w->d_desc) cudaFree(w->d_desc);
    if (w->d_ebase) cudaFree(w->d_ebase);
    if (w->h_desc) cudaFreeHost(w->h_desc);
    if (w->h_ebase) cudaFreeHost(w->h_ebase);
    if (w->stream) cudaStreamDestroy(w->stream);
}

}  // namespace

extern "C" {

int grid_serve_create(int device, const grid_serve_opts *opts, grid_server **out)
{
    if (!out) return GRID_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GRID_EINVAL;
    }
    grid_serve_opts o{};
    if (opts) o = *opts;
    if (o.nworkers < 0 || o.nworkers > 64 || o.max_batch < 0 || o.max_batch > 4096 || o.batch_pairs < 0 ||
        o.hbm_budget < 0 || (o.arrival_order != 0 && o.arrival_order != 1) || o.small_workers < -1 ||
        o.small_workers > 8 || (o.tune_meshes != 0 && o.tune_meshes != -1))
        return GRID_EINVAL;
    if (o.nworkers == 0) o.nworkers = 2;
    if (o.small_workers == 0) o.small_workers = 1;
    if (o.max_batch == 0) o.max_batch = 32;
    if (o.batch_pairs == 0) o.batch_pairs = 1ll << 24;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    grid_server *S = new (std::nothrow) grid_server();
    if (!S) return GRID_ENOMEM;
    S->device = device;
    S->opts = o;
    int rc = GRID_OK;
    if (o.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        rc = cuda_rc(cudaMemGetInfo(&fr, &tot));
        S->budget = (int64_t)(fr / 4 * 3);
    } else {
        S->budget = o.hbm_budget;
    }
    if (rc == GRID_OK) rc = cuda_rc(cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking));
    if (rc == GRID_OK) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        rc = cuda_rc(cudaMemPoolCreate(&S->upool, &props));
        uint64_t thr = UINT64_MAX;   // keep freed blocks for the next updates
        if (rc == GRID_OK) rc = cuda_rc(cudaMemPoolSetAttribute(S->upool, cudaMemPoolAttrReleaseThreshold, &thr));
    }
    const int nsmall = o.small_workers > 0 ? o.small_workers : 0;
    S->n_small_workers = nsmall;
    int prio_least = 0, prio_greatest = 0;
    if (rc == GRID_OK) rc = cuda_rc(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    for (int i = 0; rc == GRID_OK && i < o.nworkers + nsmall; ++i) {
        auto w = std::make_unique<Worker>();
        w->small_only = i >= o.nworkers;
        grid_opts go{};
        go.radix_bits = o.radix_bits;
        void *p = nullptr;
        if ((rc = grid_ctx_create(device, &go, &w->ctx)) != GRID_OK) break;
        // a reserved worker's kernels go ahead of the large rebuilds' when SMs free up
        if ((rc = cuda_rc(cudaStreamCreateWithPriority(&w->stream, cudaStreamNonBlocking,
                                                       w->small_only ? prio_greatest : prio_least))) != GRID_OK)
            break;
        if ((rc = grid_ctx_set_stream(w->ctx, w->stream)) != GRID_OK) break;
        if ((rc = cuda_rc(cudaMallocHost(&p, sizeof(gg::JitterDesc) * o.max_batch))) != GRID_OK) break;
        w->h_desc = (gg::JitterDesc *)p;
        if ((rc = cuda_rc(cudaMallocHost(&p, sizeof(long long) * (o.max_batch + 1)))) != GRID_OK) break;
        w->h_ebase = (long long *)p;
        if ((rc = cuda_rc(cudaMalloc(&p, sizeof(gg::JitterDesc) * o.max_batch))) != GRID_OK) break;
        w->d_desc = (gg::JitterDesc *)p;
        if ((rc = cuda_rc(cudaMalloc(&p, sizeof(long long) * (o.max_batch + 1)))) != GRID_OK) break;
        w->d_ebase = (long long *)p;
        S->workers.push_back(std::move(w));
    }
    if (rc == GRID_OK) {
        for (auto &w : S->workers) w->th = std::thread(worker_main, S, w.get());
        *out = S;
    } else {
        grid_serve_destroy(S);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

void grid_serve_destroy(grid_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &w : S->workers)
        if (w->th.joinable()) w->th.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto &kv : S->reqs)   // updates of requests that never ran
        if (kv.second->uverts) cudaFreeAsync(kv.second->uverts, S->upload);
    S->reqs.clear();   // results free their buffers through the workers' contexts
    for (auto &w : S->workers) destroy_worker(w.get());
    S->workers.clear();
    if (S->upload) {
        cudaStreamSynchronize(S->upload);
        cudaStreamDestroy(S->upload);
    }
    if (S->upool) cudaMemPoolDestroy(S->upool);
    for (Mesh &m : S->meshes) {
        if (m.verts) cudaFree(m.verts);
        if (m.tris) cudaFree(m.tris);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

int grid_serve_register(grid_server *S, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                        float lambda, int32_t *mesh_id)
{
    if (!S || !mesh_id || n < 0 || nverts < 0 || !std::isfinite(lambda) || lambda <= 0.0f) return GRID_EINVAL;
    if ((n > 0 && !tris) || (nverts > 0 && !verts)) return GRID_EINVAL;
    std::lock_guard<std::mutex> reg(S->register_mu);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    Mesh m;
    m.nverts = nverts;
    m.n = n;
    m.lambda = lambda;
    int rc = GRID_OK;
    grid_ctx *probe = nullptr;
    do {
        void *p = nullptr;
        if (nverts > 0) {
            if ((rc = cuda_rc(cudaMalloc(&p, (size_t)nverts * 12))) != GRID_OK) break;
            m.verts = (float *)p;
            if ((rc = cuda_rc(cudaMemcpy(m.verts, verts, (size_t)nverts * 12, cudaMemcpyDefault))) != GRID_OK) break;
        }
        if (n > 0) {
            if ((rc = cuda_rc(cudaMalloc(&p, (size_t)n * 12))) != GRID_OK) break;
            m.tris = (int32_t *)p;
            if ((rc = cuda_rc(cudaMemcpy(m.tris, tris, (size_t)n * 12, cudaMemcpyDefault))) != GRID_OK) break;
        }
        // one build validates the mesh and measures it; its context (and
        // scratch) goes away with it
        grid_opts go{};
        go.radix_bits = S->opts.radix_bits;
        if ((rc = grid_ctx_create(S->device, &go, &probe)) != GRID_OK) break;
        grid_buf cells{}, refs{};
        grid_info info{};
        rc = grid_build(probe, m.verts, nverts, m.tris, n, lambda, &cells, &refs, &info);
        grid_buf_free(probe, &cells);
        grid_buf_free(probe, &refs);
        if (rc != GRID_OK) break;
        const int64_t pairs = info.nrefs + info.nrefs / 10 + 1024;
        const int64_t ncells = info.ncells + info.ncells / 10 + 64;
        m.est_pairs = pairs;
        m.est_bytes = estimate_bytes(pairs, ncells, n, nverts);
        // the fastest setting for rebuilds of this mesh alone (every setting
        // gives the same grid)
        if (S->opts.tune_meshes == 0 && n > 0) {
            grid_opts chosen{};
            if ((rc = grid_ctx_autotune(probe, m.verts, nverts, m.tris, n, lambda, 2, &chosen, nullptr)) != GRID_OK)
                break;
            chosen.cull = 0;
            m.opts = chosen;
            m.tuned = true;
        }
    } while (0);
    if (probe) grid_ctx_destroy(probe);
    if (rc == GRID_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->meshes.size() >= (size_t)0x7FFFFFFF) {
            rc = GRID_ELIMIT;
        } else {
            *mesh_id = (int32_t)S->meshes.size();
            S->meshes.push_back(m);
        }
    }
    if (rc != GRID_OK) {
        if (m.verts) cudaFree(m.verts);
        if (m.tris) cudaFree(m.tris);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

int grid_serve_submit(grid_server *S, int32_t mesh_id, const float *new_verts, float sigma, uint64_t seed,
                      uint64_t *ticket)
{
    if (!S || !ticket || !std::isfinite(sigma) || sigma < 0.0f) return GRID_EINVAL;
    const Clock::time_point t_submit = Clock::now();   // the update's copy counts in the latency
    int64_t est = 0, nverts = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (mesh_id < 0 || (size_t)mesh_id >= S->meshes.size()) return GRID_EINVAL;
        nverts = S->meshes[mesh_id].nverts;
        est = S->meshes[mesh_id].est_bytes + (new_verts && nverts > 0 ? (int64_t)align256((size_t)nverts * 12) : 0);
        if (est > S->budget) return GRID_ELIMIT;   // would not fit even with nothing else admitted
        if (S->reserved + est > S->budget) {
            S->refused += 1;
            return GRID_EAGAIN;
        }
        S->reserved += est;   // held from here, so concurrent submissions see it
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
    }
    auto r = std::make_unique<Request>();
    if (new_verts && nverts > 0) {
        // copy the update now: the caller may reuse its buffer once this returns
        r->ubytes = (size_t)nverts * 12;
        int rc = GRID_OK;
        {
            std::lock_guard<std::mutex> up(S->upload_mu);
            int prev = -1;
            cudaGetDevice(&prev);
            cudaSetDevice(S->device);
            void *p = nullptr;
            rc = cuda_rc(cudaMallocFromPoolAsync(&p, r->ubytes, S->upool, S->upload));
            if (rc == GRID_OK) {
                r->uverts = (float *)p;
                rc = cuda_rc(cudaMemcpyAsync(r->uverts, new_verts, r->ubytes, cudaMemcpyDefault, S->upload));
                const int rc2 = cuda_rc(cudaStreamSynchronize(S->upload));
                if (rc == GRID_OK) rc = rc2;
                if (rc != GRID_OK) {
                    cudaFreeAsync(r->uverts, S->upload);
                    cudaStreamSynchronize(S->upload);
                    r->uverts = nullptr;
                }
            }
            if (prev >= 0) cudaSetDevice(prev);
        }
        if (rc != GRID_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->reserved -= est;
            return rc;
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        r->mesh = mesh_id;
        r->sigma = sigma;
        r->seed = seed;
        r->est_bytes = est;
        r->t_submit = t_submit;
        if (!S->have_first) {
            S->have_first = true;
            S->t_first = r->t_submit;
        }
        S->submitted += 1;
        *ticket = r->ticket;
        S->queue.push_back(r->ticket);
        S->reqs.emplace(r->ticket, std::move(r));
    }
    S->cv_work.notify_all();   // a reserved worker may not take it: let every idle worker look
    return GRID_OK;
}

int grid_serve_poll(grid_server *S, uint64_t ticket, grid_buf *cells, grid_buf *refs, grid_info *info)
{
    if (!S) return GRID_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return GRID_EINVAL;
    const Request &r = *it->second;
    if (r.state != Q_DONE) return GRID_ENOTREADY;
    if (r.rc != GRID_OK) return r.rc;
    fill_result(r, cells, refs, info);
    return GRID_OK;
}

int grid_serve_wait(grid_server *S, uint64_t ticket, int64_t timeout_us, grid_buf *cells, grid_buf *refs,
                    grid_info *info)
{
    if (!S) return GRID_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->reqs.find(ticket) == S->reqs.end()) return GRID_EINVAL;
    // The request is looked up again on every wake-up, never held across the
    // wait: another thread may release the ticket between the request
    // finishing and this thread taking the lock back.
    auto done = [&] {
        auto it = S->reqs.find(ticket);
        return it == S->reqs.end() || it->second->state == Q_DONE;
    };
    if (timeout_us < 0) {
        S->cv_done.wait(lk, done);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
        return GRID_ETIMEOUT;
    }
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return GRID_EINVAL;   // released by another thread meanwhile
    const Request &r = *it->second;
    if (r.rc != GRID_OK) return r.rc;
    fill_result(r, cells, refs, info);
    return GRID_OK;
}

int grid_serve_release(grid_server *S, uint64_t ticket)
{
    if (!S) return GRID_EINVAL;
    std::shared_ptr<BatchOut> out;   // dropped after the lock: may free device memory
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return GRID_EINVAL;
        Request &r = *it->second;
        if (r.state != Q_DONE) return GRID_ENOTREADY;
        S->reserved -= r.est_bytes;
        out = std::move(r.out);
        S->reqs.erase(it);
    }
    if (out) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(S->device);
        out.reset();
        if (prev >= 0) cudaSetDevice(prev);
    }
    return GRID_OK;
}

int grid_serve_get_stats(grid_server *S, grid_serve_stats *o, int reset)
{
    if (!S || !o) return GRID_EINVAL;
    std::memset(o, 0, sizeof(*o));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        o->submitted = S->submitted;
        o->completed = S->completed;
        o->failed = S->failed;
        o->refused = S->refused;
        o->batches = S->batches;
        o->batched_requests = S->batched_requests;
        o->queued = (int64_t)S->queue.size();
        o->reserved_bytes = S->reserved;
        o->peak_reserved_bytes = S->peak_reserved;
        o->budget_bytes = S->budget;
        if (S->have_first && S->completed > 0 && S->t_last > S->t_first) {
            o->elapsed_s = std::chrono::duration<double>(S->t_last - S->t_first).count();
            o->builds_per_s = (double)S->completed / o->elapsed_s;
        }
        if (S->lat_us.n) {
            o->mean_us = S->lat_us.sum / (double)S->lat_us.n;
            o->max_us = S->lat_us.max;
            o->p50_us = S->lat_us.percentile(0.50);
            o->p99_us = S->lat_us.percentile(0.99);
            o->p50_service_us = S->service_us.percentile(0.50);
        }
        if (reset) {
            S->submitted = S->completed = S->failed = S->refused = S->batches = S->batched_requests = 0;
            S->lat_us.clear();
            S->service_us.clear();
            S->have_first = false;
            S->peak_reserved = S->reserved;
        }
    }
    return GRID_OK;
}

}  // extern "C"
