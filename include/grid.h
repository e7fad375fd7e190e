/*
 * grid.h - C ABI of the GB300 (sm_103a) parallel uniform-grid builder.
 *
 * The library builds the compact uniform grid (G, O) of a triangle mesh with
 * the parallel construction of Costa, Pereira and Jorge, "Building An
 * Efficient Grid On GPU" (Algorithm 1, Sec. 3):
 *
 *   boxes -> CountCells -> ExclusiveSum -> MakeObjectIds -> InclusiveSum ->
 *   SegmentedExclusiveSum -> MakeCellIds (GlobalCoords) -> RadixSort(C, O) ->
 *   RunLengthEncode / NonEmptyCells / ExclusiveSum -> (G, O)
 *
 * Every step runs in the library's own CUDA kernels.  Signatures use plain
 * pointers and sizes only.  Unless stated otherwise pointers are DEVICE
 * pointers on the context's device, read or written in stream order on the
 * context's current stream (grid_ctx_set_stream); the call returns after the
 * work is enqueued, except where a host value must be produced (documented
 * per call), in which case it synchronises that stream.
 *
 * Output format (Sec. 3, Fig. 4d, "compact format"):
 *   cells  int32 [ncells + 1]: cell c's object ids are refs[cells[c] ..
 *          cells[c + 1]); cells[ncells] == nrefs.  Cell id of grid coordinate
 *          (x, y, z) is x + res_x * (y + res_y * z).
 *   refs   int32 [nrefs]: object (triangle) ids in cell order, ascending
 *          inside each cell.
 *
 * World-to-grid mapping (the paper gives the data flow, not the arithmetic;
 * this is the library's fixed reading):
 *   res_a   = clamp(ceil(e_a * k), 1, GRID_RES_MAX) with e_a = hi_a - lo_a
 *             (FP32), k = (lambda * n / prod_nonzero e)^(1/d) in FP64 over the
 *             d axes of non-zero extent; a zero-extent axis gets res 1.
 *   scale_a = (float)res_a / e_a (FP32, round to nearest), 0 on a flat axis.
 *   cell_a(p) = clamp(floor((p - lo_a) * scale_a), 0, res_a - 1) with the
 *             subtraction and the product each rounded to FP32 (no FMA);
 *             NaN maps to 0.
 *   An object's box in grid coordinates is [cell(min vertex), cell(max
 *   vertex)] per axis, inclusive (GlobalCoords, Sec. 3).
 *
 * Error codes: every int-returning call returns GRID_OK (0) or a negative
 * code below; no call aborts the process.
 */
#ifndef GB300_GRID_H
#define GB300_GRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRID_OK 0
#define GRID_EINVAL (-1)     /* bad argument, vertex index out of range, non-finite coordinate */
#define GRID_ENOMEM (-2)     /* device or host allocation failed */
#define GRID_EOVERFLOW (-3)  /* ncells or nrefs above INT32_MAX */
#define GRID_EAGAIN (-4)     /* serving: admission refused, retry later */
#define GRID_ETIMEOUT (-5)   /* a bounded device wait or a host wait ran out */
#define GRID_ECUDA (-6)      /* a CUDA runtime call failed */
#define GRID_ENOSPC (-7)     /* caller's host buffer too small; info holds the sizes */
#define GRID_ENOTREADY (-8)  /* serving: result not finished yet */
#define GRID_ELIMIT (-9)     /* request larger than a fixed-size scratch buffer allows */

#define GRID_RES_MAX 65535

typedef struct grid_ctx grid_ctx;

/* Grid metadata M plus the build's sizes. */
typedef struct {
    float lo[3];          /* scene bounds: union of the triangle boxes */
    float hi[3];
    float scale[3];       /* res / extent per axis (0 on a flat axis) */
    int32_t res[3];       /* cells per axis */
    int32_t key_bits;     /* bits of the largest cell id: ceil(log2(ncells)) */
    int64_t ncells;       /* res_x * res_y * res_z */
    int64_t nrefs;        /* NO: number of <object, cell> pairs */
    int64_t n;            /* number of objects (triangles) */
} grid_info;

/* Library-allocated device memory.  Release with grid_buf_free. */
typedef struct {
    void *ptr;            /* device pointer, 256-byte aligned; NULL when count == 0 */
    int64_t count;        /* elements (int32) */
    size_t bytes;
} grid_buf;

/* One object's box in grid coordinates plus its pair offset: the per-object
 * record CountCells + ExclusiveSum produce (16 bytes, 16-byte aligned). */
typedef struct {
    uint16_t lo[3];       /* first covered cell per axis */
    uint16_t hi[3];       /* last covered cell per axis (inclusive) */
    uint32_t start;       /* exclusive prefix sum of the cell counts V */
} grid_objrec;

/* How grid_build produces the object-order pairs (C, O) of MakeObjectIds ..
 * MakeCellIds.  The pairs, and so the grid, are the same in every mode. */
#define GRID_PAIRS_FUSED 0       /* one thread per pair, generated by the first radix-sort pass's
                                    counting kernel, which stores them once for the pass's scatter
                                    to read (default) */
#define GRID_PAIRS_EMIT 1        /* one thread per pair, written to device memory by a kernel of its
                                    own, then sorted (the paper's chain of separate steps) */
#define GRID_PAIRS_PER_OBJECT 2  /* ablation: one thread per object writes all its pairs (the
                                    sorted grid's MakePairs, Sec. 2), then sorted */
#define GRID_PAIRS_REGEN 3       /* one thread per pair, generated again by each kernel of the first
                                    radix-sort pass, so (C, O) never reach device memory */

/* Tuning knobs; zero means "library default / autotuned". */
typedef struct {
    int32_t radix_bits;   /* widest digit of the LSD radix sort: 8..11 (default 9) */
    int32_t pair_gen;     /* GRID_PAIRS_*; single-mesh builds only (batched builds always fuse) */
    int32_t cull;         /* 1: drop the pairs whose cell the triangle does not touch before the
                             sort (grid_cull_pairs' test); single-mesh builds only.  The grid is
                             then the culled grid: nrefs counts the kept pairs.  0: box placement
                             (Algorithm 1 as published, the default) */
    int32_t tile_shape;   /* block shape of the radix-sort kernels; both sort 3,072-pair tiles and
                             give the same grid.  0: 256 threads x 12 pairs (the default; fastest
                             on large, dense scenes), 1: 384 threads x 8 pairs (more warps per tile;
                             faster on sparse and small scenes).  grid_ctx_autotune picks one */
    int32_t local_bits;   /* how builds finish RadixSort and the range steps.  The hybrid: radix
                             passes over the high key bits only, then one counting sort per bucket
                             of 2^L consecutive cells in shared memory, which also writes the
                             bucket's cell ranges.  The chain: radix passes over every key bit,
                             then range extraction (the paper's).  0 (default): the hybrid at up to
                             6 pairs per cell, with L chosen per build from the key width and the
                             pairs per cell, the chain otherwise.  -2: the hybrid always, L chosen
                             per build.  1..11: the hybrid always with that L (fewer radix passes,
                             larger buckets).  -1: the chain always.  Every setting gives the same
                             grid */
    int32_t reserved[3];
} grid_opts;

/* ---- context -------------------------------------------------------------- */

/* Creates a context on CUDA device `device`: a stream-ordered memory pool,
 * a control block and the kernels' scratch.  opts may be NULL. */
int grid_ctx_create(int device, const grid_opts *opts, grid_ctx **out);
void grid_ctx_destroy(grid_ctx *ctx);
/* The context's current settings (as grid_opts; radix_bits is the digit
 * width in use), and a change of them for its later builds (radix_bits 0
 * keeps the current width; values checked as grid_ctx_create does,
 * GRID_EINVAL otherwise).  Not to be called while another thread builds
 * with the context. */
int grid_ctx_get_opts(grid_ctx *ctx, grid_opts *out);
int grid_ctx_set_opts(grid_ctx *ctx, const grid_opts *opts);
/* Binds a cudaStream_t (passed as void*).  NULL selects the context's own
 * stream, a non-blocking stream: work on it is not ordered with the legacy
 * default stream.  To run in order with work on the legacy default stream
 * (stream handle 0 in most frameworks), pass cudaStreamLegacy, (void *)1. */
int grid_ctx_set_stream(grid_ctx *ctx, void *stream);
/* Device bytes currently held by the context's pool for outputs + scratch. */
int grid_ctx_mem_in_use(grid_ctx *ctx, int64_t *bytes);
const char *grid_strerror(int code);
/* Library version string. */
const char *grid_version(void);

/* Per-kernel accounting.  With profiling on, the library brackets each of its
 * kernel launches with a pair of CUDA events on the launching stream and
 * records the kernel's algorithmic bytes (the bytes the step must move:
 * inputs read once, outputs written once).  Launches are counted always. */
typedef struct {
    char name[32];        /* kernel family: bounds, count_scan, tile_search, emit, upsweep_gen,
                             downsweep_gen, upsweep, downsweep, downsweep_first, extract_split,
                             extract, bucket_split, local_sort, localize, make_pairs_per_object,
                             cull_emit */
    int64_t launches;
    double total_ms;      /* sum of event-timed durations (0 when profiling is off) */
    double bytes;         /* sum of algorithmic bytes */
} grid_kernel_stat;

/* Autotuner: builds the given mesh (device pointers, as grid_build) with
 * every candidate configuration and keeps the fastest for the context's
 * later builds.  First every radix digit width (8, 9, 10, 11 bits) x pair
 * generation (GRID_PAIRS_FUSED, GRID_PAIRS_EMIT) with the context's block
 * shape, then the other block shape (grid_opts.tile_shape) with the best of
 * those, then the other end of the sort (grid_opts.local_bits: radix passes
 * over every key bit and range extraction if the context's setting picks
 * the hybrid for this mesh, the hybrid otherwise: local_bits -1 or -2).  Each
 * candidate is timed with CUDA events on the context's stream: the median of
 * `reps` builds after one warm-up (reps <= 0 means 3).  Every candidate gives
 * the same grid, so tuning changes speed only.  *chosen (may be NULL) gets
 * the kept radix_bits, pair_gen, tile_shape and local_bits; times (may be
 * NULL, 10 entries) the median ms of each candidate: radix 8..11 x (FUSED,
 * EMIT), then the other shape, then the other sort end.  The culling setting
 * is left as it is.  Errors as grid_build; on error the context keeps its
 * previous setting. */
int grid_ctx_autotune(grid_ctx *ctx, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                      float lambda, int32_t reps, grid_opts *chosen, double *times);

/* How the context's builds would finish RadixSort for `count` pairs over
 * `ncells` cells with key_bits-bit keys (grid_opts.local_bits): *local_bits
 * gets L (the cell bits each per-bucket counting sort covers; -1 when every
 * key bit goes through radix passes, the paper's chain with range
 * extraction) and *passes the number of radix passes over the key bits
 * above L (may be NULL).  Host only. */
int grid_ctx_sort_plan(grid_ctx *ctx, int32_t key_bits, int64_t count, int64_t ncells, int32_t *local_bits,
                       int32_t *passes);

/* How often the context's builds took a slower way to the same grid since it
 * was created (either pointer may be NULL): *fallbacks, hybrid placements
 * redone by radix passes over every key bit (a cell beyond what a block
 * sorts); *plan_redos, builds whose grid metadata computed on the device
 * (to spare a host round trip between the bounds and CountCells) differed
 * from the host's, so CountCells and ExclusiveSum ran again with the host's.
 * Host only. */
int grid_ctx_counters(grid_ctx *ctx, int64_t *fallbacks, int64_t *plan_redos);

/* Turns event timing on (1) or off (0) and clears the statistics. */
int grid_ctx_profile(grid_ctx *ctx, int enable);
/* Synchronises the stream, resolves pending events and copies up to max
 * entries (one per kernel family that launched) into out; *count gets the
 * number written. */
int grid_ctx_kernel_stats(grid_ctx *ctx, grid_kernel_stat *out, int max, int *count);

/* ---- whole build (Algorithm 1) ------------------------------------------- */

/* BuildParallelGrid (Algorithm 1, Sec. 3) of the triangles tris[n][3]
 * (int32 vertex indices into verts[nverts][3], float32 xyz) at density
 * lambda (> 0, finite).  Outputs are allocated from the context's pool:
 * out_cells (int32 [ncells + 1]) and out_refs (int32 [nrefs]); info may be
 * NULL.  Synchronises the stream once to size the outputs (the scene bounds,
 * the grid metadata, computed on the device and checked against the host's
 * from the same bounds, and NO come back together) and once at the end; the
 * rest stays on the device.  n == 0 gives res (1,1,1),
 * cells = [0, 0], refs empty.  Errors: GRID_EINVAL (bad index, non-finite
 * coordinate, bad lambda, NULL pointer), GRID_EOVERFLOW, GRID_ENOMEM,
 * GRID_ETIMEOUT, GRID_ECUDA; outputs are left empty on error. */
int grid_build(grid_ctx *ctx, const float *verts, int64_t nverts, const int32_t *tris,
               int64_t n, float lambda, grid_buf *out_cells, grid_buf *out_refs,
               grid_info *info);

/* The same build (Algorithm 1, Sec. 3) from and to HOST memory: copies the
 * inputs to the device, builds, copies cells (int32 [ncells + 1]) and refs
 * (int32 [nrefs]) back into caller buffers of cells_cap / refs_cap
 * elements.  If either is too small the call returns GRID_ENOSPC with info
 * holding the needed sizes.
 * Pinned host memory gives asynchronous copies; pageable memory works too.
 * Returns after the results are in host memory. */
int grid_build_host(grid_ctx *ctx, const float *h_verts, int64_t nverts, const int32_t *h_tris,
                    int64_t n, float lambda, int32_t *h_cells, int64_t cells_cap,
                    int32_t *h_refs, int64_t refs_cap, grid_info *info);

void grid_buf_free(grid_ctx *ctx, grid_buf *buf);

/* ---- many meshes in one build ---------------------------------------------- */

/* One mesh of a batch: device pointers as in grid_build, its own lambda. */
typedef struct {
    const float *verts;   /* [nverts][3] */
    int64_t nverts;
    const int32_t *tris;  /* [n][3] */
    int64_t n;
    float lambda;
    int32_t reserved;
} grid_mesh;

/* BuildParallelGrid (Algorithm 1) of every mesh of a batch at once: the
 * meshes' triangles and pairs form one flattened problem (one launch per step
 * for the whole batch), keyed by (mesh, cell) so one stable sort orders every
 * mesh's pairs.  The result per mesh is bit-identical to grid_build of that
 * mesh alone.  out_cells holds every mesh's cells array back to back (mesh
 * m's int32 [ncells_m + 1] at cells_offsets[m], values local to the mesh);
 * out_refs every mesh's refs (int32 [nrefs_m] at refs_offsets[m], object ids
 * local to the mesh).  infos[m] gets mesh m's metadata and sizes.  The sum of
 * the meshes' cells and the sum of their pairs must each fit int32
 * (GRID_EOVERFLOW); errors as grid_build.  Synchronises the stream twice
 * (bounds, pair count) and at the end. */
int grid_build_batched(grid_ctx *ctx, const grid_mesh *meshes, int32_t nmeshes, grid_buf *out_cells,
                       grid_buf *out_refs, grid_info *infos, int64_t *cells_offsets, int64_t *refs_offsets);

/* The autotuner for batches (the many-mesh builds of grid_build_batched):
 * times the batch `meshes` built as one with every radix digit width (8..11
 * bits), then the other block shape with the best width, then the other end
 * of the sort (as grid_ctx_autotune), and keeps the fastest for the
 * context's later builds.  Timing, reps, chosen and errors as
 * grid_ctx_autotune (pair_gen is reported as GRID_PAIRS_FUSED: batched
 * builds always generate the pairs in the first radix pass); times (may be
 * NULL, 6 entries): radix 8..11, the other shape, the other sort end. */
int grid_ctx_autotune_batched(grid_ctx *ctx, const grid_mesh *meshes, int32_t nmeshes, int32_t reps,
                              grid_opts *chosen, double *times);

/* ---- the steps one by one (device pointers, caller-allocated outputs) ----- */

/* a0, "boxes" of Algorithm 1: union of the per-triangle boxes, written to host
 * lo[3], hi[3].  Checks every index and coordinate (GRID_EINVAL).
 * Synchronises the stream. */
int grid_bounds(grid_ctx *ctx, const float *verts, int64_t nverts, const int32_t *tris,
                int64_t n, float lo[3], float hi[3]);

/* a1, grid metadata M (host only), the grid description that Algorithm 1
 * (Sec. 3) takes as given: resolution, scale and ncells from the bounds and
 * the density rule above (the paper leaves the cell-size rule open, Sec. 6);
 * fills info (nrefs = 0, n set).
 * GRID_EINVAL for lambda <= 0 or non-finite, GRID_EOVERFLOW if
 * ncells > INT32_MAX. */
int grid_plan(const float lo[3], const float hi[3], int64_t n, float lambda, grid_info *info);

/* a2 + a3, CountCells and ExclusiveSum (Algorithm 1, Sec. 3): recs[n] gets
 * each triangle's box in grid coordinates and the exclusive prefix sum of
 * the cell counts V; *nrefs = NO = sum of V (host value; synchronises).
 * info must come from grid_plan for the same triangles.  GRID_EINVAL if a
 * vertex index is outside [0, nverts) (no vertex is read out of range),
 * GRID_EOVERFLOW if NO > INT32_MAX. */
int grid_count_scan(grid_ctx *ctx, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                    const grid_info *info, grid_objrec *recs, int64_t *nrefs);

/* a4 - a7, MakeObjectIds + InclusiveSum + SegmentedExclusiveSum + MakeCellIds
 * (Algorithm 1, GlobalCoords, Fig. 4a/4b): one thread per pair writes the
 * object-order lists C (cell id) and O (object id), int32 [nrefs] each. */
int grid_emit_pairs(grid_ctx *ctx, const grid_objrec *recs, int64_t n, int64_t nrefs,
                    const grid_info *info, int32_t *C, int32_t *O);

/* The same object-order lists as grid_emit_pairs, written by one thread per
 * object (the sorted grid's MakePairs, Sec. 2): an ablation of the pair
 * generation, not a step of Algorithm 1.  Same arguments and result. */
int grid_emit_pairs_per_object(grid_ctx *ctx, const grid_objrec *recs, int64_t n, int64_t nrefs,
                               const grid_info *info, int32_t *C, int32_t *O);

/* False-intersection culling (the overlap test ahead of the sort that Sec. 6
 * names as future work; not a step of Algorithm 1): from the records of
 * grid_count_scan, writes the object-order pairs of the box placement that a
 * triangle/cell test keeps, compacted in the same order, into C and O (int32,
 * capacity nrefs = the box placement's NO); *nkept gets their number
 * (synchronises).  The test, in grid coordinates q = min((v - lo) * scale,
 * res) (the cell mapping's two FP32 operations and its clamp to the far face):
 * cell (x, y, z) is the closed unit cube
 * centred at c = (x, y, z) + 1/2; with w_k = q_k - c, edges e_0 = q_1 - q_0,
 * e_1 = q_2 - q_1, e_2 = q_0 - q_2, axes n = e_0 x e_1 and (0, -e_z, e_y),
 * (e_z, 0, -e_x), (-e_y, e_x, 0) for each edge, projections
 * p_k = (a_x w_kx + a_y w_ky) + a_z w_kz, S = (|a_x| + |a_y|) + |a_z| and
 * slack t = max|w| * 2^-16 + 2^-10, a cell is dropped iff for some axis
 * min p > S/2 + S t or max p < -(S/2 + S t), each operation one FP32
 * round-to-nearest step in that order.  The slack exceeds the rounding error,
 * so a triangle touching the cell always keeps it.  A triangle whose box has at
 * most two cells keeps them without a test (each holds a vertex), so its
 * vertices are not read.  GRID_EINVAL if a tested triangle has a vertex index
 * outside [0, nverts); no vertex is read out of range. */
int grid_cull_pairs(grid_ctx *ctx, const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
                    const grid_info *info, const grid_objrec *recs, int64_t nrefs, int32_t *C, int32_t *O,
                    int64_t *nkept);

/* a8, RadixSort(C, O) (Algorithm 1, Fig. 4c): stable LSD sort of the pairs by
 * the low key_bits bits of C (0..31; keys must be < 2^key_bits).  Writes
 * C_out, O_out (int32 [count]); the inputs are not modified.  The outputs
 * must not alias the inputs. */
int grid_sort_pairs(grid_ctx *ctx, const int32_t *C, const int32_t *O, int64_t count,
                    int32_t key_bits, int32_t *C_out, int32_t *O_out);

/* a9, RunLengthEncode + NonEmptyCells + ExclusiveSum (Algorithm 1, Fig. 4d):
 * from the cell-sorted C (int32 [count], values in [0, ncells)) writes
 * cells (int32 [ncells + 1]), cells[c] = number of entries < c.  A key
 * >= ncells gives GRID_EINVAL; so does a key found out of order (unsorted
 * input is caught where a block of keys leaves its expected cell range,
 * not always: the contents of cells are then unspecified). */
int grid_extract_ranges(grid_ctx *ctx, const int32_t *C_sorted, int64_t count, int64_t ncells,
                        int32_t *cells);

/* ---- failure detection ------------------------------------------------------ */

/* Self-test of the kernels' bounded waits (not a step of the method).  Every
 * decoupled look-back (pair count scan, radix-sort passes, culling
 * compaction) polls a predecessor's status word at most 2^20 times with a
 * back-off. If the word never arrives, the kernel records a timeout, stops
 * waiting and finishes, and the call returns GRID_ETIMEOUT with the context
 * still usable.  This runs the sort passes' look-back against a
 * predecessor that never publishes, on the context's stream, and returns
 * what a build would: GRID_ETIMEOUT (the expected answer), or GRID_OK /
 * GRID_ECUDA if the wait did not behave.  *elapsed_ms (may be NULL) gets the
 * wait's device time (about a second or less).  Synchronises. */
int grid_selftest_wait_timeout(grid_ctx *ctx, double *elapsed_ms);

/* ---- per-request vertex jitter ------------------------------------------- */

/* Not a step of the method: the perturbation the serving loop applies to a
 * registered mesh before each rebuild (a moving scene).  out[e] = verts[e] +
 * d(e) for the 3 * nverts floats e, where d(e) = n(e) * (sigma * sqrt(3))
 * with the factor rounded to float once and n(e) = ((u0 + u1) + (u2 + u3)) -
 * 2, u_k = (x_k >> 8) * 2^-24 and (x_0..x_3) = Philox4x32-10 (Salmon et al.,
 * SC'11) of counter (e / 3, e % 3, 0, 0) under key (seed & 0xffffffff,
 * seed >> 32).  Every operation is one float32 add or multiply rounded to
 * nearest, so a host implementation of the same definition gives the same
 * bits.  n has mean 0, variance 1/3 * 3 = 1, and |n| <= 2.  verts and out
 * (float32 [nverts][3]) are device pointers; out may equal verts.
 * GRID_EINVAL for negative nverts, NULL pointers with nverts > 0, or sigma
 * negative or non-finite.  Enqueued on the context's stream; does not
 * synchronise. */
int grid_jitter(grid_ctx *ctx, const float *verts, float *out, int64_t nverts, float sigma, uint64_t seed);

/* ---- rebuild-serving loop --------------------------------------------------- */

/* A server keeps registered meshes resident on one GPU and rebuilds them on
 * request: each request names a mesh and may carry the mesh's new vertex
 * positions, a jitter sigma and a seed; the server takes the new vertices
 * (or the registered ones), jitters them on the device if sigma > 0
 * (grid_jitter's definition) and builds their grid with Algorithm 1.
 * Worker threads, each with its own stream and context, take queued requests
 * in arrival order (reserved workers, grid_serve_opts.small_workers, only
 * those that fit a batch); a free worker takes every queued request up to
 * max_batch (and up to batch_pairs estimated pairs) and builds them as one
 * batch (grid_build_batched; grid_build for a batch of one).  A request's result is bit-identical whichever batch,
 * worker or stream builds it.
 *
 * Admission: every admitted request reserves an estimate of the device bytes
 * its rebuild needs (outputs plus scratch, from the mesh's pair and cell
 * counts measured at registration, with 10% headroom) until it is released;
 * grid_serve_submit refuses with GRID_EAGAIN when the reservations would pass
 * hbm_budget. */
typedef struct grid_server grid_server;

typedef struct {
    int32_t nworkers;     /* worker threads / streams; 0 -> 2 */
    int32_t max_batch;    /* requests per batched build; 0 -> 32 */
    int64_t batch_pairs;  /* cap on a batch's estimated pairs (a larger single request runs alone);
                             0 -> 2^24: batching pays for small meshes (fewer launches and
                             synchronisations), while a batch of large ones sorts wider keys */
    int64_t hbm_budget;   /* bytes that admitted requests may reserve; 0 -> 3/4 of the device's free
                             memory when the server is created */
    int32_t radix_bits;   /* as grid_opts.radix_bits; 0 -> default */
    int32_t arrival_order; /* without reserved workers (small_workers -1): 0 (default): while every
                             other worker runs a request too large to batch (estimated pairs above
                             batch_pairs), a free worker takes the oldest requests that fit a batch
                             first, so they do not queue behind the large ones; large requests keep
                             their order among themselves and run as soon as no smaller one waits.
                             1: strict arrival order */
    int32_t small_workers; /* workers besides nworkers reserved for requests that fit a batch, each
                             on a stream of the highest priority, so small rebuilds neither queue
                             behind large ones nor wait for their kernels' SMs: 0 -> 1, -1 -> none,
                             1..8 */
    int32_t tune_meshes;  /* 0 (default): grid_serve_register runs grid_ctx_autotune on the mesh
                             and every rebuild of it alone (a batch of one) uses the kept
                             setting; -1: the workers' default setting for every build */
    int32_t reserved[2];
} grid_serve_opts;

typedef struct {
    int64_t submitted;    /* admitted requests */
    int64_t completed;    /* finished (successfully or not) */
    int64_t failed;       /* finished with an error */
    int64_t refused;      /* GRID_EAGAIN answers */
    int64_t batches;      /* builds run (a batch of one counts) */
    int64_t batched_requests;  /* requests built in batches of two or more */
    int64_t queued;       /* waiting for a worker now */
    int64_t reserved_bytes;     /* admission reservations now */
    int64_t peak_reserved_bytes;
    int64_t budget_bytes;
    double p50_us, p99_us, mean_us, max_us;   /* latency, submit -> result ready; the
                                                 percentiles to 1% (log-bucketed counts) */
    double p50_service_us;      /* build time of a request's batch, median */
    double builds_per_s;        /* completed / (last completion - first submission) */
    double elapsed_s;           /* that interval */
} grid_serve_stats;

/* Starts a server on CUDA device `device`; opts may be NULL. */
int grid_serve_create(int device, const grid_serve_opts *opts, grid_server **out);
/* Stops the workers after their current batch, drops queued requests and
 * frees every result and registered mesh. */
void grid_serve_destroy(grid_server *srv);
/* Copies a mesh (verts float32 [nverts][3], tris int32 [n][3]; host or device
 * pointers) into server-owned device memory, validates it with one build at
 * `lambda` and measures its pair and cell counts for admission; unless
 * tune_meshes is -1, also times the autotuner's candidates on it (a few
 * dozen builds).  Errors as grid_build.  Synchronous; safe to call while
 * requests run. */
int grid_serve_register(grid_server *srv, const float *verts, int64_t nverts, const int32_t *tris,
                        int64_t n, float lambda, int32_t *mesh_id);
/* Queues a rebuild of mesh_id; *ticket identifies it.  The paper's case for
 * the parallel construction is rebuilding a deforming scene's grid at
 * interactive rates (Abstract; Sec. 6): new_verts carries the mesh's new
 * vertex positions as they arrive, float32 [nverts][3] with the registered
 * mesh's nverts and triangle indices, in host memory (pageable or pinned) or
 * device memory of the server's device; NULL rebuilds the registered
 * vertices.  The update is copied into server-owned device memory before the
 * call returns (the caller may reuse or free its buffer at once; a device
 * buffer must already hold its values, as the copy does not wait on the
 * caller's streams), and the request's latency includes that copy.  It
 * applies to this request only; the registered vertices stay as they are.
 * sigma (>= 0) and seed add grid_jitter's perturbation on top of the
 * request's vertices (sigma 0: none).  Admission counts the update's copy
 * (12 * nverts bytes) besides the rebuild's estimate.  GRID_EAGAIN when
 * admission refuses for now (nothing queued), GRID_ELIMIT when the request's
 * estimate alone exceeds the budget (it can never be admitted), GRID_EINVAL
 * for an unknown mesh or bad sigma, GRID_ENOMEM / GRID_ECUDA if the update
 * cannot be copied (nothing queued). */
int grid_serve_submit(grid_server *srv, int32_t mesh_id, const float *new_verts, float sigma, uint64_t seed,
                      uint64_t *ticket);
/* If the request has finished: GRID_OK with views of its result (device
 * pointers owned by the server, valid until grid_serve_release; never pass
 * them to grid_buf_free) or the build's error code.  GRID_ENOTREADY while it
 * is queued or running, GRID_EINVAL for an unknown or released ticket.  Any
 * output pointer may be NULL. */
int grid_serve_poll(grid_server *srv, uint64_t ticket, grid_buf *cells, grid_buf *refs, grid_info *info);
/* As grid_serve_poll, waiting up to timeout_us (< 0: no limit) for the
 * request to finish; GRID_ETIMEOUT if it has not, GRID_EINVAL if another
 * thread released the ticket while this one waited. */
int grid_serve_wait(grid_server *srv, uint64_t ticket, int64_t timeout_us, grid_buf *cells, grid_buf *refs,
                    grid_info *info);
/* Frees a finished request's result and its admission reservation.
 * GRID_ENOTREADY while it is queued or running, GRID_EINVAL if unknown. */
int grid_serve_release(grid_server *srv, uint64_t ticket);
/* Counters and latency percentiles since creation or the last reset
 * (reset != 0 clears them after copying; the gauges queued / reserved_bytes /
 * budget_bytes are never cleared). */
int grid_serve_get_stats(grid_server *srv, grid_serve_stats *out, int reset);

/* ---- without allocation -------------------------------------------------- */

/* The same cell ranges as grid_extract_ranges, for callers that cannot
 * allocate device memory when they call it: code running under another
 * runtime's memory manager (which owns the device budget and forbids foreign
 * allocations), loops where cudaMalloc / cudaFree would synchronise the
 * device, paths that must not fail for lack of memory once initialised.  The
 * paper has no counterpart; this is a deployment entry point.  It needs no
 * context and allocates nothing: its scratch (a merge-path split table of
 * 2^18 + 1 words, 1 MiB, and an error word) is a fixed-size device array of
 * the library that every GPU which loads the library keeps until the process
 * exits.
 *
 * C_sorted (int32 [count], cell ids sorted ascending, each < ncells) and
 * cells (int32 [ncells + 1]) are device pointers on the calling thread's
 * current device; the work runs on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and the call returns after it has finished.  The
 * first call on a device looks up the scratch's device address and keeps it
 * for the life of the process; make that first call before any stream
 * capture, and make no call on a device after cudaDeviceReset has torn down
 * its context in this process (the kept address would be stale).  The error
 * word is cleared at the start of every call.  All calls share the one scratch
 * array, which keeps the last call's contents: calls that overlap on the GPU
 * (different streams or threads at the same time) race and must be
 * serialised by the caller.
 *
 * Limit: count + ncells + 1 <= 2^18 * 4096 (about 1.07e9); larger requests
 * return GRID_ELIMIT without touching the GPU.  GRID_EINVAL for bad
 * arguments or a key >= ncells, GRID_ECUDA for a failed CUDA call. */
int grid_extract_ranges_noalloc(const int32_t *C_sorted, int64_t count, int64_t ncells, int32_t *cells,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_GRID_H */
