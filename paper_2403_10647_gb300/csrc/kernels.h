// Launch interface between the host runtime and the grid kernels.
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"

namespace gg {

// Tile shapes.  COUNT: objects per count/scan tile.  PAIR: pairs per tile of
// the pair-generation, histogram and radix-sort-pass kernels.  EXTRACT:
// merged (key, cell) items per range-extraction block.
#ifndef GG_PAIR_BLOCK
#define GG_PAIR_BLOCK 256
#endif
#ifndef GG_PAIR_ITEMS
#define GG_PAIR_ITEMS 12
#endif
#ifndef GG_PASS_MIN_BLOCKS
#define GG_PASS_MIN_BLOCKS 5
#endif
#ifndef GG_GROUP_TILES
#define GG_GROUP_TILES 16
#endif
#ifndef GG_GEN_MIN_BLOCKS
#define GG_GEN_MIN_BLOCKS 6
#endif
#ifndef GG_COUNT_BLOCK
#define GG_COUNT_BLOCK 256
#endif
#ifndef GG_COUNT_TILE
#define GG_COUNT_TILE 2048
#endif
#ifndef GG_COUNT_MIN_BLOCKS
#define GG_COUNT_MIN_BLOCKS 6
#endif
constexpr int COUNT_BLOCK = GG_COUNT_BLOCK;
constexpr int COUNT_TILE = GG_COUNT_TILE;
constexpr int COUNT_MIN_BLOCKS = GG_COUNT_MIN_BLOCKS;   // resident count/scan blocks per SM compiled for
constexpr int PAIR_BLOCK = GG_PAIR_BLOCK;
constexpr int PAIR_TILE = GG_PAIR_BLOCK * GG_PAIR_ITEMS;
constexpr int PASS_MIN_BLOCKS = GG_PASS_MIN_BLOCKS;
constexpr int GROUP_TILES = GG_GROUP_TILES;   // most tiles per upsweep block
// resident blocks per SM the pair-generating upsweep is compiled for: its
// per-tile chain (object marks, records, stores) is latency-bound, so more
// blocks in flight beat the few registers spilled
constexpr int GEN_MIN_BLOCKS = GG_GEN_MIN_BLOCKS;
// Block shapes of the radix-sort kernels, chosen per context (grid_opts
// tile_shape): PAIR_BLOCK threads x PAIR_TILE / PAIR_BLOCK pairs, or
// ALT_BLOCK threads with fewer pairs each.  Both cover the same PAIR_TILE
// pairs per tile, so everything outside these kernels is shared.
enum { SHAPE_MAIN = 0, SHAPE_ALT = 1 };
constexpr int ALT_BLOCK = 384;
static_assert(PAIR_TILE % ALT_BLOCK == 0, "the alternative shape covers whole tiles");
constexpr int ALT_PASS_MIN_BLOCKS = 3;   // 56 registers, no spill
constexpr int ALT_GEN_MIN_BLOCKS = 4;
static_assert(GROUP_TILES * PAIR_TILE <= 65536, "tile offsets inside a group fit 16 bits");
constexpr int EXTRACT_BLOCK = 256;
constexpr int EXTRACT_TILE = 4096;

enum { SRC_MEM = 0, SRC_GEN = 1 };

// A batch of meshes built as one flattened problem: mesh m owns objects
// [obj_base[m], obj_base[m + 1]) and global cell ids [cell_base,
// cell_base + ncells); a pair's key is cell_base + its local cell id and its
// value the object's index inside its mesh.
struct MeshDesc {
    const float *verts;
    const int *tris;
    long long nverts;
    long long n;
    float lo[3];
    float scale[3];
    int res[3];
    unsigned cell_base;
};

struct MeshTab {
    const MeshDesc *md;             // [nm] device; nullptr for a single mesh
    const long long *obj_base;      // [nm + 1] device
    int nm;
};

struct CountArgs {
    const float *verts;
    long long nverts;
    const int *tris;
    long long n;
    float lo[3];
    float scale[3];
    int res[3];
    ObjRec *recs;                   // [n] out
    unsigned long long *status;     // [ceil(n / COUNT_TILE)] look-back words, zeroed
    Ctl *ctl;
    MeshTab mt;                     // batched: per-object mesh (verts, tris, plan)
    unsigned *pair_base;            // batched: [nm] out, pair offset of each mesh's first object
    bool device_plan;               // single mesh: take lo / scale / res from ctl->plan_* instead
    unsigned *tile_obj;             // single mesh, optional: [tile_cap] the first object of every
    unsigned tile_cap;              // PAIR_TILE-pair tile and, after the last tile, n - 1 (tile_search's
                                    // result), or ERR_TILE_REDO when it did not fit
};

struct EmitArgs {
    const ObjRec *recs;
    const unsigned *tile_obj;       // [ntiles + 1]
    MeshTab mt;
    unsigned res_x, res_y;
    unsigned count;                 // NO
    unsigned *C;
    unsigned *O;
};

// Culling emit: the object-order pairs of the box placement minus those the
// triangle/cell separating-axis test rejects, compacted in object order.
struct CullArgs {
    const ObjRec *recs;
    const unsigned *tile_obj;       // [ntiles + 1]
    const float *verts;
    long long nverts;
    const int *tris;
    float lo[3], scale[3];
    float res_f[3];                 // res per axis as float: grid coordinates are clamped to it
    unsigned res_x, res_y;
    unsigned count;                 // NO of the box placement
    unsigned *C;                    // [count] out, first nkept entries used
    unsigned *O;
    unsigned long long *status;     // [ntiles] look-back words, zero on entry
    Ctl *ctl;                       // nkept out
};

// Upsweep of one radix-sort pass: digit counts per tile, offsets of each
// tile inside its group of gtiles tiles, offsets of each group, and,
// from the last group's inclusive prefixes, the pass's digit starts.
struct UpArgs {
    const unsigned *keys_in;        // SRC_MEM
    const ObjRec *recs;             // SRC_GEN
    const unsigned *tile_obj;       // SRC_GEN
    MeshTab mt;                     // SRC_GEN, batched
    unsigned res_x, res_y;          // SRC_GEN
    unsigned *gen_keys;             // SRC_GEN: if set, the generated pairs are stored here
    unsigned *gen_vals;             //   (object order, [count] each) for the first downsweep
    unsigned count;
    unsigned ntiles;
    int shift, bits;                // this pass's digit
    unsigned short *intra;          // [ntiles][2^RBITS] out: tile offsets inside its group
                                    // (< GROUP_TILES * PAIR_TILE <= 65536)
    unsigned *gpref;                // [ngroups][2^RBITS] out: group offsets
    unsigned *status;               // [ngroups][2^RBITS] look-back words, zero on entry
    unsigned *dbase;                // [2^bits] out: the pass's digit starts (written by the last group)
    Ctl *ctl;
    unsigned gtiles;                // tiles per group, 1 .. GROUP_TILES (group_tiles)
};

// Downsweep of one pass: rank and scatter of each tile.  IN_PAIR_ANY reads
// stored pairs like IN_PAIR but may rank equal digits of a warp out of
// element order (the hybrid placement's first pass; see downsweep_kernel).
// IN_PAIR_KEEP needs equal digits to keep only the order of key bits
// [keep_lo, shift) (the hybrid placement's later passes: the order inside a
// bucket is restored by the placement): a tile whose elements all share
// those bits ranks like IN_PAIR_ANY, any other tile like IN_PAIR.
enum { IN_GEN = 0, IN_PAIR = 1, IN_PAIR_ANY = 2, IN_PAIR_KEEP = 3 };

struct DownArgs {
    const unsigned *keys_in;        // IN_PAIR
    const unsigned *vals_in;        // IN_PAIR
    const ObjRec *recs;             // IN_GEN
    const unsigned *tile_obj;       // IN_GEN
    MeshTab mt;                     // IN_GEN, batched
    unsigned res_x, res_y;          // IN_GEN
    unsigned *keys_out;
    unsigned *vals_out;
    unsigned count;
    int shift, bits;
    int keep_lo;                    // IN_PAIR_KEEP: lowest key bit whose order equal digits keep
    const unsigned *dbase;          // [2^bits] digit starts of this pass
    const unsigned *gpref;          // from the upsweep
    const unsigned short *intra;    // from the upsweep
    Ctl *ctl;
};

struct ExtractArgs {
    const unsigned *keys;           // sorted
    unsigned long long count;
    unsigned long long ncells;
    unsigned *G;                    // [ncells + 1]
    unsigned *splits;               // [extract_blocks + 1] merge-path splits (scratch)
    Ctl *ctl;
};

// Per-request vertex jitter of the serving loop: dst[e] = src[e] + s * n(e)
// for the floats e of a mesh's vertex array, n(e) a unit-variance
// Irwin-Hall normal from Philox4x32-10 at counter (e / 3, e % 3, 0, 0) and
// key (seed low, seed high) words.
struct JitterDesc {
    const float *src;
    float *dst;
    unsigned long long seed;
    float s;                        // sigma * sqrt(3), rounded to float once
    int pad;
};

// Meshes k = 0 .. nm-1 own floats [ebase[k], ebase[k + 1]) of the flattened
// element range [0, total).  With d == nullptr, `one` is the only mesh and
// ebase is not read.
cudaError_t launch_jitter(const JitterDesc &one, const JitterDesc *d, const long long *ebase, int nm,
                          long long total, cudaStream_t s);

cudaError_t launch_bounds(const float *verts, long long nverts, const int *tris, long long n, Ctl *ctl,
                          int nsm, cudaStream_t s);
// Batched: per-mesh bounds into bstate[m * 6 + (lo_inv x, y, z, hi x, y, z)].
cudaError_t launch_bounds_batched(const MeshTab &mt, long long ntot, unsigned *bstate, Ctl *ctl, cudaStream_t s);
// Batched: out[q] = G[q - m] - pair_base[m] for q in mesh m's slice
// [cells_off[m], cells_off[m + 1]) of the per-mesh cell arrays.
// Batched builds sorted in segments: recs[o].start -= seg_p0[s] for the
// segment s holding object o (the last s with seg_obj0[s] <= o).
cudaError_t launch_rebase_recs(ObjRec *recs, long long n, const long long *seg_obj0, const unsigned *seg_p0, int nseg,
                               cudaStream_t s);
cudaError_t launch_localize(const unsigned *G, const long long *cells_off, const unsigned *pair_base, int nm,
                            long long total, unsigned *out, cudaStream_t s);
cudaError_t launch_count_scan(const CountArgs &a, cudaStream_t s);
// Grid metadata M on the device (one thread): from ctl's bounds, n and
// lambda, the resolution and scale of the density rule (the host plan's
// formula and operation order; k's cube root is the device's cbrt), into
// ctl->plan_*.  With an error bit already set it writes a harmless plan
// (one cell, scale 0).
cudaError_t launch_plan(Ctl *ctl, long long n, float lambda, cudaStream_t s);
cudaError_t launch_tile_search(const ObjRec *recs, long long n, unsigned tile, unsigned ntiles,
                               unsigned *tile_obj, cudaStream_t s);
cudaError_t launch_emit(const EmitArgs &a, cudaStream_t s);
cudaError_t launch_cull_emit(const CullArgs &a, cudaStream_t s);
// Runs the look-back wait on col[0], which must be zero and stay zero.
cudaError_t launch_wait_selftest(const unsigned *col, Ctl *ctl, unsigned *out, cudaStream_t s);
// Pair-generation ablation (sorted_grid.cu): one thread per object writes its
// pairs C[start ..], O[start ..] (single mesh).
cudaError_t launch_make_pairs_per_object(const ObjRec *recs, long long n, unsigned res_x, unsigned res_y,
                                         unsigned count, unsigned *C, unsigned *O, Ctl *ctl, cudaStream_t s);
// Tiles per upsweep group for a pass of ntiles tiles on nsm SMs: GROUP_TILES
// when there are enough groups to fill the GPU, fewer (down to 1) when the
// groups would not: a group's tiles are walked by one block in sequence.
unsigned group_tiles(unsigned ntiles, int nsm);
cudaError_t launch_upsweep(const UpArgs &a, int rbits, int src, int shape, cudaStream_t s);
// gtiles: the tiles per group of the pass's upsweep
cudaError_t launch_downsweep(const DownArgs &a, int rbits, int in, unsigned ntiles, unsigned gtiles, int shape,
                             cudaStream_t s);
// Hybrid placement: once the radix passes have ordered the pairs by the high
// key bits (key >> lbits), every bucket of 2^lbits consecutive cells is a
// contiguous run of pairs.  One block per bucket sorts its run by cell with a
// counting sort in shared memory (RadixSort's low digits) and writes the
// bucket's cell ranges G (RunLengthEncode + NonEmptyCells + ExclusiveSum)
// and its object ids in cell order.
#ifndef GG_LOCAL_BLOCK
#define GG_LOCAL_BLOCK 512
#endif
#ifndef GG_LOCAL_CAP
#define GG_LOCAL_CAP 12288
#endif
#ifndef GG_LOCAL_MIN_BLOCKS
#define GG_LOCAL_MIN_BLOCKS 3
#endif
constexpr int LOCAL_BLOCK = GG_LOCAL_BLOCK;
constexpr int LOCAL_CAP = GG_LOCAL_CAP;                 // pairs a block places at once
constexpr int LOCAL_MIN_BLOCKS = GG_LOCAL_MIN_BLOCKS;   // resident blocks per SM it is compiled for
constexpr int LOCAL_LMAX = 11;                          // at most 2^11 cells per bucket
constexpr unsigned LOCAL_RUN_MAX = 512;                // longest cell run a block sorts
constexpr unsigned LOCAL_GROUP_PAIRS = LOCAL_CAP / 2;  // pairs at which a group of buckets closes

struct LocalArgs {
    const unsigned *keys;           // [count] sorted by key >> lbits
    const unsigned *vals;           // [count]
    unsigned count;
    unsigned long long ncells;
    int lbits;                      // a bucket covers 2^lbits cells
    unsigned nbuckets;
    unsigned *starts;               // [nbuckets + 1]: first pair of each bucket (bucket_split)
    unsigned *groups;               // [max_groups]: first bucket of each group, in no order
    unsigned group_pairs;           // LOCAL_GROUP_PAIRS
    unsigned max_groups;            // bound on the groups: blocks of the local sort
    unsigned *refs;                 // [count] out: object ids in cell order
    unsigned *G;                    // [ncells + 1] out
    Ctl *ctl;                       // tickets[2] counts the groups (zero on entry)
};

// starts[b] = number of keys whose key >> lbits is below b, b = 0 .. nbuckets;
// G[ncells] = count; the first bucket of every group appended to groups.
cudaError_t launch_bucket_split(const LocalArgs &a, cudaStream_t s);
cudaError_t launch_local_sort(const LocalArgs &a, cudaStream_t s);

unsigned long long extract_blocks(unsigned long long count, unsigned long long ncells);
cudaError_t launch_extract_split(const ExtractArgs &a, cudaStream_t s);
cudaError_t launch_extract(const ExtractArgs &a, cudaStream_t s);

}  // namespace gg
