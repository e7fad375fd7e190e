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
#define GG_PAIR_ITEMS 16
#endif
#ifndef GG_PASS_MIN_BLOCKS
#define GG_PASS_MIN_BLOCKS 3
#endif
constexpr int COUNT_BLOCK = 256;
constexpr int COUNT_TILE = 2048;
constexpr int PAIR_BLOCK = GG_PAIR_BLOCK;
constexpr int PAIR_TILE = GG_PAIR_BLOCK * GG_PAIR_ITEMS;
constexpr int PASS_MIN_BLOCKS = GG_PASS_MIN_BLOCKS;
constexpr int EXTRACT_BLOCK = 256;
constexpr int EXTRACT_TILE = 2048;

enum { SRC_MEM = 0, SRC_GEN = 1 };

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
};

struct EmitArgs {
    const ObjRec *recs;
    const unsigned *tile_obj;       // [ntiles + 1]
    unsigned res_x, res_y;
    unsigned count;                 // NO
    unsigned *C;
    unsigned *O;
};

struct HistArgs {
    const unsigned *keys_in;        // SRC_MEM
    const ObjRec *recs;             // SRC_GEN
    const unsigned *tile_obj;       // SRC_GEN
    unsigned res_x, res_y;          // SRC_GEN
    unsigned count;
    unsigned ntiles;
    int npasses;
    int shift[MAX_PASSES];
    int bits[MAX_PASSES];
    unsigned *hist;                 // [MAX_PASSES][MAX_RADIX], zero on entry, zero on exit
    unsigned *dbase;                // [MAX_PASSES][MAX_RADIX] out: exclusive digit starts
    unsigned *status0;              // [ntiles][status_row] zeroed here for the first pass
    int status_row;
    Ctl *ctl;
};

// Element layouts of a radix-sort pass.  Between passes an element travels
// as one 64-bit word (key << 32 | value); the first pass may instead read two
// int32 arrays or generate the object-order pairs itself, the last may write
// two arrays.
enum { IN_GEN = 0, IN_PAIR = 1, IN_PACKED = 2 };
enum { OUT_PACKED = 0, OUT_PAIR = 1 };

struct PassArgs {
    const unsigned *keys_in;        // IN_PAIR
    const unsigned *vals_in;        // IN_PAIR
    const unsigned long long *elems_in;   // IN_PACKED
    const ObjRec *recs;             // IN_GEN
    const unsigned *tile_obj;       // IN_GEN
    unsigned res_x, res_y;          // IN_GEN
    unsigned long long *elems_out;  // OUT_PACKED
    unsigned *keys_out;             // OUT_PAIR
    unsigned *vals_out;             // OUT_PAIR
    unsigned count;
    int shift, bits;
    const unsigned *dbase;          // [2^bits] global digit starts of this pass
    unsigned *status;               // [ntiles][2^RBITS] zero on entry
    unsigned *status_next;          // zeroed here for the next pass (nullable)
    unsigned *ticket;               // zero on entry
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

cudaError_t launch_bounds(const float *verts, long long nverts, const int *tris, long long n, Ctl *ctl,
                          int nsm, cudaStream_t s);
cudaError_t launch_count_scan(const CountArgs &a, cudaStream_t s);
cudaError_t launch_tile_search(const ObjRec *recs, long long n, unsigned tile, unsigned ntiles,
                               unsigned *tile_obj, cudaStream_t s);
cudaError_t launch_emit(const EmitArgs &a, cudaStream_t s);
cudaError_t launch_hist(const HistArgs &a, int rbits, int src, int nsm, cudaStream_t s);
cudaError_t launch_pass(const PassArgs &a, int rbits, int in, int out, unsigned ntiles, cudaStream_t s);
unsigned long long extract_blocks(unsigned long long count, unsigned long long ncells);
cudaError_t launch_extract_split(const ExtractArgs &a, cudaStream_t s);
cudaError_t launch_extract(const ExtractArgs &a, cudaStream_t s);

}  // namespace gg
