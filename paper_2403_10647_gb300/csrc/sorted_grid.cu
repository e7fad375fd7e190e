// Ablation of the pair generation: the "sorted grid" placement the paper
// compares against (Sec. 2, Kalojanov et al.), where one thread per object
// writes all of that object's <cell, object> pairs (MakePairs).  The paper
// attributes the sorted grid's cost on architectural scenes to this step: a
// thread whose triangle covers thousands of cells works alone while the rest
// of its warp idles, and each thread's stores form its own run, so a warp's
// stores do not coalesce.  Algorithm 1 instead spends one thread per pair
// (fused here into the first radix-sort pass).
//
// The pairs and their object order are the same as Algorithm 1's (object
// ascending, cells in GlobalCoords order within an object), so the rest of
// the build - radix sort and range extraction - and the result are unchanged.
#include <cuda_runtime.h>

#include "kernels.h"

namespace gg {

__global__ void __launch_bounds__(256) make_pairs_per_object_kernel(const ObjRec *__restrict__ recs, long long n,
                                                                   unsigned res_x, unsigned res_y, unsigned count,
                                                                   unsigned *__restrict__ C,
                                                                   unsigned *__restrict__ O, Ctl *ctl)
{
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const ObjRec r = recs[i];
    unsigned pos = r.start;
    for (unsigned z = r.lo[2]; z <= r.hi[2]; ++z) {
        for (unsigned y = r.lo[1]; y <= r.hi[1]; ++y) {
            const unsigned row = res_x * (y + res_y * z);
            for (unsigned x = r.lo[0]; x <= r.hi[0]; ++x) {
                if (pos >= count) {   // a record inconsistent with NO: skip the store, report
                    atomicOr(&ctl->err, ERR_RANGE);
                    return;
                }
                C[pos] = row + x;
                O[pos] = (unsigned)i;
                ++pos;
            }
        }
    }
}

cudaError_t launch_make_pairs_per_object(const ObjRec *recs, long long n, unsigned res_x, unsigned res_y,
                                         unsigned count, unsigned *C, unsigned *O, Ctl *ctl, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    make_pairs_per_object_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(recs, n, res_x, res_y, count, C, O,
                                                                             ctl);
    return cudaGetLastError();
}

}  // namespace gg
