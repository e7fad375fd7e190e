// Device-side definitions shared by the grid-construction kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gg {

// Error bits raised by kernels into Ctl::err and turned into GRID_* codes on
// the host.  No kernel traps: a failed check records a bit and skips the
// offending access.
constexpr unsigned ERR_BADINDEX = 1u;   // triangle references a vertex outside [0, nverts)
constexpr unsigned ERR_NONFINITE = 2u;  // NaN / Inf vertex coordinate
constexpr unsigned ERR_OVERFLOW = 4u;   // a prefix sum passed INT32_MAX
constexpr unsigned ERR_TIMEOUT = 8u;    // a bounded look-back wait gave up
constexpr unsigned ERR_RANGE = 16u;     // a key outside [0, ncells) or out of order reached range
                                        // extraction, or a sort scatter fell outside the output
constexpr unsigned ERR_TILE_REDO = 64u;        // not an error: count/scan could not record every pair
                                               // tile's first object; the host runs tile_search
constexpr unsigned ERR_LOCAL_FALLBACK = 32u;   // not an error: a group of buckets too large for the
                                               // per-bucket counting sort; the host places the build
                                               // by radix passes over every key bit instead

// Spin limit of every look-back wait (each iteration sleeps ~0.1-1 us).
constexpr unsigned SPIN_LIMIT = 1u << 20;

constexpr int MAX_PASSES = 4;
constexpr int MAX_RADIX = 1 << 11;

// Per-build control block, zeroed by one memset before the first kernel.
struct Ctl {
    unsigned lo_inv[3];         // atomicMax of ~ordered(min coordinate) per axis
    unsigned hi_ord[3];         // atomicMax of ordered(max coordinate) per axis
    unsigned err;               // ERR_* bits
    unsigned spare;             // unused (keeps the layout)
    unsigned long long nrefs;   // NO, written by the last count/scan tile
    unsigned tickets[8];        // tile tickets: [0] count/scan, [7] culling emit; [2] counts the
                                // hybrid placement's bucket groups
    unsigned long long nkept;   // pairs the culling emit kept, written by its last tile
    unsigned pad[4];
    // grid metadata M computed on the device from the bounds above (plan_kernel),
    // for count/scan to read without a host round trip; the host checks it
    // against its own plan from the same bounds
    float plan_lo[3];
    float plan_scale[3];
    int plan_res[3];
    unsigned plan_pad;
};
static_assert(sizeof(Ctl) == 136, "Ctl layout");

// One object's box in grid coordinates and its pair offset (grid_objrec).
struct __align__(16) ObjRec {
    uint16_t lo[3];
    uint16_t hi[3];
    uint32_t start;
};
static_assert(sizeof(ObjRec) == 16, "ObjRec layout");

// Order-preserving map float -> uint32 (larger float, larger key).
__host__ __device__ __forceinline__ unsigned float_to_ordered(float f)
{
#ifdef __CUDA_ARCH__
    unsigned b = __float_as_uint(f);
#else
    unsigned b;
    __builtin_memcpy(&b, &f, 4);
#endif
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__host__ __device__ __forceinline__ float ordered_to_float(unsigned k)
{
    unsigned b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, 4);
    return f;
#endif
}

#ifdef __CUDACC__

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Four consecutive 32-bit words, each read with relaxed gpu-scope semantics
// (16-byte aligned address).
__device__ __forceinline__ uint4 ld_relaxed_v4(const unsigned *p)
{
    uint4 v;
    asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Grid coordinate of world value p on one axis: floor((p - lo) * scale) with
// both operations rounded to FP32 separately (the intrinsics are never
// contracted into an FMA), clamped to [0, res - 1]; NaN maps to 0.
__device__ __forceinline__ int cell_coord(float p, float lo, float scale, int res)
{
    float u = __fmul_rn(__fsub_rn(p, lo), scale);
    if (!(u >= 1.0f)) return 0;                 // u < 1 (incl. negative) or NaN
    if (u >= (float)res) return res - 1;        // floor(u) > res - 1
    return __float2int_rz(u);                   // u in [1, res): truncation == floor
}

#endif  // __CUDACC__

}  // namespace gg
