// Range extraction without any allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the cell ranges: code that runs under another runtime's memory manager
// (which owns the whole device budget and forbids foreign allocations),
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device and stall every other stream, and code paths that must not fail
// for lack of memory once initialised.  grid_extract_ranges_noalloc serves
// them: it needs no context and no allocation; its only scratch (the
// merge-path split table and an error word) lives in fixed-size device
// arrays of this file, which every GPU that loads the library keeps until
// the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "grid.h"
#include "kernels.h"

namespace {

// Split table capacity: one entry per extraction block plus one.  A block
// covers gg::EXTRACT_TILE merged items (keys + cells + 1), so this bounds
// count + ncells + 1 by NOALLOC_MAX_BLOCKS * EXTRACT_TILE (about 1.07e9).
constexpr unsigned long long NOALLOC_MAX_BLOCKS = 1ull << 18;

static __device__ __align__(256) unsigned g_noalloc_splits[NOALLOC_MAX_BLOCKS + 1];
static __device__ __align__(256) gg::Ctl g_noalloc_ctl;

constexpr int kMaxDevices = 64;

struct SymbolAddrs {
    unsigned *splits = nullptr;
    gg::Ctl *ctl = nullptr;
    bool ready = false;
};

SymbolAddrs g_addrs[kMaxDevices];
std::mutex g_addrs_mutex;

// Device addresses of the scratch arrays on the current device, looked up
// once per device (the host-side names are not device addresses) and kept
// for the life of the process: a cudaDeviceReset in between would leave them
// stale, which the header documents as a limit of this entry point.
int scratch_addresses(int dev, SymbolAddrs *out)
{
    if (dev < 0 || dev >= kMaxDevices) return GRID_EINVAL;
    std::lock_guard<std::mutex> lock(g_addrs_mutex);
    SymbolAddrs &a = g_addrs[dev];
    if (!a.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_splits) != cudaSuccess) {
            cudaGetLastError();
            return GRID_ECUDA;
        }
        a.splits = static_cast<unsigned *>(p);
        if (cudaGetSymbolAddress(&p, g_noalloc_ctl) != cudaSuccess) {
            cudaGetLastError();
            return GRID_ECUDA;
        }
        a.ctl = static_cast<gg::Ctl *>(p);
        a.ready = true;
    }
    *out = a;
    return GRID_OK;
}

}  // namespace

extern "C" int grid_extract_ranges_noalloc(const int32_t *C_sorted, int64_t count, int64_t ncells,
                                           int32_t *cells, void *stream)
{
    if (count < 0 || count > 0x7FFFFFFFll || ncells < 1 || ncells > 0x7FFFFFFFll || !cells) return GRID_EINVAL;
    if (count > 0 && !C_sorted) return GRID_EINVAL;
    const unsigned long long nb = gg::extract_blocks((unsigned long long)count, (unsigned long long)ncells);
    if (nb > NOALLOC_MAX_BLOCKS) return GRID_ELIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GRID_ECUDA;
    }
    SymbolAddrs addr;
    const int rc = scratch_addresses(dev, &addr);
    if (rc != GRID_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the error word is shared by every call and keeps the last one's value
    if (cudaMemsetAsync(&addr.ctl->err, 0, sizeof(unsigned), s) != cudaSuccess) return GRID_ECUDA;
    gg::ExtractArgs xa{};
    xa.keys = reinterpret_cast<const unsigned *>(C_sorted);
    xa.count = (unsigned long long)count;
    xa.ncells = (unsigned long long)ncells;
    xa.G = reinterpret_cast<unsigned *>(cells);
    xa.splits = addr.splits;   // every entry is rewritten before it is read
    xa.ctl = addr.ctl;
    if (gg::launch_extract_split(xa, s) != cudaSuccess) return GRID_ECUDA;
    if (gg::launch_extract(xa, s) != cudaSuccess) return GRID_ECUDA;
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, &addr.ctl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GRID_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GRID_ECUDA;
    return err ? GRID_EINVAL : GRID_OK;
}
