// Allocation-free forward voxelization: pg_voxelize_noalloc.
//
// The regular entry points allocate a small amount of device memory of their own the first
// time they run on a device (the error word and the work counters of the direct kernel).
// Some callers cannot let a library allocate: code that runs while a stream capture in
// global mode is open elsewhere in the process (cudaMalloc is not permitted then), programs
// whose device memory is entirely reserved up front by a framework's caching allocator or
// an external budget, and embedded or real-time hosts that freeze their device-memory
// footprint after start-up.  This entry point runs the same direct kernel with its scratch
// taken from a fixed array compiled into the library instead.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "pg.h"
#include "pg_internal.h"

namespace {

// Scratch of pg_voxelize_noalloc.  Bytes [0, 16): the direct kernel's work counter and
// retired-warp counter; bytes [16, 20): its error word.  Every GPU that loads the library
// holds these PG_NOALLOC_SCRATCH_BYTES bytes until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PG_NOALLOC_SCRATCH_BYTES];

constexpr size_t kCounterBytes = 2 * sizeof(unsigned long long);
constexpr size_t kScratchNeeded = kCounterBytes + sizeof(unsigned);
static_assert(kScratchNeeded <= PG_NOALLOC_SCRATCH_BYTES, "scratch array too small");

struct Setup {
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
};

std::mutex g_mu;
std::map<int, Setup> g_setup;  // host-side bookkeeping only

// Once per device, with that device current: resolve the device address of the scratch
// array (in host code its name is only a host-side stand-in) and the SM count.
pg_status setup_device(int dev, Setup *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_setup.find(dev);
    if (it == g_setup.end()) {
        Setup s;
        cudaError_t e = cudaGetSymbolAddress((void **)&s.scratch, g_noalloc_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return pgi::set_last_error(PG_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s",
                                       cudaGetErrorString(e));
        }
        e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return pgi::set_last_error(PG_ERR_CUDA, "cudaDeviceGetAttribute: %s",
                                       cudaGetErrorString(e));
        }
        it = g_setup.emplace(dev, s).first;
    }
    *out = it->second;
    return PG_OK;
}

// Bytes of scratch one launch of the direct kernel needs.  It does not grow with the batch.
size_t scratch_bytes_needed(const pg_batch *, const pg_grid *) { return kScratchNeeded; }

}  // namespace

extern "C" pg_status pg_voxelize_noalloc(const pg_batch *batch, const pg_grid *grid,
                                         int32_t out_dtype, void *out, void *stream,
                                         uint32_t *bits_out)
{
    if (bits_out) *bits_out = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return pgi::set_last_error(PG_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    Setup s;
    pg_status st = setup_device(dev, &s);
    if (st) return st;
    if (batch && grid && scratch_bytes_needed(batch, grid) > PG_NOALLOC_SCRATCH_BYTES)
        return pgi::set_last_error(PG_ERR_INVALID_ARG,
                                   "this launch needs %zu bytes of scratch; the fixed array "
                                   "holds %d",
                                   scratch_bytes_needed(batch, grid), PG_NOALLOC_SCRATCH_BYTES);
    unsigned long long *sched = reinterpret_cast<unsigned long long *>(s.scratch);
    unsigned *err = reinterpret_cast<unsigned *>(s.scratch + kCounterBytes);
    pgi::KernelLaunch kl;
    st = pgi::direct_launch_with_scratch(batch, grid, out_dtype, out, err, sched, s.sms, &kl);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    // The array keeps the previous call's contents: the counters and the error word must
    // start at zero.
    e = cudaMemsetAsync(s.scratch, 0, kScratchNeeded, cs);
    if (e == cudaSuccess && kl.func) e = pgi::launch(kl, cs);
    unsigned bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return pgi::set_last_error(PG_ERR_CUDA, "pg_voxelize_noalloc: %s", cudaGetErrorString(e));
    }
    if (bits_out) *bits_out = bits;
    if (bits)
        return pgi::set_last_error(PG_ERR_DEVICE_VALIDATION,
                                   "device validation failed (bits 0x%x)", bits);
    pgi::set_last_error(PG_OK, "");
    return PG_OK;
}
