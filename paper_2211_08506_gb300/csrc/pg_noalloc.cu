// Allocation-free forward voxelization: pg_voxelize_noalloc.
//
// The regular entry points allocate a small amount of device memory of their own the first
// time they run on a device (the error word and the work counters of the direct kernel).
// Some callers cannot let a library allocate: code that runs while another thread holds a
// stream capture open in global mode (cudaMalloc is refused then, and the attempt
// invalidates that capture), programs whose device memory is entirely reserved up front by
// a framework's caching allocator or an external budget, and embedded or real-time hosts
// that freeze their device-memory footprint after start-up.  This entry point runs the same
// direct kernel with its scratch taken from a fixed array compiled into the library instead.
//
// Under another thread's global-mode capture the runtime also refuses synchronizing calls
// (cudaStreamSynchronize, copies into pageable memory).  So the call learns that its work has
// finished from the copy itself: after the kernel, one 8-byte copy brings the error word
// together with a marker word into page-locked host memory, and the host waits for the
// marker to arrive.
#include <cuda_runtime.h>

#include <chrono>
#include <map>
#include <mutex>
#include <thread>

#include "pg.h"
#include "pg_internal.h"

namespace {

// Scratch of pg_voxelize_noalloc.  Bytes [0, 16): the direct kernel's work counter and
// retired-warp counter; bytes [16, 20): its error word; bytes [20, 24): the completion
// marker.  Every GPU that loads the library holds these PG_NOALLOC_SCRATCH_BYTES bytes until
// the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PG_NOALLOC_SCRATCH_BYTES];

constexpr size_t kCounterBytes = 2 * sizeof(unsigned long long);
constexpr size_t kErrOffset = kCounterBytes;
constexpr size_t kMarkerOffset = kErrOffset + sizeof(unsigned);
constexpr size_t kScratchNeeded = kMarkerOffset + sizeof(unsigned);
static_assert(kScratchNeeded <= PG_NOALLOC_SCRATCH_BYTES, "scratch array too small");
static_assert(kErrOffset % 8 == 0, "error word and marker are copied as one aligned 8 bytes");
// Marker bytes written by a memset: the word 0x01010101, never 0.
constexpr unsigned char kMarkerByte = 0x01;
constexpr unsigned kMarkerWord = 0x01010101u;
// Longest wait for a call's work to finish before the call reports PG_ERR_TIMEOUT.
constexpr double kWaitLimitSeconds = 600.0;

struct Setup {
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
};

std::mutex g_mu;
std::map<int, Setup> g_setup;  // host-side bookkeeping only

// Host words, one per device, that receive {error word, marker} (little-endian: the error
// word in the low half).  Page-locked once (cudaHostRegister, no allocation) so that the
// copy into them is a plain asynchronous transfer.
constexpr int kMaxDevices = 32;
alignas(64) unsigned long long g_done_host[kMaxDevices];
static_assert(sizeof g_done_host == 256, "the header documents 256 bytes of host words");
bool g_host_registered = false;

// Once per device, with that device current: resolve the device address of the scratch
// array (in host code its name is only a host-side stand-in) and the SM count; once per
// process, page-lock the host words.
pg_status setup_device(int dev, Setup *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices)
        return pgi::set_last_error(PG_ERR_INVALID_ARG, "device ordinal %d outside 0..%d", dev,
                                   kMaxDevices - 1);
    if (!g_host_registered) {
        cudaError_t e = cudaHostRegister(g_done_host, sizeof g_done_host,
                                         cudaHostRegisterPortable);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return pgi::set_last_error(PG_ERR_CUDA, "cudaHostRegister(completion words): %s",
                                       cudaGetErrorString(e));
        }
        g_host_registered = true;
    }
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
    cudaStream_t cs = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(cs, &cap);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return pgi::set_last_error(PG_ERR_CUDA, "cudaStreamIsCapturing: %s",
                                   cudaGetErrorString(e));
    }
    if (cap != cudaStreamCaptureStatusNone)
        return pgi::set_last_error(PG_ERR_INVALID_ARG, "pg_voxelize_noalloc is synchronous: "
                                                       "its stream must not be capturing");
    unsigned long long *sched = reinterpret_cast<unsigned long long *>(s.scratch);
    unsigned *err = reinterpret_cast<unsigned *>(s.scratch + kErrOffset);
    pgi::KernelLaunch kl;
    st = pgi::direct_launch_with_scratch(batch, grid, out_dtype, out, err, sched, s.sms, &kl);
    if (st) return st;
    // The array keeps the previous call's contents: the counters and the error word must
    // start at zero; the marker is set so that the copy after the kernel carries it.
    unsigned long long *done = &g_done_host[dev];
    __atomic_store_n(done, 0ull, __ATOMIC_RELEASE);
    const char *what = "scratch clear";
    e = cudaMemsetAsync(s.scratch, 0, kMarkerOffset, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.scratch + kMarkerOffset, kMarkerByte, 4, cs);
    if (e == cudaSuccess && kl.func) {
        what = "launch";
        e = pgi::launch(kl, cs);
    }
    if (e == cudaSuccess) {
        what = "completion copy";
        e = cudaMemcpyAsync(done, s.scratch + kErrOffset, sizeof *done, cudaMemcpyDeviceToHost,
                            cs);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return pgi::set_last_error(PG_ERR_CUDA, "pg_voxelize_noalloc (%s): %s", what,
                                   cudaGetErrorString(e));
    }
    // Wait for the copy, which stream order places after the kernel, to deliver the marker.
    const auto t0 = std::chrono::steady_clock::now();
    unsigned long long word = 0;
    for (unsigned spin = 0;; ++spin) {
        word = __atomic_load_n(done, __ATOMIC_ACQUIRE);
        if ((unsigned)(word >> 32) == kMarkerWord) break;
        if (spin >= 1024) {
            std::this_thread::yield();
            if ((spin & 1023u) == 0 &&
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
                    kWaitLimitSeconds)
                return pgi::set_last_error(PG_ERR_TIMEOUT,
                                           "pg_voxelize_noalloc: the work did not finish within "
                                           "%.0f s; it may still be running on the stream",
                                           kWaitLimitSeconds);
        }
    }
    const unsigned bits = (unsigned)(word & 0xffffffffull);
    if (bits_out) *bits_out = bits;
    if (bits)
        return pgi::set_last_error(PG_ERR_DEVICE_VALIDATION,
                                   "device validation failed (bits 0x%x)", bits);
    pgi::set_last_error(PG_OK, "");
    return PG_OK;
}
