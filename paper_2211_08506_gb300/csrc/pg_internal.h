// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pg.h"

namespace pgi {

constexpr int kMaxC = PG_MAX_CHANNELS;
// Candidate atoms one warp stages in shared memory for one (molecule, channel, x-plane)
// item.  Items with more candidates take the unstaged path (same result, bit for bit).
constexpr int kStageCap = 128;
constexpr int kChanCap = 128;  // one channel's atoms of a molecule, staged per chunk

// Per-call constants (kernel parameter space; uniform across the grid).
struct Geometry {
    int n_mol, n_atoms;
    int nx, ny, nz, C;
    int cutoff;    // pg_cutoff
    int periodic;  // 0/1
    float q[kMaxC];      // log2(e) / (2 sigma_c^2): G = 2^(-q d^2)
    float r2[kMaxC];     // r_c^2, the exact per-voxel cutoff test
    float rcull[kMaxC];  // r_c widened by a relative 1e-5 for conservative culling
    float inv_s2[kMaxC]; // 1 / sigma_c^2 (adjoint)
    int form;            // pg_form
    float kerf[kMaxC];   // 1 / (sqrt(2) sigma_c): erf argument scale of the integral form
    float kdmu[kMaxC];   // kerf / sqrt(pi): scale of the integral form's derivative
};

#ifdef __CUDACC__
// Voxel-integrated form (Sec. III-A, per-axis erf integrals): the normalised Gaussian's
// integral along one axis over the voxel whose centre lies at displacement d from the atom,
// with k = 1 / (sqrt(2) sigma).  The factor is even in d; when both edges lie on the same
// side of the atom it is taken as a difference of erfc values, which does not cancel.
__device__ __forceinline__ float erf_axis(float d, float h, float k)
{
    const float a = fabsf(d);
    const float lo = (a - 0.5f * h) * k, hi = (a + 0.5f * h) * k;
    return lo > 0.0f ? 0.5f * (erfcf(lo) - erfcf(hi)) : 0.5f * (erff(hi) + erff(-lo));
}

// Derivative of erf_axis with respect to the atom coordinate (d = centre - atom), from
// d/dt erf(t) = (2 / sqrt(pi)) exp(-t^2); kd = k / sqrt(pi).
__device__ __forceinline__ float erf_axis_dmu(float d, float h, float k, float kd)
{
    const float lo = (d - 0.5f * h) * k, hi = (d + 0.5f * h) * k;
    return kd * (expf(-lo * lo) - expf(-hi * hi));
}
#endif

struct Inputs {
    const float *coords;
    const int *elem;
    const int *mol_off;
    const float *origin;
    const float *spacing;
    const float *weight;  // per-atom weights, or null (all ones)
    const float *cell;    // per-molecule 3x3 box edges (rows), or null (axis-aligned box)
};

// Largest per-warp factor table of the voxel-integrated form (floats).
constexpr int kErfTabCap = 4096;

// Row stride of the voxel-integrated form's per-atom factor table: the y factors, then the z
// factors, each padded to a multiple of 4 floats so that a lane's z factors load as float4.
__host__ __device__ inline int erf_table_stride(int ny, int nz)
{
    return ((ny + 3) & ~3) + ((nz + 3) & ~3);
}

// 32-bit words of dynamic shared memory per warp of the direct kernel: kStageCap staged
// candidates and kChanCap channel atoms (float4 each), or, if larger, the voxel-integrated
// form's factor table (erf_tab words: molecules of at most 32 atoms use it from the start,
// larger ones past the staging area), then, with a factor table, the staged candidates' x
// factors (kStageCap words).  A multiple of 4 words.
__host__ __device__ inline int direct_warp_floats(int erf_tab)
{
    const int staging = 4 * (kStageCap + kChanCap);
    return (erf_tab > staging ? erf_tab : staging) + (erf_tab > 0 ? kStageCap : 0);
}

struct DirectArgs {
    Inputs in;
    void *out;
    unsigned *err;
    unsigned long long *sched;  // {next chunk, retired warps}; zero between launches
    int lane_lists;             // 1: lane-list mode for large molecules (its instantiation)
    int chunk_planes;           // x-planes per dynamically scheduled chunk (>= 1)
    int chunk_order;            // 0: (molecule, channel) order; 1: channel-major
    int erf_tab;                // floats of per-warp factor table, voxel-integrated form (0: off)
    Geometry geo;
};

// Work counters for dynamically scheduled kernels: a small pool per device, handed out
// round-robin to launches so that launches in flight on different streams do not share one.
constexpr int kSchedSlots = 64;

struct BackwardArgs {
    Inputs in;
    const void *grad_out;
    float *grad_coords;  // [n_atoms][3], or null
    float *grad_weight;  // [n_atoms] dL/dw, or null
    unsigned *err;
    unsigned long long *sched;  // {next atom, retired warps}; zero between launches
    Geometry geo;
};

struct SeparableArgs {
    CUtensorMap out_map;  // TMA view of `out` (pipelined): 3D [n_mol][C nx][ny nz], or 2D
                          // [n_mol C nx][ny nz] rows when molecules are packed
    Inputs in;
    void *out;
    unsigned *err;
    Geometry geo;
    int m_tiles;  // 128-row tiles of the (channel, x) axis per molecule
    int n_tile;   // output columns per tensor-core tile
    int pack;     // pipelined: molecules per 128-row tile when C nx divides 128 (else 0)
    int kslots;   // pipelined: K chunks whose atom tables stay resident per tile (>= 1)
    unsigned long long wait_ns;  // wall-time limit of each bounded mbarrier wait
    int stall;    // test of the bounded waits: stop before the first handoff (0: off)
};

// A fully resolved kernel launch (function, shape, single by-value argument struct), so
// the same description can be launched directly or added to a CUDA graph.
struct KernelLaunch {
    const void *func = nullptr;
    dim3 grid, block;
    size_t smem = 0;
    size_t args_size = 0;
    alignas(64) unsigned char args[2048];
    void *params[1];
};

// Direct per-voxel gather (pg_direct.cu).
// Grid reversal (pg_refine.cu): residual 2 (F - T) in place with per-molecule squared error,
// and the per-atom descent step.
cudaError_t refine_residual(float *F, const float *T, int n_mol, long long per_mol, float *loss,
                            int sm_count, cudaStream_t s);
cudaError_t refine_update(float *coords, const float *grad, const int *mol_off, int n_mol,
                          int n_atoms, const float *loss, int *steps, float lr, float eps,
                          cudaStream_t s);

// The direct kernel's voxel-integrated instantiation for one launch (pg_direct_integral.cu),
// and its weighted instantiations, either voxel form (pg_direct_weighted.cu).
const void *pick_direct_integral(int dtype, bool vec_ok, int cutoff, int periodic, int hint);
const void *pick_direct_weighted(int dtype, bool vec_ok, int cutoff, int periodic, int form);
cudaError_t direct_plan(const DirectArgs &a, int dtype, int vec_ok, const pg_tuning &t,
                        int sm_count, KernelLaunch *kl);

// Coordinate (and weight) adjoint (pg_backward.cu); batches with cells go to the general-cell
// adjoint.
cudaError_t backward_plan(const BackwardArgs &a, int grad_dtype, int sm_count, KernelLaunch *kl);

// General cells (pg_cell.cu): forward over a DirectArgs description (lane_lists unused) and
// the adjoint.  cudaErrorNotSupported for a periodic cell without a cutoff.
cudaError_t cell_plan(const DirectArgs &a, int dtype, int vec_ok, const pg_tuning &t,
                      int sm_count, KernelLaunch *kl);
cudaError_t cell_backward_plan(const BackwardArgs &a, int grad_dtype, int sm_count,
                               KernelLaunch *kl);

// Separable tcgen05 contraction (pg_separable.cu).  Returns cudaErrorNotSupported for
// shapes it does not cover.
cudaError_t separable_plan(const SeparableArgs &a, int dtype, const pg_tuning &t, int sm_count,
                           KernelLaunch *kl);
bool separable_supported(const Geometry &g, int dtype);

// Autotuner helpers (pg_tune.cu): order-independent 64-bit hash of a buffer's bits, and
// the max-abs difference / max-abs reference of two dtype buffers.
cudaError_t buffer_hash(const void *buf, size_t bytes, unsigned long long *d_out,
                        cudaStream_t s);
cudaError_t buffer_compare(const void *a, const void *b, size_t n, int dtype, float *d_out2,
                           cudaStream_t s);

// Validate a direct-path forward call and describe its launch with a caller-supplied
// error word and work counter (no device state of the library is touched).  Sets the
// thread's last-error message on failure; kl->func stays null when there is nothing to run.
pg_status direct_launch_with_scratch(const pg_batch *b, const pg_grid *g, int dtype, void *out,
                                     unsigned *err, unsigned long long *sched, int sm_count,
                                     KernelLaunch *kl);

// Raise kernel `func`'s dynamic shared-memory limit on the current device to at least `smem`
// bytes.  Never lowered: a launch planned earlier with a larger size must still be valid.
cudaError_t raise_smem_limit(const void *func, size_t smem);

// Resident CTAs per SM of kernel `func` at `threads` threads and `smem` bytes of dynamic shared
// memory on the current device, after raising the kernel's dynamic shared-memory limit to
// `smem`.  Cached per (device, kernel, threads, smem): the driver calls cost microseconds,
// which every launch would otherwise pay.
cudaError_t occupancy(const void *func, int threads, size_t smem, int *per_sm);

// Record a failure message for pg_last_error() and return `status`.
pg_status set_last_error(pg_status status, const char *fmt, ...);

// PG_DEBUG_LAUNCH=1 in the environment prints every launch shape to stderr, and a line
// whenever the library allocates its per-device state.
void debug_launch(const KernelLaunch &kl);

inline cudaError_t launch(KernelLaunch &kl, cudaStream_t s)
{
    kl.params[0] = kl.args;
    debug_launch(kl);
    return cudaLaunchKernel(kl.func, kl.grid, kl.block, kl.params, kl.smem, s);
}

template <class A>
inline void set_args(KernelLaunch *kl, const A &a)
{
    static_assert(sizeof(A) <= sizeof(kl->args), "kernel argument struct too large");
    __builtin_memcpy(kl->args, &a, sizeof(A));
    kl->args_size = sizeof(A);
}

}  // namespace pgi
