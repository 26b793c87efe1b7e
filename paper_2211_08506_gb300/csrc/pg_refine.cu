// Grid reversal by gradient descent (Sec. IV-A steps 2-5, Sec. IV-C), the two small kernels
// it adds to the forward and adjoint kernels (sm_103a):
//
//   residual_kernel  per molecule: r = F - T over its voxels, L = sum r^2, F <- 2 r in place
//                    (the adjoint's upstream gradient dL/dF); one CTA per molecule at a time,
//                    fixed-order partial sums and tree, so L is deterministic.
//   update_kernel    per atom: x <- x - lr * dL/dx unless the molecule's L is below eps
//                    (or not finite); the molecule's first atom counts the step.
#include "pg_internal.h"

namespace pgi {

namespace {

constexpr int kResThreads = 256;

__global__ void __launch_bounds__(kResThreads) residual_kernel(float *F, const float *T,
                                                               int n_mol, long long per_mol,
                                                               float *loss)
{
    __shared__ float part[kResThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = blockIdx.x; b < n_mol; b += gridDim.x) {
        float *f = F + (long long)b * per_mol;
        const float *t = T + (long long)b * per_mol;
        float s = 0.0f;
        if (per_mol % 4 == 0 && ((uintptr_t)f % 16) == 0 && ((uintptr_t)t % 16) == 0) {
            float4 *f4 = reinterpret_cast<float4 *>(f);
            const float4 *t4 = reinterpret_cast<const float4 *>(t);
            for (long long i = threadIdx.x; i < per_mol / 4; i += kResThreads) {
                const float4 a = f4[i], c = __ldg(t4 + i);
                const float r0 = a.x - c.x, r1 = a.y - c.y, r2 = a.z - c.z, r3 = a.w - c.w;
                s = fmaf(r0, r0, s);
                s = fmaf(r1, r1, s);
                s = fmaf(r2, r2, s);
                s = fmaf(r3, r3, s);
                f4[i] = make_float4(2.0f * r0, 2.0f * r1, 2.0f * r2, 2.0f * r3);
            }
        } else {
            for (long long i = threadIdx.x; i < per_mol; i += kResThreads) {
                const float r = f[i] - __ldg(t + i);
                s = fmaf(r, r, s);
                f[i] = 2.0f * r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float L = 0.0f;
            for (int w = 0; w < kResThreads / 32; ++w) L += part[w];
            loss[b] = L;
        }
        __syncthreads();
    }
}

__global__ void update_kernel(float *coords, const float *grad, const int *mol_off, int n_mol,
                              int n_atoms, const float *loss, int *steps, float lr, float eps)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_atoms || n_mol <= 0) return;
    // Molecule of atom a: the last b with mol_off[b] <= a; atoms outside [mol_off[0],
    // mol_off[n_mol]) belong to none and stay put.
    if (a < __ldg(mol_off) || a >= __ldg(mol_off + n_mol)) return;
    int lo = 0, hi = n_mol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(mol_off + mid) <= a) lo = mid;
        else hi = mid - 1;
    }
    const float L = loss[lo];
    if (!(L >= eps) || !(L < INFINITY)) return;  // converged, or nothing finite to follow
    coords[3 * a] = fmaf(-lr, grad[3 * a], coords[3 * a]);
    coords[3 * a + 1] = fmaf(-lr, grad[3 * a + 1], coords[3 * a + 1]);
    coords[3 * a + 2] = fmaf(-lr, grad[3 * a + 2], coords[3 * a + 2]);
    if (a == __ldg(mol_off + lo)) steps[lo] += 1;
}

}  // namespace

cudaError_t refine_residual(float *F, const float *T, int n_mol, long long per_mol, float *loss,
                            int sm_count, cudaStream_t s)
{
    if (n_mol <= 0) return cudaSuccess;
    const int blocks = n_mol < 8 * sm_count ? n_mol : 8 * sm_count;
    residual_kernel<<<blocks, kResThreads, 0, s>>>(F, T, n_mol, per_mol, loss);
    return cudaGetLastError();
}

cudaError_t refine_update(float *coords, const float *grad, const int *mol_off, int n_mol,
                          int n_atoms, const float *loss, int *steps, float lr, float eps,
                          cudaStream_t s)
{
    if (n_atoms <= 0) return cudaSuccess;
    update_kernel<<<(n_atoms + 255) / 256, 256, 0, s>>>(coords, grad, mol_off, n_mol, n_atoms,
                                                        loss, steps, lr, eps);
    return cudaGetLastError();
}

}  // namespace pgi
