// Coordinate adjoint of the voxelization (sm_103a).
//
// Sec. IV-C differentiates the MSE between two grids with respect to an atom position
// through the separable voxel function.  Generalised to any upstream gradient
// g = dL/dG and to the point-sampled Gaussian, the derivative of
//     G_c(v) = sum_a chi(d) exp(-|d|^2 / 2 sigma_c^2),   d = v - x_a,
// with respect to x_a is chi(d) exp(-|d|^2 / 2 sigma^2) d / sigma^2, so
//     dL/dx_a = (1/sigma^2) sum_{v : chi} g_{c(a)}(v) exp(-|d|^2 / 2 sigma^2) d.
// (The indicator is piecewise constant; its jump at the cutoff surface is not part of the
// derivative.)  In the voxel-integrated form (Sec. III-A) each term is a product of per-axis
// erf integrals, and the derivative along an axis replaces that axis's factor by its
// derivative (Sec. IV-C's separable-product rule), which is a difference of the Gaussian at
// the voxel's two edges.
//
// With per-atom weights w_a (weighted grids) the coordinate gradient is w_a times the sum
// above, and the weight gradient dL/dw_a is the same sum of g times the atom's unweighted
// terms, without the factor d / sigma^2.
//
// One warp owns one atom at a time (atoms handed out from a per-launch counter) and walks the
// voxels of the atom's cutoff box (clamped to the grid, or wrapped for periodic cells), 32
// voxels per step with z fastest so the reads of g are coalesced.  Each lane keeps a partial sum; a fixed butterfly reduction combines them.  Each
// atom's output is written by exactly one lane, so there are no atomics and the result is
// deterministic.  Reads are ~(2 r_c / h)^3 voxels per atom: this kernel is latency-bound and
// small next to the forward pass.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pg_internal.h"

namespace pgi {

namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float wrap(float d, float L, float invL)
{
    return fmaf(-L, rintf(d * invL), d);
}

template <typename T>
__device__ __forceinline__ float to_float(T v);
template <>
__device__ __forceinline__ float to_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_float<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}

// Support of one axis: first unwrapped index and count of voxels to visit.
template <int CUT, bool PER>
__device__ __forceinline__ void axis_support(float a, float o, float h, int n, float rc,
                                             int &lo, int &cnt)
{
    if (CUT == PG_CUTOFF_NONE) {
        lo = 0;
        cnt = n;
        return;
    }
    // Voxel centres o + (i + 1/2) h within rc of a (rc is already widened by a relative 1e-5,
    // and 1e-3 of a voxel of slack covers the rounding of the bounds themselves).
    const float inv_h = 1.0f / h;
    int l = (int)fmaxf(ceilf((a - rc - o) * inv_h - 0.5f - 1e-3f), -1e8f);
    int u = (int)fminf(floorf((a + rc - o) * inv_h - 0.5f + 1e-3f), 1e8f);
    if (PER) {
        if (u - l + 1 > n) u = l + n - 1;
    } else {
        l = max(l, 0);
        u = min(u, n - 1);
    }
    lo = l;
    cnt = max(u - l + 1, 0);
}

__device__ __forceinline__ int wrap_index(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

template <typename GT, int CUT, bool PER, int FORM>
__global__ void __launch_bounds__(256) backward_kernel(const BackwardArgs A)
{
    const Geometry &G = A.geo;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const GT *gout = reinterpret_cast<const GT *>(A.grad_out);
    // Either output may be absent (null).
    auto put = [&](int a, float gx, float gy, float gz, float gw) {
        if (A.grad_coords) {
            A.grad_coords[3 * a] = gx;
            A.grad_coords[3 * a + 1] = gy;
            A.grad_coords[3 * a + 2] = gz;
        }
        if (A.grad_weight) A.grad_weight[a] = gw;
    };

    // Atoms before the first molecule or after the last one belong to no molecule.
    {
        const int first = G.n_mol > 0 ? __ldg(A.in.mol_off) : 0;
        const int last = G.n_mol > 0 ? __ldg(A.in.mol_off + G.n_mol) : 0;
        for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < G.n_atoms;
             a += gridDim.x * blockDim.x)
            if (G.n_mol == 0 || a < first || a >= last) put(a, 0.0f, 0.0f, 0.0f, 0.0f);
    }

    const long long plane = (long long)G.ny * G.nz;
    const long long grid_elems = (long long)G.nx * plane;
    const unsigned long long total_warps = (unsigned long long)gridDim.x * warps;
    // Atoms of the batch, clamped to the array (bad offsets are flagged per atom below).
    const int first = G.n_mol > 0 ? max(__ldg(A.in.mol_off), 0) : 0;
    const int last = G.n_mol > 0 ? min(__ldg(A.in.mol_off + G.n_mol), G.n_atoms) : 0;
    // Atoms are handed out one per grab from a per-launch counter (the last warp to retire
    // resets it), so molecules of uneven size balance across the GPU.
    while (true) {
        unsigned long long grab = 0;
        if (lane == 0) grab = atomicAdd(A.sched, 1ull);
        grab = __shfl_sync(0xffffffffu, grab, 0);
        const long long ga = (long long)first + (long long)grab;
        if (G.n_mol == 0 || ga >= last) break;
        const int a = (int)ga;
        // Molecule of atom a: the last b with mol_off[b] <= a (offsets are checked below).
        int lo = 0, hi = G.n_mol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(A.in.mol_off + mid) <= a) lo = mid;
            else hi = mid - 1;
        }
        const int b = lo;
        const int a0 = __ldg(A.in.mol_off + b), a1 = __ldg(A.in.mol_off + b + 1);
        const float ox = __ldg(A.in.origin + 3 * b), oy = __ldg(A.in.origin + 3 * b + 1),
                    oz = __ldg(A.in.origin + 3 * b + 2);
        const float hx = __ldg(A.in.spacing + 3 * b), hy = __ldg(A.in.spacing + 3 * b + 1),
                    hz = __ldg(A.in.spacing + 3 * b + 2);
        const bool off_ok = (a0 >= 0) && (a0 <= a) && (a < a1) && (a1 <= G.n_atoms);
        const bool sp_ok = (hx > 0.0f) && (hy > 0.0f) && (hz > 0.0f) && (hx < INFINITY) &&
                           (hy < INFINITY) && (hz < INFINITY);
        const float Lx = G.nx * hx, Ly = G.ny * hy, Lz = G.nz * hz;
        const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
        {
            const int c = __ldg(A.in.elem + a);
            if (!off_ok || (unsigned)c >= (unsigned)G.C || !sp_ok) {
                if (lane == 0) {
                    atomicOr(A.err, !off_ok ? PG_DEVERR_OFFSETS
                                            : (sp_ok ? PG_DEVERR_ELEMENT : PG_DEVERR_SPACING));
                    put(a, 0.0f, 0.0f, 0.0f, 0.0f);
                }
                continue;
            }
            const float ax = __ldg(A.in.coords + 3 * a), ay = __ldg(A.in.coords + 3 * a + 1),
                        az = __ldg(A.in.coords + 3 * a + 2);
            const float q = G.q[c], r2 = G.r2[c], rc = G.rcull[c];
            const float kf = G.kerf[c], kd = G.kdmu[c];
            int ilo, ni, jlo, nj, klo, nk;
            axis_support<CUT, PER>(ax, ox, hx, G.nx, rc, ilo, ni);
            axis_support<CUT, PER>(ay, oy, hy, G.ny, rc, jlo, nj);
            axis_support<CUT, PER>(az, oz, hz, G.nz, rc, klo, nk);
            const GT *g = gout + ((long long)b * G.C + c) * grid_elems;
            // Each lane starts at flat voxel `lane` of the (ni x nj x nk) box, z fastest, and
            // advances 32 voxels per step with carries (no division in the loop).  For periodic
            // cells the box start is first brought into [0, n) so one conditional wrap suffices.
            if (PER) {
                ilo = wrap_index(ilo, G.nx);
                jlo = wrap_index(jlo, G.ny);
                klo = wrap_index(klo, G.nz);
            }
            const int njk = nj * nk;
            const long long total = (long long)ni * njk;
            int fi = 0, fj = 0, fk = 0, si = 0, sj = 0, sk = 0;
            if (total > 0) {
                fi = lane / njk;
                fj = (lane - fi * njk) / nk;
                fk = lane - fi * njk - fj * nk;
                si = 32 / njk;
                sj = (32 - si * njk) / nk;
                sk = 32 - si * njk - sj * nk;
            }
            float sx = 0.0f, sy = 0.0f, sz = 0.0f, sw = 0.0f;
            constexpr int U = 4;  // voxels in flight per lane
            for (long long f0 = lane; f0 < total; f0 += 32 * U) {
                // gv: g times the term (FORM 0); FORM 1 keeps the derivative terms in d*v
                // and g times the term in tv.
                float gv[U], dxv[U], dyv[U], dzv[U], tv[U];
                bool inv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool valid = f0 + 32LL * u < total;
                    int i = ilo + fi, j = jlo + fj, k = klo + fk;
                    if (PER) {
                        if (i >= G.nx) i -= G.nx;
                        if (j >= G.ny) j -= G.ny;
                        if (k >= G.nz) k -= G.nz;
                    }
                    float dx = fmaf((float)i + 0.5f, hx, ox) - ax;
                    float dy = fmaf((float)j + 0.5f, hy, oy) - ay;
                    float dz = fmaf((float)k + 0.5f, hz, oz) - az;
                    if (PER) {
                        dx = wrap(dx, Lx, iLx);
                        dy = wrap(dy, Ly, iLy);
                        dz = wrap(dz, Lz, iLz);
                    }
                    dxv[u] = dx;
                    dyv[u] = dy;
                    dzv[u] = dz;
                    const float dx2 = dx * dx;
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx2));
                    bool in;
                    if (CUT == PG_CUTOFF_SPHERE)
                        in = d2 <= r2;
                    else if (CUT == PG_CUTOFF_BOX)
                        in = fmaxf(dx2, fmaxf(dy * dy, dz * dz)) <= r2;
                    else
                        in = true;
                    inv[u] = valid && in;
                    gv[u] = valid ? to_float<GT>(g[(long long)i * plane + (long long)j * G.nz + k])
                                  : 0.0f;
                    if (FORM == 0) {
                        gv[u] *= inv[u] ? ex2_approx(-q * d2) : 0.0f;
                        tv[u] = gv[u];
                    } else {
                        const float w = inv[u] ? gv[u] : 0.0f;
                        const float fx = erf_axis(dx, hx, kf), fy = erf_axis(dy, hy, kf),
                                    fz = erf_axis(dz, hz, kf);
                        tv[u] = w * fx * fy * fz;
                        dxv[u] = w * erf_axis_dmu(dx, hx, kf, kd) * fy * fz;
                        dyv[u] = w * fx * erf_axis_dmu(dy, hy, kf, kd) * fz;
                        dzv[u] = w * fx * fy * erf_axis_dmu(dz, hz, kf, kd);
                    }
                    // advance this lane by 32 voxels
                    fk += sk;
                    if (fk >= nk) {
                        fk -= nk;
                        ++fj;
                    }
                    fj += sj;
                    if (fj >= nj) {
                        fj -= nj;
                        ++fi;
                    }
                    fi += si;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (FORM == 0) {
                        sx = fmaf(gv[u], dxv[u], sx);
                        sy = fmaf(gv[u], dyv[u], sy);
                        sz = fmaf(gv[u], dzv[u], sz);
                    } else {
                        sx += dxv[u];
                        sy += dyv[u];
                        sz += dzv[u];
                    }
                    sw += tv[u];
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
                sz += __shfl_xor_sync(0xffffffffu, sz, o);
                sw += __shfl_xor_sync(0xffffffffu, sw, o);
            }
            if (lane == 0) {
                const float w = A.in.weight ? __ldg(A.in.weight + a) : 1.0f;
                const float s = w * (FORM == 0 ? G.inv_s2[c] : 1.0f);
                put(a, sx * s, sy * s, sz * s, sw);
            }
        }
    }

    // Retire (see the forward kernel): the last warp resets the counter.
    if (lane == 0) {
        __threadfence();
        const unsigned long long done = atomicAdd(A.sched + 1, 1ull);
        if (done == total_warps - 1) {
            __threadfence();
            atomicExch(A.sched, 0ull);
            atomicExch(A.sched + 1, 0ull);
        }
    }
}

template <typename GT, int FORM>
const void *pick_form(int cutoff, int periodic)
{
    if (periodic) {
        if (cutoff == PG_CUTOFF_SPHERE)
            return (const void *)backward_kernel<GT, PG_CUTOFF_SPHERE, true, FORM>;
        if (cutoff == PG_CUTOFF_BOX)
            return (const void *)backward_kernel<GT, PG_CUTOFF_BOX, true, FORM>;
        return (const void *)backward_kernel<GT, PG_CUTOFF_NONE, true, FORM>;
    }
    if (cutoff == PG_CUTOFF_SPHERE)
        return (const void *)backward_kernel<GT, PG_CUTOFF_SPHERE, false, FORM>;
    if (cutoff == PG_CUTOFF_BOX) return (const void *)backward_kernel<GT, PG_CUTOFF_BOX, false, FORM>;
    return (const void *)backward_kernel<GT, PG_CUTOFF_NONE, false, FORM>;
}

template <typename GT>
const void *pick(int cutoff, int periodic, int form)
{
    return form == PG_FORM_INTEGRAL ? pick_form<GT, 1>(cutoff, periodic)
                                    : pick_form<GT, 0>(cutoff, periodic);
}

}  // namespace

cudaError_t backward_plan(const BackwardArgs &a, int grad_dtype, int sm_count, KernelLaunch *kl)
{
    if (a.in.cell) return cell_backward_plan(a, grad_dtype, sm_count, kl);
    const int cut = a.geo.cutoff, per = a.geo.periodic, form = a.geo.form;
    const void *f = grad_dtype == PG_F32   ? pick<float>(cut, per, form)
                    : grad_dtype == PG_F16 ? pick<__half>(cut, per, form)
                                           : pick<__nv_bfloat16>(cut, per, form);
    const int threads = 256;
    int per_sm = 0;
    cudaError_t e = occupancy(f, threads, 0, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // Persistent grid: atoms come from the work counter; never more warps than atoms.
    long long blocks = (long long)sm_count * per_sm;
    const long long need = ((long long)a.geo.n_atoms + threads / 32 - 1) / (threads / 32);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kl->func = f;
    kl->grid = dim3((unsigned)blocks);
    kl->block = dim3((unsigned)threads);
    kl->smem = 0;
    set_args(kl, a);
    return cudaSuccess;
}

}  // namespace pgi
