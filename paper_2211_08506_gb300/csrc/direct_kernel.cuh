// Direct per-voxel gather for batched Gaussian-density voxelization (sm_103a).
//
// Computes Sec. III-A Eq. 1 in its point-sampled, unnormalised, explicitly truncated form
// (Sec. VI-B): G[b][c][v] = sum_{a in b, elem a = c} chi(d) 2^(-q_c |d|^2), d = v - x_a.
//
// Work decomposition.  The output is a dense [B][C][nx][ny][nz] array and, with ~1% of
// voxels non-zero, writing it is the whole cost: the kernel is a write-bandwidth-bound
// fill with sparse splats.  One work item is one contiguous (y, z) plane of one
// (molecule b, channel c, x index) triple.  Persistent warps take chunks of consecutive
// planes from a per-launch atomic counter, so uneven molecules balance out.
//
// Per item, one warp
//   1. culls the molecule's atoms 32 at a time with a warp ballot: an atom survives if it
//      belongs to channel c and its (nearest-image) x distance to the plane is within the
//      cutoff; survivors are compacted, in atom order, into the warp's shared-memory stage
//      as {dx, y, z};
//   2. walks the plane 32 lanes x VEC voxels at a time (VEC = 16 bytes of output per
//      lane).  For each such row group it ballots the staged atoms against the group's
//      (y, z) bounding box, then every lane adds the survivors' contributions to its VEC
//      voxels, applying the exact cutoff test per voxel;
//   3. stores the VEC values with one 16-byte store per lane (FP32, or FP16/BF16 rounded
//      to nearest even), zeros included.
// Culls are conservative and survivors are visited in atom order, so every voxel sums the
// same terms in the same order whatever the launch shape: results are bitwise identical
// across block sizes, occupancy, store hints and chunk sizes, and equal to the unstaged
// fallback used when an item has more than kStageCap candidates.
//
// Dense planes (kScatterMin or more staged candidates) can instead be accumulated in scatter
// mode (see scatter_plane), in a kernel instantiation of its own.  Scatter mode adds the same
// terms in exact fixed point, so its results differ from the gather's float sums only by the
// rounding of those sums (a few units in the last place of FP32); across launch shapes they are
// again bitwise identical.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pg_internal.h"

namespace pgi {

namespace {

// Staged candidates from which a plane is accumulated in scatter mode instead of gathered.
constexpr int kScatterMin = 6;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Nearest-image displacement on a ring of length L (invL = 1/L).
__device__ __forceinline__ float wrap(float d, float L, float invL)
{
    return fmaf(-L, rintf(d * invL), d);
}

template <typename T>
__device__ __forceinline__ T from_float(float v);
template <>
__device__ __forceinline__ float from_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

template <typename T, int VEC>
__device__ __forceinline__ uint4 pack16(const float (&acc)[VEC]);

template <>
__device__ __forceinline__ uint4 pack16<float, 4>(const float (&a)[4])
{
    return make_uint4(__float_as_uint(a[0]), __float_as_uint(a[1]), __float_as_uint(a[2]),
                      __float_as_uint(a[3]));
}

__device__ __forceinline__ unsigned h2u(__half2 h) { return *reinterpret_cast<unsigned *>(&h); }
__device__ __forceinline__ unsigned b2u(__nv_bfloat162 h)
{
    return *reinterpret_cast<unsigned *>(&h);
}

template <>
__device__ __forceinline__ uint4 pack16<__half, 8>(const float (&a)[8])
{
    return make_uint4(h2u(__floats2half2_rn(a[0], a[1])), h2u(__floats2half2_rn(a[2], a[3])),
                      h2u(__floats2half2_rn(a[4], a[5])), h2u(__floats2half2_rn(a[6], a[7])));
}

template <>
__device__ __forceinline__ uint4 pack16<__nv_bfloat16, 8>(const float (&a)[8])
{
    return make_uint4(b2u(__floats2bfloat162_rn(a[0], a[1])),
                      b2u(__floats2bfloat162_rn(a[2], a[3])),
                      b2u(__floats2bfloat162_rn(a[4], a[5])),
                      b2u(__floats2bfloat162_rn(a[6], a[7])));
}

template <int HINT>
__device__ __forceinline__ void store16(void *p, uint4 v)
{
    if (HINT == 1)
        __stcs(reinterpret_cast<uint4 *>(p), v);
    else
        *reinterpret_cast<uint4 *>(p) = v;
}

// Per-voxel z factor of a term: 2^(-q dz^2) for the point sample (FORM 0), or the voxel's
// erf integral along z (FORM 1, Sec. III-A); zero outside a box cutoff.
template <int CUT, int FORM>
__device__ __forceinline__ float z_factor(float dz, float q, float r2, float kf, float hz)
{
    const float dz2 = dz * dz;
    const float e = FORM ? erf_axis(dz, hz, kf) : ex2_approx(-q * dz2);
    return (CUT == PG_CUTOFF_BOX && dz2 > r2) ? 0.0f : e;
}

// Per-row factor of a term: 2^(-q (dx^2 + dy^2)) for the point sample, or the product of the
// x and y erf integrals (fx passed in, computed once per atom and plane); zero when the row
// is outside a box cutoff.
template <int CUT, int FORM>
__device__ __forceinline__ float row_factor(float fx, float dy, float dx2, float dxy2, float q,
                                            float r2, float kf, float hy)
{
    float e = FORM ? fx * erf_axis(dy, hy, kf) : ex2_approx(-q * dxy2);
    if (CUT == PG_CUTOFF_BOX && fmaxf(dx2, dy * dy) > r2) e = 0.0f;
    return e;
}

// Per-lane accumulation of one atom's contribution into the lane's VEC voxels: each term is
// the product of the atom's row factor (times its weight w, exactly 1 for unweighted grids)
// and the voxel's z factor, under the exact per-voxel cutoff test for a sphere.
template <int VEC, int CUT, bool PER, int FORM>
struct LaneVoxels {
    float vy;        // voxel-centre y of the lane's row
    float vz[VEC];   // voxel-centre z of the lane's voxels
    float acc[VEC];

    __device__ __forceinline__ void add(float dx, float ay, float az, float w, float q, float r2,
                                        float kf, float hx, float hy, float hz, float Ly,
                                        float iLy, float Lz, float iLz)
    {
        float dy = vy - ay;
        if (PER) dy = wrap(dy, Ly, iLy);
        const float dx2 = dx * dx;
        const float dxy2 = fmaf(dy, dy, dx2);
        const float fx = FORM ? erf_axis(dx, hx, kf) : 0.0f;
        const float exy = w * row_factor<CUT, FORM>(fx, dy, dx2, dxy2, q, r2, kf, hy);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            float dz = vz[k] - az;
            if (PER) dz = wrap(dz, Lz, iLz);
            const float ez = z_factor<CUT, FORM>(dz, q, r2, kf, hz);
            if (CUT == PG_CUTOFF_SPHERE)
                acc[k] = (fmaf(dz, dz, dxy2) <= r2) ? fmaf(exy, ez, acc[k]) : acc[k];
            else
                acc[k] = fmaf(exy, ez, acc[k]);
        }
    }
};

// Conservative test: can an atom at (dx, ay, az) reach the box of voxel centres
// [cy +- wy] x [cz +- wz] of the current row group?
template <int CUT, bool PER>
__device__ __forceinline__ bool reaches(float dx, float ay, float az, float cy, float wy,
                                        float cz, float wz, float rc, float Ly, float iLy,
                                        float Lz, float iLz)
{
    if (CUT == PG_CUTOFF_NONE) return true;
    float ey = cy - ay, ez = cz - az;
    if (PER) {
        ey = wrap(ey, Ly, iLy);
        ez = wrap(ez, Lz, iLz);
    }
    const float gy = fmaxf(fabsf(ey) - wy, 0.0f);
    const float gz = fmaxf(fabsf(ez) - wz, 0.0f);
    if (CUT == PG_CUTOFF_SPHERE) return fmaf(dx, dx, fmaf(gy, gy, gz * gz)) <= rc * rc;
    return fmaxf(gy, gz) <= rc;
}

// Zero-fill one plane slice: lanes store 16-byte (or scalar) zeros.
template <typename T, int VEC, int HINT>
__device__ __forceinline__ void zero_plane(T *out, int nvec, int lane)
{
#pragma unroll 4
    for (int v = lane; v < nvec; v += 32) {
        if constexpr (VEC * sizeof(T) == 16)
            store16<HINT>(out + (long long)v * VEC, make_uint4(0u, 0u, 0u, 0u));
        else
            out[v] = from_float<T>(0.0f);
    }
}

template <typename T, int VEC, int HINT>
__device__ __forceinline__ void store_lane(T *out, int v, const float (&acc)[VEC])
{
    if constexpr (VEC * sizeof(T) == 16)
        store16<HINT>(out + (long long)v * VEC, pack16<T, VEC>(acc));
    else
        out[v] = from_float<T>(acc[0]);
}

// Gather of one plane in passes of two lane groups, for planes whose lane columns repeat
// from group to group: with lpr = nz / VEC lanes per row, lane l < act = rpg * lpr owns the
// columns z0 .. z0 + VEC - 1 of rows y0 + l / lpr and y0 + l / lpr + rpg of each pass of
// 2 * rpg rows.  Each surviving atom's z factors are computed once per pass and shared by both
// rows.  for_each(cy, wy, cz, wz, f) calls f(dx, ay, az, w), w the atom's weight, for the
// candidates that can reach the pass's box of voxel centres, in atom order.  Every voxel adds
// the same terms in the same order as LaneVoxels::add does (atoms culled for one of the two rows add exact zeros or are
// skipped by the same test), so both give identical bits.
template <typename T, int VEC, int CUT, bool PER, int HINT, int FORM, typename ForEach>
__device__ __forceinline__ void blocked_plane(T *out, int ny, int nz, int rpg, int act,
                                              int my_row, int z0, int lane, float q, float r2,
                                              float kf, float hx, float oy, float oz, float hy,
                                              float hz, float Ly, float iLy, float Lz, float iLz,
                                              ForEach for_each)
{
    float vz[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) vz[k] = fmaf((float)(z0 + k) + 0.5f, hz, oz);
    const float cz = fmaf(0.5f * (float)(nz - 1) + 0.5f, hz, oz);
    const float wz = 0.5f * (float)(nz - 1) * hz;
    for (int y0 = 0; y0 < ny; y0 += 2 * rpg) {
        const int y_end = min(y0 + 2 * rpg, ny) - 1;
        const float cy = fmaf(0.5f * (float)(y0 + y_end) + 0.5f, hy, oy);
        const float wy = 0.5f * (float)(y_end - y0) * hy;
        const int ya = y0 + my_row, yb = ya + rpg;
        const float vya = fmaf((float)ya + 0.5f, hy, oy);
        const float vyb = fmaf((float)yb + 0.5f, hy, oy);
        float acc0[VEC], acc1[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc0[k] = acc1[k] = 0.0f;
        for_each(cy, wy, cz, wz, [&](float dx, float ay, float az, float w) {
            const float dx2 = dx * dx;
            float dya = vya - ay, dyb = vyb - ay;
            if (PER) {
                dya = wrap(dya, Ly, iLy);
                dyb = wrap(dyb, Ly, iLy);
            }
            const float dxya = fmaf(dya, dya, dx2), dxyb = fmaf(dyb, dyb, dx2);
            const float fx = FORM ? erf_axis(dx, hx, kf) : 0.0f;
            const float ea = w * row_factor<CUT, FORM>(fx, dya, dx2, dxya, q, r2, kf, hy);
            const float eb = w * row_factor<CUT, FORM>(fx, dyb, dx2, dxyb, q, r2, kf, hy);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                float dz = vz[k] - az;
                if (PER) dz = wrap(dz, Lz, iLz);
                const float ez = z_factor<CUT, FORM>(dz, q, r2, kf, hz);
                if (CUT == PG_CUTOFF_SPHERE) {
                    acc0[k] = (fmaf(dz, dz, dxya) <= r2) ? fmaf(ea, ez, acc0[k]) : acc0[k];
                    acc1[k] = (fmaf(dz, dz, dxyb) <= r2) ? fmaf(eb, ez, acc1[k]) : acc1[k];
                } else {
                    acc0[k] = fmaf(ea, ez, acc0[k]);
                    acc1[k] = fmaf(eb, ez, acc1[k]);
                }
            }
        });
        if (lane < act) {
            if (ya < ny) store_lane<T, VEC, HINT>(out, (ya * nz + z0) / VEC, acc0);
            if (yb < ny) store_lane<T, VEC, HINT>(out, (yb * nz + z0) / VEC, acc1);
        }
    }
}

__device__ __forceinline__ int wrap_index(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Index range [lo, hi] of voxel centres o + (i+1/2)h within rho of a (widened by one voxel
// each side): clamped to the grid, or for periodic cells at most n consecutive (unwrapped)
// indices so that no voxel is visited twice.
template <bool PER>
__device__ __forceinline__ void disc_range(float a, float rho, float o, float inv_h, int n,
                                           int &lo, int &hi)
{
    lo = (int)fmaxf(floorf((a - rho - o) * inv_h - 0.5f), -1e8f) - 1;
    hi = (int)fminf(ceilf((a + rho - o) * inv_h - 0.5f), 1e8f) + 1;
    if (PER) {
        if (hi - lo + 1 > n) hi = lo + n - 1;
    } else {
        lo = max(lo, 0);
        hi = min(hi, n - 1);
    }
}

// Scatter mode for dense planes (Sec. VI-A visits each atom's non-zero box; here the box is cut
// down to the exact disc row by row).  Work unit: one "run", the voxels of one row of one
// candidate's disc in this plane.  The runs of all candidates are numbered consecutively
// (per-candidate row counts, prefix-summed across the warp), and lane i takes runs i, i+32, ...
// so lanes stay busy however many rows a disc has.  For its run a lane finds the exact z span
// of the disc in that row and adds each in-cutoff term to the warp's plane accumulator with a
// shared-memory integer atomic.  The accumulator is fixed point, scaled so that a voxel's sum
// of at most `count` terms (each <= 1) stays below 2^30: integer addition is exact and
// associative, so the result does not depend on the order in which lanes and runs land, and
// every term is the same ex2 of the same d^2 as in the gather mode.
template <typename T, int VEC, int CUT, bool PER, int HINT>
__device__ __forceinline__ void scatter_plane(T *out, int *acc_i, int *run_off, int *run_ylo,
                                              const float4 *stage, int count, int ny, int nz,
                                              int lane, float q, float r2, float rc, float oy,
                                              float oz, float hy, float hz, float Ly, float iLy,
                                              float Lz, float iLz)
{
    const int nvec = ny * nz / VEC;
    const float inv_hy = 1.0f / hy, inv_hz = 1.0f / hz;
    // count < 2^bits, so a voxel's scaled sum is below 2^30.
    const int bits = 32 - __clz(count);
    const float scale = __int_as_float((127 + 30 - bits) << 23);
    const float inv_scale = __int_as_float((127 - 30 + bits) << 23);

    // 1. Row range of each candidate's disc, and the prefix offsets of its runs.
    int total = 0;
    for (int cb = 0; cb < count; cb += 32) {
        const int j = cb + lane;
        int nrows = 0, ylo = 0;
        if (j < count) {
            const float4 st = stage[j];
            float rho = rc;
            if (CUT == PG_CUTOFF_SPHERE) rho = sqrtf(fmaxf(fmaf(-st.x, st.x, rc * rc), 0.0f));
            int lo, hi;
            disc_range<PER>(st.y, rho, oy, inv_hy, ny, lo, hi);
            nrows = max(hi - lo + 1, 0);
            ylo = PER ? wrap_index(lo, ny) : lo;
        }
        int incl = nrows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (j < count) {
            run_off[j] = total + incl - nrows;
            run_ylo[j] = ylo;
        }
        total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) run_off[count] = total;
    __syncwarp();

    // 2. Runs.
    int j = 0;
    for (int u = lane; u < total; u += 32) {
        while (run_off[j + 1] <= u) ++j;
        const float4 st = stage[j];
        const float dx = st.x, ay = st.y, az = st.z;
        const float dx2 = dx * dx;
        int y = run_ylo[j] + (u - run_off[j]);
        if (PER && y >= ny) y -= ny;
        float dy = fmaf((float)y + 0.5f, hy, oy) - ay;
        if (PER) dy = wrap(dy, Ly, iLy);
        const float dy2 = dy * dy;
        const float dxy2 = fmaf(dy, dy, dx2);
        float w = rc;
        if (CUT == PG_CUTOFF_SPHERE) {
            const float rem = fmaf(rc, rc, -dxy2);
            if (rem < 0.0f) continue;
            w = sqrtf(rem);
        } else if (fmaxf(dx2, dy2) > r2) {
            continue;
        }
        int zlo, zhi;
        disc_range<PER>(az, w, oz, inv_hz, nz, zlo, zhi);
        int *row = acc_i + y * nz;
        int z = PER ? wrap_index(zlo, nz) : zlo;
        const float exy = ex2_approx(-q * dxy2);
        // Fixed-point term of voxel zz of this run (0 when outside the cutoff): the product
        // of the same row and z factors, under the same test, as the gather mode adds.
        auto term = [&](int zz) -> int {
            float dz = fmaf((float)zz + 0.5f, hz, oz) - az;
            if (PER) dz = wrap(dz, Lz, iLz);
            if (CUT == PG_CUTOFF_SPHERE && fmaf(dz, dz, dxy2) > r2) return 0;
            return __float2int_rn(exy * z_factor<CUT, 0>(dz, q, r2, 0.0f, hz) * scale);
        };
        int k = zhi - zlo + 1;
        // Four voxels at a time: independent terms first, then their atomics.
        for (; k >= 4; k -= 4) {
            int zz[4], tv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                zz[i] = z + i;
                if (PER && zz[i] >= nz) zz[i] -= nz;
                tv[i] = term(zz[i]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (tv[i]) atomicAdd(row + zz[i], tv[i]);
            z += 4;
            if (PER && z >= nz) z -= nz;
        }
        for (; k > 0; --k) {
            const int tv = term(z);
            if (tv) atomicAdd(row + z, tv);
            ++z;
            if (PER && z >= nz) z -= nz;
        }
    }
    __syncwarp();

    // 3. Convert, store, and leave the accumulator zeroed for the next plane.
    for (int v = lane; v < nvec; v += 32) {
        float a[VEC];
        if constexpr (VEC % 4 == 0) {
#pragma unroll
            for (int k = 0; k < VEC; k += 4) {
                int4 *p = reinterpret_cast<int4 *>(acc_i + v * VEC) + k / 4;
                const int4 w = *p;
                *p = make_int4(0, 0, 0, 0);
                a[k] = (float)w.x * inv_scale;
                a[k + 1] = (float)w.y * inv_scale;
                a[k + 2] = (float)w.z * inv_scale;
                a[k + 3] = (float)w.w * inv_scale;
            }
        } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                a[k] = (float)acc_i[v * VEC + k] * inv_scale;
                acc_i[v * VEC + k] = 0;
            }
        }
        store_lane<T, VEC, HINT>(out, v, a);
    }
    __syncwarp();
}

// WGT: per-atom weights (weighted grids).  Unweighted batches run the instantiation without
// them, which carries no weight loads, shuffles or multiplies.
template <typename T, int VEC, int CUT, bool PER, int HINT, bool SCAT, int FORM, bool WGT>
__global__ void __launch_bounds__(512, (SCAT || VEC == 8) ? 1 : 2) direct_kernel(const DirectArgs A)
{
    extern __shared__ float4 smem_all[];
    const Geometry &G = A.geo;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps_per_block = blockDim.x >> 5;
    // Per warp (layout in direct_warp_floats): the plane's staged candidates, the chunk's
    // channel atoms, then in scatter mode the plane accumulator and the run bookkeeping.
    float4 *stage = smem_all + (size_t)warp * (direct_warp_floats(A.plane_stride) / 4);
    float4 *chan = stage + kStageCap;
    int *acc_i = reinterpret_cast<int *>(chan + kChanCap);
    int *run_off = acc_i + A.plane_stride;
    int *run_ylo = run_off + kStageCap + 4;
    if (SCAT) {  // the scatter accumulator starts zeroed and each plane leaves it so
        for (int i = lane; i < A.plane_stride; i += 32) acc_i[i] = 0;
        __syncwarp();
    }
    const unsigned lt_mask = (1u << lane) - 1u;

    // Work is handed out dynamically in chunks of up to chunk_planes consecutive x-planes of
    // one (molecule, channel) grid: lane 0 takes the next chunk index from a per-launch
    // counter.  The molecule's header and, for molecules of at most 32 atoms, the atoms
    // themselves stay in registers across the chunk's planes (and across chunks of the same
    // molecule).  The last warp to finish resets the counter for the next launch.
    const int chunk_planes = A.chunk_planes;
    const int x_chunks = (G.nx + chunk_planes - 1) / chunk_planes;
    const unsigned long long n_chunks = (unsigned long long)G.n_mol * G.C * x_chunks;
    const unsigned long long total_warps = (unsigned long long)gridDim.x * warps_per_block;

    const int plane = G.ny * G.nz;
    const int nvec = plane / VEC;
    const int y_start = (lane * VEC) / G.nz, z_start = (lane * VEC) % G.nz;
    const int y_step = (32 * VEC) / G.nz, z_step = (32 * VEC) % G.nz;
    // Two-group passes (blocked_plane) when whole rows fill at least 28 of the 32 lanes.
    const int lpr = G.nz / VEC;
    const int rpg = (lpr >= 1 && lpr <= 32) ? 32 / lpr : 0;
    const int act = rpg * lpr;
    const bool blocked = act >= 28;
    const int my_row = blocked ? lane / lpr : 0;
    const int my_z0 = blocked ? (lane - my_row * lpr) * VEC : 0;

    int cur_b = -1;
    int a0 = 0, a1 = 0;
    float ox = 0.f, oy = 0.f, oz = 0.f, hx = 1.f, hy = 1.f, hz = 1.f;
    float Lx = 1.f, Ly = 1.f, Lz = 1.f, iLx = 1.f, iLy = 1.f, iLz = 1.f;
    bool small = true;
    // Lane-held atom of a small molecule (lane < a1 - a0).
    float my_x = 0.f, my_y = 0.f, my_z = 0.f, my_w = 1.f;
    int my_e = -1;

    while (true) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(A.sched, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= n_chunks) break;
        // Chunk order 0 walks (molecule, channel) in memory order, so concurrent stores stay
        // close together; order 1 runs channel-major (channel 0 of every molecule first),
        // which hands out the largest chunks first when channels are listed by decreasing
        // atom frequency.  The output item is (molecule, channel, x) either way.
        const unsigned long long grid_q = chunk / (unsigned)x_chunks;
        const int xc = (int)(chunk - grid_q * x_chunks);
        int b, c;
        if (A.chunk_order) {
            c = (int)(grid_q / (unsigned)G.n_mol);
            b = (int)(grid_q - (unsigned long long)c * G.n_mol);
        } else {
            b = (int)(grid_q / (unsigned)G.C);
            c = (int)(grid_q - (unsigned long long)b * G.C);
        }
        const unsigned long long bc = (unsigned long long)b * G.C + c;
        const int x_begin = xc * chunk_planes;
        const int x_end = min(G.nx, x_begin + chunk_planes);
        if (b != cur_b) {
            cur_b = b;
            a0 = __ldg(A.in.mol_off + b);
            a1 = __ldg(A.in.mol_off + b + 1);
            ox = __ldg(A.in.origin + 3 * b);
            oy = __ldg(A.in.origin + 3 * b + 1);
            oz = __ldg(A.in.origin + 3 * b + 2);
            hx = __ldg(A.in.spacing + 3 * b);
            hy = __ldg(A.in.spacing + 3 * b + 1);
            hz = __ldg(A.in.spacing + 3 * b + 2);
            const bool off_ok = (a0 >= 0) && (a0 <= a1) && (a1 <= G.n_atoms);
            const bool sp_ok = (hx > 0.0f) && (hy > 0.0f) && (hz > 0.0f) && (hx < INFINITY) &&
                               (hy < INFINITY) && (hz < INFINITY);
            if (!off_ok || !sp_ok) {
                if (lane == 0)
                    atomicOr(A.err, (off_ok ? 0u : PG_DEVERR_OFFSETS) |
                                        (sp_ok ? 0u : PG_DEVERR_SPACING));
                a0 = a1 = 0;
            }
            Lx = G.nx * hx;
            Ly = G.ny * hy;
            Lz = G.nz * hz;
            iLx = 1.0f / Lx;
            iLy = 1.0f / Ly;
            iLz = 1.0f / Lz;
            small = (a1 - a0) <= 32;
            my_e = -1;
            bool bad = false;
            if (small && a0 + lane < a1) {
                const int ai = a0 + lane;
                my_e = __ldg(A.in.elem + ai);
                if (WGT) my_w = __ldg(A.in.weight + ai);
                my_x = __ldg(A.in.coords + 3 * ai);
                my_y = __ldg(A.in.coords + 3 * ai + 1);
                my_z = __ldg(A.in.coords + 3 * ai + 2);
                if ((unsigned)my_e >= (unsigned)G.C) {
                    bad = true;
                    my_e = -1;
                }
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(A.err, PG_DEVERR_ELEMENT);
        }
        // Large molecule: this channel's atoms, in atom order, staged in shared memory once
        // per chunk when they fit, so that each plane culls them from there.
        int n_chan = -1;
        if (!small) {
            int cnt = 0;
            // 64 atoms per step, all loads issued before any is used.
            for (int base = a0; base < a1; base += 64) {
                int e[2];
                float ax[2], ay[2], az[2], aw[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ai = base + 32 * h + lane;
                    e[h] = -1;
                    ax[h] = ay[h] = az[h] = 0.0f;
                    aw[h] = 1.0f;
                    if (ai < a1) {
                        e[h] = __ldg(A.in.elem + ai);
                        if (WGT) aw[h] = __ldg(A.in.weight + ai);
                        ax[h] = __ldg(A.in.coords + 3 * ai);
                        ay[h] = __ldg(A.in.coords + 3 * ai + 1);
                        az[h] = __ldg(A.in.coords + 3 * ai + 2);
                        if ((unsigned)e[h] >= (unsigned)G.C && c == 0 && x_begin == 0)
                            atomicOr(A.err, PG_DEVERR_ELEMENT);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool ok = e[h] == c;
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) {
                        const int pos = cnt + __popc(m & lt_mask);
                        if (pos < kChanCap) chan[pos] = make_float4(ax[h], ay[h], az[h], aw[h]);
                    }
                    cnt += __popc(m);
                }
            }
            __syncwarp();
            n_chan = cnt <= kChanCap ? cnt : -1;
        }
        for (int x = x_begin; x < x_end; ++x) {
            const long long item = (long long)bc * G.nx + x;
            T *out = reinterpret_cast<T *>(A.out) + item * (long long)plane;
            const float q = G.q[c], r2 = G.r2[c], rc = G.rcull[c], kf = G.kerf[c];
            if (PER && CUT != PG_CUTOFF_NONE && lane == 0 && x == 0 && a1 > a0 &&
                (2.0f * rc >= fminf(Lx, fminf(Ly, Lz))))
                atomicOr(A.err, PG_DEVERR_PERIODIC);
            const float vx = fmaf((float)x + 0.5f, hx, ox);

            if (small) {
                // Candidates of this plane: the lane's own atom if it has channel c and lies
                // within the cutoff of the plane in x.
                float dx = vx - my_x;
                if (PER) dx = wrap(dx, Lx, iLx);
                const bool cand = (my_e == c) && ((CUT == PG_CUTOFF_NONE) || (fabsf(dx) <= rc));
                const unsigned cmask = __ballot_sync(0xffffffffu, cand);
                if (cmask == 0u) {
                    zero_plane<T, VEC, HINT>(out, nvec, lane);
                } else if (blocked) {
                    blocked_plane<T, VEC, CUT, PER, HINT, FORM>(
                        out, G.ny, G.nz, rpg, act, my_row, my_z0, lane, q, r2, kf, hx, oy, oz, hy,
                        hz, Ly, iLy, Lz, iLz, [&](float cy, float wy, float cz, float wz, auto &&f) {
                            const bool hit = cand && reaches<CUT, PER>(dx, my_y, my_z, cy, wy, cz,
                                                                       wz, rc, Ly, iLy, Lz, iLz);
                            unsigned m = __ballot_sync(0xffffffffu, hit);
                            while (m) {
                                const int src = __ffs(m) - 1;
                                m &= m - 1;
                                f(__shfl_sync(0xffffffffu, dx, src),
                                  __shfl_sync(0xffffffffu, my_y, src),
                                  __shfl_sync(0xffffffffu, my_z, src),
                                  WGT ? __shfl_sync(0xffffffffu, my_w, src) : 1.0f);
                            }
                        });
                } else {
                    int y = y_start, z0 = z_start;
                    for (int g = 0; g < nvec; g += 32) {
                        const int last = min(31, nvec - 1 - g);
                        const int y_lo = __shfl_sync(0xffffffffu, y, 0);
                        const int y_hi = __shfl_sync(0xffffffffu, y, last);
                        int z_lo = 0, z_hi = G.nz - 1;
                        if (y_lo == y_hi) {
                            z_lo = __shfl_sync(0xffffffffu, z0, 0);
                            z_hi = __shfl_sync(0xffffffffu, z0, last) + VEC - 1;
                        }
                        const float cy = fmaf(0.5f * (float)(y_lo + y_hi) + 0.5f, hy, oy);
                        const float wy = 0.5f * (float)(y_hi - y_lo) * hy;
                        const float cz = fmaf(0.5f * (float)(z_lo + z_hi) + 0.5f, hz, oz);
                        const float wz = 0.5f * (float)(z_hi - z_lo) * hz;
                        const bool hit = cand && reaches<CUT, PER>(dx, my_y, my_z, cy, wy, cz, wz,
                                                                   rc, Ly, iLy, Lz, iLz);
                        unsigned m = __ballot_sync(0xffffffffu, hit);
                        LaneVoxels<VEC, CUT, PER, FORM> lv;
    #pragma unroll
                        for (int k = 0; k < VEC; ++k) lv.acc[k] = 0.0f;
                        if (m) {
                            lv.vy = fmaf((float)y + 0.5f, hy, oy);
    #pragma unroll
                            for (int k = 0; k < VEC; ++k)
                                lv.vz[k] = fmaf((float)(z0 + k) + 0.5f, hz, oz);
                            while (m) {
                                const int src = __ffs(m) - 1;
                                m &= m - 1;
                                const float sdx = __shfl_sync(0xffffffffu, dx, src);
                                const float sy = __shfl_sync(0xffffffffu, my_y, src);
                                const float sz = __shfl_sync(0xffffffffu, my_z, src);
                                const float sw = WGT ? __shfl_sync(0xffffffffu, my_w, src) : 1.0f;
                                lv.add(sdx, sy, sz, sw, q, r2, kf, hx, hy, hz, Ly, iLy, Lz,
                                       iLz);
                            }
                        }
                        if (g + lane < nvec) store_lane<T, VEC, HINT>(out, g + lane, lv.acc);
                        y += y_step;
                        z0 += z_step;
                        if (z0 >= G.nz) {
                            z0 -= G.nz;
                            ++y;
                        }
                    }
                }
            } else {
                // Large molecule: cull and stage this channel's atoms near the plane, in order,
                // from the chunk's channel list, or else from global memory.
                int count = 0;
                for (int cb = 0; cb < n_chan; cb += 32) {
                    const int j = cb + lane;
                    bool ok = false;
                    float dx = 0.0f, ay = 0.0f, az = 0.0f, aw = 1.0f;
                    if (j < n_chan) {
                        const float4 a = chan[j];
                        ay = a.y;
                        az = a.z;
                        if (WGT) aw = a.w;
                        dx = vx - a.x;
                        if (PER) dx = wrap(dx, Lx, iLx);
                        ok = (CUT == PG_CUTOFF_NONE) || (fabsf(dx) <= rc);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) stage[count + __popc(m & lt_mask)] = make_float4(dx, ay, az, aw);
                    count += __popc(m);
                }
                for (int base = n_chan >= 0 ? a1 : a0; base < a1; base += 32) {
                    const int ai = base + lane;
                    bool ok = false;
                    float dx = 0.0f, ay = 0.0f, az = 0.0f, aw = 1.0f;
                    if (ai < a1) {
                        // Loads issued together, used after.
                        const int e = __ldg(A.in.elem + ai);
                        if (WGT) aw = __ldg(A.in.weight + ai);
                        const float ax = __ldg(A.in.coords + 3 * ai);
                        ay = __ldg(A.in.coords + 3 * ai + 1);
                        az = __ldg(A.in.coords + 3 * ai + 2);
                        if ((unsigned)e >= (unsigned)G.C) {
                            if (c == 0 && x == 0) atomicOr(A.err, PG_DEVERR_ELEMENT);
                        } else if (e == c) {
                            dx = vx - ax;
                            if (PER) dx = wrap(dx, Lx, iLx);
                            ok = (CUT == PG_CUTOFF_NONE) || (fabsf(dx) <= rc);
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) {
                        const int pos = count + __popc(m & lt_mask);
                        if (pos < kStageCap) stage[pos] = make_float4(dx, ay, az, aw);
                    }
                    count += __popc(m);
                }
                __syncwarp();
                if (count == 0) {
                    zero_plane<T, VEC, HINT>(out, nvec, lane);
                } else if (SCAT && count >= kScatterMin && count <= kStageCap) {
                    scatter_plane<T, VEC, CUT, PER, HINT>(out, acc_i, run_off, run_ylo, stage,
                                                         count, G.ny, G.nz, lane, q, r2, rc, oy,
                                                         oz, hy, hz, Ly, iLy, Lz, iLz);
                } else if (blocked && count <= kStageCap) {
                    blocked_plane<T, VEC, CUT, PER, HINT, FORM>(
                        out, G.ny, G.nz, rpg, act, my_row, my_z0, lane, q, r2, kf, hx, oy, oz, hy,
                        hz, Ly, iLy, Lz, iLz, [&](float cy, float wy, float cz, float wz, auto &&f) {
                            for (int cb = 0; cb < count; cb += 32) {
                                const int j = cb + lane;
                                bool ok = false;
                                if (j < count) {
                                    const float4 st = stage[j];
                                    ok = reaches<CUT, PER>(st.x, st.y, st.z, cy, wy, cz, wz, rc, Ly,
                                                           iLy, Lz, iLz);
                                }
                                unsigned m = __ballot_sync(0xffffffffu, ok);
                                while (m) {
                                    const int src = __ffs(m) - 1;
                                    m &= m - 1;
                                    const float4 st = stage[cb + src];
                                    f(st.x, st.y, st.z, WGT ? st.w : 1.0f);
                                }
                            }
                        });
                } else {
                    int y = y_start, z0 = z_start;
                    for (int g = 0; g < nvec; g += 32) {
                        const int v = g + lane;
                        LaneVoxels<VEC, CUT, PER, FORM> lv;
    #pragma unroll
                        for (int k = 0; k < VEC; ++k) lv.acc[k] = 0.0f;
                        const int last = min(31, nvec - 1 - g);
                        const int y_lo = __shfl_sync(0xffffffffu, y, 0);
                        const int y_hi = __shfl_sync(0xffffffffu, y, last);
                        int z_lo = 0, z_hi = G.nz - 1;
                        if (y_lo == y_hi) {
                            z_lo = __shfl_sync(0xffffffffu, z0, 0);
                            z_hi = __shfl_sync(0xffffffffu, z0, last) + VEC - 1;
                        }
                        const float cy = fmaf(0.5f * (float)(y_lo + y_hi) + 0.5f, hy, oy);
                        const float wy = 0.5f * (float)(y_hi - y_lo) * hy;
                        const float cz = fmaf(0.5f * (float)(z_lo + z_hi) + 0.5f, hz, oz);
                        const float wz = 0.5f * (float)(z_hi - z_lo) * hz;
                        lv.vy = fmaf((float)y + 0.5f, hy, oy);
    #pragma unroll
                        for (int k = 0; k < VEC; ++k) lv.vz[k] = fmaf((float)(z0 + k) + 0.5f, hz, oz);

                        if (count <= kStageCap) {
                            for (int cb = 0; cb < count; cb += 32) {
                                const int j = cb + lane;
                                bool ok = false;
                                if (j < count) {
                                    const float4 st = stage[j];
                                    ok = reaches<CUT, PER>(st.x, st.y, st.z, cy, wy, cz, wz, rc, Ly,
                                                           iLy, Lz, iLz);
                                }
                                unsigned m = __ballot_sync(0xffffffffu, ok);
                                while (m) {
                                    const int src = __ffs(m) - 1;
                                    m &= m - 1;
                                    const float4 st = stage[cb + src];
                                    lv.add(st.x, st.y, st.z, WGT ? st.w : 1.0f, q, r2, kf, hx, hy,
                                           hz, Ly, iLy, Lz, iLz);
                                }
                            }
                        } else {
                            // Unstaged fallback: the same atoms in the same order, from global.
                            for (int base = a0; base < a1; base += 32) {
                                const int ai = base + lane;
                                bool ok = false;
                                float dx = 0.0f, ay = 0.0f, az = 0.0f, aw = 1.0f;
                                if (ai < a1 && __ldg(A.in.elem + ai) == c) {
                                    if (WGT) aw = __ldg(A.in.weight + ai);
                                    const float ax = __ldg(A.in.coords + 3 * ai);
                                    ay = __ldg(A.in.coords + 3 * ai + 1);
                                    az = __ldg(A.in.coords + 3 * ai + 2);
                                    dx = vx - ax;
                                    if (PER) dx = wrap(dx, Lx, iLx);
                                    ok = ((CUT == PG_CUTOFF_NONE) || (fabsf(dx) <= rc)) &&
                                         reaches<CUT, PER>(dx, ay, az, cy, wy, cz, wz, rc, Ly, iLy,
                                                           Lz, iLz);
                                }
                                unsigned m = __ballot_sync(0xffffffffu, ok);
                                while (m) {
                                    const int src = __ffs(m) - 1;
                                    m &= m - 1;
                                    const float sdx = __shfl_sync(0xffffffffu, dx, src);
                                    const float sy = __shfl_sync(0xffffffffu, ay, src);
                                    const float sz = __shfl_sync(0xffffffffu, az, src);
                                    const float sw = WGT ? __shfl_sync(0xffffffffu, aw, src) : 1.0f;
                                    lv.add(sdx, sy, sz, sw, q, r2, kf, hx, hy, hz, Ly, iLy, Lz,
                                           iLz);
                                }
                            }
                        }
                        if (v < nvec) store_lane<T, VEC, HINT>(out, v, lv.acc);
                        y += y_step;
                        z0 += z_step;
                        if (z0 >= G.nz) {
                            z0 -= G.nz;
                            ++y;
                        }
                    }
                }
                __syncwarp();
            }

        }  // planes of the chunk
    }

    // Retire: the final failed grab above is ordered before this arrival, so when the last
    // warp arrives no other warp touches the counter again and it can be reset.
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

// Scatter-capable instantiations (SCAT) exist only for the point form and where a cutoff
// bounds each atom's disc; the gather-only ones carry no scatter code and so keep their
// register allocation.
template <typename T, int VEC, int CUT, bool PER, int HINT, int FORM>
const void *pick_scat(bool scat)
{
    if constexpr (CUT != PG_CUTOFF_NONE && FORM == 0)
        if (scat) return (const void *)direct_kernel<T, VEC, CUT, PER, HINT, true, FORM, false>;
    return (const void *)direct_kernel<T, VEC, CUT, PER, HINT, false, FORM, false>;
}

template <typename T, int VEC, int CUT, bool PER, int FORM>
const void *pick_hint(int hint, bool scat)
{
    return hint == 1 ? pick_scat<T, VEC, CUT, PER, 1, FORM>(scat)
                     : pick_scat<T, VEC, CUT, PER, 0, FORM>(scat);
}

template <typename T, int VEC, int FORM>
const void *pick_shape(int cutoff, int periodic, int hint, bool scat)
{
    if (periodic) {
        if (cutoff == PG_CUTOFF_SPHERE)
            return pick_hint<T, VEC, PG_CUTOFF_SPHERE, true, FORM>(hint, scat);
        if (cutoff == PG_CUTOFF_BOX) return pick_hint<T, VEC, PG_CUTOFF_BOX, true, FORM>(hint, scat);
        return pick_hint<T, VEC, PG_CUTOFF_NONE, true, FORM>(hint, scat);
    }
    if (cutoff == PG_CUTOFF_SPHERE)
        return pick_hint<T, VEC, PG_CUTOFF_SPHERE, false, FORM>(hint, scat);
    if (cutoff == PG_CUTOFF_BOX) return pick_hint<T, VEC, PG_CUTOFF_BOX, false, FORM>(hint, scat);
    return pick_hint<T, VEC, PG_CUTOFF_NONE, false, FORM>(hint, scat);
}

// Weighted instantiations: gather mode (scatter mode assumes unit terms) and default stores.
template <typename T, int VEC, int FORM>
const void *pick_weighted_shape(int cutoff, int periodic)
{
    if (periodic) {
        if (cutoff == PG_CUTOFF_SPHERE)
            return (const void *)direct_kernel<T, VEC, PG_CUTOFF_SPHERE, true, 0, false, FORM, true>;
        if (cutoff == PG_CUTOFF_BOX)
            return (const void *)direct_kernel<T, VEC, PG_CUTOFF_BOX, true, 0, false, FORM, true>;
        return (const void *)direct_kernel<T, VEC, PG_CUTOFF_NONE, true, 0, false, FORM, true>;
    }
    if (cutoff == PG_CUTOFF_SPHERE)
        return (const void *)direct_kernel<T, VEC, PG_CUTOFF_SPHERE, false, 0, false, FORM, true>;
    if (cutoff == PG_CUTOFF_BOX)
        return (const void *)direct_kernel<T, VEC, PG_CUTOFF_BOX, false, 0, false, FORM, true>;
    return (const void *)direct_kernel<T, VEC, PG_CUTOFF_NONE, false, 0, false, FORM, true>;
}

template <int FORM>
const void *pick_weighted(int dtype, bool vec_ok, int cut, int per)
{
    if (dtype == PG_F32)
        return vec_ok ? pick_weighted_shape<float, 4, FORM>(cut, per)
                      : pick_weighted_shape<float, 1, FORM>(cut, per);
    if (dtype == PG_F16)
        return vec_ok ? pick_weighted_shape<__half, 8, FORM>(cut, per)
                      : pick_weighted_shape<__half, 1, FORM>(cut, per);
    return vec_ok ? pick_weighted_shape<__nv_bfloat16, 8, FORM>(cut, per)
                  : pick_weighted_shape<__nv_bfloat16, 1, FORM>(cut, per);
}

// The instantiation for one launch: dtype, vector stores, cutoff, boundary, store hint,
// scatter mode and voxel form.
template <int FORM>
const void *pick_direct(int dtype, bool vec_ok, int cut, int per, int hint, bool scat)
{
    if (dtype == PG_F32)
        return vec_ok ? pick_shape<float, 4, FORM>(cut, per, hint, scat)
                      : pick_shape<float, 1, FORM>(cut, per, hint, scat);
    if (dtype == PG_F16)
        return vec_ok ? pick_shape<__half, 8, FORM>(cut, per, hint, scat)
                      : pick_shape<__half, 1, FORM>(cut, per, hint, scat);
    return vec_ok ? pick_shape<__nv_bfloat16, 8, FORM>(cut, per, hint, scat)
                  : pick_shape<__nv_bfloat16, 1, FORM>(cut, per, hint, scat);
}

}  // namespace

}  // namespace pgi
