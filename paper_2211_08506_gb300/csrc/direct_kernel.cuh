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
// Planes of large molecules can instead give each lane its own list of the candidates that
// reach its voxels (lane-list mode, see lane_plane), in a kernel instantiation of its own.  It
// adds the same terms in the same order, so its results are bitwise identical to the
// gather's.
#pragma once

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

// One atom's terms on a lane's VEC columns of two rows (voxel centres vz[], rows vya and vyb):
// the row factors once per row, each z factor once for both rows, the exact per-voxel test for
// a sphere.  Every voxel adds the same terms in the same order of operations as
// LaneVoxels::add.
template <int VEC, int CUT, bool PER, int FORM>
__device__ __forceinline__ void add_pair(float (&acc0)[VEC], float (&acc1)[VEC],
                                         const float (&vz)[VEC], float vya, float vyb, float dx,
                                         float ay, float az, float w, float q, float r2, float kf,
                                         float hx, float hy, float hz, float Ly, float iLy,
                                         float Lz, float iLz)
{
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
}

// Gather of one plane in passes of two lane groups, for planes whose lane columns repeat
// from group to group: with lpr = nz / VEC lanes per row, lane l < act = rpg * lpr owns the
// columns z0 .. z0 + VEC - 1 of rows y0 + l / lpr and y0 + l / lpr + rpg of each pass of
// 2 * rpg rows.  Each surviving atom's z factors are computed once per pass and shared by both
// rows.  for_each(cy, wy, cz, wz, f) calls f(dx, ay, az, w), w the atom's weight, for the
// candidates that can reach the pass's box of voxel centres, in atom order.  Every voxel adds
// the same terms in the same order as LaneVoxels::add does (atoms culled for one of the two
// rows add exact zeros or are skipped by the same test), so both give identical bits.
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
            add_pair<VEC, CUT, PER, FORM>(acc0, acc1, vz, vya, vyb, dx, ay, az, w, q, r2, kf, hx,
                                          hy, hz, Ly, iLy, Lz, iLz);
        });
        if (lane < act) {
            if (ya < ny) store_lane<T, VEC, HINT>(out, (ya * nz + z0) / VEC, acc0);
            if (yb < ny) store_lane<T, VEC, HINT>(out, (yb * nz + z0) / VEC, acc1);
        }
    }
}

// Voxel-integrated form with a separable cutoff (none or box): the per-axis factors do not
// depend on the plane, so the warp computes them once per chunk into a table in shared memory
// (Sec. VI-A's per-axis tables): for the chunk's i-th atom of the channel, row i of the table
// (erf_table_stride floats) holds its y factor on each row y and then its z factor on each
// column z, each exactly the value erf_axis gives for that row or column, zeroed outside a box
// cutoff.  A plane is then walked in the passes of blocked_plane, and every term is the atom's
// x factor times its table entries in the same order of operations as blocked_plane uses, so
// the two give identical bits.  for_each(cy, wy, cz, wz, f) calls f(dx, fx, w, ti) - the
// candidate's x displacement, x factor, weight and table row - for the candidates that can
// reach the pass's box of voxel centres, in atom order.
template <typename T, int VEC, int CUT, bool PER, int HINT, typename ForEach>
__device__ __forceinline__ void table_plane(T *out, const float *tab, int ny, int nz, int rpg,
                                            int act, int my_row, int z0, int lane, float r2,
                                            float oy, float oz, float hy, float hz,
                                            ForEach for_each)
{
    const int tw = erf_table_stride(ny, nz);
    const int tyw = (ny + 3) & ~3;
    const float cz = fmaf(0.5f * (float)(nz - 1) + 0.5f, hz, oz);
    const float wz = 0.5f * (float)(nz - 1) * hz;
    for (int y0 = 0; y0 < ny; y0 += 2 * rpg) {
        const int y_end = min(y0 + 2 * rpg, ny) - 1;
        const float cy = fmaf(0.5f * (float)(y0 + y_end) + 0.5f, hy, oy);
        const float wy = 0.5f * (float)(y_end - y0) * hy;
        const int ya = y0 + my_row, yb = ya + rpg;
        // Rows past the grid are computed but not stored; read a valid entry for them.
        const int ra = min(ya, ny - 1), rb = min(yb, ny - 1);
        float acc0[VEC], acc1[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc0[k] = acc1[k] = 0.0f;
        for_each(cy, wy, cz, wz, [&](float dx, float fx, float w, int ti) {
            const float *ty = tab + ti * tw;
            const float *tz = ty + tyw;
            const bool xout = CUT == PG_CUTOFF_BOX && dx * dx > r2;
            const float ea = w * (xout ? 0.0f : fx * ty[ra]);
            const float eb = w * (xout ? 0.0f : fx * ty[rb]);
            float ez[VEC];
            if constexpr (VEC % 4 == 0) {
#pragma unroll
                for (int k = 0; k < VEC; k += 4) {
                    const float4 f = *reinterpret_cast<const float4 *>(tz + z0 + k);
                    ez[k] = f.x;
                    ez[k + 1] = f.y;
                    ez[k + 2] = f.z;
                    ez[k + 3] = f.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) ez[k] = tz[z0 + k];
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                acc0[k] = fmaf(ea, ez[k], acc0[k]);
                acc1[k] = fmaf(eb, ez[k], acc1[k]);
            }
        });
        if (lane < act) {
            if (ya < ny) store_lane<T, VEC, HINT>(out, (ya * nz + z0) / VEC, acc0);
            if (yb < ny) store_lane<T, VEC, HINT>(out, (yb * nz + z0) / VEC, acc1);
        }
    }
}

// Fills rows 0 .. n - 1 of a voxel-integrated factor table (see table_plane), 32 entries per
// step across the warp; atom(i) gives row i's atom position {y, z} (a float2).
template <int CUT, bool PER, typename AtomYZ>
__device__ __forceinline__ void build_erf_table(float *tab, int n, int ny, int nz, int lane,
                                                float q, float r2, float kf, float oy, float oz,
                                                float hy, float hz, float Ly, float iLy, float Lz,
                                                float iLz, AtomYZ atom)
{
    const int tw = erf_table_stride(ny, nz);
    const int tyw = (ny + 3) & ~3;
    const int total = n * tw;
    for (int base = 0; base < total; base += 32) {
        const int idx = base + lane;
        const int row = idx / tw;
        const int j = idx - row * tw;
        const float2 a = atom(min(row, n - 1));
        if (idx < total) {
            float v = 0.0f;
            if (j < tyw) {
                if (j < ny) {
                    float dy = fmaf((float)j + 0.5f, hy, oy) - a.x;
                    if (PER) dy = wrap(dy, Ly, iLy);
                    v = erf_axis(dy, hy, kf);
                    if (CUT == PG_CUTOFF_BOX && dy * dy > r2) v = 0.0f;
                }
            } else if (j - tyw < nz) {
                float dz = fmaf((float)(j - tyw) + 0.5f, hz, oz) - a.y;
                if (PER) dz = wrap(dz, Lz, iLz);
                v = z_factor<CUT, 1>(dz, q, r2, kf, hz);
            }
            tab[idx] = v;
        }
    }
}

// Index i wrapped into [0, n) (periodic axes).
__device__ __forceinline__ int wrap_index(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Lane-list mode, for planes of large molecules (staged candidates) with a cutoff: the passes
// of blocked_plane, but each lane adds only the candidates that can reach its own voxels.  A
// lane owns VEC columns of two adjacent rows, a box of 2 x VEC voxel centres; for every
// candidate that reaches the pass's box the warp tests, per lane, whether the candidate also
// reaches the lane's box, and each lane then walks its own list in atom order.  On dense
// planes a disc covers a small part of the 2 * rpg rows x nz columns of a pass, so the lane
// lists are much shorter than the pass list: the warp runs as many terms as the longest lane
// list rather than one per candidate of the pass.  The lists are conservative and in atom
// order, and each term is add_pair's, as in blocked_plane: identical bits.
template <typename T, int VEC, int CUT, bool PER, int HINT, int FORM, bool WGT>
__device__ __forceinline__ void lane_plane(T *out, const float4 *stage, int count, int ny,
                                           int nz, int rpg, int act, int my_row, int z0, int lane,
                                           float q, float r2, float rc, float kf, float hx,
                                           float oy, float oz, float hy, float hz, float Ly,
                                           float iLy, float Lz, float iLz)
{
    float vz[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) vz[k] = fmaf((float)(z0 + k) + 0.5f, hz, oz);
    // Pass box: whole rows.  Lane box: the lane's VEC columns of its two rows.
    const float cz = fmaf(0.5f * (float)(nz - 1) + 0.5f, hz, oz);
    const float wz = 0.5f * (float)(nz - 1) * hz;
    const float lcz = fmaf((float)z0 + 0.5f * (float)(VEC - 1) + 0.5f, hz, oz);
    const float lwz = 0.5f * (float)(VEC - 1) * hz;
    const float lwy = 0.5f * hy;
    for (int y0 = 0; y0 < ny; y0 += 2 * rpg) {
        const int y_end = min(y0 + 2 * rpg, ny) - 1;
        const float cy = fmaf(0.5f * (float)(y0 + y_end) + 0.5f, hy, oy);
        const float wy = 0.5f * (float)(y_end - y0) * hy;
        const int ya = y0 + 2 * my_row, yb = ya + 1;
        const float vya = fmaf((float)ya + 0.5f, hy, oy);
        const float vyb = fmaf((float)yb + 0.5f, hy, oy);
        const float lcy = fmaf((float)ya + 1.0f, hy, oy);
        float acc0[VEC], acc1[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc0[k] = acc1[k] = 0.0f;
        for (int cb = 0; cb < count; cb += 32) {
            const int j = cb + lane;
            bool ok = false;
            if (j < count) {
                const float4 st = stage[j];
                ok = reaches<CUT, PER>(st.x, st.y, st.z, cy, wy, cz, wz, rc, Ly, iLy, Lz, iLz);
            }
            unsigned m = __ballot_sync(0xffffffffu, ok);
            // The lane's list: bit i for candidate cb + i.
            unsigned lm = 0u;
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1;
                const float4 st = stage[cb + i];
                if (reaches<CUT, PER>(st.x, st.y, st.z, lcy, lwy, lcz, lwz, rc, Ly, iLy, Lz,
                                      iLz))
                    lm |= 1u << i;
            }
            if (lane >= act) lm = 0u;
            while (lm) {
                const int i = __ffs(lm) - 1;
                lm &= lm - 1;
                const float4 st = stage[cb + i];
                add_pair<VEC, CUT, PER, FORM>(acc0, acc1, vz, vya, vyb, st.x, st.y, st.z,
                                              WGT ? st.w : 1.0f, q, r2, kf, hx, hy, hz, Ly, iLy,
                                              Lz, iLz);
            }
        }
        if (lane < act) {
            if (ya < ny) store_lane<T, VEC, HINT>(out, (ya * nz + z0) / VEC, acc0);
            if (yb < ny) store_lane<T, VEC, HINT>(out, (yb * nz + z0) / VEC, acc1);
        }
    }
}

// WGT: per-atom weights (weighted grids).  Unweighted batches run the instantiation without
// them, which carries no weight loads, shuffles or multiplies.
template <typename T, int VEC, int CUT, bool PER, int HINT, bool LANE, int FORM, bool WGT>
__global__ void __launch_bounds__(512, (LANE || VEC == 8) ? 1 : 2) direct_kernel(const DirectArgs A)
{
    extern __shared__ float4 smem_all[];
    const Geometry &G = A.geo;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps_per_block = blockDim.x >> 5;
    // Per warp (layout in direct_warp_floats): the plane's staged candidates, then the
    // chunk's channel atoms.
    float4 *stage = smem_all + (size_t)warp * (direct_warp_floats(A.erf_tab) / 4);
    float4 *chan = stage + kStageCap;
    // Voxel-integrated form with a separable cutoff: per-chunk factor tables (table_plane).
    // Molecules of at most 32 atoms keep theirs in the staging area, which they do not use;
    // larger molecules keep theirs after their staged candidates and channel atoms, with each
    // staged candidate's x factor in sfx.
    constexpr bool TAB = FORM == 1 && CUT != PG_CUTOFF_SPHERE;
    constexpr int kStaging = 4 * (kStageCap + kChanCap);
    float *tab = reinterpret_cast<float *>(stage);
    float *stab = reinterpret_cast<float *>(stage) + kStaging;
    float *sfx = reinterpret_cast<float *>(stage) + max(kStaging, A.erf_tab);
    long long tab_bc = -1;  // (molecule, channel) whose factors the table holds
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
        // Small molecule, voxel-integrated form, separable cutoff: the factor table of this
        // (molecule, channel), built unless the warp already holds it.  my_ti is the lane's atom's
        // row in it (its rank among the channel's atoms).
        bool use_tab = false;
        int my_ti = -1;
        if constexpr (TAB) {
            if (small && blocked && A.erf_tab > 0) {
                const unsigned chm = __ballot_sync(0xffffffffu, my_e == c);
                const int nch = __popc(chm);
                const int tw = erf_table_stride(G.ny, G.nz);
                use_tab = nch > 0 && nch * tw <= A.erf_tab;
                if (use_tab) {
                    my_ti = (my_e == c) ? __popc(chm & lt_mask) : -1;
                    if (tab_bc != (long long)bc) {
                        __syncwarp();
                        build_erf_table<CUT, PER>(
                            tab, nch, G.ny, G.nz, lane, G.q[c], G.r2[c], G.kerf[c], oy, oz, hy, hz,
                            Ly, iLy, Lz, iLz, [&](int i) {
                                const int src = __fns(chm, 0, i + 1);
                                return make_float2(__shfl_sync(0xffffffffu, my_y, src),
                                                   __shfl_sync(0xffffffffu, my_z, src));
                            });
                        __syncwarp();
                        tab_bc = (long long)bc;
                    }
                }
            }
        }
        // Large molecule: this channel's atoms that can reach a plane of the chunk, in atom
        // order, staged in shared memory once per chunk when they fit, so that each plane culls
        // them from there.  An atom can reach a plane only if its x distance (nearest image
        // when periodic) to the chunk's centre is within the chunk's half width plus the
        // widened cutoff, with a margin for rounding.
        int n_chan = -1;
        if (!small) {
            tab_bc = -1;  // the staging below overwrites the factor table
            int cnt = 0;
            const float xc = fmaf(0.5f * (float)(x_begin + x_end - 1) + 0.5f, hx, ox);
            const float xreach = fmaf(0.5f * (float)(x_end - 1 - x_begin), hx, G.rcull[c]) +
                                 1e-3f * hx + 1e-5f * (fabsf(xc) + (PER ? Lx : 0.0f));
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
                    bool ok = e[h] == c;
                    if (CUT != PG_CUTOFF_NONE) {
                        const float ex = PER ? wrap(ax[h] - xc, Lx, iLx) : ax[h] - xc;
                        ok = ok && fabsf(ex) <= xreach;
                    }
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
        // Larger molecule, voxel-integrated form, separable cutoff: the factor table of the
        // chunk's channel atoms, when it fits after the staging area.
        bool use_stab = false;
        if constexpr (TAB) {
            if (!small && blocked && n_chan > 0 &&
                n_chan * erf_table_stride(G.ny, G.nz) <= A.erf_tab - kStaging) {
                use_stab = true;
                build_erf_table<CUT, PER>(stab, n_chan, G.ny, G.nz, lane, G.q[c], G.r2[c],
                                          G.kerf[c], oy, oz, hy, hz, Ly, iLy, Lz, iLz,
                                          [&](int i) {
                                              const float4 a = chan[i];
                                              return make_float2(a.y, a.z);
                                          });
                __syncwarp();
            }
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
                } else if (TAB && use_tab) {
                    const float fx = cand ? erf_axis(dx, hx, kf) : 0.0f;
                    table_plane<T, VEC, CUT, PER, HINT>(
                        out, tab, G.ny, G.nz, rpg, act, my_row, my_z0, lane, r2, oy, oz, hy, hz,
                        [&](float cy, float wy, float cz, float wz, auto &&f) {
                            const bool hit = cand && reaches<CUT, PER>(dx, my_y, my_z, cy, wy, cz,
                                                                       wz, rc, Ly, iLy, Lz, iLz);
                            unsigned m = __ballot_sync(0xffffffffu, hit);
                            while (m) {
                                const int src = __ffs(m) - 1;
                                m &= m - 1;
                                f(__shfl_sync(0xffffffffu, dx, src),
                                  __shfl_sync(0xffffffffu, fx, src),
                                  WGT ? __shfl_sync(0xffffffffu, my_w, src) : 1.0f,
                                  __shfl_sync(0xffffffffu, my_ti, src));
                            }
                        });
                } else if (blocked) {
                    blocked_plane<T, VEC, CUT, PER, HINT, FORM>(
                        out, G.ny, G.nz, rpg, act, my_row, my_z0, lane, q, r2, kf, hx, oy, oz,
                        hy, hz, Ly, iLy, Lz, iLz,
                        [&](float cy, float wy, float cz, float wz, auto &&f) {
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
                    if (ok) {
                        const int pos = count + __popc(m & lt_mask);
                        if (TAB && use_stab) {
                            // With a factor table: the atom's table row instead of its weight,
                            // and its x factor beside.
                            stage[pos] = make_float4(dx, ay, az, __int_as_float(j));
                            sfx[pos] = erf_axis(dx, hx, kf);
                        } else {
                            stage[pos] = make_float4(dx, ay, az, aw);
                        }
                    }
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
                } else if (TAB && use_stab) {
                    table_plane<T, VEC, CUT, PER, HINT>(
                        out, stab, G.ny, G.nz, rpg, act, my_row, my_z0, lane, r2, oy, oz, hy, hz,
                        [&](float cy, float wy, float cz, float wz, auto &&f) {
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
                                    const int ti = __float_as_int(st.w);
                                    f(st.x, sfx[cb + src], WGT ? chan[ti].w : 1.0f, ti);
                                }
                            }
                        });
                } else if (LANE && blocked && count <= kStageCap) {
                    lane_plane<T, VEC, CUT, PER, HINT, FORM, WGT>(
                        out, stage, count, G.ny, G.nz, rpg, act, my_row, my_z0, lane, q, r2,
                        rc, kf, hx, oy, oz, hy, hz, Ly, iLy, Lz, iLz);
                } else if (blocked && count <= kStageCap) {
                    blocked_plane<T, VEC, CUT, PER, HINT, FORM>(
                        out, G.ny, G.nz, rpg, act, my_row, my_z0, lane, q, r2, kf, hx, oy, oz,
                        hy, hz, Ly, iLy, Lz, iLz,
                        [&](float cy, float wy, float cz, float wz, auto &&f) {
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

// Lane-list instantiations exist only for the point form and where a cutoff bounds each
// atom's disc; the gather-only ones carry no lane-list code and so keep their register
// allocation.
template <typename T, int VEC, int CUT, bool PER, int HINT, int FORM>
const void *pick_lane(bool lanes)
{
    if constexpr (CUT != PG_CUTOFF_NONE && FORM == 0)
        if (lanes) return (const void *)direct_kernel<T, VEC, CUT, PER, HINT, true, FORM, false>;
    return (const void *)direct_kernel<T, VEC, CUT, PER, HINT, false, FORM, false>;
}

template <typename T, int VEC, int CUT, bool PER, int FORM>
const void *pick_hint(int hint, bool lanes)
{
    return hint == 1 ? pick_lane<T, VEC, CUT, PER, 1, FORM>(lanes)
                     : pick_lane<T, VEC, CUT, PER, 0, FORM>(lanes);
}

template <typename T, int VEC, int FORM>
const void *pick_shape(int cutoff, int periodic, int hint, bool lanes)
{
    if (periodic) {
        if (cutoff == PG_CUTOFF_SPHERE)
            return pick_hint<T, VEC, PG_CUTOFF_SPHERE, true, FORM>(hint, lanes);
        if (cutoff == PG_CUTOFF_BOX) return pick_hint<T, VEC, PG_CUTOFF_BOX, true, FORM>(hint, lanes);
        return pick_hint<T, VEC, PG_CUTOFF_NONE, true, FORM>(hint, lanes);
    }
    if (cutoff == PG_CUTOFF_SPHERE)
        return pick_hint<T, VEC, PG_CUTOFF_SPHERE, false, FORM>(hint, lanes);
    if (cutoff == PG_CUTOFF_BOX) return pick_hint<T, VEC, PG_CUTOFF_BOX, false, FORM>(hint, lanes);
    return pick_hint<T, VEC, PG_CUTOFF_NONE, false, FORM>(hint, lanes);
}

// Weighted instantiations: gather mode and default stores.
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
// lane-list mode and voxel form.
template <int FORM>
const void *pick_direct(int dtype, bool vec_ok, int cut, int per, int hint, bool lanes)
{
    if (dtype == PG_F32)
        return vec_ok ? pick_shape<float, 4, FORM>(cut, per, hint, lanes)
                      : pick_shape<float, 1, FORM>(cut, per, hint, lanes);
    if (dtype == PG_F16)
        return vec_ok ? pick_shape<__half, 8, FORM>(cut, per, hint, lanes)
                      : pick_shape<__half, 1, FORM>(cut, per, hint, lanes);
    return vec_ok ? pick_shape<__nv_bfloat16, 8, FORM>(cut, per, hint, lanes)
                  : pick_shape<__nv_bfloat16, 1, FORM>(cut, per, hint, lanes);
}

}  // namespace

}  // namespace pgi
