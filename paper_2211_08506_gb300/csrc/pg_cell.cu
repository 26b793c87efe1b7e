// Voxelization in general cells (sm_103a): grids whose x, y, z axes run along the rows a, b,
// c of a per-molecule 3x3 matrix M (Sec. III-A: the box's orientation and size are the
// user's choice, voxels need not be cubic; periodic crystals use the nearest image over the
// lattice translations).  Voxel (i, j, k) sits at fractional position
// u = ((i + 1/2) / nx, (j + 1/2) / ny, (k + 1/2) / nz) of the box, that is at o + u M.
//
// Nearest image.  With p = (x - o) M^-1 the atom's fractional position and e = u - p, the
// displacement is d = (e - t) M for the lattice translation t.  Let g_k be column k of M^-1.
// A cutoff region whose reach along fractional axis k, rho |g_k|, is below one half admits
// at most one image of an atom per voxel: any image inside it has |e_k - t_k| < 1/2 on every
// axis, so t = round(e) axis by axis.  rho is r_c for the sphere, and for the box the
// radius sqrt(3) r_c of its circumscribed sphere, so that the image chosen is also the
// nearest one.  The kernels therefore wrap e per fractional axis and, where that condition
// fails for some molecule and channel, set PG_DEVERR_PERIODIC.  Without a cutoff the
// nearest image is not found by rounding in a skewed cell, and the host rejects that case.
//
// Forward kernel.  Work items are (molecule, channel, x-plane) as in the direct kernel,
// handed out in chunks of planes from a per-launch counter, in either chunk order.  Per chunk a warp stages the
// channel's atoms as {p, w}.  Per plane it keeps the candidates within the cutoff's
// fractional reach of the plane as {e_x a, w} and {p_y, p_z}.  For a lane's voxels of row j
// the displacement is d = base + e_z c with base = e_x a + e_y b, so
//     |d|^2 = |base|^2 + e_z (2 base.c + e_z |c|^2),
// one quadratic per row and two FMAs per voxel.  Candidates are visited in atom order after
// a conservative fractional-box cull, so results do not depend on the launch shape.
//
// Adjoint kernel.  One warp per atom (atom counter) walks the voxels of the atom's fractional
// support box, 32 per step with z fastest, and sums g * w * exp(-|d|^2 / 2 sigma^2) * d /
// sigma^2 (and, for the weight gradient, g * exp(...)) with a fixed butterfly reduction.
#include "direct_kernel.cuh"

namespace pgi {

namespace {

constexpr int kCellCap = 256;     // channel atoms staged per warp and chunk
constexpr int kCellThreads = 128;

// Shared memory per warp: kCellCap {p, w} + kCellCap {e_x a, w} + kCellCap {p_y, p_z}.
constexpr size_t kCellWarpBytes = (size_t)kCellCap * (16 + 16 + 8);

// A molecule's box: edges M (rows a, b, c), inverse, origin, and per fractional axis the
// Euclidean and L1 lengths of the columns of M^-1.
struct Frame {
    float M[9], Mi[9], o[3], g2[3], g1[3];
    bool ok;
};

__device__ __forceinline__ Frame load_frame(const Inputs &in, int b)
{
    Frame f;
#pragma unroll
    for (int i = 0; i < 9; ++i) f.M[i] = __ldg(in.cell + 9 * b + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) f.o[i] = __ldg(in.origin + 3 * b + i);
    const float *M = f.M;
    // Every product and sum is spelled out (fmaf, __fmul_rn), so that the compiler cannot
    // contract them differently in different kernel instantiations: forward and adjoint
    // kernels of any store width get the same bits of the inverse.
    auto cof = [](float a, float b, float c, float d) {  // a b - c d
        return fmaf(a, b, -__fmul_rn(c, d));
    };
    const float c0 = cof(M[4], M[8], M[5], M[7]), c1 = cof(M[5], M[6], M[3], M[8]),
                c2 = cof(M[3], M[7], M[4], M[6]);
    const float det = fmaf(M[0], c0, fmaf(M[1], c1, __fmul_rn(M[2], c2)));
    f.ok = isfinite(det) && det != 0.0f;
    const float id = f.ok ? 1.0f / det : 0.0f;
    f.Mi[0] = __fmul_rn(c0, id);
    f.Mi[1] = __fmul_rn(cof(M[2], M[7], M[1], M[8]), id);
    f.Mi[2] = __fmul_rn(cof(M[1], M[5], M[2], M[4]), id);
    f.Mi[3] = __fmul_rn(c1, id);
    f.Mi[4] = __fmul_rn(cof(M[0], M[8], M[2], M[6]), id);
    f.Mi[5] = __fmul_rn(cof(M[2], M[3], M[0], M[5]), id);
    f.Mi[6] = __fmul_rn(c2, id);
    f.Mi[7] = __fmul_rn(cof(M[1], M[6], M[0], M[7]), id);
    f.Mi[8] = __fmul_rn(cof(M[0], M[4], M[1], M[3]), id);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float x = f.Mi[k], y = f.Mi[3 + k], z = f.Mi[6 + k];
        f.g2[k] = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
        f.g1[k] = __fadd_rn(__fadd_rn(fabsf(x), fabsf(y)), fabsf(z));
        f.ok = f.ok && isfinite(f.g2[k]);
    }
    return f;
}

// Fractional position of x in the molecule's box.
__device__ __forceinline__ void to_frac(const Frame &f, float x, float y, float z, float &px,
                                        float &py, float &pz)
{
    const float dx = x - f.o[0], dy = y - f.o[1], dz = z - f.o[2];
    px = fmaf(dx, f.Mi[0], fmaf(dy, f.Mi[3], dz * f.Mi[6]));
    py = fmaf(dx, f.Mi[1], fmaf(dy, f.Mi[4], dz * f.Mi[7]));
    pz = fmaf(dx, f.Mi[2], fmaf(dy, f.Mi[5], dz * f.Mi[8]));
}

template <bool PER>
__device__ __forceinline__ float wrap1(float e)
{
    return PER ? e - rintf(e) : e;
}

// Fractional reach of channel c's cutoff along axis k (for culls and supports).
template <int CUT>
__device__ __forceinline__ float reach(const Frame &f, int k, float rc)
{
    if (CUT == PG_CUTOFF_NONE) return INFINITY;
    return rc * (CUT == PG_CUTOFF_BOX ? f.g1[k] : f.g2[k]);
}

// Whether a periodic box admits at most one image per voxel for cutoff radius r_c.
template <int CUT>
__device__ __forceinline__ bool images_unique(const Frame &f, float rc)
{
    const float rho = CUT == PG_CUTOFF_BOX ? 1.7320508f * rc : rc;
    return rho * f.g2[0] < 0.5f && rho * f.g2[1] < 0.5f && rho * f.g2[2] < 0.5f;
}

template <typename T, int VEC, int CUT, bool PER>
__global__ void __launch_bounds__(kCellThreads) cell_kernel(const DirectArgs A)
{
    extern __shared__ float4 cell_smem[];
    const Geometry &G = A.geo;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps_per_block = blockDim.x >> 5;
    float4 *chan = cell_smem + (size_t)warp * (kCellWarpBytes / 16);
    float4 *stage = chan + kCellCap;
    float2 *stage2 = reinterpret_cast<float2 *>(stage + kCellCap);
    const unsigned lt_mask = (1u << lane) - 1u;

    const int chunk_planes = A.chunk_planes;
    const int x_chunks = (G.nx + chunk_planes - 1) / chunk_planes;
    const unsigned long long n_chunks = (unsigned long long)G.n_mol * G.C * x_chunks;
    const unsigned long long total_warps = (unsigned long long)gridDim.x * warps_per_block;
    const int plane = G.ny * G.nz;
    const int nvec = plane / VEC;
    const int y_start = (lane * VEC) / G.nz, z_start = (lane * VEC) % G.nz;
    const int y_step = (32 * VEC) / G.nz, z_step = (32 * VEC) % G.nz;
    const float inx = 1.0f / G.nx, iny = 1.0f / G.ny, inz = 1.0f / G.nz;
    // Two-row passes when whole rows fill at least 28 of the 32 lanes: with lpr = nz / VEC
    // lanes per row, lane l < act = rpg * lpr owns columns z0 .. z0 + VEC - 1 of rows
    // y0 + l / lpr and y0 + l / lpr + rpg of each pass of 2 * rpg rows.
    const int lpr = G.nz / VEC;
    const int rpg = (lpr >= 1 && lpr <= 32) ? 32 / lpr : 0;
    const int act = rpg * lpr;
    const bool blocked = act >= 28;
    const int my_row = blocked ? lane / lpr : 0;
    const int my_z0 = blocked ? (lane - my_row * lpr) * VEC : 0;

    int cur_b = -1;
    int a0 = 0, a1 = 0;
    Frame F;
    F.ok = false;

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
            F = load_frame(A.in, b);
            const bool off_ok = (a0 >= 0) && (a0 <= a1) && (a1 <= G.n_atoms);
            if (!off_ok || !F.ok) {
                if (lane == 0 && c == 0 && x_begin == 0)
                    atomicOr(A.err, (off_ok ? 0u : PG_DEVERR_OFFSETS) |
                                        (F.ok ? 0u : PG_DEVERR_SPACING));
                a0 = a1 = 0;
            }
        }
        const float q = G.q[c], r2 = G.r2[c], rc = G.rcull[c];
        const float ext_x = reach<CUT>(F, 0, rc), ext_y = reach<CUT>(F, 1, rc),
                    ext_z = reach<CUT>(F, 2, rc);
        if (PER && lane == 0 && x_begin == 0 && a1 > a0 && !images_unique<CUT>(F, rc))
            atomicOr(A.err, PG_DEVERR_PERIODIC);
        // The channel's atoms in atom order as {fractional position, weight}.
        int n_chan = 0;
        for (int base = a0; base < a1; base += 32) {
            const int ai = base + lane;
            bool ok = false;
            float4 v = make_float4(0.f, 0.f, 0.f, 1.f);
            if (ai < a1) {
                const int e = __ldg(A.in.elem + ai);
                if ((unsigned)e >= (unsigned)G.C) {
                    if (c == 0 && x_begin == 0) atomicOr(A.err, PG_DEVERR_ELEMENT);
                } else if (e == c) {
                    ok = true;
                    to_frac(F, __ldg(A.in.coords + 3 * ai), __ldg(A.in.coords + 3 * ai + 1),
                            __ldg(A.in.coords + 3 * ai + 2), v.x, v.y, v.z);
                    if (A.in.weight) v.w = __ldg(A.in.weight + ai);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            const int pos = n_chan + __popc(m & lt_mask);
            if (ok && pos < kCellCap) chan[pos] = v;
            n_chan += __popc(m);
        }
        __syncwarp();
        const bool staged = n_chan <= kCellCap;
        const float ax = F.M[0], ay = F.M[1], az = F.M[2];
        const float bx = F.M[3], by = F.M[4], bz = F.M[5];
        const float cx = F.M[6], cy = F.M[7], cz = F.M[8];
        const float cc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));

        for (int x = x_begin; x < x_end; ++x) {
            const long long item = (long long)bc * G.nx + x;
            T *out = reinterpret_cast<T *>(A.out) + item * (long long)plane;
            const float ux = ((float)x + 0.5f) * inx;
            // Candidates of the plane: {e_x a, w} and {p_y, p_z}, in atom order.
            int count = 0;
            if (staged) {
                for (int cb = 0; cb < n_chan; cb += 32) {
                    const int j = cb + lane;
                    bool ok = false;
                    float4 v;
                    float ex = 0.0f;
                    if (j < n_chan) {
                        v = chan[j];
                        ex = wrap1<PER>(ux - v.x);
                        ok = fabsf(ex) <= ext_x;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) {
                        const int pos = count + __popc(m & lt_mask);
                        stage[pos] = make_float4(ex * ax, ex * ay, ex * az, v.w);
                        stage2[pos] = make_float2(v.y, v.z);
                    }
                    count += __popc(m);
                }
                __syncwarp();
                if (count == 0) {
                    zero_plane<T, VEC, 0>(out, nvec, lane);
                    continue;
                }
            }
            // One atom's terms for this lane's VEC voxels of row y (fractional uy, uz[]).
            auto add = [&](const float4 &s, const float2 &s2, float uy, const float (&uz)[VEC],
                           float (&acc)[VEC]) {
                const float ey = wrap1<PER>(uy - s2.x);
                const float px = fmaf(ey, bx, s.x), py = fmaf(ey, by, s.y),
                            pz = fmaf(ey, bz, s.z);
                const float A2 = fmaf(px, px, fmaf(py, py, pz * pz));
                const float B2 = 2.0f * fmaf(px, cx, fmaf(py, cy, pz * cz));
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const float ez = wrap1<PER>(uz[k] - s2.y);
                    const float d2 = fmaf(ez, fmaf(ez, cc, B2), A2);
                    bool in = true;
                    if (CUT == PG_CUTOFF_SPHERE) {
                        in = d2 <= r2;
                    } else if (CUT == PG_CUTOFF_BOX) {
                        const float dx = fmaf(ez, cx, px), dy = fmaf(ez, cy, py),
                                    dz = fmaf(ez, cz, pz);
                        in = fmaxf(dx * dx, fmaxf(dy * dy, dz * dz)) <= r2;
                    }
                    acc[k] = in ? fmaf(s.w, ex2_approx(-q * d2), acc[k]) : acc[k];
                }
            };
            if (staged && blocked) {
                // Two-row passes: each candidate's e_z terms are formed once per column and
                // shared by the lane's two rows.  Every voxel adds the same terms, formed by
                // the same operations, in the same order as with add().
                float uz[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) uz[k] = ((float)(my_z0 + k) + 0.5f) * inz;
                const float czf = (0.5f * (float)(G.nz - 1) + 0.5f) * inz;
                const float wzf = 0.5f * (float)(G.nz - 1) * inz;
                for (int y0 = 0; y0 < G.ny; y0 += 2 * rpg) {
                    const int y_end = min(y0 + 2 * rpg, G.ny) - 1;
                    const float cyf = (0.5f * (float)(y0 + y_end) + 0.5f) * iny;
                    const float wyf = 0.5f * (float)(y_end - y0) * iny;
                    const int ya = y0 + my_row, yb = ya + rpg;
                    const float uya = ((float)ya + 0.5f) * iny, uyb = ((float)yb + 0.5f) * iny;
                    float acc0[VEC], acc1[VEC];
#pragma unroll
                    for (int k = 0; k < VEC; ++k) acc0[k] = acc1[k] = 0.0f;
                    for (int cb = 0; cb < count; cb += 32) {
                        const int j = cb + lane;
                        bool ok = false;
                        if (j < count) {
                            const float2 s2 = stage2[j];
                            const float gy = fmaxf(fabsf(wrap1<PER>(cyf - s2.x)) - wyf, 0.0f);
                            const float gz = fmaxf(fabsf(wrap1<PER>(czf - s2.y)) - wzf, 0.0f);
                            ok = gy <= ext_y && gz <= ext_z;
                        }
                        unsigned m = __ballot_sync(0xffffffffu, ok);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1;
                            const float4 sv = stage[cb + src];
                            const float2 s2 = stage2[cb + src];
                            const float eya = wrap1<PER>(uya - s2.x);
                            const float eyb = wrap1<PER>(uyb - s2.x);
                            const float pxa = fmaf(eya, bx, sv.x), pya = fmaf(eya, by, sv.y),
                                        pza = fmaf(eya, bz, sv.z);
                            const float pxb = fmaf(eyb, bx, sv.x), pyb = fmaf(eyb, by, sv.y),
                                        pzb = fmaf(eyb, bz, sv.z);
                            const float A2a = fmaf(pxa, pxa, fmaf(pya, pya, pza * pza));
                            const float A2b = fmaf(pxb, pxb, fmaf(pyb, pyb, pzb * pzb));
                            const float B2a = 2.0f * fmaf(pxa, cx, fmaf(pya, cy, pza * cz));
                            const float B2b = 2.0f * fmaf(pxb, cx, fmaf(pyb, cy, pzb * cz));
#pragma unroll
                            for (int k = 0; k < VEC; ++k) {
                                const float ez = wrap1<PER>(uz[k] - s2.y);
                                const float d2a = fmaf(ez, fmaf(ez, cc, B2a), A2a);
                                const float d2b = fmaf(ez, fmaf(ez, cc, B2b), A2b);
                                bool ina = true, inb = true;
                                if (CUT == PG_CUTOFF_SPHERE) {
                                    ina = d2a <= r2;
                                    inb = d2b <= r2;
                                } else if (CUT == PG_CUTOFF_BOX) {
                                    const float dxa = fmaf(ez, cx, pxa), dya = fmaf(ez, cy, pya),
                                                dza = fmaf(ez, cz, pza);
                                    const float dxb = fmaf(ez, cx, pxb), dyb = fmaf(ez, cy, pyb),
                                                dzb = fmaf(ez, cz, pzb);
                                    ina = fmaxf(dxa * dxa, fmaxf(dya * dya, dza * dza)) <= r2;
                                    inb = fmaxf(dxb * dxb, fmaxf(dyb * dyb, dzb * dzb)) <= r2;
                                }
                                acc0[k] = ina ? fmaf(sv.w, ex2_approx(-q * d2a), acc0[k]) : acc0[k];
                                acc1[k] = inb ? fmaf(sv.w, ex2_approx(-q * d2b), acc1[k]) : acc1[k];
                            }
                        }
                    }
                    if (lane < act) {
                        if (ya < G.ny) store_lane<T, VEC, 0>(out, (ya * G.nz + my_z0) / VEC, acc0);
                        if (yb < G.ny) store_lane<T, VEC, 0>(out, (yb * G.nz + my_z0) / VEC, acc1);
                    }
                }
                __syncwarp();
                continue;
            }
            int y = y_start, z0 = z_start;
            for (int g = 0; g < nvec; g += 32) {
                const int v = g + lane;
                const int last = min(31, nvec - 1 - g);
                const int y_lo = __shfl_sync(0xffffffffu, y, 0);
                const int y_hi = __shfl_sync(0xffffffffu, y, last);
                int z_lo = 0, z_hi = G.nz - 1;
                if (y_lo == y_hi) {
                    z_lo = __shfl_sync(0xffffffffu, z0, 0);
                    z_hi = __shfl_sync(0xffffffffu, z0, last) + VEC - 1;
                }
                // Fractional centre and half-width of the group's rows and columns.
                const float cyf = (0.5f * (float)(y_lo + y_hi) + 0.5f) * iny;
                const float wyf = 0.5f * (float)(y_hi - y_lo) * iny;
                const float czf = (0.5f * (float)(z_lo + z_hi) + 0.5f) * inz;
                const float wzf = 0.5f * (float)(z_hi - z_lo) * inz;
                const float uy = ((float)y + 0.5f) * iny;
                float uz[VEC], acc[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    uz[k] = ((float)(z0 + k) + 0.5f) * inz;
                    acc[k] = 0.0f;
                }
                auto near = [&](float py, float pz) {
                    const float gy = fmaxf(fabsf(wrap1<PER>(cyf - py)) - wyf, 0.0f);
                    const float gz = fmaxf(fabsf(wrap1<PER>(czf - pz)) - wzf, 0.0f);
                    return gy <= ext_y && gz <= ext_z;
                };
                if (staged) {
                    for (int cb = 0; cb < count; cb += 32) {
                        const int j = cb + lane;
                        bool ok = false;
                        if (j < count) {
                            const float2 s2 = stage2[j];
                            ok = near(s2.x, s2.y);
                        }
                        unsigned m = __ballot_sync(0xffffffffu, ok);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1;
                            add(stage[cb + src], stage2[cb + src], uy, uz, acc);
                        }
                    }
                } else {
                    // More channel atoms than the stage holds: the same candidates in the same
                    // order, read and transformed from global memory per row group.
                    for (int base = a0; base < a1; base += 32) {
                        const int ai = base + lane;
                        bool ok = false;
                        float4 s = make_float4(0.f, 0.f, 0.f, 1.f);
                        float2 s2 = make_float2(0.f, 0.f);
                        if (ai < a1 && __ldg(A.in.elem + ai) == c) {
                            float px, py, pz;
                            to_frac(F, __ldg(A.in.coords + 3 * ai),
                                    __ldg(A.in.coords + 3 * ai + 1),
                                    __ldg(A.in.coords + 3 * ai + 2), px, py, pz);
                            const float ex = wrap1<PER>(ux - px);
                            s = make_float4(ex * ax, ex * ay, ex * az,
                                            A.in.weight ? __ldg(A.in.weight + ai) : 1.0f);
                            s2 = make_float2(py, pz);
                            ok = fabsf(ex) <= ext_x && near(py, pz);
                        }
                        unsigned m = __ballot_sync(0xffffffffu, ok);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1;
                            const float4 ss = make_float4(
                                __shfl_sync(0xffffffffu, s.x, src),
                                __shfl_sync(0xffffffffu, s.y, src),
                                __shfl_sync(0xffffffffu, s.z, src),
                                __shfl_sync(0xffffffffu, s.w, src));
                            const float2 ss2 = make_float2(__shfl_sync(0xffffffffu, s2.x, src),
                                                           __shfl_sync(0xffffffffu, s2.y, src));
                            add(ss, ss2, uy, uz, acc);
                        }
                    }
                }
                if (v < nvec) store_lane<T, VEC, 0>(out, v, acc);
                y += y_step;
                z0 += z_step;
                if (z0 >= G.nz) {
                    z0 -= G.nz;
                    ++y;
                }
            }
            __syncwarp();
        }
    }

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

template <typename GT>
__device__ __forceinline__ float grad_value(GT v);
template <>
__device__ __forceinline__ float grad_value<float>(float v) { return v; }
template <>
__device__ __forceinline__ float grad_value<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float grad_value<__nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}

// Voxels of one fractional axis within reach ext of fractional position p: first unwrapped
// index and count (whole axis without a cutoff; clamped, or at most n when periodic).
template <int CUT, bool PER>
__device__ __forceinline__ void frac_support(float p, float ext, int n, int &lo, int &cnt)
{
    if (CUT == PG_CUTOFF_NONE) {
        lo = 0;
        cnt = n;
        return;
    }
    int l = (int)fmaxf(ceilf((p - ext) * n - 0.5f - 1e-3f), -1e8f);
    int u = (int)fminf(floorf((p + ext) * n - 0.5f + 1e-3f), 1e8f);
    if (PER) {
        if (u - l + 1 > n) u = l + n - 1;
    } else {
        l = max(l, 0);
        u = min(u, n - 1);
    }
    lo = l;
    cnt = max(u - l + 1, 0);
}

template <typename GT, int CUT, bool PER>
__global__ void __launch_bounds__(256) cell_backward_kernel(const BackwardArgs A)
{
    const Geometry &G = A.geo;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const GT *gout = reinterpret_cast<const GT *>(A.grad_out);
    auto put = [&](int a, float gx, float gy, float gz, float gw) {
        if (A.grad_coords) {
            A.grad_coords[3 * a] = gx;
            A.grad_coords[3 * a + 1] = gy;
            A.grad_coords[3 * a + 2] = gz;
        }
        if (A.grad_weight) A.grad_weight[a] = gw;
    };
    {
        const int first = G.n_mol > 0 ? __ldg(A.in.mol_off) : 0;
        const int last = G.n_mol > 0 ? __ldg(A.in.mol_off + G.n_mol) : 0;
        for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < G.n_atoms;
             a += gridDim.x * blockDim.x)
            if (G.n_mol == 0 || a < first || a >= last) put(a, 0.f, 0.f, 0.f, 0.f);
    }
    const long long plane = (long long)G.ny * G.nz;
    const long long grid_elems = (long long)G.nx * plane;
    const unsigned long long total_warps = (unsigned long long)gridDim.x * warps;
    const int first = G.n_mol > 0 ? max(__ldg(A.in.mol_off), 0) : 0;
    const int last = G.n_mol > 0 ? min(__ldg(A.in.mol_off + G.n_mol), G.n_atoms) : 0;
    const float inx = 1.0f / G.nx, iny = 1.0f / G.ny, inz = 1.0f / G.nz;
    while (true) {
        unsigned long long grab = 0;
        if (lane == 0) grab = atomicAdd(A.sched, 1ull);
        grab = __shfl_sync(0xffffffffu, grab, 0);
        const long long ga = (long long)first + (long long)grab;
        if (G.n_mol == 0 || ga >= last) break;
        const int a = (int)ga;
        int lo = 0, hi = G.n_mol - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(A.in.mol_off + mid) <= a) lo = mid;
            else hi = mid - 1;
        }
        const int b = lo;
        const int a0 = __ldg(A.in.mol_off + b), a1 = __ldg(A.in.mol_off + b + 1);
        const Frame F = load_frame(A.in, b);
        const bool off_ok = (a0 >= 0) && (a0 <= a) && (a < a1) && (a1 <= G.n_atoms);
        const int c = __ldg(A.in.elem + a);
        if (!off_ok || (unsigned)c >= (unsigned)G.C || !F.ok) {
            if (lane == 0) {
                atomicOr(A.err, !off_ok ? PG_DEVERR_OFFSETS
                                        : (F.ok ? PG_DEVERR_ELEMENT : PG_DEVERR_SPACING));
                put(a, 0.f, 0.f, 0.f, 0.f);
            }
            continue;
        }
        const float q = G.q[c], r2 = G.r2[c], rc = G.rcull[c];
        if (PER && lane == 0 && !images_unique<CUT>(F, rc)) atomicOr(A.err, PG_DEVERR_PERIODIC);
        float px, py, pz;
        to_frac(F, __ldg(A.in.coords + 3 * a), __ldg(A.in.coords + 3 * a + 1),
                __ldg(A.in.coords + 3 * a + 2), px, py, pz);
        int ilo, ni, jlo, nj, klo, nk;
        frac_support<CUT, PER>(px, reach<CUT>(F, 0, rc), G.nx, ilo, ni);
        frac_support<CUT, PER>(py, reach<CUT>(F, 1, rc), G.ny, jlo, nj);
        frac_support<CUT, PER>(pz, reach<CUT>(F, 2, rc), G.nz, klo, nk);
        if (PER) {
            ilo = wrap_index(ilo, G.nx);
            jlo = wrap_index(jlo, G.ny);
            klo = wrap_index(klo, G.nz);
        }
        const GT *g = gout + ((long long)b * G.C + c) * grid_elems;
        const int njk = nj * nk;
        const long long total = (long long)ni * njk;
        float sx = 0.f, sy = 0.f, sz = 0.f, sw = 0.f;
        for (long long f = lane; f < total; f += 32) {
            const int fi = (int)(f / njk);
            const int rem = (int)(f - (long long)fi * njk);
            const int fj = rem / nk, fk = rem - (rem / nk) * nk;
            int i = ilo + fi, j = jlo + fj, k = klo + fk;
            if (PER) {
                if (i >= G.nx) i -= G.nx;
                if (j >= G.ny) j -= G.ny;
                if (k >= G.nz) k -= G.nz;
            }
            const float ex = wrap1<PER>(((float)i + 0.5f) * inx - px);
            const float ey = wrap1<PER>(((float)j + 0.5f) * iny - py);
            const float ez = wrap1<PER>(((float)k + 0.5f) * inz - pz);
            const float dx = fmaf(ex, F.M[0], fmaf(ey, F.M[3], ez * F.M[6]));
            const float dy = fmaf(ex, F.M[1], fmaf(ey, F.M[4], ez * F.M[7]));
            const float dz = fmaf(ex, F.M[2], fmaf(ey, F.M[5], ez * F.M[8]));
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            bool in = true;
            if (CUT == PG_CUTOFF_SPHERE) in = d2 <= r2;
            else if (CUT == PG_CUTOFF_BOX) in = fmaxf(dx * dx, fmaxf(dy * dy, dz * dz)) <= r2;
            if (!in) continue;
            const float t = grad_value<GT>(g[(long long)i * plane + (long long)j * G.nz + k]) *
                            ex2_approx(-q * d2);
            sx = fmaf(t, dx, sx);
            sy = fmaf(t, dy, sy);
            sz = fmaf(t, dz, sz);
            sw += t;
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
            const float s = w * G.inv_s2[c];
            put(a, sx * s, sy * s, sz * s, sw);
        }
    }
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

template <typename T, int VEC>
const void *pick_cell_shape(int cutoff, int periodic)
{
    if (periodic)
        return cutoff == PG_CUTOFF_BOX ? (const void *)cell_kernel<T, VEC, PG_CUTOFF_BOX, true>
                                       : (const void *)cell_kernel<T, VEC, PG_CUTOFF_SPHERE, true>;
    if (cutoff == PG_CUTOFF_SPHERE) return (const void *)cell_kernel<T, VEC, PG_CUTOFF_SPHERE, false>;
    if (cutoff == PG_CUTOFF_BOX) return (const void *)cell_kernel<T, VEC, PG_CUTOFF_BOX, false>;
    return (const void *)cell_kernel<T, VEC, PG_CUTOFF_NONE, false>;
}

template <typename GT>
const void *pick_cell_backward(int cutoff, int periodic)
{
    if (periodic)
        return cutoff == PG_CUTOFF_BOX
                   ? (const void *)cell_backward_kernel<GT, PG_CUTOFF_BOX, true>
                   : (const void *)cell_backward_kernel<GT, PG_CUTOFF_SPHERE, true>;
    if (cutoff == PG_CUTOFF_SPHERE)
        return (const void *)cell_backward_kernel<GT, PG_CUTOFF_SPHERE, false>;
    if (cutoff == PG_CUTOFF_BOX) return (const void *)cell_backward_kernel<GT, PG_CUTOFF_BOX, false>;
    return (const void *)cell_backward_kernel<GT, PG_CUTOFF_NONE, false>;
}

}  // namespace

cudaError_t cell_plan(const DirectArgs &a, int dtype, int vec_ok, const pg_tuning &t,
                      int sm_count, KernelLaunch *kl)
{
    if (a.geo.periodic && a.geo.cutoff == PG_CUTOFF_NONE) return cudaErrorNotSupported;
    const int cut = a.geo.cutoff, per = a.geo.periodic;
    const void *f;
    if (dtype == PG_F32)
        f = vec_ok ? pick_cell_shape<float, 4>(cut, per) : pick_cell_shape<float, 1>(cut, per);
    else if (dtype == PG_F16)
        f = vec_ok ? pick_cell_shape<__half, 8>(cut, per) : pick_cell_shape<__half, 1>(cut, per);
    else
        f = vec_ok ? pick_cell_shape<__nv_bfloat16, 8>(cut, per)
                   : pick_cell_shape<__nv_bfloat16, 1>(cut, per);
    const int threads = kCellThreads;
    const size_t smem = (size_t)(threads / 32) * kCellWarpBytes;
    int per_sm = 0;
    cudaError_t e = occupancy(f, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < per_sm) per_sm = t.blocks_per_sm;
    const long long items = (long long)a.geo.n_mol * a.geo.C * a.geo.nx;
    const long long need = (items + threads / 32 - 1) / (threads / 32);
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kl->func = f;
    kl->grid = dim3((unsigned)blocks);
    kl->block = dim3((unsigned)threads);
    kl->smem = smem;
    set_args(kl, a);
    return cudaSuccess;
}

cudaError_t cell_backward_plan(const BackwardArgs &a, int grad_dtype, int sm_count,
                               KernelLaunch *kl)
{
    if (a.geo.periodic && a.geo.cutoff == PG_CUTOFF_NONE) return cudaErrorNotSupported;
    const int cut = a.geo.cutoff, per = a.geo.periodic;
    const void *f = grad_dtype == PG_F32   ? pick_cell_backward<float>(cut, per)
                    : grad_dtype == PG_F16 ? pick_cell_backward<__half>(cut, per)
                                           : pick_cell_backward<__nv_bfloat16>(cut, per);
    const int threads = 256;
    int per_sm = 0;
    cudaError_t e = occupancy(f, threads, 0, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
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
