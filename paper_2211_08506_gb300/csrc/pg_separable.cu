// Separable tcgen05 contraction for batched Gaussian-density voxelization (sm_103a).
//
// With a per-axis cutoff (none, or the box |d_axis| <= r_c) the point-sampled Gaussian of
// Sec. III-A factors per axis, which is the separability the paper exploits with per-axis
// tables (Sec. III-A after Eq. 5; Sec. VI-A).  For one molecule the grid is then a matrix
// product over atoms a:
//
//     G[(c,x), (y,z)] = sum_a A[(c,x), a] * B[a, (y,z)],
//     A[(c,x), a] = [elem a == c] g_x(a, x),   B[a, (y,z)] = g_y(a, y) g_z(a, z),
//     g_axis(a, i) = chi_axis(d) 2^(-q_c d^2),  d = voxel centre - atom (nearest image),
//
// M = C nx rows, N = ny nz columns (the output [C][nx][ny][nz] is this matrix, row-major),
// K = the molecule's atoms.  The operands are generated in shared memory and never touch
// HBM: A is rounded once from FP32 g_x, B once from the FP32 product g_y g_z (BF16, round
// to nearest even); the tensor cores accumulate in FP32 in tensor memory.
//
// One CTA of 128 threads owns one 128-row M tile of one molecule at a time (persistent loop
// over (molecule, M tile) items).  Thread t is accumulator row t (TMEM lane t).  Per item the
// CTA builds per-axis tables and the A tile once, then for each N tile of n_tile columns:
//   builds B (n_tile x 32 atoms, BF16) -> one thread issues two K=16 tcgen05.mma into a TMEM
//   accumulator of n_tile FP32 columns and commits to an mbarrier -> every thread loads its
//   row with tcgen05.ld, converts to the output type and writes it to a padded shared
//   staging row -> each warp then writes its 32 rows to global memory with coalesced
//   16-byte stores (one bulk copy per row was measured to be limited by the rate at which
//   the copy engine accepts requests).
// Molecules with more than 32 atoms loop over 32-atom K chunks, accumulating in TMEM.
// Both operands use the K-major, no-swizzle canonical layout: 8-row x 16-byte core matrices,
// 128 bytes apart along K (leading byte offset) and 512 bytes apart along M/N (stride byte
// offset).
//
// Every mbarrier wait is bounded; on expiry the kernel sets PG_DEVERR_TIMEOUT and returns.
// Before a CTA frees its tensor memory, the thread that issued its MMAs commits once more to a
// drain barrier and waits for it (bounded), so no MMA can still be writing the columns; if
// that never arrives the columns stay allocated and PG_DEVERR_TMEM_HELD is set.
#include <cstdlib>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include <cmath>

#include "pg_internal.h"

namespace pgi {

namespace {

constexpr int kKC = 32;         // atoms per K chunk (two K=16 MMA steps)
constexpr int kTab = 36;        // floats per table row: 32 atoms + 4 pad (conflict-free reads)
constexpr int kTabX = 33;       // g_x rows: A-tile threads read one atom across 32 rows
constexpr int kRows = 128;      // M tile = CTA threads = TMEM lanes
constexpr unsigned kWaitLimit = 1u << 24;  // polls of one mbarrier wait, at most; and at most
                                           // SeparableArgs::wait_ns of wall time

struct SepLayout {
    int bar, drain, tmem, atoms, a, b, gy, gz, stage, stage_stride, total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SepLayout sep_layout(int ny, int nz, int n_tile, int esz)
{
    SepLayout L;
    int o = 0;
    L.bar = o;
    o += 8;
    L.drain = o;  // the final commit before tensor memory is freed
    o += 8;
    L.tmem = o;
    o += 8;
    o = align_up(o, 128);
    L.atoms = o;
    o += kKC * 2 * 16;
    o = align_up(o, 1024);
    L.a = o;
    o += kRows * kKC * 2;
    o = align_up(o, 1024);
    L.b = o;
    o += n_tile * kKC * 2;
    o = align_up(o, 128);
    L.gy = o;
    o += ny * kTab * 4;
    o = align_up(o, 128);
    L.gz = o;
    o += nz * kTab * 4;
    o = align_up(o, 128);
    L.stage = o;
    L.stage_stride = n_tile * esz + 16;
    o += kRows * L.stage_stride;
    L.total = align_up(o, 128);
    return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

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

// ---- mbarrier, tcgen05 and bulk-copy wrappers (inline PTX) ----

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// As mbar_try_wait, but a thread whose phase has not completed is suspended by the hardware
// until it completes or about kSuspendNs have passed, instead of polling: the waiting warps
// issue almost nothing and wake as soon as the phase completes.
constexpr unsigned kSuspendNs = 2000;
__device__ __forceinline__ bool mbar_wait_suspend(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(kSuspendNs)
        : "memory");
    return ok != 0u;
}

// Bounded wait, at most kDrainNs, for phase 0 of the drain barrier: the final tcgen05.commit a
// CTA issues before it frees its tensor memory, which arrives once every MMA the committing
// thread issued has completed (at once when none is outstanding).
constexpr unsigned long long kDrainNs = 2000000000ull;
__device__ __forceinline__ bool drain_wait(uint32_t bar)
{
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        if (mbar_wait_suspend(bar, 0u)) return true;
        if ((it & 3u) == 3u && global_ns() - t0 > kDrainNs) return false;
    }
    return false;
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     dst_smem),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16_f32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// TMA tensor store of one box from shared memory; coordinates innermost first.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y,
                                             int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(src), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(src), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void bulk_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
    return d;                // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    return (1u << 4)                        // D format: F32
           | (1u << 7)                      // A format: BF16
           | (1u << 10)                     // B format: BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(kRows >> 4) << 24);  // M / 16
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Per-axis factor: chi_axis(d) 2^(-q d^2) for the point sample, or chi_axis(d) times the
// voxel's erf integral along the axis (spacing h, k = 1 / (sqrt(2) sigma)) for the
// voxel-integrated form of Sec. III-A.
template <int CUT, int FORM>
__device__ __forceinline__ float axis_factor(float d, float q, float r2, float h, float k)
{
    const float d2 = d * d;
    const float v = FORM ? erf_axis(d, h, k) : ex2_approx(-q * d2);
    return (CUT == PG_CUTOFF_BOX && d2 > r2) ? 0.0f : v;
}

template <typename T>
__device__ __forceinline__ void store_row_chunk(unsigned char *dst, const uint32_t (&r)[32]);

template <>
__device__ __forceinline__ void store_row_chunk<float>(unsigned char *dst, const uint32_t (&r)[32])
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
}

template <>
__device__ __forceinline__ void store_row_chunk<__half>(unsigned char *dst, const uint32_t (&r)[32])
{
    uint32_t p[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        __half2 h = __floats2half2_rn(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        p[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = make_uint4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
}

template <>
__device__ __forceinline__ void store_row_chunk<__nv_bfloat16>(unsigned char *dst,
                                                               const uint32_t (&r)[32])
{
    uint32_t p[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        p[i] = pack_bf16x2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = make_uint4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
}

// Staging of 32 accumulator columns [cb, cb+32) of row `lane` for a TMA store box of
// 32 rows x 128 bytes with the 128-byte swizzle: 16-byte chunk j of a row sits at chunk
// j ^ (row % 8), so the 8 rows sharing a bank group write to 8 different chunks.
template <typename T>
__device__ __forceinline__ void stage_swizzled(unsigned char *warp_stage, int lane, int cb,
                                               const uint32_t (&r)[32])
{
    constexpr int chunks = 32 * (int)sizeof(T) / 16;  // 16-byte chunks in 32 columns
    uint32_t p[4 * chunks];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < 32; ++i) p[i] = r[i];
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if constexpr (std::is_same<T, __half>::value) {
                __half2 h = __floats2half2_rn(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                p[i] = *reinterpret_cast<uint32_t *>(&h);
            } else {
                p[i] = pack_bf16x2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
            }
        }
    }
    const int c0 = cb * (int)sizeof(T) / 16;  // first 16-byte chunk of this column block
#pragma unroll
    for (int i = 0; i < chunks; ++i) {
        const int c = c0 + i;
        const int slab = c >> 3, j = c & 7;
        *reinterpret_cast<uint4 *>(warp_stage + slab * 4096 + lane * 128 + ((j ^ (lane & 7)) << 4)) =
            make_uint4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
    }
}

// Coalesced write-out of one warp's 32 staged rows: row segment bytes are spread over lanes
// 16 bytes each (several rows per step when a segment is shorter than 512 bytes), so every
// store instruction covers whole 32-byte sectors.  Rows at or past M and columns at or past
// N are skipped.  `stage` is the warp's first staging row, `stride` the staging row pitch.
template <typename T>
__device__ __forceinline__ void store_warp_rows(T *out, const unsigned char *stage, int stride,
                                                int row0, int M, long long row_base, int N,
                                                int n0, int n_tile, int lane)
{
    const int seg16 = n_tile * (int)sizeof(T) / 16;  // 16-byte pieces per row segment
    const int cols = min(n_tile, N - n0);
    const int valid16 = cols * (int)sizeof(T) / 16;
    constexpr int per16 = 16 / (int)sizeof(T);      // elements per 16-byte piece
    if (seg16 <= 32) {
        const int rows_per_step = 32 / seg16;
        const int rr = lane / seg16, c16 = lane - (lane / seg16) * seg16;
        for (int r = rr; r < 32; r += rows_per_step) {
            const int R = row0 + r;
            if (R < M && c16 < valid16) {
                const uint4 v = *reinterpret_cast<const uint4 *>(stage + r * stride + c16 * 16);
                __stcs(reinterpret_cast<uint4 *>(out + (row_base + R) * (long long)N + n0 +
                                                 c16 * per16),
                       v);
            }
        }
    } else {
        for (int r = 0; r < 32; ++r) {
            const int R = row0 + r;
            if (R >= M) break;
            for (int c16 = lane; c16 < valid16; c16 += 32) {
                const uint4 v = *reinterpret_cast<const uint4 *>(stage + r * stride + c16 * 16);
                __stcs(reinterpret_cast<uint4 *>(out + (row_base + R) * (long long)N + n0 +
                                                 c16 * per16),
                       v);
            }
        }
    }
}

template <typename T, int CUT, bool PER, int FORM>
__global__ void __launch_bounds__(128, 1) separable_kernel(const SeparableArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const Geometry &G = A.geo;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int n_tile = A.n_tile;
    const SepLayout L = sep_layout(G.ny, G.nz, n_tile, (int)sizeof(T));
    float4 *atom_pos = reinterpret_cast<float4 *>(smem + L.atoms);  // {x, y, z, q}
    float4 *atom_aux = atom_pos + kKC;                               // {r2, elem, -, -}
    unsigned char *sa = smem + L.a;
    unsigned char *sb = smem + L.b;
    float *tgy = reinterpret_cast<float *>(smem + L.gy);
    float *tgz = reinterpret_cast<float *>(smem + L.gz);
    unsigned char *srow = smem + L.stage + tid * L.stage_stride;
    const uint32_t bar = smem_u32(smem + L.bar);
    const uint32_t drain = smem_u32(smem + L.drain);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
    volatile uint32_t *drained = tmem_slot + 1;  // the drain barrier arrived

    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(drain, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), (uint32_t)n_tile);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = instr_desc(n_tile);
    const uint32_t sa_addr = smem_u32(sa), sb_addr = smem_u32(sb);
    uint32_t phase = 0;
    bool timed_out = false;

    const int M = G.C * G.nx;
    const int N = G.ny * G.nz;
    const int n_chunks = (N + n_tile - 1) / n_tile;
    const long long n_items = (long long)G.n_mol * A.m_tiles;
    T *out = reinterpret_cast<T *>(A.out);

    for (long long item = blockIdx.x; item < n_items && !timed_out; item += gridDim.x) {
        const int b = (int)(item / A.m_tiles);
        const int m0 = (int)(item % A.m_tiles) * kRows;
        int a0 = __ldg(A.in.mol_off + b), a1 = __ldg(A.in.mol_off + b + 1);
        const float ox = __ldg(A.in.origin + 3 * b), oy = __ldg(A.in.origin + 3 * b + 1),
                    oz = __ldg(A.in.origin + 3 * b + 2);
        const float hx = __ldg(A.in.spacing + 3 * b), hy = __ldg(A.in.spacing + 3 * b + 1),
                    hz = __ldg(A.in.spacing + 3 * b + 2);
        const bool off_ok = (a0 >= 0) && (a0 <= a1) && (a1 <= G.n_atoms);
        const bool sp_ok = (hx > 0.0f) && (hy > 0.0f) && (hz > 0.0f) && (hx < INFINITY) &&
                           (hy < INFINITY) && (hz < INFINITY);
        if (!off_ok || !sp_ok) {
            if (tid == 0 && m0 == 0)
                atomicOr(A.err, (off_ok ? 0u : PG_DEVERR_OFFSETS) | (sp_ok ? 0u : PG_DEVERR_SPACING));
            a0 = a1 = 0;
        }
        const float Lx = G.nx * hx, Ly = G.ny * hy, Lz = G.nz * hz;
        const float iLx = 1.0f / Lx, iLy = 1.0f / Ly, iLz = 1.0f / Lz;
        const int n_atoms = a1 - a0;
        const int n_kc = n_atoms > 0 ? (n_atoms + kKC - 1) / kKC : 1;
        const int R = m0 + tid;
        const bool row_ok = R < M;
        const int row_c = row_ok ? R / G.nx : -2;
        const int row_x = row_ok ? R - (R / G.nx) * G.nx : 0;
        const float vx = fmaf((float)row_x + 0.5f, hx, ox);

        for (int nc = 0; nc < n_chunks && !timed_out; ++nc) {
            const int n0 = nc * n_tile;
            for (int kc = 0; kc < n_kc && !timed_out; ++kc) {
                if (n_kc > 1 || nc == 0) {
                    // Atoms of this K chunk, their per-axis tables and the A tile.
                    if (tid < kKC) {
                        const int ai = a0 + kc * kKC + tid;
                        float4 pos = make_float4(0.f, 0.f, 0.f, 0.f);
                        float4 aux = make_float4(0.f, -1.f, 0.f, 0.f);
                        if (ai < a1) {
                            const int e = __ldg(A.in.elem + ai);
                            if ((unsigned)e < (unsigned)G.C) {
                                pos = make_float4(__ldg(A.in.coords + 3 * ai),
                                                  __ldg(A.in.coords + 3 * ai + 1),
                                                  __ldg(A.in.coords + 3 * ai + 2), G.q[e]);
                                aux = make_float4(G.r2[e], (float)e, G.kerf[e],
                                                  A.in.weight ? __ldg(A.in.weight + ai) : 1.0f);
                            } else if (m0 == 0) {
                                atomicOr(A.err, PG_DEVERR_ELEMENT);
                            }
                        }
                        atom_pos[tid] = pos;
                        atom_aux[tid] = aux;
                    }
                    __syncthreads();
                    for (int i = tid; i < G.ny * kKC; i += kRows) {
                        const int y = i / kKC, j = i - (i / kKC) * kKC;
                        const float4 p = atom_pos[j];
                        float v = 0.0f;
                        if (atom_aux[j].y >= 0.0f) {
                            float d = fmaf((float)y + 0.5f, hy, oy) - p.y;
                            if (PER) d = wrap(d, Ly, iLy);
                            v = axis_factor<CUT, FORM>(d, p.w, atom_aux[j].x, hy,
                                                 atom_aux[j].z);
                        }
                        tgy[y * kTab + j] = v;
                    }
                    for (int i = tid; i < G.nz * kKC; i += kRows) {
                        const int z = i / kKC, j = i - (i / kKC) * kKC;
                        const float4 p = atom_pos[j];
                        float v = 0.0f;
                        if (atom_aux[j].y >= 0.0f) {
                            float d = fmaf((float)z + 0.5f, hz, oz) - p.z;
                            if (PER) d = wrap(d, Lz, iLz);
                            v = axis_factor<CUT, FORM>(d, p.w, atom_aux[j].x, hz,
                                                 atom_aux[j].z);
                        }
                        tgz[z * kTab + j] = v;
                    }
                    // A row `tid`: [elem a == c] w_a g_x(a, x), 4 core-matrix chunks of 8 atoms.
#pragma unroll
                    for (int jg = 0; jg < kKC / 8; ++jg) {
                        float v[8];
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const int j = jg * 8 + t;
                            const float4 p = atom_pos[j];
                            const float4 aux = atom_aux[j];
                            v[t] = 0.0f;
                            if (row_ok && (int)aux.y == row_c) {
                                float d = vx - p.x;
                                if (PER) d = wrap(d, Lx, iLx);
                                v[t] = aux.w * axis_factor<CUT, FORM>(d, p.w, aux.x, hx, aux.z);
                            }
                        }
                        const uint4 w = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                                   pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
                        *reinterpret_cast<uint4 *>(sa + (tid >> 3) * 512 + jg * 128 +
                                                   (tid & 7) * 16) = w;
                    }
                    __syncthreads();
                }
                // B tile: column n = n0 + nl of B is (y, z); 16-byte chunk qi holds atoms
                // kg*8 .. kg*8+7 of column nl at byte qi*16 of the canonical layout.
                for (int qi = tid; qi < n_tile * (kKC / 8); qi += kRows) {
                    const int nl = (qi >> 5) * 8 + (qi & 7);
                    const int kg = (qi >> 3) & 3;
                    const int n = n0 + nl;
                    uint4 w = make_uint4(0u, 0u, 0u, 0u);
                    if (n < N) {
                        const int y = n / G.nz, z = n - (n / G.nz) * G.nz;
                        const float4 *gy4 = reinterpret_cast<const float4 *>(tgy + y * kTab + kg * 8);
                        const float4 *gz4 = reinterpret_cast<const float4 *>(tgz + z * kTab + kg * 8);
                        const float4 y0 = gy4[0], y1 = gy4[1], z0 = gz4[0], z1 = gz4[1];
                        w = make_uint4(pack_bf16x2(y0.x * z0.x, y0.y * z0.y),
                                       pack_bf16x2(y0.z * z0.z, y0.w * z0.w),
                                       pack_bf16x2(y1.x * z1.x, y1.y * z1.y),
                                       pack_bf16x2(y1.z * z1.z, y1.w * z1.w));
                    }
                    *reinterpret_cast<uint4 *>(sb + qi * 16) = w;
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                if (tid == 0 && !A.stall) {
                    tc_fence_after();
#pragma unroll
                    for (int s = 0; s < kKC / 16; ++s) {
                        const uint64_t ad = smem_desc(sa_addr + s * 256, 128, 512);
                        const uint64_t bd = smem_desc(sb_addr + s * 256, 128, 512);
                        mma_bf16_f32(tmem, ad, bd, idesc, (kc > 0 || s > 0) ? 1u : 0u);
                    }
                    mma_commit(bar);
                }
                bool done = false;
                const unsigned long long t0 = global_ns();
                for (unsigned it = 0; it < kWaitLimit && !done; ++it) {
                    done = mbar_try_wait(bar, phase);
                    if (!done && (it & 63u) == 63u && global_ns() - t0 > A.wait_ns) break;
                }
                phase ^= 1u;
                timed_out = __syncthreads_or(!done) != 0;
                tc_fence_after();
            }
            if (timed_out) break;
            // Epilogue: TMEM row -> registers -> output type -> staging row, then the warp
            // writes its 32 rows out with coalesced stores.
            for (int cb = 0; cb < n_tile; cb += 32) {
                uint32_t r[32];
                tmem_ld32(tmem_row + cb, r);
                tmem_ld_wait();
                store_row_chunk<T>(srow + cb * (int)sizeof(T), r);
            }
            tc_fence_before();
            __syncwarp();
            store_warp_rows<T>(out, smem + L.stage + warp * 32 * L.stage_stride, L.stage_stride,
                               m0 + warp * 32, M, (long long)b * M, N, n0, n_tile, tid & 31);
            __syncwarp();
        }
    }
    if (timed_out && tid == 0) atomicOr(A.err, PG_DEVERR_TIMEOUT);
    // The tensor memory is freed only once every MMA of the CTA has completed: thread 0, which
    // issued them, commits to the drain barrier and waits for it.  If it never arrives, the
    // columns stay allocated rather than be freed under an MMA that may still write them.
    if (tid == 0) {
        mma_commit(drain);
        *drained = drain_wait(drain) ? 1u : 0u;
        if (!*drained) atomicOr(A.err, PG_DEVERR_TIMEOUT | PG_DEVERR_TMEM_HELD);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && *drained) {
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)n_tile);
    }
}

// ---------------------------------------------------------------------------------------
// Pipelined variant.  Three warp roles overlap the work of consecutive N tiles:
//   warps 0-3  epilogue: thread t owns accumulator row t; drains one of two TMEM accumulators
//              (tcgen05.ld -> output type -> staging row -> coalesced stores) while the other
//              fills;
//   warps 4-7 (4-19 for packed tiles) producer: per item builds atoms and per-axis tables,
//              then for every step
//              (N tile, K chunk) writes the B operand into one of two shared-memory stages.
//              The A operand does not depend on the N tile: when the item's K chunks fit the
//              resident slots it is written once per K chunk into a slot of its own, else
//              into the stage with B at every step;
//   warp 8 (20) MMA: one thread issues the tcgen05.mma pair of each step and commits to the
//              stage's "empty" barrier and, after a tile's last K chunk, to the accumulator's
//              "full" barrier.
// All three walk the same (item, N tile, K chunk) sequence, so every handoff is a
// full/empty mbarrier pair with phase parities derived from a step counter.  Waits are
// bounded: a role that gives up raises a shared flag the others poll, then all drain and
// the CTA frees its tensor memory.
constexpr int kPipeStages = 2;
// Producer warps: 16 for packed tiles (molecules of a few dozen atoms, where building the
// operands is the critical path and each producer warp waits on long dependent chains) with
// 2-byte outputs, 8 with FP32 outputs (whose epilogue needs more registers than a 21-warp CTA
// leaves), else 4 so that two CTAs fit an SM.
__host__ __device__ constexpr int pipe_prod_warps(bool pack, int esz)
{
    return pack ? (esz == 4 ? 8 : 16) : 4;
}
// Threads of the pipelined kernel: epilogue, producers, MMA issuer.
__host__ __device__ constexpr int pipe_threads(bool pack, int esz)
{
    return 128 + 32 * pipe_prod_warps(pack, esz) + 32;
}

struct PipeLayout {
    int bars, tmem, flag, tile, atoms, stage0, stage_bytes, a_bytes, aslots, gx, gy, gz, out,
        out_stride, total;
};

__host__ __device__ inline PipeLayout pipe_layout(int nx, int ny, int nz, int n_tile, int esz,
                                               int kslots, int pack)
{
    PipeLayout L;
    int o = 0;
    L.bars = o;  // b_full[2], b_empty[2], acc_full[2], acc_empty[2], drain
    o += 9 * 8;
    L.tmem = o;
    o += 8;
    L.flag = o;  // {a role gave up, the drain arrived}
    o += 8;
    o = align_up(o, 16);
    // Packed tiles: the tile's CSR offsets (pack + 1) and each molecule's origin and spacing.
    L.tile = o;
    o += pack > 0 ? (pack + 1) * 4 + pack * 24 : 0;
    o = align_up(o, 128);
    L.atoms = o;
    o += kKC * 4 * 16;  // the K chunk being built: pos, aux, geometry (2)
    o = align_up(o, 1024);
    L.a_bytes = kRows * kKC * 2;
    L.stage_bytes = align_up(L.a_bytes + n_tile * kKC * 2, 1024);
    L.stage0 = o;
    o += kPipeStages * L.stage_bytes;
    L.aslots = o;  // resident A tiles, one per K chunk slot
    o += kslots * L.a_bytes;
    L.gx = o;
    o += nx * kTabX * 4;  // read only while the chunk's A tile is built
    o = align_up(o, 128);
    L.gy = o;
    o += kslots * ny * kTab * 4;
    o = align_up(o, 128);
    L.gz = o;
    o += kslots * nz * kTab * 4;
    o = align_up(o, 1024);
    L.out = o;
    L.out_stride = (n_tile * esz / 128) * 4096;  // per warp: slabs of 32 rows x 128 bytes
    o += 4 * L.out_stride;
    L.total = align_up(o, 1024);
    return L;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

template <int NPROD>
__device__ __forceinline__ void producer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory");
}

// True for every producer thread iff it is true for all of them (named barrier 1, all
// producer threads), so the producers always take the same branch after a bounded wait.
template <int NPROD>
__device__ __forceinline__ bool producers_all(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NPROD)
        : "memory");
    return r != 0u;
}

// Bounded wait on `parity`; false if it gave up or another role already did.
__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity, volatile int *flag,
                                          unsigned long long wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        if (mbar_wait_suspend(bar, parity)) return true;
        if ((it & 3u) == 3u && (*flag || global_ns() - t0 > wait_ns)) break;
    }
    *flag = 1;
    return false;
}

// One lane of the warp polls the barrier; __syncwarp then orders the other lanes after its
// acquire.  Returns the same value on every lane.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *flag,
                                          unsigned long long wait_ns)
{
    bool got = true;
    if ((threadIdx.x & 31) == 0) got = pipe_wait(bar, parity, flag, wait_ns);
    return __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
}

// Every lane's prior shared-memory writes (and tcgen05 loads, fenced by the caller) are
// ordered before one arrival made by lane 0.
__device__ __forceinline__ void warp_arrive(uint32_t bar)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

struct PipeItem {
    int b, nb, m0, a0, a1, n_kc;  // first molecule, molecules in the tile (packed), rows
    float ox, oy, oz, hx, hy, hz;
    unsigned bad;  // PG_DEVERR_* bits of this molecule (its grid is then all zeros)
};

// Packed tiles (A.pack > 0): item i holds molecules i*pack .. i*pack + nb - 1, whose rows
// (molecule-major, C nx each) fill the 128-row tile and whose atoms are one contiguous CSR
// range.  If any of them has bad offsets the whole tile is left without atoms (its grids
// are written as zeros) and flagged; a molecule with bad spacing loses only its own atoms.
__device__ __forceinline__ PipeItem pipe_item_packed(const SeparableArgs &A, long long item)
{
    const Geometry &G = A.geo;
    PipeItem it;
    it.b = (int)(item * A.pack);
    it.nb = min(A.pack, G.n_mol - it.b);
    it.m0 = 0;
    it.ox = it.oy = it.oz = 0.0f;
    it.hx = it.hy = it.hz = 1.0f;
    it.a0 = __ldg(A.in.mol_off + it.b);
    it.a1 = __ldg(A.in.mol_off + it.b + it.nb);
    bool off_ok = (it.a0 >= 0) && (it.a1 <= G.n_atoms);
    for (int k = 0; k < it.nb && off_ok; ++k)
        off_ok = __ldg(A.in.mol_off + it.b + k) <= __ldg(A.in.mol_off + it.b + k + 1);
    it.bad = off_ok ? 0u : PG_DEVERR_OFFSETS;
    if (it.bad) it.a0 = it.a1 = 0;
    const int n = it.a1 - it.a0;
    it.n_kc = n > 0 ? (n + kKC - 1) / kKC : 1;
    return it;
}

template <bool PACK>
__device__ __forceinline__ PipeItem pipe_item(const SeparableArgs &A, long long item)
{
    if (PACK) return pipe_item_packed(A, item);
    const Geometry &G = A.geo;
    PipeItem it;
    it.b = (int)(item / A.m_tiles);
    it.nb = 1;
    it.m0 = (int)(item % A.m_tiles) * kRows;
    it.a0 = __ldg(A.in.mol_off + it.b);
    it.a1 = __ldg(A.in.mol_off + it.b + 1);
    it.ox = __ldg(A.in.origin + 3 * it.b);
    it.oy = __ldg(A.in.origin + 3 * it.b + 1);
    it.oz = __ldg(A.in.origin + 3 * it.b + 2);
    it.hx = __ldg(A.in.spacing + 3 * it.b);
    it.hy = __ldg(A.in.spacing + 3 * it.b + 1);
    it.hz = __ldg(A.in.spacing + 3 * it.b + 2);
    const bool off_ok = (it.a0 >= 0) && (it.a0 <= it.a1) && (it.a1 <= G.n_atoms);
    const bool sp_ok = (it.hx > 0.0f) && (it.hy > 0.0f) && (it.hz > 0.0f) &&
                       (it.hx < INFINITY) && (it.hy < INFINITY) && (it.hz < INFINITY);
    it.bad = (off_ok ? 0u : PG_DEVERR_OFFSETS) | (sp_ok ? 0u : PG_DEVERR_SPACING);
    if (it.bad) it.a0 = it.a1 = 0;
    const int n = it.a1 - it.a0;
    it.n_kc = n > 0 ? (n + kKC - 1) / kKC : 1;
    return it;
}

template <typename T, int CUT, bool PER, int FORM, bool PACK>
__global__ void __launch_bounds__(pipe_threads(PACK, (int)sizeof(T)), PACK ? 1 : 2)
    separable_pipe_kernel(const __grid_constant__ SeparableArgs A)
{
    constexpr int kProdWarps = pipe_prod_warps(PACK, (int)sizeof(T));
    constexpr int kProducers = 32 * kProdWarps;
    extern __shared__ __align__(1024) unsigned char smem[];
    const Geometry &G = A.geo;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int n_tile = A.n_tile;
    const PipeLayout L = pipe_layout(G.nx, G.ny, G.nz, n_tile, (int)sizeof(T), A.kslots,
                                     PACK ? A.pack : 0);
    const uint32_t bars = smem_u32(smem + L.bars);
    auto b_full = [&](int s) { return bars + 8u * s; };
    auto b_empty = [&](int s) { return bars + 8u * (2 + s); };
    auto acc_full = [&](int s) { return bars + 8u * (4 + s); };
    auto acc_empty = [&](int s) { return bars + 8u * (6 + s); };
    const uint32_t drain = bars + 8u * 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L.tmem);
    volatile int *flag = reinterpret_cast<volatile int *>(smem + L.flag);
    volatile int *drained = flag + 1;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(b_full(s), kProdWarps);  // one elected lane per producer warp
            mbar_init(b_empty(s), 1);    // tcgen05.commit
            mbar_init(acc_full(s), 1);   // tcgen05.commit
            mbar_init(acc_empty(s), 4);  // one elected lane per epilogue warp
        }
        mbar_init(drain, 1);             // tcgen05.commit before the tensor memory is freed
        *flag = 0;
        *drained = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), (uint32_t)(2 * n_tile));
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int M = G.C * G.nx;
    const int N = G.ny * G.nz;
    const int n_chunks = (N + n_tile - 1) / n_tile;
    const long long n_items = PACK ? ((long long)G.n_mol + A.pack - 1) / A.pack
                                         : (long long)G.n_mol * A.m_tiles;

    if (warp >= 4 && warp < 4 + kProdWarps) {
        // ------------------------------------------------------------------ producer
        const int p = tid - 128;  // 0 .. kProducers - 1
        // A-tile work: producer p builds row p % 128 of the tile, its kAGroups atom groups of 8
        // starting at group (p / 128) * kAGroups.
        constexpr int kAGroups = (kKC / 8) / (kProducers / kRows);
        const int arow = p & (kRows - 1);
        const int ag0 = (p / kRows) * kAGroups;
        // Per atom of the K chunk: {x, y, z, q}, {r2, elem, k_erf, molecule within the tile},
        // and its molecule's grid geometry {ox, oy, oz, hx} with {hy, hz, weight, -}.  The
        // weight scales the atom's A entries (its g_x), exactly 1 for unweighted grids.
        // The g_y, g_z tables and the A tiles of up to A.kslots K chunks stay resident for a
        // tile, so a tile with several chunks builds each once instead of once per N chunk.
        // The atoms and g_x are only read while a chunk's A tile is built, in the step that
        // builds its tables, so one copy serves every slot.
        float4 *const atoms0 = reinterpret_cast<float4 *>(smem + L.atoms);
        float *const tgx0 = reinterpret_cast<float *>(smem + L.gx);
        float *const tgy0 = reinterpret_cast<float *>(smem + L.gy);
        float *const tgz0 = reinterpret_cast<float *>(smem + L.gz);
        constexpr int kColStep = kProducers / 4;  // B columns between a producer's chunks
        const int dyc = kColStep / G.nz, dzc = kColStep - (kColStep / G.nz) * G.nz;
        unsigned step = 0;
        bool ok = true;
        for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const PipeItem it = pipe_item<PACK>(A, item);
            if (it.bad && p == 0 && it.m0 == 0) atomicOr(A.err, it.bad);
            // This producer's A row: molecule lm of the tile (0 unless packed), channel, x.
            const int R = it.m0 + arow;
            const int lm = PACK ? R / M : 0;
            const int r = R - lm * M;
            const bool row_ok = PACK ? lm < it.nb : R < M;
            const int row_c = row_ok ? r / G.nx : -2;
            const int row_x = row_ok ? r - (r / G.nx) * G.nx : 0;
            // The row's voxel-centre x for a one-molecule tile (packed tiles take it from the
            // atom's own molecule below).
            const float vx_item = fmaf((float)row_x + 0.5f, it.hx, it.ox);
            // Packed tiles: the molecules' offsets and geometry, read once per tile so that
            // staging a K chunk needs no dependent global loads.  The barrier orders these
            // writes after every producer's use of the previous tile's; the barrier that opens
            // the first chunk's staging orders them before the reads.
            int *const t_off = reinterpret_cast<int *>(smem + L.tile);
            float *const t_geo = reinterpret_cast<float *>(t_off + (PACK ? A.pack + 1 : 0));
            if (PACK) {
                producer_sync<kProducers>();
                for (int k = p; k <= it.nb; k += kProducers)
                    t_off[k] = __ldg(A.in.mol_off + it.b + k);
                for (int k = p; k < 6 * it.nb; k += kProducers) {
                    const int m = it.b + k / 6, f = k % 6;
                    t_geo[k] = f < 3 ? __ldg(A.in.origin + 3 * m + f)
                                     : __ldg(A.in.spacing + 3 * m + f - 3);
                }
            }
            for (int nc = 0; nc < n_chunks && ok; ++nc) {
                const int n0 = nc * n_tile;
                for (int kc = 0; kc < it.n_kc && ok; ++kc, ++step) {
                    const int s = (int)(step % kPipeStages);
                    const uint32_t ph = (step / kPipeStages) & 1u;
                    const bool got = warp_wait(b_empty(s), ph ^ 1u, flag, A.wait_ns);
                    // A.stall (a test of the bounded waits) stops the producers before their
                    // first arrive: no MMA is issued and no store starts, and every wait gives up.
                    if (!producers_all<kProducers>(got) || A.stall) {
                        ok = false;
                        break;
                    }
                    unsigned char *sa = smem + L.stage0 + s * L.stage_bytes;
                    unsigned char *sb = sa + L.a_bytes;
                    const bool resident = it.n_kc <= A.kslots;
                    const int slot = resident ? kc : 0;
                    // Resident tiles keep each K chunk's A in a slot of its own, written at the
                    // first N chunk.  Before a tile overwrites the slots, every MMA of the
                    // previous tile (up to the step just handed over) must have completed.
                    if (resident && nc == 0 && kc == 0 && step > 0) {
                        const unsigned u = step - 1;
                        const bool done = warp_wait(b_empty((int)(u % kPipeStages)),
                                                    (u / kPipeStages) & 1u, flag, A.wait_ns);
                        if (!producers_all<kProducers>(done)) {
                            ok = false;
                            break;
                        }
                    }
                    unsigned char *a_dst = resident ? smem + L.aslots + kc * L.a_bytes : sa;
                    float4 *atom_pos = atoms0;
                    float4 *atom_aux = atom_pos + kKC;
                    float4 *atom_g0 = atom_pos + 2 * kKC;
                    float4 *atom_g1 = atom_pos + 3 * kKC;
                    float *tgx = tgx0;
                    float *tgy = tgy0 + slot * G.ny * kTab;
                    float *tgz = tgz0 + slot * G.nz * kTab;
                    const bool new_atoms =
                        resident ? nc == 0 : ((nc == 0 && kc == 0) || it.n_kc > 1);
                    if (new_atoms) {
                        producer_sync<kProducers>();  // every producer is done reading the old tables
                        if (p < kKC) {
                            const int ai = it.a0 + kc * kKC + p;
                            float4 pos = make_float4(0.f, 0.f, 0.f, 0.f);
                            float4 aux = make_float4(0.f, -1.f, 0.f, 0.f);
                            float4 g0 = make_float4(0.f, 0.f, 0.f, 1.f);
                            float4 g1 = make_float4(1.f, 1.f, 1.f, 0.f);
                            if (ai < it.a1) {
                                // Loads issued together, used after.
                                const int e = __ldg(A.in.elem + ai);
                                const float cx = __ldg(A.in.coords + 3 * ai),
                                            cy = __ldg(A.in.coords + 3 * ai + 1),
                                            cz = __ldg(A.in.coords + 3 * ai + 2);
                                const float wgt = A.in.weight ? __ldg(A.in.weight + ai) : 1.0f;
                                // The atom's molecule: the item's, or in a packed tile the last
                                // k with mol_off[b + k] <= ai.
                                int k = 0;
                                if (PACK) {
                                    int lo = 0, hi = it.nb - 1;
                                    while (lo < hi) {
                                        const int mid = (lo + hi + 1) >> 1;
                                        if (t_off[mid] <= ai) lo = mid;
                                        else hi = mid - 1;
                                    }
                                    k = lo;
                                }
                                if (PACK) {
                                    const float *gk = t_geo + 6 * k;
                                    g0 = make_float4(gk[0], gk[1], gk[2], gk[3]);
                                    g1 = make_float4(gk[4], gk[5], 1.f, 0.f);
                                } else {
                                    g0 = make_float4(it.ox, it.oy, it.oz, it.hx);
                                    g1 = make_float4(it.hy, it.hz, 1.f, 0.f);
                                }
                                const bool sp_ok = g0.w > 0.0f && g1.x > 0.0f && g1.y > 0.0f &&
                                                   g0.w < INFINITY && g1.x < INFINITY &&
                                                   g1.y < INFINITY;
                                if (!sp_ok) {
                                    if (ai == (PACK ? t_off[k] : it.a0))
                                        atomicOr(A.err, PG_DEVERR_SPACING);
                                } else if ((unsigned)e < (unsigned)G.C) {
                                    pos = make_float4(cx, cy, cz, G.q[e]);
                                    aux = make_float4(G.r2[e], (float)e, G.kerf[e], (float)k);
                                    g1.z = wgt;
                                } else if (it.m0 == 0) {
                                    atomicOr(A.err, PG_DEVERR_ELEMENT);
                                }
                            }
                            atom_pos[p] = pos;
                            atom_aux[p] = aux;
                            atom_g0[p] = g0;
                            atom_g1[p] = g1;
                        }
                        producer_sync<kProducers>();
                        // Per-axis tables of this K chunk: g_y, g_z, and for the erf form also
                        // g_x (an erf per A entry would cost more than the table).
                        if (FORM == 1 && !PER) {
                            // Open boundaries: neighbouring voxels share an edge, so each lane
                            // evaluates erf at one lower edge and takes the upper one from the
                            // next lane (Sec. VI-A's reuse of the subtrahend): n + n/32 erf
                            // evaluations per atom and axis instead of 2n.
                            const int pw = p >> 5;
                            auto erf_table = [&](float *tab, int n, int stride, int axis) {
                                const int blocks = (n + 31) >> 5;
#pragma unroll 2
                                for (int task = pw; task < kKC * blocks; task += kProdWarps) {
                                    const int j = task % kKC, i = (task / kKC) * 32 + lane;
                                    const float4 q4 = atom_pos[j];
                                    const float4 aux = atom_aux[j];
                                    const float4 g0 = atom_g0[j], g1 = atom_g1[j];
                                    const float mu = axis == 0 ? q4.x : (axis == 1 ? q4.y : q4.z);
                                    const float o = axis == 0 ? g0.x : (axis == 1 ? g0.y : g0.z);
                                    const float h = axis == 0 ? g0.w : (axis == 1 ? g1.x : g1.y);
                                    const float e_lo = erff((fmaf((float)i, h, o) - mu) * aux.z);
                                    float e_hi = __shfl_down_sync(0xffffffffu, e_lo, 1);
                                    if (lane == 31)
                                        e_hi = erff((fmaf((float)(i + 1), h, o) - mu) * aux.z);
                                    float v = 0.5f * (e_hi - e_lo);
                                    const float d = fmaf((float)i + 0.5f, h, o) - mu;
                                    if (aux.y < 0.0f || (CUT == PG_CUTOFF_BOX && d * d > aux.x))
                                        v = 0.0f;
                                    if (axis == 0) v *= g1.z;
                                    if (i < n) tab[i * stride + j] = v;
                                }
                            };
                            erf_table(tgx, G.nx, kTabX, 0);
                            erf_table(tgy, G.ny, kTab, 1);
                            erf_table(tgz, G.nz, kTab, 2);
                        }
                        for (int i = p; FORM == 1 && PER && i < G.nx * kKC; i += kProducers) {
                            const int x = i / kKC, j = i - (i / kKC) * kKC;
                            const float4 q4 = atom_pos[j];
                            const float4 g0 = PACK ? atom_g0[j]
                                                         : make_float4(it.ox, 0.f, 0.f, it.hx);
                            float v = 0.0f;
                            if (atom_aux[j].y >= 0.0f) {
                                float d = fmaf((float)x + 0.5f, g0.w, g0.x) - q4.x;
                                if (PER) {
                                    const float Lx = G.nx * g0.w;
                                    d = wrap(d, Lx, 1.0f / Lx);
                                }
                                v = atom_g1[j].z * axis_factor<CUT, FORM>(d, q4.w, atom_aux[j].x,
                                                                          g0.w, atom_aux[j].z);
                            }
                            tgx[x * kTabX + j] = v;
                        }
                        for (int i = p; (FORM == 0 || PER) && i < G.ny * kKC; i += kProducers) {
                            const int y = i / kKC, j = i - (i / kKC) * kKC;
                            const float4 q4 = atom_pos[j];
                            const float oy = PACK ? atom_g0[j].y : it.oy;
                            const float hy = PACK ? atom_g1[j].x : it.hy;
                            float v = 0.0f;
                            if (atom_aux[j].y >= 0.0f) {
                                float d = fmaf((float)y + 0.5f, hy, oy) - q4.y;
                                if (PER) {
                                    const float Ly = G.ny * hy;
                                    d = wrap(d, Ly, 1.0f / Ly);
                                }
                                v = axis_factor<CUT, FORM>(d, q4.w, atom_aux[j].x, hy,
                                                     atom_aux[j].z);
                            }
                            tgy[y * kTab + j] = v;
                        }
                        for (int i = p; (FORM == 0 || PER) && i < G.nz * kKC; i += kProducers) {
                            const int z = i / kKC, j = i - (i / kKC) * kKC;
                            const float4 q4 = atom_pos[j];
                            const float oz = PACK ? atom_g0[j].z : it.oz;
                            const float hz = PACK ? atom_g1[j].y : it.hz;
                            float v = 0.0f;
                            if (atom_aux[j].y >= 0.0f) {
                                float d = fmaf((float)z + 0.5f, hz, oz) - q4.z;
                                if (PER) {
                                    const float Lz = G.nz * hz;
                                    d = wrap(d, Lz, 1.0f / Lz);
                                }
                                v = axis_factor<CUT, FORM>(d, q4.w, atom_aux[j].x, hz,
                                                     atom_aux[j].z);
                            }
                            tgz[z * kTab + j] = v;
                        }
                        producer_sync<kProducers>();
                    }
                    // A tile: once per K chunk of a resident tile, else every step.
                    if (!resident || nc == 0) {
#pragma unroll
                        for (int jh = 0; jh < kAGroups; ++jh) {
                            const int jg = ag0 + jh;
                            float v[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int j = jg * 8 + t;
                                const float4 aux = atom_aux[j];
                                v[t] = 0.0f;
                                if (row_ok && (int)aux.y == row_c && (int)aux.w == lm) {
                                    if (FORM == 1) {
                                        v[t] = tgx[row_x * kTabX + j];
                                    } else {
                                        const float hx = PACK ? atom_g0[j].w : it.hx;
                                        const float vx =
                                            PACK
                                                ? fmaf((float)row_x + 0.5f, hx, atom_g0[j].x)
                                                : vx_item;
                                        float d = vx - atom_pos[j].x;
                                        if (PER) {
                                            const float Lx = G.nx * hx;
                                            d = wrap(d, Lx, 1.0f / Lx);
                                        }
                                        v[t] = atom_g1[j].z *
                                               axis_factor<CUT, FORM>(d, atom_pos[j].w, aux.x, hx,
                                                                      aux.z);
                                    }
                                }
                            }
                            *reinterpret_cast<uint4 *>(a_dst + (arow >> 3) * 512 + jg * 128 +
                                                       (arow & 7) * 16) =
                                make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                           pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
                        }
                    }
                    // B tile (layout as in the single-stage kernel).  Producer p always
                    // writes atom group kg = (p/8)%4 of columns nl = (p/32)*8 + p%8 + 32i, so
                    // its (y, z) advance by a fixed step: no division per chunk.
                    {
                        const int kg = (p >> 3) & 3;
                        int n = n0 + (p >> 5) * 8 + (p & 7);
                        int y = n / G.nz, z = n - (n / G.nz) * G.nz;
                        for (int qi = p; qi < n_tile * (kKC / 8); qi += kProducers) {
                            uint4 w = make_uint4(0u, 0u, 0u, 0u);
                            if (n < N) {
                                const float4 *gy4 =
                                    reinterpret_cast<const float4 *>(tgy + y * kTab + kg * 8);
                                const float4 *gz4 =
                                    reinterpret_cast<const float4 *>(tgz + z * kTab + kg * 8);
                                const float4 y0 = gy4[0], y1 = gy4[1], z0 = gz4[0], z1 = gz4[1];
                                w = make_uint4(pack_bf16x2(y0.x * z0.x, y0.y * z0.y),
                                               pack_bf16x2(y0.z * z0.z, y0.w * z0.w),
                                               pack_bf16x2(y1.x * z1.x, y1.y * z1.y),
                                               pack_bf16x2(y1.z * z1.z, y1.w * z1.w));
                            }
                            *reinterpret_cast<uint4 *>(sb + qi * 16) = w;
                            n += kColStep;
                            z += dzc;
                            y += dyc;
                            if (z >= G.nz) {
                                z -= G.nz;
                                ++y;
                            }
                        }
                    }
                    fence_proxy_async_smem();
                    warp_arrive(b_full(s));
                }
            }
        }
    } else if (warp == 4 + kProdWarps) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc(n_tile);
            unsigned step = 0, tile = 0;
            bool ok = true;
            for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const PipeItem it = pipe_item<PACK>(A, item);
                for (int nc = 0; nc < n_chunks && ok; ++nc, ++tile) {
                    const int buf = (int)(tile & 1u);
                    const uint32_t aph = (tile >> 1) & 1u;
                    for (int kc = 0; kc < it.n_kc && ok; ++kc, ++step) {
                        const int s = (int)(step % kPipeStages);
                        const uint32_t ph = (step / kPipeStages) & 1u;
                        if (!pipe_wait(b_full(s), ph, flag, A.wait_ns)) {
                            ok = false;
                            break;
                        }
                        if (kc == 0 && !pipe_wait(acc_empty(buf), aph ^ 1u, flag, A.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = smem_u32(smem + L.stage0 + s * L.stage_bytes);
                        const uint32_t sb = st + L.a_bytes;
                        const uint32_t sa = it.n_kc <= A.kslots
                                                ? smem_u32(smem + L.aslots + kc * L.a_bytes)
                                                : st;
#pragma unroll
                        for (int k = 0; k < kKC / 16; ++k)
                            mma_bf16_f32(tmem + buf * n_tile, smem_desc(sa + k * 256, 128, 512),
                                         smem_desc(sb + k * 256, 128, 512), idesc,
                                         (kc > 0 || k > 0) ? 1u : 0u);
                        mma_commit(b_empty(s));
                        if (kc == it.n_kc - 1) mma_commit(acc_full(buf));
                    }
                }
            }
            // Every MMA issued here must complete before the tensor memory is freed.
            mma_commit(drain);
            *drained = drain_wait(drain) ? 1 : 0;
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        unsigned char *wstage = smem + L.out + warp * L.out_stride;
        const int slabs = n_tile * (int)sizeof(T) / 128;
        const int slab_cols = 128 / (int)sizeof(T);
        const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
        unsigned tile = 0;
        bool ok = true;
        for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
            const PipeItem it = pipe_item<PACK>(A, item);
            for (int nc = 0; nc < n_chunks && ok; ++nc, ++tile) {
                const int buf = (int)(tile & 1u);
                const uint32_t ph = (tile >> 1) & 1u;
                // tcgen05.ld is warp-collective: the whole warp continues or stops together
                // (warp_wait returns the same value on every lane).
                if (!warp_wait(acc_full(buf), ph, flag, A.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // The previous tile's TMA stores must have read this warp's staging.
                if (lane == 0) bulk_wait_read_all();
                __syncwarp();
                for (int cb = 0; cb < n_tile; cb += 64) {
                    uint32_t r0[32], r1[32];
                    tmem_ld32(tmem_row + buf * n_tile + cb, r0);
                    tmem_ld32(tmem_row + buf * n_tile + cb + 32, r1);
                    tmem_ld_wait();
                    stage_swizzled<T>(wstage, lane, cb, r0);
                    stage_swizzled<T>(wstage, lane, cb + 32, r1);
                }
                tc_fence_before();
                fence_proxy_async_smem();
                warp_arrive(acc_empty(buf));  // includes __syncwarp: the warp's rows are staged
                // One TMA tensor store per 32-row x 128-byte slab; the tensor map clips rows
                // past M and columns past N.  Boxes lying wholly outside are skipped.
                if (PACK) {
                    // Packed: rows are global (molecule-major); the map clips past the batch.
                    const long long grow = (long long)it.b * M + warp * 32;
                    if (lane == 0 && grow < (long long)G.n_mol * M) {
                        for (int sl = 0; sl < slabs; ++sl) {
                            const int x = nc * n_tile + sl * slab_cols;
                            if (x < N)
                                tma_store_2d(&A.out_map, smem_u32(wstage + sl * 4096), x,
                                             (int)grow);
                        }
                        bulk_commit();
                    }
                } else {
                    const int row0 = it.m0 + warp * 32;
                    if (lane == 0 && row0 < M) {
                        for (int sl = 0; sl < slabs; ++sl) {
                            const int x = nc * n_tile + sl * slab_cols;
                            if (x < N)
                                tma_store_3d(&A.out_map, smem_u32(wstage + sl * 4096), x, row0,
                                             it.b);
                        }
                        bulk_commit();
                    }
                }
            }
        }
        if (lane == 0) bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    // If the drain never arrived, the columns stay allocated rather than be freed under an
    // MMA that may still write them.
    if (tid == 0 && (*flag || !*drained))
        atomicOr(A.err, PG_DEVERR_TIMEOUT | (*drained ? 0u : PG_DEVERR_TMEM_HELD));
    if (warp == 0 && *drained) {
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)(2 * n_tile));
    }
}

template <typename T, int CUT, int FORM>
const void *pick_per(int periodic, bool pipe, bool pack)
{
    if (pipe && pack)
        return periodic ? (const void *)separable_pipe_kernel<T, CUT, true, FORM, true>
                        : (const void *)separable_pipe_kernel<T, CUT, false, FORM, true>;
    if (pipe)
        return periodic ? (const void *)separable_pipe_kernel<T, CUT, true, FORM, false>
                        : (const void *)separable_pipe_kernel<T, CUT, false, FORM, false>;
    return periodic ? (const void *)separable_kernel<T, CUT, true, FORM>
                    : (const void *)separable_kernel<T, CUT, false, FORM>;
}

// Point-sampled (FORM 0) and voxel-integrated (FORM 1, Sec. III-A) operand factors are
// separate instantiations, so the point form carries no erf code.
template <typename T>
const void *pick_cut(int cutoff, int periodic, bool pipe, int form, bool pack)
{
    if (form == PG_FORM_INTEGRAL)
        return cutoff == PG_CUTOFF_BOX ? pick_per<T, PG_CUTOFF_BOX, 1>(periodic, pipe, pack)
                                       : pick_per<T, PG_CUTOFF_NONE, 1>(periodic, pipe, pack);
    return cutoff == PG_CUTOFF_BOX ? pick_per<T, PG_CUTOFF_BOX, 0>(periodic, pipe, pack)
                                   : pick_per<T, PG_CUTOFF_NONE, 0>(periodic, pipe, pack);
}

}  // namespace

bool separable_supported(const Geometry &g, int dtype)
{
    (void)dtype;
    if (g.cutoff == PG_CUTOFF_SPHERE) return false;
    const long long N = (long long)g.ny * g.nz;
    // Row segments go out as bulk copies: 16-byte multiples; tables must fit shared memory.
    if (N % 16 != 0) return false;
    if (g.nx > 256 || g.ny > 256 || g.nz > 256) return false;
    return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 3D tensor map over the output, dims innermost first {N = ny nz, M = C nx, n_mol}; boxes of
// 128 bytes x 32 rows x 1 molecule with the 128-byte swizzle.
cudaError_t encode_out_map(SeparableArgs &a, int dtype)
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    const int esz = dtype == PG_F32 ? 4 : 2;
    const CUtensorMapDataType dt = dtype == PG_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == PG_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t N = (cuuint64_t)a.geo.ny * a.geo.nz, M = (cuuint64_t)a.geo.C * a.geo.nx;
    // Packed tiles store global rows (2D); otherwise rows of one molecule (3D), so that a
    // molecule's last tile cannot spill into the next molecule.
    const cuuint32_t rank = a.pack > 0 ? 2 : 3;
    const cuuint64_t dims[3] = {N, a.pack > 0 ? M * (cuuint64_t)a.geo.n_mol : M,
                                (cuuint64_t)a.geo.n_mol};
    const cuuint64_t strides[2] = {N * esz, N * M * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(128 / esz), 32, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(&a.out_map, dt, rank, a.out, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t separable_plan(const SeparableArgs &a0, int dtype, const pg_tuning &t, int sm_count,
                           KernelLaunch *kl)
{
    if (!separable_supported(a0.geo, dtype)) return cudaErrorNotSupported;
    if ((uintptr_t)a0.out % 16 != 0) return cudaErrorNotSupported;
    SeparableArgs a = a0;
    const bool pipe = t.separable_simple == 0;
    // PG_DEBUG_STALL_PRODUCERS=1 (read at every call; for tests of the bounded waits) stops
    // the operand producers (single-stage kernel: the MMA issue) before the first handoff and
    // shortens every wait to 2 ms, so that the launch ends with PG_DEVERR_TIMEOUT having
    // issued no MMA and started no store.
    const char *stall = std::getenv("PG_DEBUG_STALL_PRODUCERS");
    a.stall = (stall && stall[0] == '1') ? 1 : 0;
    a.wait_ns = a.stall ? 2000000ull : 2000000000ull;
    int n_tile = t.n_tile;
    if (n_tile != 64 && n_tile != 128 && n_tile != 256) n_tile = 128;
    const int esz = dtype == PG_F32 ? 4 : 2;
    // Molecules with fewer than 128 (channel, x) rows share a tile when their rows divide it.
    const int Mrows = a.geo.C * a.geo.nx;
    a.pack = (pipe && Mrows < kRows && kRows % Mrows == 0) ? kRows / Mrows : 0;
    // Resident K chunks: enough for a tile of twice the average atoms, at most 8, within the
    // shared memory of one CTA, or of blocks_per_sm CTAs per SM when the tuning asks for more.
    const double atoms_per_tile = (a.pack > 0 ? a.pack : 1) * (a.geo.n_mol > 0
                                      ? (double)a.geo.n_atoms / a.geo.n_mol : 0.0);
    int kslots = (int)std::ceil(2.0 * atoms_per_tile / kKC);
    kslots = kslots < 1 ? 1 : (kslots > 8 ? 8 : kslots);
    auto bytes = [&](int nt, int ks) {
        return pipe ? pipe_layout(a.geo.nx, a.geo.ny, a.geo.nz, nt, esz, ks, a.pack).total
                    : sep_layout(a.geo.ny, a.geo.nz, nt, esz).total;
    };
    const int budget = (pipe && t.blocks_per_sm >= 2) ? 228 * 1024 / t.blocks_per_sm - 1024
                                                      : 227 * 1024;
    while (kslots > 1 && bytes(n_tile, kslots) > budget) --kslots;
    // Largest requested tile whose shared-memory footprint fits one SM's 227 KB.
    while (n_tile > 64 && bytes(n_tile, kslots) > 227 * 1024) n_tile /= 2;
    const int smem = bytes(n_tile, kslots);
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    a.n_tile = n_tile;
    a.kslots = kslots;
    a.m_tiles = (a.geo.C * a.geo.nx + kRows - 1) / kRows;
    if (pipe) {
        cudaError_t em = encode_out_map(a, dtype);
        if (em != cudaSuccess) return em;
    }
    const int cut = a.geo.cutoff, per = a.geo.periodic, form = a.geo.form;
    const bool pack = a.pack > 0;
    const void *f = dtype == PG_F32   ? pick_cut<float>(cut, per, pipe, form, pack)
                    : dtype == PG_F16 ? pick_cut<__half>(cut, per, pipe, form, pack)
                                      : pick_cut<__nv_bfloat16>(cut, per, pipe, form, pack);
    const int threads = pipe ? pipe_threads(a.pack > 0, esz) : kRows;
    const int tmem_cols = pipe ? 2 * n_tile : n_tile;
    cudaError_t e = raise_smem_limit(f, (size_t)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // Resident CTAs per SM from the three limits that bind here: shared memory (with the
    // per-block reservation), registers, and the SM's 512 tensor-memory columns.
    int dev = 0, smem_sm = 0, smem_reserved = 0, regs_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)))
        return e;
    if ((e = cudaDeviceGetAttribute(&smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)))
        return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)))
        return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, f)) != cudaSuccess) return e;
    const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * (threads + 31) / 32 * 32;
    int per_sm = smem_sm / (smem + smem_reserved);
    if (regs_cta > 0 && regs_sm / regs_cta < per_sm) per_sm = regs_sm / regs_cta;
    if (512 / tmem_cols < per_sm) per_sm = 512 / tmem_cols;
    if (per_sm < 1) return cudaErrorNotSupported;
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < per_sm) per_sm = t.blocks_per_sm;
    const long long items = a.pack > 0 ? ((long long)a.geo.n_mol + a.pack - 1) / a.pack
                                       : (long long)a.geo.n_mol * a.m_tiles;
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > items) blocks = items;
    if (blocks < 1) blocks = 1;
    kl->func = f;
    kl->grid = dim3((unsigned)blocks);
    kl->block = dim3(threads);
    kl->smem = (size_t)smem;
    set_args(kl, a);
    return cudaSuccess;
}

}  // namespace pgi
