// Host runtime behind the C ABI in pg.h: argument validation, per-call constants, kernel
// dispatch, the device error word, the launch autotuner with its cache, and plans
// (CUDA graphs holding the host-to-device copy of a batch plus the launch).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>  // header-only NVTX v3: inert unless a profiler injects itself

#include "pg.h"
#include "pg_internal.h"

using namespace pgi;

namespace {

thread_local std::string t_last_error;

// An NVTX range over one API call, so that profiler timelines show where each call's host
// work (and, for plan runs, the graph replay it waits for) begins and ends.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

pg_status fail(pg_status s, const char *fmt, ...)
{
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

pg_status cuda_fail(cudaError_t e, const char *what)
{
    (void)cudaGetLastError();  // clear the non-sticky error state
    return fail(PG_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define PG_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------- per-device state

struct Device {
    int id = -1;
    int sms = 0;
    unsigned *err = nullptr;                // device error word (PG_DEVERR_* bits)
    unsigned long long *sched = nullptr;    // kSchedSlots work counters, 4 words apart
    std::atomic<unsigned> *next_slot = nullptr;
    std::string name;
    // A separable launch reported PG_DEVERR_TMEM_HELD: a CTA kept tensor memory it could not
    // safely free, so a later launch's allocation might never be granted.
    std::atomic<bool> *tmem_held = nullptr;

    unsigned long long *take_slot()
    {
        const unsigned i = next_slot->fetch_add(1u, std::memory_order_relaxed) % kSchedSlots;
        return sched + 4 * (size_t)i;
    }
};

std::mutex g_mu;
std::map<int, Device> g_devices;

// PG_DEBUG_LAUNCH=1 in the environment traces launches and per-device allocations to stderr.
bool debug_trace_on()
{
    static const bool on = [] {
        const char *v = std::getenv("PG_DEBUG_LAUNCH");
        return v && v[0] == '1';
    }();
    return on;
}

pg_status get_device(Device **out)
{
    int id = 0;
    PG_CUDA(cudaGetDevice(&id), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devices.find(id);
    if (it == g_devices.end()) {
        Device d;
        d.id = id;
        PG_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, id),
                "cudaDeviceGetAttribute");
        cudaDeviceProp prop;
        PG_CUDA(cudaGetDeviceProperties(&prop, id), "cudaGetDeviceProperties");
        d.name = prop.name;
        for (char &ch : d.name)
            if (ch == ' ') ch = '_';
        PG_CUDA(cudaMalloc(&d.err, sizeof(unsigned)), "cudaMalloc(error word)");
        PG_CUDA(cudaMemset(d.err, 0, sizeof(unsigned)), "cudaMemset(error word)");
        const size_t sched_bytes = sizeof(unsigned long long) * 4 * kSchedSlots;
        PG_CUDA(cudaMalloc(&d.sched, sched_bytes), "cudaMalloc(work counters)");
        PG_CUDA(cudaMemset(d.sched, 0, sched_bytes), "cudaMemset(work counters)");
        d.next_slot = new std::atomic<unsigned>(0u);
        d.tmem_held = new std::atomic<bool>(false);
        PG_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize(setup)");
        if (debug_trace_on())
            std::fprintf(stderr, "[pg] per-device state allocated on device %d\n", id);
        it = g_devices.emplace(id, d).first;
    }
    *out = &it->second;
    return PG_OK;
}

// ---------------------------------------------------------------- validation

size_t dtype_size(int dtype) { return dtype == PG_F32 ? 4 : 2; }

pg_status validate(const pg_batch *b, const pg_grid *g)
{
    if (!b || !g) return fail(PG_ERR_INVALID_ARG, "batch and grid must not be NULL");
    if (b->n_mol < 0 || b->n_atoms < 0)
        return fail(PG_ERR_INVALID_ARG, "negative n_mol (%d) or n_atoms (%d)", b->n_mol,
                    b->n_atoms);
    if (b->n_mol > 0 && (!b->mol_off || !b->origin || (!b->spacing && !b->cell)))
        return fail(PG_ERR_INVALID_ARG,
                    "mol_off, origin and spacing (or cell) are required when n_mol > 0");
    if (b->n_atoms > 0 && (!b->coords || !b->elem))
        return fail(PG_ERR_INVALID_ARG, "coords and elem are required when n_atoms > 0");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(PG_ERR_INVALID_ARG, "grid shape %dx%dx%d must be positive", g->nx, g->ny,
                    g->nz);
    if (g->n_channels < 1 || g->n_channels > kMaxC)
        return fail(PG_ERR_INVALID_ARG, "n_channels %d outside 1..%d", g->n_channels, kMaxC);
    if (!g->sigma) return fail(PG_ERR_INVALID_ARG, "sigma must not be NULL");
    for (int c = 0; c < g->n_channels; ++c)
        if (!(g->sigma[c] > 0.0f) || !std::isfinite(g->sigma[c]))
            return fail(PG_ERR_INVALID_ARG, "sigma[%d] = %g must be positive and finite", c,
                        (double)g->sigma[c]);
    if (g->cutoff != PG_CUTOFF_SPHERE && g->cutoff != PG_CUTOFF_NONE && g->cutoff != PG_CUTOFF_BOX)
        return fail(PG_ERR_INVALID_ARG, "unknown cutoff mode %d", g->cutoff);
    if (g->cutoff != PG_CUTOFF_NONE && (!(g->cutoff_k > 0.0f) || !std::isfinite(g->cutoff_k)))
        return fail(PG_ERR_INVALID_ARG, "cutoff_k = %g must be positive and finite",
                    (double)g->cutoff_k);
    if (g->periodic != 0 && g->periodic != 1)
        return fail(PG_ERR_INVALID_ARG, "periodic must be 0 or 1");
    if (g->voxel_form != PG_FORM_POINT && g->voxel_form != PG_FORM_INTEGRAL)
        return fail(PG_ERR_INVALID_ARG, "unknown voxel_form %d", g->voxel_form);
    if (b->cell && g->voxel_form != PG_FORM_POINT)
        return fail(PG_ERR_UNSUPPORTED, "the voxel-integrated form needs an axis-aligned box "
                                        "(cell must be NULL)");
    if (b->cell && g->periodic && g->cutoff == PG_CUTOFF_NONE)
        return fail(PG_ERR_UNSUPPORTED, "a periodic cell matrix needs a cutoff (SPHERE or BOX): "
                                        "without one the nearest image is not found by "
                                        "rounding");
    const long long plane = (long long)g->ny * g->nz;
    if (plane > INT32_MAX || (long long)g->nx * plane > INT32_MAX)
        return fail(PG_ERR_INVALID_ARG, "one channel grid must hold fewer than 2^31 voxels");
    const long long per_mol = (long long)g->n_channels * g->nx * plane;
    if (b->n_mol > 0 && per_mol > (1ll << 60) / b->n_mol)
        return fail(PG_ERR_INVALID_ARG, "output too large");
    return PG_OK;
}

pg_status check_dtype(int dtype)
{
    if (dtype != PG_F32 && dtype != PG_F16 && dtype != PG_BF16)
        return fail(PG_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    return PG_OK;
}

void make_geometry(const pg_batch *b, const pg_grid *g, Geometry *G)
{
    std::memset(G, 0, sizeof *G);
    G->n_mol = b->n_mol;
    G->n_atoms = b->n_atoms;
    G->nx = g->nx;
    G->ny = g->ny;
    G->nz = g->nz;
    G->C = g->n_channels;
    G->cutoff = g->cutoff;
    G->periodic = g->periodic;
    G->form = g->voxel_form;
    const double log2e = 1.4426950408889634;
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < g->n_channels; ++c) {
        const double s = g->sigma[c];
        const double r = (double)g->cutoff_k * s;
        G->q[c] = (float)(log2e / (2.0 * s * s));
        G->inv_s2[c] = (float)(1.0 / (s * s));
        G->kerf[c] = (float)(1.0 / (std::sqrt(2.0) * s));
        G->kdmu[c] = (float)(1.0 / (std::sqrt(2.0 * pi) * s));
        if (g->cutoff == PG_CUTOFF_NONE) {
            G->r2[c] = INFINITY;
            G->rcull[c] = INFINITY;
        } else {
            G->r2[c] = (float)(r * r);
            G->rcull[c] = (float)(r * (1.0 + 1e-5) + 1e-6);
        }
    }
}

Inputs make_inputs(const pg_batch *b)
{
    return Inputs{b->coords, b->elem, b->mol_off, b->origin, b->spacing, b->weight, b->cell};
}

pg_tuning default_tuning(int path)
{
    pg_tuning t;
    std::memset(&t, 0, sizeof t);
    t.path = path == PG_PATH_SEPARABLE ? PG_PATH_SEPARABLE : PG_PATH_DIRECT;
    t.block_threads = 256;
    t.blocks_per_sm = 0;
    t.store_hint = 0;
    t.n_tile = 128;
    t.chunk_planes = 8;
    return t;
}

// Whether the direct kernel runs in lane-list mode (its lane-list instantiation): the point
// form with a cutoff, unweighted axis-aligned boxes.  Molecules of at most 32 atoms never
// reach it (they take the register path), so a batch whose mean is that small keeps the
// gather-only instantiation and its higher occupancy.
bool direct_lanes_on(const pg_batch *b, const pg_grid *g, const pg_tuning &t)
{
    return !t.gather_only && g->voxel_form == PG_FORM_POINT && !b->weight && !b->cell &&
           g->cutoff != PG_CUTOFF_NONE && b->n_atoms > 32LL * b->n_mol;
}

// Floats of per-warp factor table for the direct kernel's voxel-integrated form with a
// separable cutoff: room for 64 atoms' per-axis factors, at most kErfTabCap; 0 elsewhere.
int direct_erf_tab(const pg_batch *b, const pg_grid *g, const pg_tuning &t)
{
    if (t.gather_only || g->voxel_form != PG_FORM_INTEGRAL || g->cutoff == PG_CUTOFF_SPHERE ||
        b->cell)
        return 0;
    const long long need = 64LL * erf_table_stride(g->ny, g->nz);
    return (int)std::min<long long>(need, kErfTabCap);
}

bool vec_stores_ok(const void *out, const pg_grid *g, int dtype)
{
    return ((uintptr_t)out % 16 == 0) && (((size_t)g->nz * dtype_size(dtype)) % 16 == 0);
}

// Resolve one forward launch without issuing it.
pg_status plan_forward(const pg_batch *b, const pg_grid *g, int dtype, void *out,
                       const pg_tuning &t, const Device &d, unsigned *err,
                       unsigned long long *sched, KernelLaunch *kl)
{
    Geometry G;
    make_geometry(b, g, &G);
    if (t.path == PG_PATH_SEPARABLE) {
        if (d.tmem_held->load())
            return fail(PG_ERR_CUDA, "separable launches are refused on this device: an earlier "
                                     "launch kept tensor memory after a timed-out wait "
                                     "(PG_DEVERR_TMEM_HELD)");
        if (b->cell)
            return fail(PG_ERR_UNSUPPORTED, "the separable path needs an axis-aligned box; a "
                                            "cell matrix's metric does not factor per axis");
        if (g->cutoff == PG_CUTOFF_SPHERE)
            return fail(PG_ERR_UNSUPPORTED,
                        "the separable path needs a separable cutoff (NONE or BOX); the "
                        "spherical cutoff does not factor per axis");
        if (!separable_supported(G, dtype))
            return fail(PG_ERR_UNSUPPORTED, "separable path does not cover this grid/dtype");
        SeparableArgs a;
        std::memset(&a, 0, sizeof a);
        a.in = make_inputs(b);
        a.out = out;
        a.err = err;
        a.geo = G;
        a.n_tile = t.n_tile;
        cudaError_t e = separable_plan(a, dtype, t, d.sms, kl);
        if (e == cudaErrorNotSupported)
            return fail(PG_ERR_UNSUPPORTED, "separable path does not cover this grid/dtype");
        if (e != cudaSuccess) return cuda_fail(e, "separable_plan");
        return PG_OK;
    }
    DirectArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = make_inputs(b);
    a.out = out;
    a.err = err;
    a.sched = sched;
    a.lane_lists = direct_lanes_on(b, g, t) ? 1 : 0;
    a.chunk_planes = (t.chunk_planes >= 1 && t.chunk_planes <= 64) ? t.chunk_planes : 8;
    a.chunk_order = t.chunk_order == 1 ? 1 : 0;
    a.erf_tab = direct_erf_tab(b, g, t);
    a.geo = G;
    const int vec = vec_stores_ok(out, g, dtype) ? 1 : 0;
    if (b->cell) {
        a.lane_lists = 0;
        a.erf_tab = 0;
        cudaError_t e = cell_plan(a, dtype, vec, t, d.sms, kl);
        if (e != cudaSuccess) return cuda_fail(e, "cell_plan");
        return PG_OK;
    }
    cudaError_t e = direct_plan(a, dtype, vec, t, d.sms, kl);
    if (e != cudaSuccess) return cuda_fail(e, "direct_plan");
    return PG_OK;
}

pg_status forward(const pg_batch *b, const pg_grid *g, int dtype, void *out, const pg_tuning &t,
                  cudaStream_t s)
{
    pg_status st = validate(b, g);
    if (st) return st;
    if ((st = check_dtype(dtype))) return st;
    if (t.path != PG_PATH_DIRECT && t.path != PG_PATH_SEPARABLE)
        return fail(PG_ERR_INVALID_ARG, "tuning.path must be DIRECT or SEPARABLE");
    if (b->n_mol > 0 && !out) return fail(PG_ERR_INVALID_ARG, "out must not be NULL");
    if ((uintptr_t)out % dtype_size(dtype) != 0)
        return fail(PG_ERR_INVALID_ARG, "out is not aligned to its element size");
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    if (b->n_mol == 0) return PG_OK;
    KernelLaunch kl;
    if ((st = plan_forward(b, g, dtype, out, t, *d, d->err, d->take_slot(), &kl))) return st;
    PG_CUDA(launch(kl, s), "voxelize launch");
    return PG_OK;
}

// ---------------------------------------------------------------- tuning cache

std::mutex g_tune_mu;
std::map<std::string, pg_tuning> g_tune;

std::string bucket_key(const pg_batch *b, const pg_grid *g, int dtype, int path,
                       const Device &d)
{
    const double apm = b->n_mol > 0 ? (double)b->n_atoms / b->n_mol : 0.0;
    const int bucket = apm >= 1.0 ? (int)std::floor(std::log2(apm)) : 0;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%dx%dx%d|C%d|dt%d|cut%d|per%d|apm%d|path%d%s%s%s",
             d.name.c_str(), g->nx, g->ny, g->nz, g->n_channels, dtype, g->cutoff, g->periodic,
             bucket, path, g->voxel_form == PG_FORM_INTEGRAL ? "|form1" : "",
             b->cell ? "|cell" : "", b->weight ? "|wgt" : "");
    return buf;
}

// PG_TUNING_CACHE names a tuning-cache file: it is merged into the in-memory cache on first
// use, and every pg_autotune rewrites it with the whole cache.
const char *tuning_cache_path()
{
    const char *p = std::getenv("PG_TUNING_CACHE");
    return (p && *p) ? p : nullptr;
}

void tuning_cache_init()
{
    static std::once_flag once;
    std::call_once(once, [] {
        const char *p = tuning_cache_path();
        if (!p) return;
        std::ifstream probe(p);
        if (!probe) return;  // not written yet
        const std::string saved = t_last_error;
        pg_tuning_load(p);
        t_last_error = saved;
    });
}

pg_tuning resolve(const pg_batch *b, const pg_grid *g, int dtype, int path, const Device &d)
{
    tuning_cache_init();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(bucket_key(b, g, dtype, path, d));
    if (it != g_tune.end()) return it->second;
    return default_tuning(path);
}

// ---------------------------------------------------------------- plans

bool is_pinned(const void *p)
{
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeHost;
}

}  // namespace

// Host-to-device copies of a plan run: coords, elem, mol_off, origin, spacing, weight, cell.
constexpr int kPlanCopies = 7;

struct pg_plan {
    int device = -1;
    pg_grid grid;
    std::vector<float> sigma;
    int dtype = 0;
    int max_mol = 0, max_atoms = 0;
    int path = PG_PATH_AUTO;  // as requested at creation
    float *d_coords = nullptr;
    int *d_elem = nullptr;
    int *d_moloff = nullptr;
    float *d_origin = nullptr;
    float *d_spacing = nullptr;
    float *d_weight = nullptr;
    float *d_cell = nullptr;
    unsigned *d_err = nullptr;
    unsigned long long *d_sched = nullptr;
    unsigned char *h_stage = nullptr;
    size_t stage_off[kPlanCopies] = {};
    unsigned *h_err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_memset = nullptr, n_copy[kPlanCopies] = {}, n_kernel = nullptr,
                    n_errcopy = nullptr;
    const void *kernel_func = nullptr;
    // What the executable graph currently holds, so that an unchanged run skips the update.
    const void *cur_src[kPlanCopies] = {};
    size_t cur_cnt[kPlanCopies] = {};
    KernelLaunch cur_kl;
    bool cur_valid = false;
    bool in_flight = false;  // launched, not yet waited for
    cudaEvent_t done = nullptr;  // recorded after each launch's graph
};

namespace {

void plan_free(pg_plan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_coords);
    cudaFree(p->d_elem);
    cudaFree(p->d_moloff);
    cudaFree(p->d_origin);
    cudaFree(p->d_spacing);
    cudaFree(p->d_weight);
    cudaFree(p->d_cell);
    cudaFree(p->d_err);
    cudaFree(p->d_sched);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->h_err) cudaFreeHost(p->h_err);
    if (p->done) cudaEventDestroy(p->done);
    delete p;
}

pg_status plan_build_graph(pg_plan *p, const void *const src[kPlanCopies], const size_t bytes[kPlanCopies],
                           void *const dst[kPlanCopies], KernelLaunch &kl)
{
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
    }
    PG_CUDA(cudaGraphCreate(&p->graph, 0), "cudaGraphCreate");
    cudaMemsetParams ms;
    std::memset(&ms, 0, sizeof ms);
    ms.dst = p->d_err;
    ms.value = 0;
    ms.elementSize = sizeof(unsigned);
    ms.width = 1;
    ms.height = 1;
    ms.pitch = sizeof(unsigned);
    PG_CUDA(cudaGraphAddMemsetNode(&p->n_memset, p->graph, nullptr, 0, &ms), "add memset node");
    cudaGraphNode_t deps[kPlanCopies + 1];
    deps[0] = p->n_memset;
    for (int i = 0; i < kPlanCopies; ++i) {
        PG_CUDA(cudaGraphAddMemcpyNode1D(&p->n_copy[i], p->graph, nullptr, 0, dst[i], src[i],
                                         bytes[i], cudaMemcpyHostToDevice),
                "add H2D node");
        deps[i + 1] = p->n_copy[i];
    }
    kl.params[0] = kl.args;
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = const_cast<void *>(kl.func);
    kp.gridDim = kl.grid;
    kp.blockDim = kl.block;
    kp.sharedMemBytes = (unsigned)kl.smem;
    kp.kernelParams = kl.params;
    PG_CUDA(cudaGraphAddKernelNode(&p->n_kernel, p->graph, deps, kPlanCopies + 1, &kp),
            "add kernel node");
    PG_CUDA(cudaGraphAddMemcpyNode1D(&p->n_errcopy, p->graph, &p->n_kernel, 1, p->h_err,
                                     p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost),
            "add D2H node");
    PG_CUDA(cudaGraphInstantiate(&p->exec, p->graph, 0), "cudaGraphInstantiate");
    p->kernel_func = kl.func;
    return PG_OK;
}

bool same_launch(const KernelLaunch &a, const KernelLaunch &b)
{
    return a.func == b.func && a.grid.x == b.grid.x && a.grid.y == b.grid.y &&
           a.grid.z == b.grid.z && a.block.x == b.block.x && a.block.y == b.block.y &&
           a.block.z == b.block.z && a.smem == b.smem && a.args_size == b.args_size &&
           std::memcmp(a.args, b.args, a.args_size) == 0;
}

pg_status plan_update_graph_nodes(pg_plan *p, const void *const src[kPlanCopies], const size_t bytes[kPlanCopies],
                                  void *const dst[kPlanCopies], KernelLaunch &kl);

// Bring the executable graph in line with this run; nothing to do when the copies and the
// launch are those of the previous run.
pg_status plan_update_graph(pg_plan *p, const void *const src[kPlanCopies], const size_t bytes[kPlanCopies],
                            void *const dst[kPlanCopies], KernelLaunch &kl)
{
    bool same = p->exec && p->cur_valid && same_launch(kl, p->cur_kl);
    for (int i = 0; same && i < kPlanCopies; ++i)
        same = src[i] == p->cur_src[i] && bytes[i] == p->cur_cnt[i];
    if (same) return PG_OK;
    pg_status st = plan_update_graph_nodes(p, src, bytes, dst, kl);
    p->cur_valid = st == PG_OK;
    if (st == PG_OK) {
        for (int i = 0; i < kPlanCopies; ++i) {
            p->cur_src[i] = src[i];
            p->cur_cnt[i] = bytes[i];
        }
        p->cur_kl = kl;
    }
    return st;
}

pg_status plan_update_graph_nodes(pg_plan *p, const void *const src[kPlanCopies], const size_t bytes[kPlanCopies],
                                  void *const dst[kPlanCopies], KernelLaunch &kl)
{
    if (!p->exec || kl.func != p->kernel_func) return plan_build_graph(p, src, bytes, dst, kl);
    for (int i = 0; i < kPlanCopies; ++i) {
        if (cudaGraphExecMemcpyNodeSetParams1D(p->exec, p->n_copy[i], dst[i], src[i], bytes[i],
                                               cudaMemcpyHostToDevice) != cudaSuccess) {
            (void)cudaGetLastError();
            return plan_build_graph(p, src, bytes, dst, kl);
        }
    }
    kl.params[0] = kl.args;
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = const_cast<void *>(kl.func);
    kp.gridDim = kl.grid;
    kp.blockDim = kl.block;
    kp.sharedMemBytes = (unsigned)kl.smem;
    kp.kernelParams = kl.params;
    if (cudaGraphExecKernelNodeSetParams(p->exec, p->n_kernel, &kp) != cudaSuccess) {
        (void)cudaGetLastError();
        return plan_build_graph(p, src, bytes, dst, kl);
    }
    return PG_OK;
}

pg_status report_bits(unsigned bits)
{
    if (!bits) return PG_OK;
    return fail((bits & PG_DEVERR_TIMEOUT) ? PG_ERR_TIMEOUT : PG_ERR_DEVICE_VALIDATION,
                "device validation failed (bits 0x%x:%s%s%s%s%s%s)", bits,
                (bits & PG_DEVERR_ELEMENT) ? " element id outside [0, C)" : "",
                (bits & PG_DEVERR_OFFSETS) ? " bad CSR offsets" : "",
                (bits & PG_DEVERR_SPACING) ? " non-positive spacing" : "",
                (bits & PG_DEVERR_PERIODIC) ? " periodic cutoff >= half a cell edge" : "",
                (bits & PG_DEVERR_TIMEOUT) ? " tensor-core wait timed out" : "",
                (bits & PG_DEVERR_TMEM_HELD) ? " tensor memory kept" : "");
}

}  // namespace

namespace pgi {

void debug_launch(const KernelLaunch &kl)
{
    if (debug_trace_on())
        std::fprintf(stderr, "[pg] launch func=%p grid=%u block=%u smem=%zu\n", kl.func,
                     kl.grid.x, kl.block.x, kl.smem);
}

cudaError_t raise_smem_limit(const void *func, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &lim = limit[std::make_pair(dev, func)];
    if (smem > lim) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lim = smem;
    }
    return cudaSuccess;
}

cudaError_t occupancy(const void *func, int threads, size_t smem, int *per_sm)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = raise_smem_limit(func, smem)) != cudaSuccess) return e;
    const auto key = std::make_tuple(dev, func, threads, smem);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem);
    if (e != cudaSuccess) return e;
    cache[key] = n;
    *per_sm = n;
    return cudaSuccess;
}

pg_status set_last_error(pg_status status, const char *fmt, ...)
{
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return status;
}

pg_status direct_launch_with_scratch(const pg_batch *b, const pg_grid *g, int dtype, void *out,
                                     unsigned *err, unsigned long long *sched, int sm_count,
                                     KernelLaunch *kl)
{
    kl->func = nullptr;
    pg_status st = validate(b, g);
    if (st) return st;
    if ((st = check_dtype(dtype))) return st;
    if (b->n_mol > 0 && !out) return fail(PG_ERR_INVALID_ARG, "out must not be NULL");
    if ((uintptr_t)out % dtype_size(dtype) != 0)
        return fail(PG_ERR_INVALID_ARG, "out is not aligned to its element size");
    if (b->n_mol == 0) return PG_OK;
    DirectArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = make_inputs(b);
    a.out = out;
    a.err = err;
    a.sched = sched;
    const pg_tuning t = default_tuning(PG_PATH_DIRECT);
    a.lane_lists = direct_lanes_on(b, g, t) ? 1 : 0;
    a.chunk_planes = 8;
    a.erf_tab = b->cell ? 0 : direct_erf_tab(b, g, t);
    make_geometry(b, g, &a.geo);
    const int vec = vec_stores_ok(out, g, dtype) ? 1 : 0;
    cudaError_t e = b->cell ? cell_plan(a, dtype, vec, t, sm_count, kl)
                            : direct_plan(a, dtype, vec, t, sm_count, kl);
    if (e != cudaSuccess) return cuda_fail(e, "direct_plan");
    return PG_OK;
}

}  // namespace pgi

extern "C" {

int32_t pg_version(void) { return PG_ABI_VERSION; }

const char *pg_last_error(void) { return t_last_error.c_str(); }

const char *pg_status_string(int32_t s)
{
    switch (s) {
    case PG_OK: return "PG_OK";
    case PG_ERR_INVALID_ARG: return "PG_ERR_INVALID_ARG";
    case PG_ERR_UNSUPPORTED: return "PG_ERR_UNSUPPORTED";
    case PG_ERR_CUDA: return "PG_ERR_CUDA";
    case PG_ERR_DEVICE_VALIDATION: return "PG_ERR_DEVICE_VALIDATION";
    case PG_ERR_TIMEOUT: return "PG_ERR_TIMEOUT";
    default: return "PG_ERR_UNKNOWN";
    }
}

pg_status pg_voxelize_tuned(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype,
                            void *out, const pg_tuning *tuning, void *stream)
{
    if (!tuning) return fail(PG_ERR_INVALID_ARG, "tuning must not be NULL");
    t_last_error.clear();
    return forward(batch, grid, out_dtype, out, *tuning, (cudaStream_t)stream);
}

pg_status pg_voxelize(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype, void *out,
                      int32_t path, void *stream)
{
    NvtxRange range("pg_voxelize");
    t_last_error.clear();
    if (path != PG_PATH_AUTO && path != PG_PATH_DIRECT && path != PG_PATH_SEPARABLE)
        return fail(PG_ERR_INVALID_ARG, "unknown path %d", path);
    pg_status st = validate(batch, grid);
    if (st) return st;
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    pg_tuning t = resolve(batch, grid, out_dtype, path, *d);
    if (path == PG_PATH_AUTO && t.path == PG_PATH_SEPARABLE &&
        (grid->cutoff == PG_CUTOFF_SPHERE || batch->cell))
        t = default_tuning(PG_PATH_DIRECT);
    return forward(batch, grid, out_dtype, out, t, (cudaStream_t)stream);
}

pg_status pg_voxelize_backward(const pg_batch *batch, const pg_grid *grid, int32_t grad_dtype,
                               const void *grad_out, float *grad_coords, void *stream)
{
    t_last_error.clear();
    if (batch && batch->n_atoms > 0 && !grad_coords)
        return fail(PG_ERR_INVALID_ARG, "grad_coords must not be NULL");
    return pg_voxelize_backward_ex(batch, grid, grad_dtype, grad_out, grad_coords, nullptr,
                                   stream);
}

pg_status pg_voxelize_backward_ex(const pg_batch *batch, const pg_grid *grid,
                                  int32_t grad_dtype, const void *grad_out, float *grad_coords,
                                  float *grad_weight, void *stream)
{
    NvtxRange range("pg_voxelize_backward");
    t_last_error.clear();
    pg_status st = validate(batch, grid);
    if (st) return st;
    if ((st = check_dtype(grad_dtype))) return st;
    if (batch->n_mol > 0 && !grad_out)
        return fail(PG_ERR_INVALID_ARG, "grad_out must not be NULL");
    if (batch->n_atoms > 0 && !grad_coords && !grad_weight)
        return fail(PG_ERR_INVALID_ARG, "grad_coords and grad_weight must not both be NULL");
    if ((uintptr_t)grad_out % dtype_size(grad_dtype) != 0 || (uintptr_t)grad_coords % 4 != 0 ||
        (uintptr_t)grad_weight % 4 != 0)
        return fail(PG_ERR_INVALID_ARG, "grad_out / grad_coords / grad_weight misaligned");
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    if (batch->n_atoms == 0) return PG_OK;
    BackwardArgs a;
    std::memset(&a, 0, sizeof a);
    a.in = make_inputs(batch);
    a.grad_out = grad_out;
    a.grad_coords = grad_coords;
    a.grad_weight = grad_weight;
    a.err = d->err;
    a.sched = d->take_slot();
    make_geometry(batch, grid, &a.geo);
    KernelLaunch kl;
    cudaError_t be = backward_plan(a, grad_dtype, d->sms, &kl);
    if (be == cudaErrorNotSupported)
        return fail(PG_ERR_UNSUPPORTED, "the adjoint does not cover this cell/cutoff");
    PG_CUDA(be, "backward_plan");
    PG_CUDA(launch(kl, (cudaStream_t)stream), "backward launch");
    return PG_OK;
}

size_t pg_refine_work_floats(const pg_batch *batch, const pg_grid *grid)
{
    if (!batch || !grid || batch->n_mol < 0 || batch->n_atoms < 0 || grid->nx <= 0 ||
        grid->ny <= 0 || grid->nz <= 0 || grid->n_channels <= 0)
        return 0;
    return (size_t)batch->n_mol * grid->n_channels * grid->nx * grid->ny * grid->nz +
           3 * (size_t)batch->n_atoms;
}

pg_status pg_refine(const pg_batch *batch, const pg_grid *grid, const float *target,
                    float *coords, float *work, float *loss, int32_t *steps, int32_t iters,
                    float lr, float eps, void *stream)
{
    NvtxRange range("pg_refine");
    t_last_error.clear();
    if (!batch) return fail(PG_ERR_INVALID_ARG, "batch must not be NULL");
    if (iters < 0) return fail(PG_ERR_INVALID_ARG, "iters must be >= 0");
    if (!(lr >= 0.0f) || !(lr < INFINITY))
        return fail(PG_ERR_INVALID_ARG, "lr must be finite and >= 0");
    if (!(eps >= 0.0f)) return fail(PG_ERR_INVALID_ARG, "eps must be >= 0");
    pg_batch b = *batch;
    b.coords = coords;  // the coordinates being refined
    pg_status st = validate(&b, grid);
    if (st) return st;
    if (b.n_mol > 0 && (!target || !work || !loss || !steps))
        return fail(PG_ERR_INVALID_ARG, "target, work, loss and steps are required");
    if ((uintptr_t)work % 16 != 0 || (uintptr_t)target % 4 != 0 || (uintptr_t)coords % 4 != 0)
        return fail(PG_ERR_INVALID_ARG, "work must be 16-byte aligned, target and coords 4-byte");
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    if (b.n_mol == 0) return PG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const long long per_mol = (long long)grid->n_channels * grid->nx * grid->ny * grid->nz;
    float *F = work;
    float *grad = work + per_mol * b.n_mol;
    PG_CUDA(cudaMemsetAsync(steps, 0, sizeof(int32_t) * b.n_mol, s), "clear steps");
    const pg_tuning t = resolve(&b, grid, PG_F32, PG_PATH_DIRECT, *d);
    for (int it = 0;; ++it) {
        if ((st = forward(&b, grid, PG_F32, F, t, s))) return st;
        PG_CUDA(refine_residual(F, target, b.n_mol, per_mol, loss, d->sms, s), "residual");
        if (it == iters) break;
        if ((st = pg_voxelize_backward(&b, grid, PG_F32, F, grad, stream))) return st;
        PG_CUDA(refine_update(coords, grad, b.mol_off, b.n_mol, b.n_atoms, loss, steps, lr,
                              eps, s),
                "update");
    }
    return PG_OK;
}

pg_status pg_sync_status(void *stream, uint32_t *bits_out)
{
    t_last_error.clear();
    Device *d = nullptr;
    pg_status st = get_device(&d);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PG_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    unsigned bits = 0;
    PG_CUDA(cudaMemcpyAsync(&bits, d->err, sizeof bits, cudaMemcpyDeviceToHost, s),
            "read error word");
    PG_CUDA(cudaMemsetAsync(d->err, 0, sizeof(unsigned), s), "clear error word");
    PG_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (bits_out) *bits_out = bits;
    if (bits & PG_DEVERR_TMEM_HELD) d->tmem_held->store(true);
    return report_bits(bits);
}

pg_status pg_get_tuning(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype,
                        int32_t path, pg_tuning *tuning)
{
    t_last_error.clear();
    pg_status st = validate(batch, grid);
    if (st) return st;
    if (!tuning) return fail(PG_ERR_INVALID_ARG, "tuning must not be NULL");
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    *tuning = resolve(batch, grid, out_dtype, path, *d);
    return PG_OK;
}

pg_status pg_autotune(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype, void *out,
                      int32_t path, void *stream, pg_tuning *chosen)
{
    NvtxRange range("pg_autotune");
    tuning_cache_init();
    t_last_error.clear();
    pg_status st = validate(batch, grid);
    if (st) return st;
    if ((st = check_dtype(out_dtype))) return st;
    if (path != PG_PATH_AUTO && path != PG_PATH_DIRECT && path != PG_PATH_SEPARABLE)
        return fail(PG_ERR_INVALID_ARG, "unknown path %d", path);
    if (batch->n_mol > 0 && !out) return fail(PG_ERR_INVALID_ARG, "out must not be NULL");
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (batch->n_mol == 0) {
        if (chosen) *chosen = default_tuning(path);
        return PG_OK;
    }

    // Every direct candidate (any launch shape, chunk order or dense-plane setting) adds the
    // same terms in the same order, so each must match the reference's bits.
    std::vector<pg_tuning> cands;
    if (path != PG_PATH_SEPARABLE) {
        // Full product of the direct kernel's launch knobs; the default comes first and is
        // the reference every other candidate must match bit for bit.
        cands.push_back(default_tuning(PG_PATH_DIRECT));
        const pg_tuning def = default_tuning(PG_PATH_DIRECT);
        const int go_max =
            (direct_lanes_on(batch, grid, def) || direct_erf_tab(batch, grid, def) > 0) ? 1 : 0;
        // The general-cell kernel has a fixed block and no store hint or lane-list mode: only
        // the residency and the chunk size vary.
        if (batch->cell)
            for (int order : {0, 1})
                for (int bps : {0, 1, 2})
                    for (int cp : {1, 2, 4, 8, 16}) {
                        pg_tuning t = default_tuning(PG_PATH_DIRECT);
                        t.blocks_per_sm = bps;
                        t.chunk_planes = cp;
                        t.chunk_order = order;
                        cands.push_back(t);
                    }
        for (int order : {0, 1})
            for (int threads : {128, 256, 512})
                for (int bps : {0, 1, 2})
                    for (int hint : {0, 1})
                        for (int cp : {1, 2, 4, 8, 16, 32})
                            for (int go = 0; go <= go_max && !batch->cell; ++go) {
                                pg_tuning t = default_tuning(PG_PATH_DIRECT);
                                t.block_threads = threads;
                                t.blocks_per_sm = bps;
                                t.store_hint = hint;
                                t.chunk_planes = cp;
                                t.gather_only = go;
                                t.chunk_order = order;
                                cands.push_back(t);
                            }
    }
    Geometry G;
    make_geometry(batch, grid, &G);
    const bool sep_ok = grid->cutoff != PG_CUTOFF_SPHERE && !batch->cell &&
                        separable_supported(G, out_dtype);
    if (path != PG_PATH_DIRECT && sep_ok) {
        // The pipelined kernel also tries a footprint of two CTAs per SM (fewer resident K
        // chunks) against the default of as many resident chunks as one CTA holds.
        for (int simple : {0, 1})
            for (int nt : {128, 256, 64})
                for (int bps : {0, 2}) {
                    if (simple && bps) continue;
                    pg_tuning t = default_tuning(PG_PATH_SEPARABLE);
                    t.n_tile = nt;
                    t.separable_simple = simple;
                    t.blocks_per_sm = bps;
                    cands.push_back(t);
                }
    }
    if (cands.empty())
        return fail(PG_ERR_UNSUPPORTED, "no eligible candidate for path %d (separable needs a "
                                        "NONE or BOX cutoff)", path);

    // Reference: the first candidate's output, as a full-bit hash plus a copy of the first
    // few molecules for tolerance checks of candidates that round differently.
    const size_t per_mol = (size_t)grid->n_channels * grid->nx * grid->ny * grid->nz;
    const int n_sample = std::min(batch->n_mol, 8);
    const size_t sample_elems = per_mol * n_sample;
    const size_t esz = dtype_size(out_dtype);
    void *sample = nullptr;
    void *spacer = nullptr;
    constexpr size_t kSpacerBytes = 32u << 20;
    unsigned long long *d_hash = nullptr;
    float *d_cmp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    std::vector<float> times(cands.size(), INFINITY);
    auto cleanup = [&]() {
        cudaFree(sample);
        cudaFree(spacer);
        cudaFree(d_hash);
        cudaFree(d_cmp);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e2) cudaEventDestroy(e2);
    };
    auto cu = [&](cudaError_t e, const char *what) -> pg_status {
        if (e == cudaSuccess) return PG_OK;
        cleanup();
        return cuda_fail(e, what);
    };
    if ((st = cu(cudaMalloc(&sample, sample_elems * esz), "cudaMalloc(tune sample)"))) return st;
    if ((st = cu(cudaMalloc(&spacer, kSpacerBytes), "cudaMalloc(tune spacer)"))) return st;
    if ((st = cu(cudaMalloc(&d_hash, sizeof(unsigned long long)), "cudaMalloc"))) return st;
    if ((st = cu(cudaMalloc(&d_cmp, 2 * sizeof(float)), "cudaMalloc"))) return st;
    if ((st = cu(cudaEventCreate(&e0), "cudaEventCreate"))) return st;
    if ((st = cu(cudaEventCreate(&e1), "cudaEventCreate"))) return st;
    if ((st = cu(cudaEventCreate(&e2), "cudaEventCreate"))) return st;
    const size_t out_bytes = per_mol * (size_t)batch->n_mol * esz;

    unsigned long long ref_hash = 0;
    int ref_index = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        KernelLaunch kl;
        if (plan_forward(batch, grid, out_dtype, out, cands[i], *d, d->err, d->take_slot(),
                         &kl) != PG_OK) {
            t_last_error.clear();
            continue;
        }
        if ((st = cu(launch(kl, s), "tune launch"))) return st;
        // Parity against the reference candidate.
        bool pass = true;
        if (ref_index < 0) {
            if ((st = cu(buffer_hash(out, out_bytes, d_hash, s), "hash"))) return st;
            if ((st = cu(cudaMemcpyAsync(&ref_hash, d_hash, sizeof ref_hash,
                                         cudaMemcpyDeviceToHost, s), "copy hash")))
                return st;
            if ((st = cu(cudaMemcpyAsync(sample, out, sample_elems * esz,
                                         cudaMemcpyDeviceToDevice, s), "copy sample")))
                return st;
            if ((st = cu(cudaStreamSynchronize(s), "sync"))) return st;
            ref_index = (int)i;
        } else if (cands[i].path == PG_PATH_DIRECT && cands[ref_index].path == PG_PATH_DIRECT) {
            unsigned long long h = 0;
            if ((st = cu(buffer_hash(out, out_bytes, d_hash, s), "hash"))) return st;
            if ((st = cu(cudaMemcpyAsync(&h, d_hash, sizeof h, cudaMemcpyDeviceToHost, s),
                         "copy hash")))
                return st;
            if ((st = cu(cudaStreamSynchronize(s), "sync"))) return st;
            pass = (h == ref_hash);
        } else {
            float cmp[2] = {0, 0};
            if ((st = cu(buffer_compare(out, sample, sample_elems, out_dtype, d_cmp, s),
                         "compare")))
                return st;
            if ((st = cu(cudaMemcpyAsync(cmp, d_cmp, sizeof cmp, cudaMemcpyDeviceToHost, s),
                         "copy compare")))
                return st;
            if ((st = cu(cudaStreamSynchronize(s), "sync"))) return st;
            // Separable candidates round through BF16 operands.
            pass = cmp[0] <= 1e-2f * cmp[1];
        }
        if (!pass) continue;
        // Time: median of 7 single launches, each after an unrelated fill of the spacer
        // buffer (outside the timed events).  That is how a launch runs in a training step,
        // a graph replay between other kernels or a plan run.  Back-to-back launches of one
        // candidate measured small chunks faster than they run there.
        std::vector<float> ms;
        for (int r = 0; r < 7; ++r) {
            if ((st = cu(cudaMemsetAsync(spacer, r, kSpacerBytes, s), "spacer"))) return st;
            if ((st = cu(cudaEventRecord(e0, s), "event"))) return st;
            if ((st = cu(launch(kl, s), "tune launch"))) return st;
            if ((st = cu(cudaEventRecord(e1, s), "event"))) return st;
            if ((st = cu(cudaEventSynchronize(e1), "event sync"))) return st;
            float t = 0;
            if ((st = cu(cudaEventElapsedTime(&t, e0, e1), "elapsed"))) return st;
            ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        times[i] = ms[ms.size() / 2];
    }

    // Second round: the fastest few candidates of each path are timed again, 15 times each,
    // interleaved so that clock and memory-state drift affects them alike.  Each time is a
    // pair of launches after the spacer fill: the first runs as after unrelated work, the
    // second right after a launch of the same kernel, as graph replays of one step follow
    // each other.  The sum of the two medians replaces the first-round time (halved, so that
    // it stays comparable to a single launch).
    {
        std::vector<int> order;
        for (size_t i = 0; i < cands.size(); ++i)
            if (std::isfinite(times[i])) order.push_back((int)i);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return times[a] < times[b]; });
        std::vector<int> top;
        int n_direct = 0, n_sep = 0;
        for (int i : order) {
            if (cands[i].path == PG_PATH_DIRECT && n_direct < 8) {
                top.push_back(i);
                ++n_direct;
            } else if (cands[i].path == PG_PATH_SEPARABLE && n_sep < 3) {
                top.push_back(i);
                ++n_sep;
            }
        }
        std::vector<KernelLaunch> kls(top.size());
        for (size_t t = 0; t < top.size(); ++t)
            if (plan_forward(batch, grid, out_dtype, out, cands[top[t]], *d, d->err,
                             d->take_slot(), &kls[t]) != PG_OK) {
                t_last_error.clear();
                kls[t].func = nullptr;
            }
        std::vector<std::vector<float>> ms(top.size()), ms2(top.size());
        for (int r = 0; r < 15; ++r)
            for (size_t t = 0; t < top.size(); ++t) {
                if (!kls[t].func) continue;
                if ((st = cu(cudaMemsetAsync(spacer, r, kSpacerBytes, s), "spacer"))) return st;
                if ((st = cu(cudaEventRecord(e0, s), "event"))) return st;
                if ((st = cu(launch(kls[t], s), "tune launch"))) return st;
                if ((st = cu(cudaEventRecord(e1, s), "event"))) return st;
                if ((st = cu(launch(kls[t], s), "tune launch"))) return st;
                if ((st = cu(cudaEventRecord(e2, s), "event"))) return st;
                if ((st = cu(cudaEventSynchronize(e2), "event sync"))) return st;
                float ev = 0, ev2 = 0;
                if ((st = cu(cudaEventElapsedTime(&ev, e0, e1), "elapsed"))) return st;
                if ((st = cu(cudaEventElapsedTime(&ev2, e1, e2), "elapsed"))) return st;
                ms[t].push_back(ev);
                ms2[t].push_back(ev2);
            }
        for (size_t t = 0; t < top.size(); ++t) {
            if (ms[t].empty()) continue;
            std::sort(ms[t].begin(), ms[t].end());
            std::sort(ms2[t].begin(), ms2[t].end());
            times[top[t]] = 0.5f * (ms[t][ms[t].size() / 2] + ms2[t][ms2[t].size() / 2]);
        }
    }
    cleanup();

    // Fastest candidate, except that direct candidates within 5% of the fastest direct time
    // count as tied and the tie goes to the largest chunk (then to the faster): fewer grabs
    // of the shared work counter.  Launches with small chunks that timed close to the fastest
    // ran up to a third slower as graph replays beside the adjoint.
    int best = -1, best_direct = -1, best_sep = -1;
    float t_direct = INFINITY;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (!std::isfinite(times[i])) continue;
        if (cands[i].path == PG_PATH_DIRECT) t_direct = std::min(t_direct, times[i]);
        if (cands[i].path == PG_PATH_SEPARABLE && (best_sep < 0 || times[i] < times[best_sep]))
            best_sep = (int)i;
    }
    for (size_t i = 0; i < cands.size(); ++i) {
        if (!std::isfinite(times[i]) || cands[i].path != PG_PATH_DIRECT) continue;
        if (times[i] > 1.05f * t_direct) continue;
        if (best_direct < 0 || cands[i].chunk_planes > cands[best_direct].chunk_planes ||
            (cands[i].chunk_planes == cands[best_direct].chunk_planes &&
             times[i] < times[best_direct]))
            best_direct = (int)i;
    }
    if (best_direct >= 0) best = best_direct;
    if (best_sep >= 0 && (best < 0 || times[best_sep] < times[best])) best = best_sep;
    if (best < 0) return fail(PG_ERR_CUDA, "no autotune candidate ran and passed parity");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[bucket_key(batch, grid, out_dtype, path, *d)] = cands[best];
        if (best_direct >= 0)
            g_tune[bucket_key(batch, grid, out_dtype, PG_PATH_DIRECT, *d)] = cands[best_direct];
        if (best_sep >= 0)
            g_tune[bucket_key(batch, grid, out_dtype, PG_PATH_SEPARABLE, *d)] = cands[best_sep];
    }
    if (chosen) *chosen = cands[best];
    if (const char *path_file = tuning_cache_path()) {
        if (pg_tuning_save(path_file) != PG_OK)
            return fail(PG_ERR_INVALID_ARG, "tuned, but the tuning cache %s could not be "
                                            "written", path_file);
    }
    return PG_OK;
}

pg_status pg_tuning_save(const char *file)
{
    t_last_error.clear();
    if (!file) return fail(PG_ERR_INVALID_ARG, "file must not be NULL");
    std::ofstream f(file);
    if (!f) return fail(PG_ERR_INVALID_ARG, "cannot write %s", file);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : g_tune)
        f << kv.first << ' ' << kv.second.path << ' ' << kv.second.block_threads << ' '
          << kv.second.blocks_per_sm << ' ' << kv.second.store_hint << ' ' << kv.second.n_tile
          << ' ' << kv.second.gather_only << ' ' << kv.second.chunk_planes << ' '
          << kv.second.separable_simple << ' ' << kv.second.chunk_order << '\n';
    return PG_OK;
}

pg_status pg_tuning_load(const char *file)
{
    t_last_error.clear();
    if (!file) return fail(PG_ERR_INVALID_ARG, "file must not be NULL");
    std::ifstream f(file);
    if (!f) return fail(PG_ERR_INVALID_ARG, "cannot read %s", file);
    std::string line;
    std::map<std::string, pg_tuning> add;
    while (std::getline(f, line)) {
        if (line.empty()) continue;
        std::istringstream is(line);
        std::string key;
        pg_tuning t;
        std::memset(&t, 0, sizeof t);
        if (!(is >> key >> t.path >> t.block_threads >> t.blocks_per_sm >> t.store_hint >>
              t.n_tile))
            return fail(PG_ERR_INVALID_ARG, "malformed tuning line: %s", line.c_str());
        if (!(is >> t.gather_only)) t.gather_only = 0;
        if (!(is >> t.chunk_planes)) t.chunk_planes = 8;
        if (!(is >> t.separable_simple)) t.separable_simple = 0;
        if (!(is >> t.chunk_order)) t.chunk_order = 0;
        add[key] = t;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : add) g_tune[kv.first] = kv.second;
    return PG_OK;
}

pg_status pg_plan_create(pg_plan **plan, const pg_grid *grid, int32_t out_dtype, int32_t path,
                         int32_t max_mol, int32_t max_atoms)
{
    t_last_error.clear();
    if (!plan) return fail(PG_ERR_INVALID_ARG, "plan must not be NULL");
    *plan = nullptr;
    pg_batch probe;
    std::memset(&probe, 0, sizeof probe);
    pg_status st = validate(&probe, grid);
    if (st) return st;
    if ((st = check_dtype(out_dtype))) return st;
    if (max_mol < 1 || max_atoms < 0) return fail(PG_ERR_INVALID_ARG, "bad plan capacity");
    if (path != PG_PATH_AUTO && path != PG_PATH_DIRECT && path != PG_PATH_SEPARABLE)
        return fail(PG_ERR_INVALID_ARG, "unknown path %d", path);
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;
    pg_plan *p = new pg_plan();
    p->device = d->id;
    p->grid = *grid;
    p->sigma.assign(grid->sigma, grid->sigma + grid->n_channels);
    p->grid.sigma = p->sigma.data();
    p->dtype = out_dtype;
    p->max_mol = max_mol;
    p->max_atoms = max_atoms;
    p->path = path;
    const size_t A = (size_t)std::max(max_atoms, 1), M = (size_t)max_mol;
    const size_t sizes[kPlanCopies] = {A * 3 * 4, A * 4,      (M + 1) * 4, M * 3 * 4,
                                       M * 3 * 4, A * 4, M * 9 * 4};
    size_t total = 0;
    for (int i = 0; i < kPlanCopies; ++i) {
        p->stage_off[i] = total;
        total += (sizes[i] + 255) / 256 * 256;
    }
    auto bad = [&](cudaError_t e, const char *what) {
        plan_free(p);
        return cuda_fail(e, what);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_coords, sizes[0])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_elem, sizes[1])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_moloff, sizes[2])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_origin, sizes[3])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_spacing, sizes[4])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_weight, sizes[5])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_cell, sizes[6])) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_err, sizeof(unsigned))) != cudaSuccess) return bad(e, "cudaMalloc");
    if ((e = cudaMalloc(&p->d_sched, 4 * sizeof(unsigned long long))) != cudaSuccess)
        return bad(e, "cudaMalloc");
    if ((e = cudaMemset(p->d_sched, 0, 4 * sizeof(unsigned long long))) != cudaSuccess)
        return bad(e, "cudaMemset");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bad(e, "cudaDeviceSynchronize");
    if ((e = cudaHostAlloc((void **)&p->h_stage, total, cudaHostAllocDefault)) != cudaSuccess)
        return bad(e, "cudaHostAlloc");
    if ((e = cudaHostAlloc((void **)&p->h_err, sizeof(unsigned), cudaHostAllocDefault)) !=
        cudaSuccess)
        return bad(e, "cudaHostAlloc");
    if ((e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess)
        return bad(e, "cudaEventCreateWithFlags");
    std::memset(p->h_stage, 0, total);
    *p->h_err = 0;
    *plan = p;
    return PG_OK;
}

pg_status pg_plan_run(pg_plan *p, const pg_batch *hb, void *out, void *stream)
{
    NvtxRange range("pg_plan_run (copies + kernel graph replay)");
    pg_status st = pg_plan_launch(p, hb, out, stream);
    if (st) return st;
    return pg_plan_wait(p, stream);
}

pg_status pg_plan_wait(pg_plan *p, void *stream)
{
    t_last_error.clear();
    if (!p) return fail(PG_ERR_INVALID_ARG, "plan must not be NULL");
    (void)stream;
    if (!p->in_flight) return PG_OK;
    const cudaError_t e = cudaEventSynchronize(p->done);
    p->in_flight = false;
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    if (*p->h_err & PG_DEVERR_TMEM_HELD) {
        Device *d = nullptr;
        if (get_device(&d) == PG_OK) d->tmem_held->store(true);
    }
    return report_bits(*p->h_err);
}

pg_status pg_plan_launch(pg_plan *p, const pg_batch *hb, void *out, void *stream)
{
    t_last_error.clear();
    if (!p) return fail(PG_ERR_INVALID_ARG, "plan must not be NULL");
    if (p->in_flight)
        return fail(PG_ERR_INVALID_ARG, "the plan's previous launch has not been waited for "
                                        "(pg_plan_wait)");
    pg_status st = validate(hb, &p->grid);
    if (st) return st;
    if (hb->n_mol > p->max_mol || hb->n_atoms > p->max_atoms)
        return fail(PG_ERR_INVALID_ARG, "batch (%d molecules, %d atoms) exceeds plan capacity "
                                        "(%d, %d)", hb->n_mol, hb->n_atoms, p->max_mol,
                    p->max_atoms);
    if (hb->n_mol > 0 && !out) return fail(PG_ERR_INVALID_ARG, "out must not be NULL");
    if ((uintptr_t)out % dtype_size(p->dtype) != 0)
        return fail(PG_ERR_INVALID_ARG, "out is not aligned to its element size");
    int dev = -1;
    PG_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->device) return fail(PG_ERR_INVALID_ARG, "plan belongs to device %d", p->device);
    if (hb->n_mol == 0) return PG_OK;
    Device *d = nullptr;
    if ((st = get_device(&d))) return st;

    // Absent optional arrays (spacing with a cell, weight, cell) copy 16 dummy bytes, so the
    // graph keeps one shape; the launch reads them as NULL.
    const void *host[kPlanCopies] = {hb->coords, hb->elem,   hb->mol_off, hb->origin,
                                     hb->spacing, hb->weight, hb->cell};
    const size_t nA = (size_t)hb->n_atoms, nM = (size_t)hb->n_mol;
    const size_t bytes[kPlanCopies] = {nA * 12,
                                       nA * 4,
                                       (nM + 1) * 4,
                                       nM * 12,
                                       hb->spacing ? nM * 12 : 0,
                                       hb->weight ? nA * 4 : 0,
                                       hb->cell ? nM * 36 : 0};
    void *const dst[kPlanCopies] = {p->d_coords,  p->d_elem,   p->d_moloff, p->d_origin,
                                    p->d_spacing, p->d_weight, p->d_cell};
    const void *src[kPlanCopies];
    size_t cnt[kPlanCopies];
    for (int i = 0; i < kPlanCopies; ++i) {
        unsigned char *slot = p->h_stage + p->stage_off[i];
        if (bytes[i] == 0) {  // graphs take no zero-length copies: move 16 dummy bytes
            src[i] = slot;
            cnt[i] = 16;
        } else if (is_pinned(host[i])) {
            src[i] = host[i];
            cnt[i] = bytes[i];
        } else {
            std::memcpy(slot, host[i], bytes[i]);
            src[i] = slot;
            cnt[i] = bytes[i];
        }
    }
    pg_batch db = *hb;
    db.coords = p->d_coords;
    db.elem = p->d_elem;
    db.mol_off = p->d_moloff;
    db.origin = p->d_origin;
    db.spacing = hb->spacing ? p->d_spacing : nullptr;
    db.weight = hb->weight ? p->d_weight : nullptr;
    db.cell = hb->cell ? p->d_cell : nullptr;
    KernelLaunch kl;
    // A batch with cell matrices always takes the general-cell kernel.
    // The launch choice of this batch's bucket (its atoms per molecule, and whether it
    // carries weights or cell matrices), as pg_voxelize would make it.
    pg_tuning t = resolve(hb, &p->grid, p->dtype, p->path, *d);
    if (t.path == PG_PATH_SEPARABLE && (p->grid.cutoff == PG_CUTOFF_SPHERE || hb->cell))
        t = default_tuning(PG_PATH_DIRECT);
    if ((st = plan_forward(&db, &p->grid, p->dtype, out, t, *d, p->d_err, p->d_sched, &kl)))
        return st;
    if ((st = plan_update_graph(p, src, cnt, dst, kl))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PG_CUDA(cudaGraphLaunch(p->exec, s), "cudaGraphLaunch");
    PG_CUDA(cudaEventRecord(p->done, s), "cudaEventRecord");
    p->in_flight = true;
    return PG_OK;
}

pg_status pg_plan_destroy(pg_plan *p)
{
    t_last_error.clear();
    if (p) plan_free(p);
    return PG_OK;
}

void pg_shutdown(void)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        int cur = -1;
        cudaGetDevice(&cur);
        for (auto &kv : g_devices) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            cudaFree(kv.second.err);
            cudaFree(kv.second.sched);
            delete kv.second.next_slot;
            delete kv.second.tmem_held;
        }
        g_devices.clear();
        if (cur >= 0) cudaSetDevice(cur);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // extern "C"
