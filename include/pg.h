/*
 * pg.h - C ABI of a GB300 (sm_103a) library for batched Gaussian-density voxelization,
 * the grid-generation method of ParticleGrid (arXiv 2211.08506).
 *
 * What is computed (Sec. III-A, Eq. 1, point-sampled and unnormalised): for molecule b,
 * channel c, voxel (i, j, k)
 *
 *     G[b][c][i][j][k] = sum over atoms a of b with elem[a] == c of
 *                        chi(d) * exp(-|d|^2 / (2 sigma_c^2)),
 *     d = v - x_a,   v = origin_b + ((i + 1/2) h_x, (j + 1/2) h_y, (k + 1/2) h_z),
 *
 * with h = spacing_b.  For periodic cells (Sec. III-A, nearest image) every component of
 * d is replaced by d - L round(d / L), L = n h on that axis (orthorhombic cell, origin at
 * its corner).  chi is the cutoff indicator with r_c = cutoff_k * sigma_c:
 * PG_CUTOFF_SPHERE: |d|^2 <= r_c^2; PG_CUTOFF_BOX: max_axis |d_axis| <= r_c;
 * PG_CUTOFF_NONE: always 1.  Sec. VI-B truncates where the Gaussian is negligible; here
 * the truncation radius is explicit.
 *
 * With voxel_form = PG_FORM_INTEGRAL each voxel instead holds the normalised Gaussian
 * integrated over the voxel (Sec. III-A, the gridding function after Eq. 5 and its per-axis
 * erf integrals): the product over axes of
 *     (1/2) [erf((e_hi - x) / (sqrt(2) sigma_c)) - erf((e_lo - x) / (sqrt(2) sigma_c))],
 * with e_lo, e_hi the voxel's edges and x the atom coordinate (its nearest image relative to
 * the voxel centre when periodic); chi is still evaluated at the voxel centre.  Each atom
 * then adds exactly one to a grid that covers its support (the conservation law after Eq. 5).
 *
 * Weighted grids (Sec. III-A, the remark that the gridding function extends to weighted
 * grids): with per-atom weights w_a (pg_batch.weight) every term is multiplied by w_a.
 *
 * General cells (Sec. III-A: the box's orientation and size are the user's choice and
 * voxels need not be cubic; crystals use the nearest image over lattice translations): a
 * batch may give per molecule a 3x3 matrix M (pg_batch.cell) whose rows a, b, c are the box
 * edges along which the grid's x, y and z indices run.  Voxel (i, j, k) then sits at
 *     v = origin_b + ((i + 1/2) / nx) a + ((j + 1/2) / ny) b + ((k + 1/2) / nz) c,
 * and spacing is not read.  For a periodic cell, d is the displacement to the nearest
 * lattice image of the atom.  The kernels find it by rounding the fractional displacement
 * (v - x) M^-1 per axis.  That is exact when the cutoff region reaches less than half a
 * cell along every fractional axis: r_c |g_k| < 1/2 for the sphere and sqrt(3) r_c |g_k| <
 * 1/2 for the box, with g_k column k of M^-1.  The device checks this and sets
 * PG_DEVERR_PERIODIC where it fails.  Cells take the point form on the direct path.  The
 * voxel-integrated form, the separable path and a periodic cell without a cutoff return
 * PG_ERR_UNSUPPORTED.
 *
 * General conventions
 *  - All buffers belong to the caller.  The library keeps only a small per-device error
 *    word, per-plan buffers (pg_plan_*) and an in-memory tuning cache; pg_shutdown()
 *    frees them.
 *  - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream) unless stated otherwise.  Device pointers
 *    must belong to the device that is current on the calling thread.
 *  - Errors found on the host (null pointers, negative counts, unsupported combinations)
 *    return immediately with a status and a message in pg_last_error(); nothing is
 *    launched.  Errors only visible in device data (an element id outside [0, C), CSR
 *    offsets that are not monotone or exceed n_atoms, non-positive spacing, a periodic
 *    cutoff radius of half a cell edge or more) never fault: the kernels skip the bad
 *    atom or molecule (its grid is written as zeros) and set a device error word that
 *    pg_sync_status() reports and clears.
 *  - No exception crosses this ABI and no kernel traps.
 */
#ifndef PG_H_
#define PG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PG_ABI_VERSION 2
#define PG_MAX_CHANNELS 64

typedef enum {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1,       /* rejected on the host, nothing launched */
    PG_ERR_UNSUPPORTED = 2,       /* valid but not implemented (e.g. separable + sphere) */
    PG_ERR_CUDA = 3,              /* a CUDA runtime call failed; message has the detail */
    PG_ERR_DEVICE_VALIDATION = 4, /* the device error word was set (see pg_sync_status) */
    PG_ERR_TIMEOUT = 5            /* a bounded device wait gave up (PG_DEVERR_TIMEOUT) */
} pg_status;

typedef enum { PG_F32 = 0, PG_F16 = 1, PG_BF16 = 2 } pg_dtype;

typedef enum { PG_CUTOFF_SPHERE = 0, PG_CUTOFF_NONE = 1, PG_CUTOFF_BOX = 2 } pg_cutoff;

/* Voxel function: the point sample at the voxel centre, or the voxel integral (erf form). */
typedef enum { PG_FORM_POINT = 0, PG_FORM_INTEGRAL = 1 } pg_form;

typedef enum {
    PG_PATH_AUTO = 0,      /* tuned choice for this problem's bucket, else DIRECT */
    PG_PATH_DIRECT = 1,    /* per-voxel gather: any cutoff, any dtype */
    PG_PATH_SEPARABLE = 2  /* tcgen05 BF16 contraction: NONE or BOX cutoff only */
} pg_path;

/* Device-error bits reported by pg_sync_status() / pg_plan_run(). */
#define PG_DEVERR_ELEMENT 0x1u   /* elem[a] outside [0, n_channels) */
#define PG_DEVERR_OFFSETS 0x2u   /* mol_off not monotone, negative, or > n_atoms */
#define PG_DEVERR_SPACING 0x4u   /* spacing <= 0 or not finite, or a singular cell matrix */
#define PG_DEVERR_PERIODIC 0x8u  /* periodic cell whose cutoff reaches half a cell or more */
#define PG_DEVERR_TIMEOUT 0x10u  /* a bounded wait on tensor-core completion gave up */
#define PG_DEVERR_TMEM_HELD 0x20u /* with 0x10: a CTA could not confirm that its MMAs had
                                     finished and kept its tensor memory instead of freeing it;
                                     separable launches on the device are then refused */

/*
 * A batch of B molecules in CSR form (Sec. V: points carry (channel, x, y, z); Sec. III-A:
 * per-molecule box and resolution).  For pg_voxelize* all pointers are DEVICE pointers;
 * for pg_plan_run they are HOST pointers.
 *   coords   float  [n_atoms][3]  Cartesian positions, Angstrom
 *   elem     int32  [n_atoms]     channel (element) id in [0, n_channels)
 *   mol_off  int32  [n_mol + 1]   atoms of molecule b are mol_off[b] .. mol_off[b+1]-1;
 *                                 mol_off[0] >= 0, non-decreasing, mol_off[n_mol] <= n_atoms
 *   origin   float  [n_mol][3]    lower corner of molecule b's grid box
 *   spacing  float  [n_mol][3]    voxel edges (h_x, h_y, h_z) of molecule b, > 0; not read
 *                                 (may be NULL) when `cell` is given
 *   weight   float  [n_atoms]     optional per-atom weights (weighted grids); NULL = all 1
 *   cell     float  [n_mol][3][3] optional box edges of molecule b, row-major, rows a, b, c
 *                                 along the grid's x, y, z axes (non-singular); NULL = the
 *                                 axis-aligned box of `spacing`
 * A zero-initialised pg_batch leaves weight and cell NULL (ABI version 1 behaviour).
 */
typedef struct {
    int32_t n_mol;
    int32_t n_atoms;
    const float *coords;
    const int32_t *elem;
    const int32_t *mol_off;
    const float *origin;
    const float *spacing;
    const float *weight;
    const float *cell;
} pg_batch;

/*
 * Grid description shared by the whole batch.
 *   nx, ny, nz   grid shape (>= 1); the output of a batch is the dense, contiguous array
 *                out[n_mol][n_channels][nx][ny][nz] (z fastest, Sec. III-A's
 *                (Channel, H, W, D) per molecule)
 *   n_channels   C, 1 .. PG_MAX_CHANNELS
 *   sigma        HOST float[C]: Gaussian width per channel (standard deviation, Angstrom,
 *                > 0; the paper's "variance" parameter, Sec. III-A / Sec. V)
 *   cutoff_k     r_c = cutoff_k * sigma_c (> 0; ignored for PG_CUTOFF_NONE)
 *   cutoff       pg_cutoff
 *   periodic     0: open boundaries; 1: periodic cell (edges n*h, or the batch's cell
 *                matrix) with nearest-image distances (requires r_c < L/2 on every axis of
 *                an axis-aligned cell, the reach condition above for a cell matrix; checked
 *                on the device)
 *   voxel_form   pg_form (0 = point sample; zero-initialised grids keep the point form)
 */
typedef struct {
    int32_t nx, ny, nz;
    int32_t n_channels;
    const float *sigma;
    float cutoff_k;
    int32_t cutoff;
    int32_t periodic;
    int32_t voxel_form;
} pg_grid;

/*
 * Launch choice for one problem bucket.  Zeros mean "library default".
 *   path           pg_path (DIRECT or SEPARABLE; AUTO resolves through the tuning cache)
 *   block_threads  threads per CTA of the direct kernel: 128, 256 or 512
 *   blocks_per_sm  persistent CTAs per SM (0 = as many as fit); on the pipelined separable
 *                  path 2 also sizes its resident K chunks so that two CTAs fit an SM
 *   store_hint     0: default global stores; 1: streaming (evict-first) stores
 *   n_tile         separable path: output columns per tensor-core tile (64, 128 or 256)
 *   gather_only    direct path, 0 allows the dense-plane modes: in the point form with a
 *                  cutoff (batches of molecules with more than 32 atoms on average), each
 *                  lane of a plane pass adds only the candidates that reach its own voxels
 *                  (lane lists); in the voxel-integrated form with no or a box cutoff,
 *                  every chunk's atoms get y and z factor tables in shared memory.  1: every
 *                  lane adds every candidate of the pass, and every factor is computed where
 *                  it is used.  Both give identical bits.
 *   chunk_planes   direct path: x-planes per dynamically scheduled work chunk (1..64; 0 = 8)
 *   separable_simple  separable path: 0 = warp-specialized pipeline (default), 1 = one-stage
 *                  kernel.  Both accumulate the same BF16 products in the same order.
 *   chunk_order    direct and general-cell kernels: 0 = chunks in (molecule, channel) order,
 *                  so concurrent stores stay close in memory; 1 = channel-major, which hands
 *                  out the largest chunks first when channels are listed by decreasing atom
 *                  frequency.  Results are identical bit for bit.
 */
typedef struct {
    int32_t path;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t store_hint;
    int32_t n_tile;
    int32_t gather_only;
    int32_t chunk_planes;
    int32_t separable_simple;
    int32_t chunk_order;
} pg_tuning;

/* Library ABI version (PG_ABI_VERSION). */
int32_t pg_version(void);

/* Message of the last failed call on this thread ("" if none).  Valid until the next call
   on the same thread. */
const char *pg_last_error(void);

/* Static name of a status code. */
const char *pg_status_string(int32_t status);

/*
 * Forward voxelization (Sec. III-A, Eq. 1; Sec. VI-B truncation): writes every element of
 * out[n_mol][C][nx][ny][nz] (zeros included; no pre-zeroing needed).
 *   out_dtype  pg_dtype of `out` (accumulation is always FP32; FP16/BF16 are rounded to
 *              nearest even on store)
 *   out        DEVICE buffer; 16-byte alignment enables vector stores (any alignment of
 *              the element type is accepted)
 *   path       pg_path.  SEPARABLE with PG_CUTOFF_SPHERE returns PG_ERR_UNSUPPORTED.
 * Returns PG_OK once the work is enqueued.
 */
pg_status pg_voxelize(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype, void *out,
                      int32_t path, void *stream);

/* pg_voxelize with an explicit launch choice (used by the tuner and by tests that check
   every candidate). */
pg_status pg_voxelize_tuned(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype,
                            void *out, const pg_tuning *tuning, void *stream);

/*
 * Adjoint of pg_voxelize with respect to the atom coordinates (Sec. IV-C, generalised from
 * the MSE loss to any upstream gradient): for L with dL/dG = grad_out,
 *     grad_coords[a] = sum_v grad_out[b][elem[a]][v] * chi(d) * exp(-|d|^2/(2 sigma^2))
 *                      * d / sigma^2,        d = v - x_a (nearest image if periodic).
 *   grad_dtype   pg_dtype of grad_out (read and widened to FP32)
 *   grad_out     DEVICE [n_mol][C][nx][ny][nz]
 *   grad_coords  DEVICE float [n_atoms][3], overwritten (not accumulated); atoms outside
 *                every molecule's CSR range get 0
 * Deterministic: one warp per atom, fixed-order reduction, no atomics.
 */
pg_status pg_voxelize_backward(const pg_batch *batch, const pg_grid *grid, int32_t grad_dtype,
                               const void *grad_out, float *grad_coords, void *stream);

/*
 * pg_voxelize_backward with the weight gradient of a weighted grid as well:
 *     grad_weight[a] = sum_v grad_out[b][elem[a]][v] * (atom a's unweighted term at v),
 * and grad_coords[a] as above (times w_a when batch->weight is given).
 *   grad_coords  DEVICE float [n_atoms][3] or NULL (not computed)
 *   grad_weight  DEVICE float [n_atoms] or NULL (not computed); atoms outside every
 *                molecule get 0
 * At least one of the two must be non-NULL when n_atoms > 0.
 */
pg_status pg_voxelize_backward_ex(const pg_batch *batch, const pg_grid *grid,
                                  int32_t grad_dtype, const void *grad_out, float *grad_coords,
                                  float *grad_weight, void *stream);

/*
 * Grid reversal by gradient descent (Sec. IV-A steps 2-5, Sec. IV-C).  For each molecule,
 * from the coordinates in `coords`, repeat on the stream (no host synchronisation):
 *     F = grid of x (FP32, as pg_voxelize on the direct path);
 *     L = sum_v (F(v) - target(v))^2 over the molecule's voxels;
 *     stop if L < eps;  otherwise  x <- x - lr * dL/dx,
 * with dL/dx = sum_v 2 (F - target) dF/dx, the adjoint of pg_voxelize_backward for the
 * upstream gradient 2 (F - target), for at most `iters` updates.
 *   batch    DEVICE CSR batch (elem, mol_off, origin, spacing, optional weight and cell,
 *            counts); batch->coords is not read, the coordinates come from `coords`
 *   target   DEVICE float[n_mol][C][nx][ny][nz]: the grid to reverse
 *   coords   DEVICE float[n_atoms][3]: starting coordinates, overwritten with the result
 *   work     DEVICE float workspace of pg_refine_work_floats(batch, grid) floats (the
 *            current grid and the coordinate gradient), caller-owned
 *   loss     DEVICE float[n_mol]: each molecule's loss at the returned coordinates
 *   steps    DEVICE int32[n_mol]: updates applied to each molecule
 *   iters >= 0, lr >= 0 and finite, eps >= 0 (eps = 0 runs exactly `iters` updates).
 * Each iteration launches the forward, residual, adjoint and update kernels; a molecule
 * that has reached eps keeps its coordinates (its loss is recomputed each iteration).
 */
pg_status pg_refine(const pg_batch *batch, const pg_grid *grid, const float *target,
                    float *coords, float *work, float *loss, int32_t *steps, int32_t iters,
                    float lr, float eps, void *stream);

/* Floats of workspace pg_refine needs: n_mol * C * nx * ny * nz + 3 * n_atoms. */
size_t pg_refine_work_floats(const pg_batch *batch, const pg_grid *grid);

/* Synchronize `stream`, then read and clear the device error word.  Returns
   PG_ERR_DEVICE_VALIDATION (bits in *bits_out if non-NULL) if it was set. */
pg_status pg_sync_status(void *stream, uint32_t *bits_out);

/*
 * Time every launch candidate for this problem's bucket (grid shape, dtype, cutoff,
 * periodicity, atoms-per-molecule bucket), check each against the first candidate's
 * output (bitwise for the direct kernel's launch shapes, 1e-2 of the grid maximum for
 * the separable path), and record the fastest passing one for PG_PATH_AUTO.
 * Each candidate is timed as the median of single launches that each follow an unrelated
 * 32 MB device fill, as a launch runs inside a larger step; the fastest few of each path
 * are then timed again, interleaved, as 15 pairs of launches after the fill (the first of a
 * pair as after unrelated work, the second right after the same kernel, as consecutive graph
 * replays run), and the mean of the two medians decides.
 * `out` is used as scratch and holds an arbitrary candidate's result afterwards; the call
 * also allocates and frees a 32 MB spacer buffer.
 * `path` restricts the search (AUTO = all eligible paths).  Synchronizes `stream`.
 * The chosen tuning is written to *chosen if non-NULL.
 */
pg_status pg_autotune(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype, void *out,
                      int32_t path, void *stream, pg_tuning *chosen);

/* The tuning PG_PATH_AUTO (or the given path) would use for this problem. */
pg_status pg_get_tuning(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype,
                        int32_t path, pg_tuning *tuning);

/* Tuning cache as text lines "key value..."; load merges into the in-memory cache.
   If the environment variable PG_TUNING_CACHE names a file, the library merges it into the
   cache on first use (when it exists) and pg_autotune rewrites it with the whole cache after
   every successful tuning (PG_ERR_INVALID_ARG if it cannot be written). */
pg_status pg_tuning_save(const char *file);
pg_status pg_tuning_load(const char *file);

/*
 * Plans: fixed-capacity input buffers plus a CUDA graph holding the host-to-device copy
 * of a batch and the voxelization launch, for on-the-fly grid generation from host data
 * (the data-loader use of Sec. V / Sec. VI-D).
 *   pg_plan_create  capacity max_mol molecules / max_atoms atoms; grid, dtype and path fixed.
 *                   Each run launches the choice pg_voxelize would make for its batch's
 *                   bucket (atoms per molecule, weights, cell matrices).
 *   pg_plan_run     batch holds HOST pointers (pinned memory is copied directly;
 *                   pageable memory is first packed into the plan's pinned staging),
 *                   weight and cell included when given;
 *                   replays the graph on `stream`, writes `out` (DEVICE), then copies the
 *                   4-byte device error word back and waits for the graph to finish.
 *                   Returns PG_ERR_DEVICE_VALIDATION if it was set.  Not thread-safe per
 *                   plan.
 *   pg_plan_destroy frees the plan (synchronize users of it first).
 */
typedef struct pg_plan pg_plan;
pg_status pg_plan_create(pg_plan **plan, const pg_grid *grid, int32_t out_dtype, int32_t path,
                         int32_t max_mol, int32_t max_atoms);
pg_status pg_plan_run(pg_plan *plan, const pg_batch *host_batch, void *out, void *stream);
pg_status pg_plan_destroy(pg_plan *plan);

/*
 * pg_plan_run in two halves, so that more work can follow the plan on the stream before the
 * one host synchronization (in a differentiation step: the adjoint and the copy of the
 * coordinate gradient to the host).
 *   pg_plan_launch  everything pg_plan_run does up to and including the graph launch on
 *                   `stream`; returns without synchronizing.  Host inputs must stay unchanged
 *                   until the wait (pinned ones are copied by the graph).  One launch per
 *                   plan may be outstanding: a second launch before the wait returns
 *                   PG_ERR_INVALID_ARG.
 *   pg_plan_wait    waits for the plan's outstanding launch (its copies, kernel and error
 *                   word; not for later work on the stream) and reports the device error
 *                   word as pg_plan_run would (PG_OK if none is outstanding).  `stream` is
 *                   the launch's stream (kept for symmetry; the wait uses an event recorded
 *                   after the launch).
 * Two plans of the same shape can alternate (double buffering): launch one batch, then wait
 * for the previous batch's plan while the new one runs.
 */
pg_status pg_plan_launch(pg_plan *plan, const pg_batch *host_batch, void *out, void *stream);
pg_status pg_plan_wait(pg_plan *plan, void *stream);

/* Free per-device state and the tuning cache.  Later calls re-create what they need. */
void pg_shutdown(void);

/*
 * pg_voxelize_noalloc - forward voxelization that allocates no device memory.
 *
 * The paper has no counterpart: this serves callers that cannot let a library allocate.
 * The other entry points cudaMalloc a small per-device state the first time they run on a
 * device.  That is not possible while another thread holds a stream capture open in global
 * mode (cudaMalloc is then refused and the capture is invalidated), and it is not acceptable
 * when a framework's caching allocator or an external budget owns all device memory, or when
 * a host freezes its device-memory footprint after start-up.  This call runs the direct
 * kernel with its scratch - the work counter and the error word - in a fixed
 * PG_NOALLOC_SCRATCH_BYTES array compiled into the library, which every GPU that loads the
 * library holds until the process exits.  A launch needs 24 bytes of it whatever the batch
 * size; a launch that needed more than the array holds would be rejected with
 * PG_ERR_INVALID_ARG.
 * Results are identical, bit for bit, to pg_voxelize_tuned with the default launch of the
 * direct path (a zeroed pg_tuning with path = PG_PATH_DIRECT), and so to pg_voxelize with
 * PG_PATH_DIRECT: every launch choice of the direct path gives the same bits.
 *   batch, grid, out_dtype, out   as for pg_voxelize (DEVICE buffers, caller-owned)
 *   stream                        cudaStream_t as void*, not capturing (a capturing stream
 *                                 returns PG_ERR_INVALID_ARG: the call waits for its own
 *                                 work).  While another thread holds a capture open, pass a
 *                                 stream created with cudaStreamNonBlocking: work on the
 *                                 legacy default stream (NULL) would depend implicitly on the
 *                                 capturing stream and invalidate that capture.
 *   bits_out                      if non-NULL, receives the device error bits (PG_DEVERR_*)
 * Synchronous without synchronizing calls (which a global-mode capture held by another thread
 * refuses): it clears the scratch, launches, and copies the error word together with a
 * completion marker into a static page-locked host word, then waits on the host until the
 * marker arrives.  Returns PG_ERR_DEVICE_VALIDATION if an error bit was set, PG_ERR_TIMEOUT
 * if the work has not finished after 600 s (it may still be running then).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current, and the first call in the process page-locks (cudaHostRegister,
 * no allocation) the 256 bytes of static host words; make that first call before any stream
 * capture.  All calls share the one device array and host word: calls that overlap
 * (different streams or threads) race on them and must be serialized by the caller.
 */
#define PG_NOALLOC_SCRATCH_BYTES 256
pg_status pg_voxelize_noalloc(const pg_batch *batch, const pg_grid *grid, int32_t out_dtype,
                              void *out, void *stream, uint32_t *bits_out);

#ifdef __cplusplus
}
#endif

#endif /* PG_H_ */
