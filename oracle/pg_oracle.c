/*
 * pg_oracle.c - plain FP64 CPU oracle for Gaussian-density voxelization
 * (ParticleGrid, arXiv 2211.08506).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  It shares no code, header, table or
 * constant with the CUDA library; it is slow on purpose and written so each function
 * can be checked against the paper by eye.
 *
 * What it computes (Sec. III-A, Eq. 1, with the point-sampled, unnormalised reading):
 *
 *   G[b,c,i,j,k] = sum over atoms a of molecule b with elem(a) = c of
 *                  chi(d) * exp(-|d|^2 / (2 sigma_c^2)),
 *   d = v_ijk - x_a,  v_ijk = o_b + ((i+1/2) h_x, (j+1/2) h_y, (k+1/2) h_z),
 *
 * where, for periodic cells (Sec. III-A, nearest image), each component of d is replaced
 * by its minimum image d - L round(d/L) with L = n h on that axis, and chi is the cutoff
 * indicator: [|d|^2 <= r_c^2] (sphere), [max_a |d_a| <= r_c] (box) or 1 (none), with
 * r_c = k sigma_c.  Output layout [B][C][nx][ny][nz], z fastest.
 *
 * The coordinate gradient of L = <W, G> (Sec. IV-C, generalised from the MSE loss to any
 * upstream weight W = dL/dG) is
 *
 *   dL/dx_a = sum_v W[b, elem(a), v] * chi(d) * exp(-|d|^2/(2 sigma^2)) * d / sigma^2.
 *
 * Readings taken where the paper is silent or differs from the point-sampled form:
 * voxel values are sampled at voxel centres; sigma is the standard deviation; the cutoff
 * is inclusive; atoms outside the grid still contribute wherever their support reaches.
 *
 * Voxel-integrated form (Sec. III-A, the gridding function after Eq. 5 and its per-axis
 * erf integrals).  Instead of the point sample, each voxel holds the normalised Gaussian
 * integrated over the voxel, a product of one factor per axis:
 *
 *   F = (1/2)^3 * prod over axes of [erf((x_i + h - mu) / (sqrt(2) sigma))
 *                                    - erf((x_i - mu) / (sqrt(2) sigma))],
 *
 * with x_i the voxel's lower edge and mu the atom coordinate (its nearest image relative
 * to the voxel centre on a periodic axis).  The printed formula is taken in this order, the
 * upper edge first, so that each factor is positive.  The cutoff indicator chi is evaluated
 * at the voxel centre exactly as in the point form.  Its coordinate derivative (Sec. IV-C) is
 * per axis
 *
 *   d/dmu [...]/2 = (1 / (sqrt(2 pi) sigma)) [exp(-(x_i - mu)^2 / 2 sigma^2)
 *                                            - exp(-(x_i + h - mu)^2 / 2 sigma^2)],
 *
 * times the other two axes' factors.  This uses d/dt erf(t) = (2 / sqrt(pi)) exp(-t^2).
 *
 * Weighted grids (Sec. III-A, the remark that the gridding function extends to weighted
 * grids): with per-atom weights w_a every term above is multiplied by w_a, so
 *   G = sum_a w_a chi(d) exp(...),  dL/dx_a = w_a * (the unweighted sum),
 *   dL/dw_a = sum_v W(v) chi(d) exp(...)   (the atom's own unweighted grid against W).
 * A null weight array means w_a = 1.
 *
 * General cells (Sec. III-A: the box's orientation and size are the user's choice and
 * voxels need not be cubic; periodic crystals use the nearest image over the lattice
 * translations).  A molecule may give a 3x3 matrix M whose rows a, b, c are the box edges
 * along which the grid's x, y and z indices run.  Its voxel centres are then
 *   v_ijk = o + ((i+1/2)/nx) a + ((j+1/2)/ny) b + ((k+1/2)/nz) c,
 * and spacing is ignored.  For a periodic cell, d is the displacement to the nearest
 * image x + t_a a + t_b b + t_c c (t integer).  It is found exactly by enumeration: with
 * e = (v - x) M^-1 the fractional displacement and R the distance to the image t = round(e),
 * any image at most R away has |e_k - t_k| <= R |g_k|, where g_k is column k of M^-1.  All
 * such t are tried and the shortest d wins; among equals the first in (t_a, t_b, t_c)
 * lexicographic order wins.  chi and the Gaussian are evaluated at that d.  The
 * voxel-integrated and separable forms assume an axis-aligned box and reject cells.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { PGO_SPHERE = 0, PGO_NONE = 1, PGO_BOX = 2 };
enum { PGO_POINT = 0, PGO_INTEGRAL = 1 };
enum { PGO_OK = 0, PGO_BAD_ARG = 1, PGO_BAD_ELEM = 2, PGO_UNSUPPORTED = 3 };

typedef struct {
    int32_t n_mol;
    const int32_t *mol_off;  /* [B+1] */
    const double *coords;    /* [N][3] */
    const int32_t *elem;     /* [N] */
    const double *origin;    /* [B][3] */
    const double *spacing;   /* [B][3] */
    int32_t nx, ny, nz, n_channels;
    const double *sigma;     /* [C] */
    double cutoff_k;
    int32_t cutoff;          /* PGO_SPHERE / PGO_NONE / PGO_BOX */
    int32_t periodic;
    int32_t form;            /* PGO_POINT / PGO_INTEGRAL */
    const double *weight;    /* [N] per-atom weights, or NULL for all ones */
    const double *cell;      /* [B][3][3] rows = grid box edges a, b, c, or NULL */
} pgo_problem;

/* Voxel centre along one axis: o + (i + 1/2) h. */
static double centre(double o, double h, long i) { return o + ((double)i + 0.5) * h; }

/* Nearest-image displacement on a periodic axis of length L (Sec. III-A). */
static double min_image(double d, double L) { return d - L * round(d / L); }

/* Cutoff indicator chi for displacement (dx, dy, dz) and radius r. */
static int inside(int cutoff, double dx, double dy, double dz, double r)
{
    if (cutoff == PGO_SPHERE) return dx * dx + dy * dy + dz * dz <= r * r;
    if (cutoff == PGO_BOX) return fabs(dx) <= r && fabs(dy) <= r && fabs(dz) <= r;
    return 1;
}

/*
 * One axis of the voxel-integrated form: half the erf difference across the voxel whose
 * centre lies at displacement d from the atom (lower edge at d - h/2, upper at d + h/2).
 */
static double erf_factor(double d, double h, double sigma)
{
    double s = sqrt(2.0) * sigma;
    return 0.5 * (erf((d + 0.5 * h) / s) - erf((d - 0.5 * h) / s));
}

/* Derivative of erf_factor with respect to the atom coordinate (d = centre - mu). */
static double erf_factor_dmu(double d, double h, double sigma)
{
    double s2 = 2.0 * sigma * sigma;
    double lo = d - 0.5 * h, hi = d + 0.5 * h;
    return (exp(-lo * lo / s2) - exp(-hi * hi / s2)) / (sqrt(2.0 * acos(-1.0)) * sigma);
}

/*
 * The value one atom adds to a voxel at displacement d (inside the cutoff): the point
 * sample exp(-|d|^2 / 2 sigma^2), or the product of the three erf factors.
 */
static double term(const pgo_problem *p, int b, double sigma, double dx, double dy, double dz)
{
    if (p->form == PGO_INTEGRAL) {
        const double *h = p->spacing + 3 * b;
        return erf_factor(dx, h[0], sigma) * erf_factor(dy, h[1], sigma) *
               erf_factor(dz, h[2], sigma);
    }
    return exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * sigma * sigma));
}

/* Weight of atom a (1 without weights). */
static double weight_of(const pgo_problem *p, int a) { return p->weight ? p->weight[a] : 1.0; }

/* Inverse of the 3x3 row-major matrix M by its adjugate (M non-singular). */
static void inverse3(const double *M, double *Mi)
{
    double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                 M[2] * (M[3] * M[7] - M[4] * M[6]);
    Mi[0] = (M[4] * M[8] - M[5] * M[7]) / det;
    Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
    Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    Mi[3] = (M[5] * M[6] - M[3] * M[8]) / det;
    Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
    Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    Mi[6] = (M[3] * M[7] - M[4] * M[6]) / det;
    Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
    Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
}

/* |g_k| for k = 0, 1, 2: the lengths of the columns of M^-1. */
static void column_norms(const double *Mi, double *g)
{
    for (int k = 0; k < 3; ++k)
        g[k] = sqrt(Mi[k] * Mi[k] + Mi[3 + k] * Mi[3 + k] + Mi[6 + k] * Mi[6 + k]);
}

/*
 * Displacement d from atom position x to voxel (i, j, k) of molecule b in a general cell:
 * v - x, or for a periodic cell the displacement to the nearest lattice image of the atom
 * (exact enumeration, see the file header).
 */
static void cell_disp(const pgo_problem *p, int b, long i, long j, long k, const double *x,
                      double *d)
{
    const double *M = p->cell + 9 * b, *o = p->origin + 3 * b;
    const double u[3] = {((double)i + 0.5) / p->nx, ((double)j + 0.5) / p->ny,
                         ((double)k + 0.5) / p->nz};
    double d0[3];
    for (int c = 0; c < 3; ++c)
        d0[c] = o[c] + u[0] * M[c] + u[1] * M[3 + c] + u[2] * M[6 + c] - x[c];
    if (!p->periodic) {
        d[0] = d0[0];
        d[1] = d0[1];
        d[2] = d0[2];
        return;
    }
    double Mi[9], g[3], e[3];
    inverse3(M, Mi);
    column_norms(Mi, g);
    for (int c = 0; c < 3; ++c) e[c] = d0[0] * Mi[c] + d0[1] * Mi[3 + c] + d0[2] * Mi[6 + c];
    long t0[3], lo[3], hi[3];
    double R2 = 0.0;
    for (int c = 0; c < 3; ++c) t0[c] = lround(e[c]);
    for (int c = 0; c < 3; ++c) {
        double dc = d0[c] - t0[0] * M[c] - t0[1] * M[3 + c] - t0[2] * M[6 + c];
        R2 += dc * dc;
    }
    for (int c = 0; c < 3; ++c) {
        double w = sqrt(R2) * g[c];
        lo[c] = (long)ceil(e[c] - w);
        hi[c] = (long)floor(e[c] + w);
        if (lo[c] > t0[c]) lo[c] = t0[c];
        if (hi[c] < t0[c]) hi[c] = t0[c];
    }
    double best = INFINITY;
    for (long ta = lo[0]; ta <= hi[0]; ++ta)
        for (long tb = lo[1]; tb <= hi[1]; ++tb)
            for (long tc = lo[2]; tc <= hi[2]; ++tc) {
                double dt[3], r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    dt[c] = d0[c] - ta * M[c] - tb * M[3 + c] - tc * M[6 + c];
                    r2 += dt[c] * dt[c];
                }
                if (r2 < best) {
                    best = r2;
                    d[0] = dt[0];
                    d[1] = dt[1];
                    d[2] = dt[2];
                }
            }
}

/*
 * Index range [lo, hi] on axis k of a general cell that holds every voxel whose centre can
 * be within r of the atom: the fractional coordinate of such a centre is within r |g_k| of
 * the atom's (modulo 1 when periodic), widened by one voxel each side.  Clamped to the grid
 * when not periodic; at most n consecutive indices when periodic.
 */
static void cell_support(const pgo_problem *p, int b, int k, const double *x, double r,
                         long *lo, long *hi)
{
    const int n[3] = {p->nx, p->ny, p->nz};
    if (p->cutoff == PGO_NONE) {
        *lo = 0;
        *hi = n[k] - 1;
        return;
    }
    const double *M = p->cell + 9 * b, *o = p->origin + 3 * b;
    double Mi[9], g[3];
    inverse3(M, Mi);
    column_norms(Mi, g);
    double f = (x[0] - o[0]) * Mi[k] + (x[1] - o[1]) * Mi[3 + k] + (x[2] - o[2]) * Mi[6 + k];
    /* The box cutoff reaches sqrt(3) r from the atom. */
    double reach = (p->cutoff == PGO_BOX ? sqrt(3.0) : 1.0) * r * g[k];
    long l = (long)floor((f - reach) * n[k] - 0.5) - 1;
    long u = (long)ceil((f + reach) * n[k] - 0.5) + 1;
    if (p->periodic) {
        if (u - l + 1 > n[k]) u = l + n[k] - 1;
    } else {
        if (l < 0) l = 0;
        if (u > n[k] - 1) u = n[k] - 1;
    }
    *lo = l;
    *hi = u;
}

static long grid_index(const pgo_problem *p, long b, long c, long i, long j, long k)
{
    return (((b * p->n_channels + c) * p->nx + i) * p->ny + j) * p->nz + k;
}

static int check(const pgo_problem *p)
{
    if (!p || p->n_mol < 0 || p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->n_channels <= 0)
        return PGO_BAD_ARG;
    if (p->cutoff != PGO_SPHERE && p->cutoff != PGO_NONE && p->cutoff != PGO_BOX)
        return PGO_BAD_ARG;
    if (p->form != PGO_POINT && p->form != PGO_INTEGRAL) return PGO_BAD_ARG;
    if (p->cell && p->form != PGO_POINT) return PGO_UNSUPPORTED;
    for (int b = 0; b < p->n_mol; ++b)
        for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a)
            if (p->elem[a] < 0 || p->elem[a] >= p->n_channels) return PGO_BAD_ELEM;
    return PGO_OK;
}

/* Displacement d = v - x on axis ax for voxel index i of molecule b. */
static double disp(const pgo_problem *p, int b, int ax, long i, double x)
{
    const int n[3] = {p->nx, p->ny, p->nz};
    double o = p->origin[3 * b + ax], h = p->spacing[3 * b + ax];
    double d = centre(o, h, i) - x;
    if (p->periodic) d = min_image(d, n[ax] * h);
    return d;
}

/*
 * Brute force: every voxel of every channel sums over every atom of the molecule, in
 * atom order.  This is the definition with nothing skipped.
 */
static void brute_molecule(const pgo_problem *p, int b, double *out)
{
    for (int c = 0; c < p->n_channels; ++c) {
        double r = p->cutoff_k * p->sigma[c];
        for (long i = 0; i < p->nx; ++i)
            for (long j = 0; j < p->ny; ++j)
                for (long k = 0; k < p->nz; ++k) {
                    double s = 0.0;
                    for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a) {
                        if (p->elem[a] != c) continue;
                        double d[3];
                        if (p->cell) {
                            cell_disp(p, b, i, j, k, p->coords + 3 * a, d);
                        } else {
                            d[0] = disp(p, b, 0, i, p->coords[3 * a + 0]);
                            d[1] = disp(p, b, 1, j, p->coords[3 * a + 1]);
                            d[2] = disp(p, b, 2, k, p->coords[3 * a + 2]);
                        }
                        if (inside(p->cutoff, d[0], d[1], d[2], r))
                            s += weight_of(p, a) * term(p, b, p->sigma[c], d[0], d[1], d[2]);
                    }
                    out[grid_index(p, b, c, i, j, k)] = s;
                }
    }
}

/*
 * Index range [lo, hi] on one axis that holds every voxel centre within r of x
 * (widened by one voxel each side; chi decides exactly).  Non-periodic ranges are
 * clamped to the grid; periodic ranges are left unwrapped but cover at most n
 * consecutive indices, so after wrapping no voxel is visited twice.
 */
static void support(const pgo_problem *p, int b, int ax, double x, double r, long *lo, long *hi)
{
    const int n[3] = {p->nx, p->ny, p->nz};
    if (p->cutoff == PGO_NONE) {
        *lo = 0;
        *hi = n[ax] - 1;
        return;
    }
    double o = p->origin[3 * b + ax], h = p->spacing[3 * b + ax];
    long l = (long)floor((x - r - o) / h - 0.5) - 1;
    long u = (long)ceil((x + r - o) / h - 0.5) + 1;
    if (p->periodic) {
        if (u - l + 1 > n[ax]) u = l + n[ax] - 1;
    } else {
        if (l < 0) l = 0;
        if (u > n[ax] - 1) u = n[ax] - 1;
    }
    *lo = l;
    *hi = u;
}

static long wrap_index(long i, long n) { return ((i % n) + n) % n; }

/*
 * Support-box mode: the same sum, visited atom by atom over each atom's cutoff box
 * only (chi is zero outside it).  Per voxel the atoms are still added in atom order, so
 * the result equals brute force bit for bit.  With eps > 0 it instead splits the sum into
 * out (contributions inside the cutoff by more than a relative eps) and band (every
 * contribution, inside or outside, whose |d|^2 is within eps * r^2 of r^2), so that a
 * lower-precision implementation of the cutoff test can be bracketed.
 */
static void bbox_molecule(const pgo_problem *p, int b, double *out, double eps, double *band)
{
    long per_mol = (long)p->n_channels * p->nx * p->ny * p->nz;
    memset(out + b * per_mol, 0, sizeof(double) * per_mol);
    if (band) memset(band + b * per_mol, 0, sizeof(double) * per_mol);
    for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a) {
        int c = p->elem[a];
        double r = p->cutoff_k * p->sigma[c];
        double wa = weight_of(p, a);
        const double *xa = p->coords + 3 * a;
        double x = xa[0], y = xa[1], z = xa[2];
        long ilo, ihi, jlo, jhi, klo, khi;
        if (p->cell) {
            cell_support(p, b, 0, xa, r, &ilo, &ihi);
            cell_support(p, b, 1, xa, r, &jlo, &jhi);
            cell_support(p, b, 2, xa, r, &klo, &khi);
        } else {
            support(p, b, 0, x, r, &ilo, &ihi);
            support(p, b, 1, y, r, &jlo, &jhi);
            support(p, b, 2, z, r, &klo, &khi);
        }
        for (long iu = ilo; iu <= ihi; ++iu) {
            long i = p->periodic ? wrap_index(iu, p->nx) : iu;
            double dx = p->cell ? 0.0 : disp(p, b, 0, i, x);
            for (long ju = jlo; ju <= jhi; ++ju) {
                long j = p->periodic ? wrap_index(ju, p->ny) : ju;
                double dy = p->cell ? 0.0 : disp(p, b, 1, j, y);
                for (long ku = klo; ku <= khi; ++ku) {
                    long k = p->periodic ? wrap_index(ku, p->nz) : ku;
                    double dz;
                    if (p->cell) {
                        double d[3];
                        cell_disp(p, b, i, j, k, xa, d);
                        dx = d[0];
                        dy = d[1];
                        dz = d[2];
                    } else {
                        dz = disp(p, b, 2, k, z);
                    }
                    double d2 = dx * dx + dy * dy + dz * dz;
                    long v = grid_index(p, b, c, i, j, k);
                    if (eps > 0.0 && p->cutoff != PGO_NONE) {
                        /* Two-sided band: contributions within eps of the cutoff surface,
                           inside or outside, may flip in a lower-precision test. */
                        double m2 = (p->cutoff == PGO_SPHERE)
                                        ? d2
                                        : fmax(dx * dx, fmax(dy * dy, dz * dz));
                        if (fabs(m2 - r * r) <= eps * r * r) {
                            band[v] += wa * term(p, b, p->sigma[c], dx, dy, dz);
                            continue;
                        }
                    }
                    if (!inside(p->cutoff, dx, dy, dz, r)) continue;
                    out[v] += wa * term(p, b, p->sigma[c], dx, dy, dz);
                }
            }
        }
    }
}

static int threads_or_default(int n_threads)
{
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

/* mode 0: brute force, mode 1: support box.  out: [B][C][nx][ny][nz]. */
int pgo_voxelize(const pgo_problem *p, int mode, double *out, int n_threads)
{
    int st = check(p);
    if (st) return st;
    int nt = threads_or_default(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) {
        if (mode == 0)
            brute_molecule(p, b, out);
        else
            bbox_molecule(p, b, out, 0.0, NULL);
    }
    return PGO_OK;
}

/* Split into strictly-inside and cutoff-band contributions (see bbox_molecule). */
int pgo_voxelize_band(const pgo_problem *p, double eps, double *out_in, double *out_band,
                      int n_threads)
{
    int st = check(p);
    if (st) return st;
    if (!(eps > 0.0)) return PGO_BAD_ARG;
    int nt = threads_or_default(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) bbox_molecule(p, b, out_in, eps, out_band);
    return PGO_OK;
}

/*
 * Separable form (Sec. III-A after Eq. 5; Sec. VI-A): for the no-cutoff and box-cutoff
 * indicators the Gaussian factors per axis, so the grid is the per-channel sum of outer
 * products of three per-axis tables
 *   g_x[a][i] = [|d_x| <= r] exp(-d_x^2 / 2 sigma^2)  (the bracket is 1 with no cutoff),
 * or [|d_x| <= r] times the erf factor in the voxel-integrated form,
 * and G[c,i,j,k] = sum_{a: elem(a)=c} g_x[a][i] g_y[a][j] g_z[a][k].
 * With weights, g_x of atom a is multiplied by w_a.  The spherical indicator does not
 * factor, and neither does the metric of a general cell; those cases are rejected.
 */
int pgo_separable(const pgo_problem *p, double *out, int n_threads)
{
    int st = check(p);
    if (st) return st;
    if (p->cutoff == PGO_SPHERE || p->cell) return PGO_UNSUPPORTED;
    int nt = threads_or_default(n_threads);
    (void)nt;
    long per_mol = (long)p->n_channels * p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) {
        double *gx = malloc(sizeof(double) * p->nx);
        double *gy = malloc(sizeof(double) * p->ny);
        double *gz = malloc(sizeof(double) * p->nz);
        memset(out + b * per_mol, 0, sizeof(double) * per_mol);
        for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a) {
            int c = p->elem[a];
            double s2 = 2.0 * p->sigma[c] * p->sigma[c];
            double r = p->cutoff_k * p->sigma[c];
            const int n[3] = {p->nx, p->ny, p->nz};
            double *g[3] = {gx, gy, gz};
            for (int ax = 0; ax < 3; ++ax)
                for (long i = 0; i < n[ax]; ++i) {
                    double d = disp(p, b, ax, i, p->coords[3 * a + ax]);
                    int keep = (p->cutoff == PGO_NONE) || fabs(d) <= r;
                    double f = p->form == PGO_INTEGRAL
                                   ? erf_factor(d, p->spacing[3 * b + ax], p->sigma[c])
                                   : exp(-d * d / s2);
                    g[ax][i] = keep ? f : 0.0;
                }
            for (long i = 0; i < p->nx; ++i) gx[i] *= weight_of(p, a);
            for (long i = 0; i < p->nx; ++i)
                for (long j = 0; j < p->ny; ++j)
                    for (long k = 0; k < p->nz; ++k)
                        out[grid_index(p, b, c, i, j, k)] += gx[i] * gy[j] * gz[k];
        }
        free(gx);
        free(gy);
        free(gz);
    }
    return PGO_OK;
}

/*
 * Coordinate gradient of L = <W, G> (Sec. IV-C):
 *   dL/dx_a = sum_v W(v) chi(d) exp(-|d|^2/2 sigma^2) d / sigma^2,  d = v - x_a,
 * and in the voxel-integrated form, per axis, the derivative of that axis's erf factor
 * times the other two factors.
 * mode 0 visits every voxel of the atom's channel, mode 1 only its cutoff box.
 * W has the grid layout [B][C][nx][ny][nz]; grad is [N][3].
 */
/*
 * Gradient for the atoms of molecule b (see pgo_gradient); with grad_w non-null it also
 * writes dL/dw_a, the atom's unweighted terms against W.
 */
static void gradient_molecule(const pgo_problem *p, int b, int mode, const double *W,
                              double *grad, double *grad_w)
{
    for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a) {
        int c = p->elem[a];
        double sg2 = p->sigma[c] * p->sigma[c];
        double r = p->cutoff_k * p->sigma[c];
        const double *xa = p->coords + 3 * a;
        double x = xa[0], y = xa[1], z = xa[2];
        long ilo = 0, ihi = p->nx - 1, jlo = 0, jhi = p->ny - 1, klo = 0, khi = p->nz - 1;
        if (mode == 1 && p->cell) {
            cell_support(p, b, 0, xa, r, &ilo, &ihi);
            cell_support(p, b, 1, xa, r, &jlo, &jhi);
            cell_support(p, b, 2, xa, r, &klo, &khi);
        } else if (mode == 1) {
            support(p, b, 0, x, r, &ilo, &ihi);
            support(p, b, 1, y, r, &jlo, &jhi);
            support(p, b, 2, z, r, &klo, &khi);
        }
        double gx = 0.0, gy = 0.0, gz = 0.0, gw = 0.0;
        for (long iu = ilo; iu <= ihi; ++iu) {
            long i = p->periodic ? wrap_index(iu, p->nx) : iu;
            double dx = p->cell ? 0.0 : disp(p, b, 0, i, x);
            for (long ju = jlo; ju <= jhi; ++ju) {
                long j = p->periodic ? wrap_index(ju, p->ny) : ju;
                double dy = p->cell ? 0.0 : disp(p, b, 1, j, y);
                for (long ku = klo; ku <= khi; ++ku) {
                    long k = p->periodic ? wrap_index(ku, p->nz) : ku;
                    double dz;
                    if (p->cell) {
                        double d[3];
                        cell_disp(p, b, i, j, k, xa, d);
                        dx = d[0];
                        dy = d[1];
                        dz = d[2];
                    } else {
                        dz = disp(p, b, 2, k, z);
                    }
                    if (!inside(p->cutoff, dx, dy, dz, r)) continue;
                    double Wv = W[grid_index(p, b, c, i, j, k)];
                    gw += Wv * term(p, b, p->sigma[c], dx, dy, dz);
                    if (p->form == PGO_INTEGRAL) {
                        const double *h = p->spacing + 3 * b, sg = p->sigma[c];
                        double fx = erf_factor(dx, h[0], sg), fy = erf_factor(dy, h[1], sg);
                        double fz = erf_factor(dz, h[2], sg);
                        gx += Wv * erf_factor_dmu(dx, h[0], sg) * fy * fz;
                        gy += Wv * fx * erf_factor_dmu(dy, h[1], sg) * fz;
                        gz += Wv * fx * fy * erf_factor_dmu(dz, h[2], sg);
                    } else {
                        double w = Wv * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * sg2));
                        gx += w * dx;
                        gy += w * dy;
                        gz += w * dz;
                    }
                }
            }
        }
        /* The point form's common 1/sigma^2 and the weight are applied once at the end. */
        double wa = weight_of(p, a);
        if (grad) {
            grad[3 * a + 0] = wa * (p->form == PGO_INTEGRAL ? gx : gx / sg2);
            grad[3 * a + 1] = wa * (p->form == PGO_INTEGRAL ? gy : gy / sg2);
            grad[3 * a + 2] = wa * (p->form == PGO_INTEGRAL ? gz : gz / sg2);
        }
        if (grad_w) grad_w[a] = gw;
    }
}

int pgo_gradient(const pgo_problem *p, int mode, const double *W, double *grad, int n_threads)
{
    int st = check(p);
    if (st) return st;
    int nt = threads_or_default(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) gradient_molecule(p, b, mode, W, grad, NULL);
    return PGO_OK;
}

/* Weight gradient dL/dw_a of L = <W, G> (weighted grids): grad_w is [N]. */
int pgo_gradient_weight(const pgo_problem *p, int mode, const double *W, double *grad_w,
                        int n_threads)
{
    int st = check(p);
    if (st) return st;
    int nt = threads_or_default(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) gradient_molecule(p, b, mode, W, NULL, grad_w);
    return PGO_OK;
}

/*
 * Grid reversal by gradient descent (Sec. IV-A steps 2-5, Sec. IV-C).  Each molecule b, from
 * its coordinates x^0 in p->coords, repeats:
 *   F = grid of x^t;  L = sum_v (F(v) - T(v))^2 over the molecule's voxels;
 *   stop if L < eps;  otherwise x^{t+1} = x^t - lr * dL/dx^t,
 * with dL/dx = sum_v 2 (F - T) dF/dx, the gradient above with W = 2 (F - T), for at most
 * `iters` updates.  out_coords [N][3] receives the final coordinates, loss[b] the loss of
 * the final coordinates and steps[b] the number of updates applied.
 */
int pgo_refine(const pgo_problem *p, const double *target, int iters, double lr, double eps,
               double *out_coords, double *loss, int32_t *steps, int n_threads)
{
    int st = check(p);
    if (st) return st;
    if (iters < 0 || !(lr >= 0.0)) return PGO_BAD_ARG;
    int nt = threads_or_default(n_threads);
    (void)nt;
    long per_mol = (long)p->n_channels * p->nx * p->ny * p->nz;
    long n_atoms = p->n_mol > 0 ? p->mol_off[p->n_mol] : 0;
    memcpy(out_coords, p->coords, sizeof(double) * 3 * n_atoms);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) {
        /* Molecule b as a one-molecule problem (atom indices stay global), reading and
           updating its own atoms in out_coords. */
        pgo_problem q = *p;
        q.n_mol = 1;
        q.mol_off = p->mol_off + b;
        q.origin = p->origin + 3 * b;
        q.spacing = p->spacing + 3 * b;
        q.cell = p->cell ? p->cell + 9 * b : NULL;
        q.coords = out_coords;
        double *F = malloc(sizeof(double) * per_mol);
        double *W = malloc(sizeof(double) * per_mol);
        double *g = malloc(sizeof(double) * 3 * (n_atoms > 0 ? n_atoms : 1));
        const double *T = target + b * per_mol;
        int t = 0;
        double L = 0.0;
        for (;;) {
            bbox_molecule(&q, 0, F, 0.0, NULL);
            L = 0.0;
            for (long v = 0; v < per_mol; ++v) {
                double r = F[v] - T[v];
                L += r * r;
                W[v] = 2.0 * r;
            }
            if (L < eps || t == iters) break;
            gradient_molecule(&q, 0, 1, W, g, NULL);
            for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a)
                for (int ax = 0; ax < 3; ++ax) out_coords[3 * a + ax] -= lr * g[3 * a + ax];
            ++t;
        }
        loss[b] = L;
        steps[b] = t;
        free(F);
        free(W);
        free(g);
    }
    return PGO_OK;
}

/*
 * Central finite differences of L = <W, G> with the support frozen: chi and the
 * periodic image are taken at the unperturbed position, and only the Gaussian sees the
 * shifted atom.  That is the derivative of the piecewise-smooth loss away from the
 * cutoff surface, which is what the analytic gradient computes.  Only atom a's own
 * terms depend on x_a (G is a sum over atoms), so the difference is formed from them.
 */
int pgo_fd_gradient_frozen(const pgo_problem *p, const double *W, double step, double *grad,
                           int n_threads)
{
    int st = check(p);
    if (st) return st;
    if (!(step > 0.0)) return PGO_BAD_ARG;
    int nt = threads_or_default(n_threads);
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int b = 0; b < p->n_mol; ++b) {
        for (int a = p->mol_off[b]; a < p->mol_off[b + 1]; ++a) {
            int c = p->elem[a];
            double r = p->cutoff_k * p->sigma[c];
            const double *xa = p->coords + 3 * a;
            double x = xa[0], y = xa[1], z = xa[2];
            double lp[3] = {0, 0, 0}, lm[3] = {0, 0, 0};
            for (long i = 0; i < p->nx; ++i) {
                double dx = p->cell ? 0.0 : disp(p, b, 0, i, x);
                for (long j = 0; j < p->ny; ++j) {
                    double dy = p->cell ? 0.0 : disp(p, b, 1, j, y);
                    for (long k = 0; k < p->nz; ++k) {
                        double dz;
                        if (p->cell) {
                            double dv[3];
                            cell_disp(p, b, i, j, k, xa, dv);
                            dx = dv[0];
                            dy = dv[1];
                            dz = dv[2];
                        } else {
                            dz = disp(p, b, 2, k, z);
                        }
                        if (!inside(p->cutoff, dx, dy, dz, r)) continue;
                        double w = W[grid_index(p, b, c, i, j, k)] * weight_of(p, a);
                        double d[3] = {dx, dy, dz};
                        for (int ax = 0; ax < 3; ++ax) {
                            double e[3] = {d[0], d[1], d[2]};
                            e[ax] = d[ax] - step; /* atom moved by +step */
                            lp[ax] += w * term(p, b, p->sigma[c], e[0], e[1], e[2]);
                            e[ax] = d[ax] + step; /* atom moved by -step */
                            lm[ax] += w * term(p, b, p->sigma[c], e[0], e[1], e[2]);
                        }
                    }
                }
            }
            for (int ax = 0; ax < 3; ++ax) grad[3 * a + ax] = (lp[ax] - lm[ax]) / (2.0 * step);
        }
    }
    return PGO_OK;
}

/* <W, G> for the whole batch (used by the raw finite-difference driver). */
double pgo_inner(const double *W, const double *G, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += W[i] * G[i];
    return s;
}
