/*
 * vct_oracle.c -- plain, slow FP64 CPU oracle of the VCT + SPH(2) step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check of __graft_entry__ and the
 * CPU-baseline leg of bench.py use it.  It shares no code, header or table
 * with the CUDA library.
 *
 * Built with -O2 -ffp-contract=off (no FMA contraction), optional OpenMP over
 * particles.  Every reduction across particles (Krylov dot products) is a
 * serial loop in index order, so results do not depend on the thread count.
 *
 * What it computes, in the paper's order and notation:
 *   map          r -> r^ = (x, y, alpha (z + beta))            Sec. 2.1, Eq. (VCT)
 *   metric       J = det J = alpha, c_trans                    Eqs. (jacobi), (det_jacobi), (lap_VCT)
 *   map kinds    E / BF / BFE / sigma (+ alpha clamp)          Sec. 2.2
 *   kernel       cubic spline, l = 1.2 d0, r_e = 2 l           Sec. 3.1
 *   neighbours   S_i = { j != i : |r^_ij| < r_e }, brute force Eq. (SPH_neighbor_set)
 *   L_i, <grad>  corrected first-order gradient                Eqs. (gra_1st), (div_1st)
 *   SPH(2)       <D phi> = 2 M^-1 sum V F q (phi_ij - r.grad)  Eq. (sec_SPH2)
 *   predictor    VCT predictor with variable viscosity         Eq. (VCT_predictor), Sec. 3.4
 *   PPE          c_trans . <D^ p> = rho/dt J <div v*> + gamma (rho Jbar/J - rho^)/dt^2
 *                                                              Eqs. (VCT_ppe), (VCT_ppe_w0), (VCT_ppe_w)
 *   walls        no-slip v = 0, pressure Neumann extrapolation Sec. 3.5, Eq. (PNC)
 *   corrector    v = v* - dt/rho J grad^ p; r += dt v          Eqs. (VCT_predictor), (VCT_update)
 *   smoothing    Jbar exchange between neighbours              Sec. 3.6, Eq. (VCT_bar_a)
 *   regularise   dynamic stabilization, XSPH on free-surface particles and
 *                optimized particle shifting after the update  Sec. 4.1 (parameters;
 *                the formulas are restated from the cited methods, see stage_regularise)
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes): r_e = 2 l; grad w_ij = -(w'(r)/r) r_ij (gradient w.r.t. r_i,
 * pointing to j); p_ij = q_ij - sum_k V_k q_ik (r_ij . L_i grad w_ik); the
 * SPH(2) cross outputs are 2 d2phi/dxdz and are halved before the c_trans
 * product; derivative sums run over fluid + wall particles, the density and
 * the free-surface test over all particles; free surface = eigenvalue rule
 * on B_i with a scan-cone test between the thresholds; the PPE divergence is
 * tr(J <grad^ (x) v*>); wall pressure enters per pair through Eq. (PNC);
 * the PPE is solved by BiCGSTAB; the Jbar exchange has a sequential
 * (literal) and a simultaneous form.
 *
 * PPE solve: BiCGSTAB (H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13,
 * 1992) on the matrix-free operator p -> c_trans . <D^ p>, which is exactly
 * the left side of Eq. (VCT_ppe).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FLUID 0
#define ORC_WALL 1
#define ORC_VIRTUAL 2
/* smallest eigenvalue of B_i (all types, symmetrised) below which a fluid
 * particle is isolated: 1 with a full kernel support, ~0.5 at a flat free
 * surface, ~0.1 at a corner of the fluid */
#define ORC_LAM_ISOLATED 0.05

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_CAPACITY = 2, ORC_ERR_SINGULAR = 3,
       ORC_ERR_NOCONV = 4, ORC_ERR_NONFINITE = 5 };
enum { ORC_MAP_E = 0, ORC_MAP_BF = 1, ORC_MAP_BFE = 2, ORC_MAP_SIGMA = 3 };

typedef struct {
    double h0, slope_x, slope_y, cos_amp, cos_len;
    int n_gauss, pad_;
    const double *amp, *cx, *cy, *width;
} orc_bathy;

typedef struct {
    int dim, map_kind;
    double aspect;
    double rho, nu_k, g, dt, d0, l_over_d0, re_over_l, gamma_over_dt, cv_over_dt, cs, ds;
    double H, H_hat, alpha_min, alpha_max, lam_fs_lo, lam_fs_hi, ppe_rtol;
    int ppe_max_iter, smagorinsky, volume_mode, neighbour_mode, smoothing_mode, pad_;
    double ops_shift, ds_overlap, xsph_eps;   /* particle regularisation, 0 = off */
    int operators;   /* 0: ISPH(2) -- SPH(2) second derivatives (Eq. sec_SPH2), 1st-order
                      *    pressure gradient (Eq. gra_1st); 1: ISPH -- 0th-order second
                      *    derivatives (Eq. sec_0th), summation pressure gradient (Eq. gra_sum);
                      *    velocity divergence 1st-order in both (Table tab:case_names) */
    int wall_slip;   /* 0: no-slip walls, v = 0; 1: free-slip, v = (I - 2 n n) v_wall (Sec. 3.5) */
} orc_params;

typedef struct {
    int n, pad_;
    double *x, *y, *z, *u, *v, *w, *p, *jbar;
    const int32_t *type;
} orc_state;

typedef struct {
    int32_t *fs;
    double *rho_hat, *nu, *lam_min;
    double *vstar;          /* d x n, component-major */
    double *ppe_b;          /* RHS of A p = b on the unknown rows, 0 elsewhere */
    const double *x_test;   /* optional input vector */
    double *ppe_Ax;         /* A x_test */
    double *jbar_used;      /* Jbar after the smoothing of the last step */
    int n_iter, pad_;
    double resid;
    double *vwall;          /* d x n: velocity each wall particle carries (0 elsewhere) */
} orc_probe;

/* ------------------------------------------------------------------------ */
/* Bathymetry h(x,y) and its derivatives h_x, h_y, h_xx, h_yy.               */
/* Bottom shapes of Sec. 4: linear, cosine (4.2), Gaussian sums (workloads). */
/* ------------------------------------------------------------------------ */
static void bathy_eval(const orc_bathy *b, double x, double y, double h[5])
{
    double v = b->h0 + b->slope_x * x + b->slope_y * y;
    double hx = b->slope_x, hy = b->slope_y, hxx = 0.0, hyy = 0.0;
    if (b->cos_amp != 0.0) {
        double k = 2.0 * M_PI / b->cos_len;
        v += b->cos_amp * cos(k * x);
        hx += -b->cos_amp * k * sin(k * x);
        hxx += -b->cos_amp * k * k * cos(k * x);
    }
    for (int g = 0; g < b->n_gauss; ++g) {
        double dx = x - b->cx[g], dy = y - b->cy[g], s2 = b->width[g] * b->width[g];
        double e = b->amp[g] * exp(-(dx * dx + dy * dy) / (2.0 * s2));
        v += e;
        hx += -e * dx / s2;
        hy += -e * dy / s2;
        hxx += e * (dx * dx / s2 - 1.0) / s2;
        hyy += e * (dy * dy / s2 - 1.0) / s2;
    }
    h[0] = v; h[1] = hx; h[2] = hy; h[3] = hxx; h[4] = hyy;
}

/* alpha, beta and their first and second horizontal derivatives (Sec. 2.2).
 * ab = {alpha, a_x, a_y, a_xx, a_yy, beta, b_x, b_y, b_xx, b_yy}. */
static void map_ab(const orc_params *P, const orc_bathy *b, double x, double y, double ab[10])
{
    double h[5];
    bathy_eval(b, x, y, h);
    for (int k = 0; k < 10; ++k) ab[k] = 0.0;
    switch (P->map_kind) {
    case ORC_MAP_E:      /* alpha = H^/H (a constant aspect ratio), beta = 0 */
        ab[0] = P->aspect;
        break;
    case ORC_MAP_BF:     /* alpha = 1, beta = -h */
        ab[0] = 1.0;
        ab[5] = -h[0]; ab[6] = -h[1]; ab[7] = -h[2]; ab[8] = -h[3]; ab[9] = -h[4];
        break;
    case ORC_MAP_BFE:    /* alpha = H^/H, beta = -h */
        ab[0] = P->aspect;
        ab[5] = -h[0]; ab[6] = -h[1]; ab[7] = -h[2]; ab[8] = -h[3]; ab[9] = -h[4];
        break;
    case ORC_MAP_SIGMA: { /* alpha = H^/(H - h), beta = -h; alpha held constant out of range */
        double D = P->H - h[0];
        ab[5] = -h[0]; ab[6] = -h[1]; ab[7] = -h[2]; ab[8] = -h[3]; ab[9] = -h[4];
        if (D <= 0.0) {
            ab[0] = P->alpha_max;
            break;
        }
        double a = P->H_hat / D;
        if (a < P->alpha_min || a > P->alpha_max) {
            ab[0] = a < P->alpha_min ? P->alpha_min : P->alpha_max;
            break;
        }
        ab[0] = a;
        /* d/dx [H^/(H-h)] = H^ h_x/(H-h)^2 ; d2/dx2 = H^ (h_xx/D^2 + 2 h_x^2/D^3) */
        ab[1] = P->H_hat * h[1] / (D * D);
        ab[2] = P->H_hat * h[2] / (D * D);
        ab[3] = P->H_hat * (h[3] / (D * D) + 2.0 * h[1] * h[1] / (D * D * D));
        ab[4] = P->H_hat * (h[4] / (D * D) + 2.0 * h[2] * h[2] / (D * D * D));
        break;
    }
    default:
        ab[0] = 1.0;
    }
    if (P->dim == 2) {   /* a 2-D section (x, z) has no y direction: drop the y derivatives */
        ab[2] = ab[4] = ab[7] = ab[9] = 0.0;
    }
}

/* Per-particle metric: zh = alpha (z + beta), s = (s_x, s_y) the third column of
 * the Jacobian (Eq. jacobi), J = alpha (Eq. det_jacobi) and c_trans (Eq. lap_VCT).
 * met = {J, s_x, s_y, c0, c3, c4, c5}; c1 = c2 = 1. */
static void metric_at(const orc_params *P, const orc_bathy *b, double x, double y, double z,
                      double *zh, double met[7])
{
    double ab[10];
    map_ab(P, b, x, y, ab);
    double al = ab[0], zeta = z + ab[5];
    double sx = ab[1] * zeta + al * ab[6];
    double sy = ab[2] * zeta + al * ab[7];
    *zh = al * zeta;
    met[0] = al;
    met[1] = sx;
    met[2] = sy;
    met[3] = (ab[3] + ab[4]) * zeta + 2.0 * (ab[1] * ab[6] + ab[2] * ab[7]) + al * (ab[8] + ab[9]);
    met[4] = al * al + sx * sx + sy * sy;
    met[5] = 2.0 * sx;
    met[6] = 2.0 * sy;
}

/* ------------------------------------------------------------------------ */
/* Cubic spline kernel (Sec. 3.1) and its radial derivative.                 */
/* ------------------------------------------------------------------------ */
static double kern_ad(int dim, double l)
{
    return dim == 2 ? 10.0 / (7.0 * M_PI * l * l) : 1.0 / (M_PI * l * l * l);
}

static double kern_w(double r, double l, int dim)
{
    double q = r / l, ad = kern_ad(dim, l);
    if (q < 1.0) return ad * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) return ad * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    return 0.0;
}

static double kern_dw(double r, double l, int dim)
{
    double q = r / l, ad = kern_ad(dim, l);
    if (q < 1.0) return ad * (-3.0 * q + 2.25 * q * q) / l;
    if (q < 2.0) return -ad * 0.75 * (2.0 - q) * (2.0 - q) / l;
    return 0.0;
}

void orc_kernel(int dim, double l, int n, const double *r, double *w, double *dw)
{
    for (int i = 0; i < n; ++i) {
        w[i] = kern_w(r[i], l, dim);
        dw[i] = kern_dw(r[i], l, dim);
    }
}

void orc_map_coeffs(const orc_params *P, const orc_bathy *b, int n, const double *x,
                    const double *y, double *ab /* n x 10 */)
{
    for (int i = 0; i < n; ++i) map_ab(P, b, x[i], y ? y[i] : 0.0, ab + 10 * i);
}

void orc_map(const orc_params *P, const orc_bathy *b, int n, const double *x, const double *y,
             const double *z, double *zh, double *met /* n x 7 */)
{
    for (int i = 0; i < n; ++i)
        metric_at(P, b, x[i], y ? y[i] : 0.0, z[i], zh + i, met + 7 * i);
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets (Eq. SPH_neighbor_set) in projected space.                 */
/* Squared distance summed in coordinate order x, (y), z, no FMA; strict <;  */
/* j != i; each row sorted by ascending index.                               */
/* ------------------------------------------------------------------------ */
static double dist2(int dim, const double *xh, int i, int j)
{
    if (dim == 2) {
        double dx = xh[2 * j] - xh[2 * i], dz = xh[2 * j + 1] - xh[2 * i + 1];
        return dx * dx + dz * dz;
    }
    double dx = xh[3 * j] - xh[3 * i], dy = xh[3 * j + 1] - xh[3 * i + 1];
    double dz = xh[3 * j + 2] - xh[3 * i + 2];
    return dx * dx + dy * dy + dz * dz;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Build CSR rows.  mode 0 = brute force O(N^2); mode 1 = the same predicate
 * over candidates from a cell grid of edge r_e (candidates sorted by index
 * first, so the rows are identical to mode 0). */
static int64_t build_neighbours(int dim, int n, const double *xh, double re, double re2,
                                int mode, int64_t *row_ptr, int32_t **col_out)
{
    int *cnt = (int *)calloc((size_t)n, sizeof(int));
    int *cell_of = NULL, *cell_start = NULL, *cell_items = NULL;
    long ncx = 1, ncy = 1, ncz = 1;
    double lo[3] = {0, 0, 0};
    if (mode == 1 && n > 0) {
        double hi[3] = {0, 0, 0};
        for (int K = 0; K < dim; ++K) { lo[K] = xh[K]; hi[K] = xh[K]; }
        for (int i = 0; i < n; ++i)
            for (int K = 0; K < dim; ++K) {
                double c = xh[dim * i + K];
                if (c < lo[K]) lo[K] = c;
                if (c > hi[K]) hi[K] = c;
            }
        long nc[3] = {1, 1, 1};
        for (int K = 0; K < dim; ++K) nc[K] = (long)floor((hi[K] - lo[K]) / re) + 1;
        ncx = nc[0]; ncy = dim == 3 ? nc[1] : 1; ncz = dim == 3 ? nc[2] : nc[1];
        long ncell = ncx * ncy * ncz;
        cell_of = (int *)malloc(sizeof(int) * (size_t)n);
        cell_start = (int *)calloc((size_t)ncell + 1, sizeof(int));
        cell_items = (int *)malloc(sizeof(int) * (size_t)n);
        for (int i = 0; i < n; ++i) {
            long c[3] = {0, 0, 0};
            for (int K = 0; K < dim; ++K) c[K] = (long)floor((xh[dim * i + K] - lo[K]) / re);
            long cx = c[0], cy = dim == 3 ? c[1] : 0, cz = dim == 3 ? c[2] : c[1];
            cell_of[i] = (int)((cz * ncy + cy) * ncx + cx);
            cell_start[cell_of[i] + 1]++;
        }
        for (long c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
        int *fill = (int *)calloc((size_t)ncell, sizeof(int));
        for (int i = 0; i < n; ++i) cell_items[cell_start[cell_of[i]] + fill[cell_of[i]]++] = i;
        free(fill);
    }
    int maxcand = 0;
    if (mode == 1) {
        /* bound on candidates per particle: sum of the 3^d largest cells */
        long ncell = ncx * ncy * ncz;
        int big = 0;
        for (long c = 0; c < ncell; ++c) {
            int s = cell_start[c + 1] - cell_start[c];
            if (s > big) big = s;
        }
        maxcand = big * (dim == 3 ? 27 : 9);
    }
    for (int pass = 0; pass < 2; ++pass) {
        int32_t *col = pass ? *col_out : NULL;
#pragma omp parallel
        {
            int *cand = mode == 1 ? (int *)malloc(sizeof(int) * (size_t)(maxcand + 1)) : NULL;
#pragma omp for schedule(dynamic, 64)
            for (int i = 0; i < n; ++i) {
                int c = 0;
                int64_t o = pass ? row_ptr[i] : 0;
                if (mode == 0) {
                    for (int j = 0; j < n; ++j) {
                        if (j == i) continue;
                        if (dist2(dim, xh, i, j) < re2) {
                            if (pass) col[o + c] = j;
                            c++;
                        }
                    }
                } else {
                    long ci = cell_of[i];
                    long cx = ci % ncx, cy = (ci / ncx) % ncy, cz = ci / (ncx * ncy);
                    int nc = 0;
                    for (long dz = -1; dz <= 1; ++dz)
                        for (long dy = (dim == 3 ? -1 : 0); dy <= (dim == 3 ? 1 : 0); ++dy)
                            for (long dx = -1; dx <= 1; ++dx) {
                                long x2 = cx + dx, y2 = cy + dy, z2 = cz + dz;
                                if (x2 < 0 || y2 < 0 || z2 < 0 || x2 >= ncx || y2 >= ncy || z2 >= ncz)
                                    continue;
                                long cc = (z2 * ncy + y2) * ncx + x2;
                                for (int k = cell_start[cc]; k < cell_start[cc + 1]; ++k)
                                    cand[nc++] = cell_items[k];
                            }
                    qsort(cand, (size_t)nc, sizeof(int), cmp_int);
                    for (int k = 0; k < nc; ++k) {
                        int j = cand[k];
                        if (j == i) continue;
                        if (dist2(dim, xh, i, j) < re2) {
                            if (pass) col[o + c] = j;
                            c++;
                        }
                    }
                }
                if (!pass) cnt[i] = c;
            }
            free(cand);
        }
        if (!pass) {
            row_ptr[0] = 0;
            for (int i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + cnt[i];
            *col_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)(row_ptr[n] + 1));
        }
    }
    free(cnt);
    free(cell_of);
    free(cell_start);
    free(cell_items);
    return row_ptr[n];
}

/* Public: neighbour CSR from projected positions.  Returns nnz, or -1 if
 * col_cap is too small (row_ptr is still filled). */
int64_t orc_neighbours(int dim, int n, const double *xh_soa /* d x n */, double re, double re2,
                       int mode, int64_t *row_ptr, int32_t *col, int64_t col_cap)
{
    double *xh = (double *)malloc(sizeof(double) * (size_t)n * dim + 8);
    for (int i = 0; i < n; ++i)
        for (int K = 0; K < dim; ++K) xh[dim * i + K] = xh_soa[(size_t)K * n + i];
    int32_t *c = NULL;
    int64_t nnz = build_neighbours(dim, n, xh, re, re2, mode, row_ptr, &c);
    free(xh);
    if (nnz > col_cap) {
        free(c);
        return -1;
    }
    if (col && nnz) memcpy(col, c, sizeof(int32_t) * (size_t)nnz);
    free(c);
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra.                                               */
/* ------------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting, in place, nrhs right-hand
 * sides stored as columns of B (n x nrhs, row-major).  Returns 0, or 1 if a
 * pivot is below tiny * max|A|. */
static int gauss_solve(int n, double *A, int nrhs, double *B)
{
    double amax = 0.0;
    for (int k = 0; k < n * n; ++k)
        if (fabs(A[k]) > amax) amax = fabs(A[k]);
    if (!(amax > 0.0)) return 1;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > fabs(A[piv * n + k])) piv = r;
        if (!(fabs(A[piv * n + k]) > 1e-14 * amax)) return 1;
        if (piv != k) {
            for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
            for (int c = 0; c < nrhs; ++c) { double t = B[k * nrhs + c]; B[k * nrhs + c] = B[piv * nrhs + c]; B[piv * nrhs + c] = t; }
        }
        for (int r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / A[k * n + k];
            for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            for (int c = 0; c < nrhs; ++c) B[r * nrhs + c] -= f * B[k * nrhs + c];
        }
    }
    for (int k = n - 1; k >= 0; --k)
        for (int c = 0; c < nrhs; ++c) {
            double s = B[k * nrhs + c];
            for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * B[j * nrhs + c];
            B[k * nrhs + c] = s / A[k * n + k];
        }
    return 0;
}

/* Smallest eigenvalue of a symmetric d x d matrix: closed form in 2-D, cyclic
 * Jacobi rotations in 3-D. */
static double sym_lam_min(int d, const double *S)
{
    if (d == 2) {
        double a = S[0], b = S[1], c = S[3];
        double m = 0.5 * (a + c), h = 0.5 * (a - c);
        return m - sqrt(h * h + b * b);
    }
    double A[9];
    memcpy(A, S, sizeof A);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = A[p * 3 + q];
                if (apq == 0.0) continue;
                double app = A[p * 3 + p], aqq = A[q * 3 + q];
                double theta = 0.5 * (aqq - app) / apq;
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) { /* columns p, q */
                    double akp = A[k * 3 + p], akq = A[k * 3 + q];
                    A[k * 3 + p] = c * akp - s * akq;
                    A[k * 3 + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* rows p, q */
                    double apk = A[p * 3 + k], aqk = A[q * 3 + k];
                    A[p * 3 + k] = c * apk - s * aqk;
                    A[q * 3 + k] = s * apk + c * aqk;
                }
            }
    }
    double m = A[0];
    if (A[4] < m) m = A[4];
    if (A[8] < m) m = A[8];
    return m;
}

static int invert_dxd(int d, const double *B, double *L)
{
    double A[9], I[9];
    memcpy(A, B, sizeof(double) * d * d);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) I[r * d + c] = r == c ? 1.0 : 0.0;
    if (gauss_solve(d, A, d, I)) return 1;
    memcpy(L, I, sizeof(double) * d * d);
    return 0;
}

/* q_ij of Eq. (sec_SPH2): 2-D (x,z): [x^2, z^2, x z]; 3-D: [x^2, y^2, z^2, x y, y z, z x] */
static void qvec(int d, const double *r, double *q)
{
    if (d == 2) {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[0] * r[1];
    } else {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[2] * r[2];
        q[3] = r[0] * r[1]; q[4] = r[1] * r[2]; q[5] = r[2] * r[0];
    }
}

/* Coefficients of the SPH(2) output D (second derivatives with the cross
 * terms doubled) in c_trans . D^: 2-D [1, c3, c4/2]; 3-D [1, 1, c3, 0, c5/2, c4/2]. */
static void ctilde(int d, const double *met, double *ct)
{
    if (d == 2) {
        ct[0] = 1.0; ct[1] = met[4]; ct[2] = 0.5 * met[5];
    } else {
        ct[0] = 1.0; ct[1] = 1.0; ct[2] = met[4]; ct[3] = 0.0; ct[4] = 0.5 * met[6]; ct[5] = 0.5 * met[5];
    }
}

/* Weights k_a(r) of the 0th-order second derivatives of Espanol & Revenga
 * (Eq. sec_0th) in the order of the SPH(2) output D (cross entries doubled):
 *   d2 phi / dx^I dx^J ~ sum_j V_j (c r^I r^J / |r|^2 - delta^IJ) (r . grad w)/|r|^2 phi_ij,
 * c = 4 (2-D), 5 (3-D); with grad w = -(w'/|r|) r, (r . grad w)/|r|^2 = -w'/|r|. */
static void er_weights(int d, const double *r, double rr2, double dw, double *k)
{
    double rr = sqrt(rr2), f = -dw / rr, c = d == 2 ? 4.0 : 5.0;
    if (d == 2) {
        k[0] = f * (c * r[0] * r[0] / rr2 - 1.0);
        k[1] = f * (c * r[1] * r[1] / rr2 - 1.0);
        k[2] = 2.0 * f * c * r[0] * r[1] / rr2;
    } else {
        k[0] = f * (c * r[0] * r[0] / rr2 - 1.0);
        k[1] = f * (c * r[1] * r[1] / rr2 - 1.0);
        k[2] = f * (c * r[2] * r[2] / rr2 - 1.0);
        k[3] = 2.0 * f * c * r[0] * r[1] / rr2;
        k[4] = 2.0 * f * c * r[1] * r[2] / rr2;
        k[5] = 2.0 * f * c * r[2] * r[0] / rr2;
    }
}

/* Jacobian of Eq. (jacobi) restricted to the d used coordinates, row-major:
 * 2-D rows x, z: [1 s_x; 0 alpha]; 3-D: [1 0 s_x; 0 1 s_y; 0 0 alpha]. */
static void jac(int d, const double *met, double *Jm)
{
    if (d == 2) {
        Jm[0] = 1.0; Jm[1] = met[1]; Jm[2] = 0.0; Jm[3] = met[0];
    } else {
        Jm[0] = 1.0; Jm[1] = 0.0; Jm[2] = met[1];
        Jm[3] = 0.0; Jm[4] = 1.0; Jm[5] = met[2];
        Jm[6] = 0.0; Jm[7] = 0.0; Jm[8] = met[0];
    }
}

/* ------------------------------------------------------------------------ */
/* Work arrays of one step.                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int j, tj;
    double V;           /* V_j used in derivative sums */
    double r[3];        /* r^_ij = r^_j - r^_i (projected) */
    double rp[3];       /* physical r_j - r_i */
    double gw[3];       /* grad w_ij */
    double gt[3];       /* L_i grad w_ij */
    double F;           /* F_ij */
    double q[6];
    double k0[6];       /* 0th-order second-derivative weights (Eq. sec_0th) */
    double dw;          /* w'(|r^_ij|) */
} pair_t;

typedef struct {
    int dim, m, n;
    double l, re, re2, V0;
    double *xh, *xp;    /* n x d, projected / physical positions */
    double *met;        /* n x 7 */
    int64_t *row_ptr;
    int32_t *col;
    /* pass 1 */
    double *L;          /* n x d*d */
    double *Ct;         /* n x d*m : C~_i[K][a] */
    double *gv;         /* n x d*d : gv[c][K] = d v_c / d x^_K */
    double *G;          /* n x d*d : physical G[I][c] = d v_c / d x_I */
    double *rho_hat, *lam, *nu;
    int32_t *fs;
    /* pass 2 */
    double *LU;         /* n x m*m (M_i), factorised copy kept for the operator */
    double *vstar, *acc;/* n x d */
    double *vw;         /* n x 3: free-slip wall velocities (NULL: no-slip, walls at rest) */
    int64_t *pstart;    /* pair cache offsets (n+1) */
    pair_t *pairs;
    int64_t npairs;
} work_t;

static void work_free(work_t *W)
{
    free(W->xh); free(W->xp); free(W->met); free(W->row_ptr); free(W->col);
    free(W->L); free(W->Ct); free(W->gv); free(W->G); free(W->rho_hat); free(W->lam);
    free(W->nu); free(W->fs); free(W->LU); free(W->vstar); free(W->acc);
    free(W->pstart); free(W->pairs); free(W->vw);
    memset(W, 0, sizeof *W);
}

static double vol_j(const orc_params *P, const work_t *W, const orc_state *S, int j)
{
    /* V_j = V0 J_j / Jbar_j (Sec. 3.6: V_i = J_i^N / Jbar_i V); V0 under Condition A */
    if (P->volume_mode == 0) return W->V0;
    return W->V0 * W->met[7 * j] / S->jbar[j];
}

static double vel(const orc_state *S, int dim, int i, int c)
{
    if (dim == 2) return c == 0 ? S->u[i] : S->w[i];
    return c == 0 ? S->u[i] : (c == 1 ? S->v[i] : S->w[i]);
}

/* Velocity a wall particle carries in the sums of its fluid neighbours:
 * 0 under no-slip (Sec. 3.5, v = v_wall = 0), the free-slip value otherwise. */
static double wall_vel(const work_t *W, int j, int c)
{
    return W->vw ? W->vw[3 * (size_t)j + c] : 0.0;
}

/* Map + metric + neighbours for the current positions. */
static int stage_geometry(const orc_params *P, const orc_bathy *b, const orc_state *S, work_t *W)
{
    int n = S->n, d = P->dim;
    W->dim = d;
    W->m = d == 2 ? 3 : 6;
    W->n = n;
    W->l = P->l_over_d0 * P->d0;
    W->re = P->re_over_l * W->l;
    W->re2 = W->re * W->re;
    W->V0 = d == 2 ? P->d0 * P->d0 : P->d0 * P->d0 * P->d0;
    W->xh = (double *)malloc(sizeof(double) * (size_t)n * d + 8);
    W->xp = (double *)malloc(sizeof(double) * (size_t)n * d + 8);
    W->met = (double *)malloc(sizeof(double) * (size_t)n * 7 + 8);
    for (int i = 0; i < n; ++i) {
        double y = d == 3 ? S->y[i] : 0.0, zh;
        metric_at(P, b, S->x[i], y, S->z[i], &zh, W->met + 7 * i);
        if (d == 2) {
            W->xh[2 * i] = S->x[i]; W->xh[2 * i + 1] = zh;
            W->xp[2 * i] = S->x[i]; W->xp[2 * i + 1] = S->z[i];
        } else {
            W->xh[3 * i] = S->x[i]; W->xh[3 * i + 1] = S->y[i]; W->xh[3 * i + 2] = zh;
            W->xp[3 * i] = S->x[i]; W->xp[3 * i + 1] = S->y[i]; W->xp[3 * i + 2] = S->z[i];
        }
    }
    for (int i = 0; i < n; ++i)
        if (!(S->jbar[i] > 0.0)) S->jbar[i] = W->met[7 * i]; /* Jbar^0 = J^0 */
    W->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    build_neighbours(d, n, W->xh, W->re, W->re2, P->neighbour_mode, W->row_ptr, &W->col);
    return ORC_OK;
}

/* Volume smoothing, Sec. 3.6: Delta J_ij = C_V (r_e - |r^_ij|)/r_e (J_j/Jbar_j - J_i/Jbar_i);
 * V'_i = V_i + Delta V_ij, V'_j = V_j - Delta V_ij, i.e. J/Jbar gains +Delta J_ij at i
 * and -Delta J_ij at j (Eq. VCT_bar_a).  Fluid-fluid pairs only.
 * mode 0: literal sequential form -- ascending i, each neighbour j of i in
 *         ascending order, Jbar updated in place after every pair.
 * mode 1: simultaneous form -- every pair is applied once from each end
 *         (as the sequential loop does), all from the values before the sweep. */
static void stage_smoothing(const orc_params *P, const orc_state *S, const work_t *W, int mode)
{
    int n = S->n;
    double CV = P->cv_over_dt * P->dt;
    if (mode == 0) {
        for (int i = 0; i < n; ++i) {
            if (S->type[i] != ORC_FLUID) continue;
            for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
                int j = W->col[k];
                if (S->type[j] != ORC_FLUID) continue;
                double Ji = W->met[7 * i], Jj = W->met[7 * j];
                double rr = sqrt(dist2(W->dim, W->xh, i, j));
                double dJ = CV * (W->re - rr) / W->re * (Jj / S->jbar[j] - Ji / S->jbar[i]);
                S->jbar[i] = Ji * S->jbar[i] / (Ji + S->jbar[i] * dJ);
                S->jbar[j] = Jj * S->jbar[j] / (Jj - S->jbar[j] * dJ);
            }
        }
        return;
    }
    double *ratio = (double *)malloc(sizeof(double) * (size_t)n + 8);
    for (int i = 0; i < n; ++i) ratio[i] = W->met[7 * i] / S->jbar[i];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        double sum = 0.0;
        for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
            int j = W->col[k];
            if (S->type[j] != ORC_FLUID) continue;
            double rr = sqrt(dist2(W->dim, W->xh, i, j));
            sum += CV * (W->re - rr) / W->re * (ratio[j] - ratio[i]);
        }
        S->jbar[i] = W->met[7 * i] / (ratio[i] + 2.0 * sum);
    }
    free(ratio);
}

/* Free-slip wall velocities (Sec. 3.5): v_j = (I - 2 n n) v_wall,j.  v_wall,j is
 * the SPH (Shepard) interpolation of the fluid velocity at wall particle j,
 * sum_k V_k v_k w_jk / sum_k V_k w_jk over its fluid neighbours (0 without
 * any).  n is the outer unit normal in physical space: the projected normal
 * n^ points from j towards the virtual particles outside the wall,
 * n^ ~ sum_{k virtual} V0 grad w_jk, and transforms as a gradient,
 * n ~ J^T n^ (the transpose of the Jacobian of Eq. jacobi): on the bottom
 * z^ = 0 this is the surface normal (h_x, h_y, -1)/|.|, which the paper
 * builds from rotations by arctan(dh/dx), arctan(dh/dy). */
static void stage_wall_velocity(const orc_params *P, const orc_state *S, work_t *W)
{
    int n = S->n, d = W->dim;
    W->vw = (double *)calloc((size_t)n * 3 + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int j = 0; j < n; ++j) {
        if (S->type[j] != ORC_WALL) continue;
        double num[3] = {0}, den = 0.0, nh[3] = {0};
        for (int64_t q = W->row_ptr[j]; q < W->row_ptr[j + 1]; ++q) {
            int k = W->col[q], tk = S->type[k];
            double r[3], rr2 = 0.0;
            for (int K = 0; K < d; ++K) {
                r[K] = W->xh[d * k + K] - W->xh[d * j + K];
                rr2 += r[K] * r[K];
            }
            double rr = sqrt(rr2);
            if (tk == ORC_FLUID) {
                double wv = vol_j(P, W, S, k) * kern_w(rr, W->l, d);
                for (int c = 0; c < d; ++c) num[c] += wv * vel(S, d, k, c);
                den += wv;
            } else if (tk == ORC_VIRTUAL && rr > 0.0) {
                double dw = kern_dw(rr, W->l, d);
                for (int K = 0; K < d; ++K) nh[K] += W->V0 * (-dw / rr) * r[K];
            }
        }
        if (!(den > 0.0)) continue;
        double v[3] = {0}, Jm[9], nn[3] = {0}, nl = 0.0, vn = 0.0;
        for (int c = 0; c < d; ++c) v[c] = num[c] / den;
        jac(d, W->met + 7 * (size_t)j, Jm);
        for (int I = 0; I < d; ++I) {
            for (int K = 0; K < d; ++K) nn[I] += Jm[I * d + K] * nh[K];
            nl += nn[I] * nn[I];
        }
        nl = sqrt(nl);
        if (nl > 0.0)
            for (int I = 0; I < d; ++I) { nn[I] /= nl; vn += nn[I] * v[I]; }
        for (int c = 0; c < d; ++c) W->vw[3 * (size_t)j + c] = v[c] - 2.0 * vn * nn[c];
    }
}

/* Pass 1 for one fluid particle: B_i, L_i, <grad^ v>, C~_i, rho^_i, free-surface
 * flag, eddy viscosity. */
static int pass1_one(const orc_params *P, const orc_state *S, work_t *W, int i)
{
    int d = W->dim, m = W->m;
    double B[9] = {0}, Ball[9] = {0}, nsum[3] = {0}, Gv[9] = {0}, Gq[18] = {0};
    double rho = 0.0, dwall = INFINITY;
    const double *xi = W->xh + d * i;
    for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
        int j = W->col[k], tj = S->type[j];
        double r[3], rp[3], rr2 = 0.0;
        for (int K = 0; K < d; ++K) {
            r[K] = W->xh[d * j + K] - xi[K];
            rp[K] = W->xp[d * j + K] - W->xp[d * i + K];
            rr2 += r[K] * r[K];
        }
        double rr = sqrt(rr2);
        double wv = kern_w(rr, W->l, d);
        rho += W->V0 * wv;
        if (rr == 0.0) continue;
        double dw = kern_dw(rr, W->l, d), gw[3];
        for (int K = 0; K < d; ++K) gw[K] = -dw / rr * r[K];
        for (int K = 0; K < d; ++K) {
            nsum[K] += W->V0 * gw[K];
            for (int L2 = 0; L2 < d; ++L2) Ball[K * d + L2] += W->V0 * gw[K] * r[L2];
        }
        if (tj == ORC_VIRTUAL) continue;
        double Vj = vol_j(P, W, S, j), q[6];
        qvec(d, r, q);
        for (int K = 0; K < d; ++K)
            for (int L2 = 0; L2 < d; ++L2) B[K * d + L2] += Vj * gw[K] * r[L2];
        for (int c = 0; c < d; ++c) {
            double vij = (tj == ORC_FLUID ? vel(S, d, j, c) : wall_vel(W, j, c)) - vel(S, d, i, c);
            for (int K = 0; K < d; ++K) Gv[c * d + K] += Vj * vij * gw[K];
        }
        for (int K = 0; K < d; ++K)
            for (int a = 0; a < m; ++a) Gq[K * m + a] += Vj * gw[K] * q[a];
        if (tj == ORC_WALL) {
            double dp = 0.0;
            for (int K = 0; K < d; ++K) dp += rp[K] * rp[K];
            dp = sqrt(dp);
            if (dp < dwall) dwall = dp;
        }
    }
    rho += W->V0 * kern_w(0.0, W->l, d);          /* self term, j = i in S_i */
    W->rho_hat[i] = P->rho * rho;
    double *L = W->L + (size_t)9 * i;
    int iso = 0;
    if (invert_dxd(d, B, L)) {
        iso = 1;
        for (int k = 0; k < 9; ++k) L[k] = 0.0;
    }
    double *gv = W->gv + (size_t)9 * i, *Ct = W->Ct + (size_t)18 * i;
    for (int c = 0; c < d; ++c)
        for (int K = 0; K < d; ++K) {
            double s = 0.0;
            for (int L2 = 0; L2 < d; ++L2) s += L[K * d + L2] * Gv[c * d + L2];
            gv[c * d + K] = s;
        }
    for (int K = 0; K < d; ++K)
        for (int a = 0; a < m; ++a) {
            double s = 0.0;
            for (int L2 = 0; L2 < d; ++L2) s += L[K * d + L2] * Gq[L2 * m + a];
            Ct[K * m + a] = s;
        }
    /* free surface (reading of Sec. 3.5): eigenvalue rule on B over all particles */
    double Bs[9];
    for (int K = 0; K < d; ++K)
        for (int L2 = 0; L2 < d; ++L2) Bs[K * d + L2] = 0.5 * (Ball[K * d + L2] + Ball[L2 * d + K]);
    double lam = sym_lam_min(d, Bs);
    W->lam[i] = lam;
    int fs;
    if (lam <= P->lam_fs_lo) fs = 1;
    else if (lam > P->lam_fs_hi) fs = 0;
    else {
        double Lall[9], nrm[3], nn = 0.0;
        if (invert_dxd(d, Ball, Lall)) fs = 1;
        else {
            for (int K = 0; K < d; ++K) {
                double s = 0.0;
                for (int L2 = 0; L2 < d; ++L2) s += Lall[K * d + L2] * nsum[L2];
                nrm[K] = -s;
                nn += nrm[K] * nrm[K];
            }
            nn = sqrt(nn);
            if (!(nn > 0.0)) fs = 0;
            else {
                double T[3], h = W->l, c45 = sqrt(0.5);
                for (int K = 0; K < d; ++K) { nrm[K] /= nn; T[K] = xi[K] + h * nrm[K]; }
                fs = 1;
                for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1] && fs; ++k) {
                    int j = W->col[k];
                    double r[3], rr2 = 0.0, tt2 = 0.0, nr = 0.0;
                    for (int K = 0; K < d; ++K) {
                        r[K] = W->xh[d * j + K] - xi[K];
                        rr2 += r[K] * r[K];
                        double tk = W->xh[d * j + K] - T[K];
                        tt2 += tk * tk;
                        nr += nrm[K] * r[K];
                    }
                    double rr = sqrt(rr2);
                    if (rr == 0.0) continue;
                    if (rr >= sqrt(2.0) * h) {
                        if (sqrt(tt2) < h) fs = 0;
                    } else if (nr > c45 * rr) {
                        fs = 0;
                    }
                }
            }
        }
    }
    /* Isolated particle (a splash or droplet): B_i not invertible, or the
     * smallest eigenvalue of B over all particle types below ORC_LAM_ISOLATED.
     * It is a free-surface particle without corrected derivatives: L_i = 0, so
     * its gradients, SPH(2) second derivatives and pressure gradient vanish and
     * it moves under gravity alone.  Flag value 2. */
    if (!iso && lam < ORC_LAM_ISOLATED) iso = 1;
    if (iso) {
        for (int k = 0; k < 9; ++k) { L[k] = 0.0; gv[k] = 0.0; }
        for (int k = 0; k < 18; ++k) Ct[k] = 0.0;
    }
    W->fs[i] = iso ? 2 : fs;
    /* physical velocity gradient G[I][c] = sum_K J[I][K] d v_c / d x^_K (Eq. grad_VCT) */
    double Jm[9], *G = W->G + (size_t)9 * i;
    jac(d, W->met + 7 * i, Jm);
    for (int I = 0; I < d; ++I)
        for (int c = 0; c < d; ++c) {
            double s = 0.0;
            for (int K = 0; K < d; ++K) s += Jm[I * d + K] * gv[c * d + K];
            G[I * d + c] = s;
        }
    /* Smagorinsky (Sec. 3.4): nu_E = (C_s f_s Delta)^2 sqrt(2 S:S), Delta = r_e */
    double nue = 0.0;
    if (P->smagorinsky) {
        double SS = 0.0;
        for (int I = 0; I < d; ++I)
            for (int c = 0; c < d; ++c) {
                double sij = 0.5 * (G[I * d + c] + G[c * d + I]);
                SS += sij * sij;
            }
        double fsd = 1.0;
        if (dwall < INFINITY) fsd = 1.0 - exp(-10.0 * P->d0 / P->ds * dwall / W->re);
        double cdel = P->cs * fsd * W->re;
        nue = cdel * cdel * sqrt(2.0 * SS);
    }
    W->nu[i] = P->nu_k + nue;
    return ORC_OK;
}

/* Pair cache + SPH(2) moment matrix for one fluid particle, then the
 * predictor (Eq. VCT_predictor).  do_pred = 0 skips the velocity terms. */
static int pass2_one(const orc_params *P, const orc_state *S, work_t *W, int i, int do_pred)
{
    int d = W->dim, m = W->m;
    const double *L = W->L + (size_t)9 * i, *Ct = W->Ct + (size_t)18 * i;
    double M[36] = {0}, bv[18] = {0}, Gnu[3] = {0};
    const double *gv = W->gv + (size_t)9 * i;
    pair_t *pp = W->pairs + W->pstart[i];
    int np = 0;
    for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
        int j = W->col[k], tj = S->type[j];
        if (tj == ORC_VIRTUAL) continue;
        pair_t *pr = pp + np;
        double rr2 = 0.0;
        for (int K = 0; K < d; ++K) {
            pr->r[K] = W->xh[d * j + K] - W->xh[d * i + K];
            pr->rp[K] = W->xp[d * j + K] - W->xp[d * i + K];
            rr2 += pr->r[K] * pr->r[K];
        }
        double rr = sqrt(rr2);
        if (rr == 0.0) continue;
        np++;
        pr->j = j;
        pr->tj = tj;
        pr->V = vol_j(P, W, S, j);
        double dw = kern_dw(rr, W->l, d), rg = 0.0;
        pr->dw = dw;
        er_weights(d, pr->r, rr2, dw, pr->k0);
        for (int K = 0; K < d; ++K) pr->gw[K] = -dw / rr * pr->r[K];
        for (int K = 0; K < d; ++K) {
            double s = 0.0;
            for (int L2 = 0; L2 < d; ++L2) s += L[K * d + L2] * pr->gw[L2];
            pr->gt[K] = s;
            rg += pr->r[K] * s;
        }
        pr->F = rg / (rr2 * rr2);
        qvec(d, pr->r, pr->q);
        double pv[6];
        for (int a = 0; a < m; ++a) {
            double s = 0.0;
            for (int K = 0; K < d; ++K) s += Ct[K * m + a] * pr->r[K];
            pv[a] = pr->q[a] - s;
        }
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < m; ++c) M[a * m + c] += pr->V * pr->F * pr->q[a] * pv[c];
        if (do_pred) {
            for (int c = 0; c < d; ++c) {
                double vij = (tj == ORC_FLUID ? vel(S, d, j, c) : wall_vel(W, j, c)) - vel(S, d, i, c),
                       rgv = 0.0;
                for (int K = 0; K < d; ++K) rgv += pr->r[K] * gv[c * d + K];
                for (int a = 0; a < m; ++a) bv[a * d + c] += pr->V * pr->F * pr->q[a] * (vij - rgv);
            }
            double nuj = tj == ORC_FLUID ? W->nu[j] : P->nu_k;
            for (int K = 0; K < d; ++K) Gnu[K] += pr->V * (nuj - W->nu[i]) * pr->gw[K];
        }
    }
    /* terminate the pair list of i */
    for (int k = np; k < (int)(W->pstart[i + 1] - W->pstart[i]); ++k) pp[k].j = -1;
    double *LU = W->LU + (size_t)36 * i;
    memcpy(LU, M, sizeof(double) * m * m);
    if (!do_pred) return ORC_OK;
    double Mc[36];
    memcpy(Mc, M, sizeof Mc);
    if (W->fs[i] == 2) {
        /* isolated: no second derivatives */
        for (int k = 0; k < m * d; ++k) bv[k] = 0.0;
    } else if (P->operators == 1) {
        /* ISPH: D_c = the 0th-order second derivatives of v_c, stored as b = D/2 */
        for (int k = 0; k < m * d; ++k) bv[k] = 0.0;
        for (int k = 0; k < np; ++k) {
            const pair_t *pr = pp + k;
            for (int c = 0; c < d; ++c) {
                double vij = (pr->tj == ORC_FLUID ? vel(S, d, pr->j, c) : wall_vel(W, pr->j, c)) -
                             vel(S, d, i, c);
                for (int a = 0; a < m; ++a) bv[a * d + c] += 0.5 * pr->V * pr->k0[a] * vij;
            }
        }
    } else if (gauss_solve(m, Mc, d, bv)) {
        /* a free-surface particle with too few neighbours for M_i loses its
         * viscous term; anywhere else a singular M_i is an error */
        if (!W->fs[i]) return ORC_ERR_SINGULAR;
        for (int k = 0; k < m * d; ++k) bv[k] = 0.0;
    }
    /* D_c = 2 M^-1 b_c (SPH(2)) or the 0th-order second derivatives (ISPH) */
    double ct[6], Jm[9], gnh[3], gn[3];
    ctilde(d, W->met + 7 * i, ct);
    jac(d, W->met + 7 * i, Jm);
    for (int K = 0; K < d; ++K) {
        double s = 0.0;
        for (int L2 = 0; L2 < d; ++L2) s += L[K * d + L2] * Gnu[L2];
        gnh[K] = s;
    }
    for (int I = 0; I < d; ++I) {
        double s = 0.0;
        for (int K = 0; K < d; ++K) s += Jm[I * d + K] * gnh[K];
        gn[I] = s;
    }
    const double *G = W->G + (size_t)9 * i;
    for (int c = 0; c < d; ++c) {
        double lap = W->met[7 * i + 3] * gv[c * d + (d - 1)];
        for (int a = 0; a < m; ++a) lap += ct[a] * 2.0 * bv[a * d + c];
        double term = 0.0;
        for (int J2 = 0; J2 < d; ++J2) term += (G[c * d + J2] + G[J2 * d + c]) * gn[J2];
        double g = c == d - 1 ? -P->g : 0.0;
        double a = W->nu[i] * lap + term + g;
        W->acc[d * i + c] = a;
        W->vstar[d * i + c] = vel(S, d, i, c) + P->dt * a;
    }
    return ORC_OK;
}

/* Left side of Eq. (VCT_ppe) at particle i for the pressure field x (zero off
 * the unknowns), with Eq. (PNC) for wall neighbours. */
static double ppe_op_one(const orc_params *P, const work_t *W, int i, const double *x)
{
    int d = W->dim, m = W->m;
    const pair_t *pp = W->pairs + W->pstart[i];
    int np = (int)(W->pstart[i + 1] - W->pstart[i]);
    double gp[3] = {0}, b[6] = {0};
    for (int k = 0; k < np && pp[k].j >= 0; ++k) {
        const pair_t *pr = pp + k;
        double pij;
        if (pr->tj == ORC_FLUID) pij = x[pr->j] - x[i];
        else {
            double s = 0.0;
            for (int K = 0; K < d; ++K) s += pr->rp[K] * W->acc[d * i + K];
            pij = P->rho * s;
        }
        for (int K = 0; K < d; ++K) gp[K] += pr->V * pij * pr->gt[K];
    }
    for (int k = 0; k < np && pp[k].j >= 0; ++k) {
        const pair_t *pr = pp + k;
        double pij, rg = 0.0;
        if (pr->tj == ORC_FLUID) pij = x[pr->j] - x[i];
        else {
            double s = 0.0;
            for (int K = 0; K < d; ++K) s += pr->rp[K] * W->acc[d * i + K];
            pij = P->rho * s;
        }
        for (int K = 0; K < d; ++K) rg += pr->r[K] * gp[K];
        for (int a = 0; a < m; ++a) b[a] += pr->V * pr->F * pr->q[a] * (pij - rg);
    }
    if (P->operators == 1) {
        /* ISPH: D = the 0th-order second derivatives of the pressure */
        for (int a = 0; a < m; ++a) b[a] = 0.0;
        for (int k = 0; k < np && pp[k].j >= 0; ++k) {
            const pair_t *pr = pp + k;
            double pij;
            if (pr->tj == ORC_FLUID) pij = x[pr->j] - x[i];
            else {
                double s = 0.0;
                for (int K = 0; K < d; ++K) s += pr->rp[K] * W->acc[d * i + K];
                pij = P->rho * s;
            }
            for (int a = 0; a < m; ++a) b[a] += 0.5 * pr->V * pr->k0[a] * pij;
        }
    } else {
        double Mc[36];
        memcpy(Mc, W->LU + (size_t)36 * i, sizeof(double) * m * m);
        gauss_solve(m, Mc, 1, b);
    }
    double ct[6];
    ctilde(d, W->met + 7 * i, ct);
    double out = W->met[7 * i + 3] * gp[d - 1];
    for (int a = 0; a < m; ++a) out += ct[a] * 2.0 * b[a];
    return out;
}

typedef struct {
    const orc_params *P;
    const work_t *W;
    const char *unk;
    double *c0;      /* op(0) on unknown rows */
} ppe_ctx;

/* y = A x = op(x) - op(0) on unknown rows, 0 elsewhere */
static void ppe_apply(const ppe_ctx *C, const double *x, double *y)
{
    int n = C->W->n;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        y[i] = C->unk[i] ? ppe_op_one(C->P, C->W, i, x) - C->c0[i] : 0.0;
}

static double dot(int n, const char *unk, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        if (unk[i]) s += a[i] * b[i];
    return s;
}

/* BiCGSTAB (van der Vorst 1992) with initial guess x. */
static int bicgstab(const ppe_ctx *C, const double *b, double *x, double rtol, int maxit,
                    int *iters, double *resid)
{
    int n = C->W->n;
    const char *u = C->unk;
    double *r = calloc((size_t)n + 1, 8), *rh = calloc((size_t)n + 1, 8), *p = calloc((size_t)n + 1, 8);
    double *v = calloc((size_t)n + 1, 8), *s = calloc((size_t)n + 1, 8), *t = calloc((size_t)n + 1, 8);
    int rc = ORC_OK, it = 0;
    ppe_apply(C, x, t);
    for (int i = 0; i < n; ++i) { r[i] = u[i] ? b[i] - t[i] : 0.0; rh[i] = r[i]; }
    double bn = sqrt(dot(n, u, b, b)), rho_old = 1.0, alpha = 1.0, omega = 1.0;
    double rn = sqrt(dot(n, u, r, r));
    if (bn == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        rn = 0.0;
    } else {
        while (rn > rtol * bn) {
            if (it >= maxit) { rc = ORC_ERR_NOCONV; break; }
            it++;
            double rho = dot(n, u, rh, r);
            if (rho == 0.0) { rc = ORC_ERR_NOCONV; break; }
            double beta = (rho / rho_old) * (alpha / omega);
            for (int i = 0; i < n; ++i) p[i] = u[i] ? r[i] + beta * (p[i] - omega * v[i]) : 0.0;
            ppe_apply(C, p, v);
            alpha = rho / dot(n, u, rh, v);
            for (int i = 0; i < n; ++i) s[i] = u[i] ? r[i] - alpha * v[i] : 0.0;
            double sn = sqrt(dot(n, u, s, s));
            if (sn <= rtol * bn) {
                for (int i = 0; i < n; ++i) if (u[i]) x[i] += alpha * p[i];
                rn = sn;
                break;
            }
            ppe_apply(C, s, t);
            omega = dot(n, u, t, s) / dot(n, u, t, t);
            for (int i = 0; i < n; ++i)
                if (u[i]) {
                    x[i] += alpha * p[i] + omega * s[i];
                    r[i] = s[i] - omega * t[i];
                }
            rn = sqrt(dot(n, u, r, r));
            rho_old = rho;
        }
    }
    /* true relative residual */
    ppe_apply(C, x, t);
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
        if (u[i]) tr += (b[i] - t[i]) * (b[i] - t[i]);
    *resid = bn > 0 ? sqrt(tr) / bn : 0.0;
    *iters = it;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return rc;
}

static int alloc_work(work_t *W, int n, int with_pairs)
{
    W->L = calloc((size_t)n * 9 + 1, 8);
    W->Ct = calloc((size_t)n * 18 + 1, 8);
    W->gv = calloc((size_t)n * 9 + 1, 8);
    W->G = calloc((size_t)n * 9 + 1, 8);
    W->rho_hat = calloc((size_t)n + 1, 8);
    W->lam = calloc((size_t)n + 1, 8);
    W->nu = calloc((size_t)n + 1, 8);
    W->fs = calloc((size_t)n + 1, 4);
    W->LU = calloc((size_t)n * 36 + 1, 8);
    W->vstar = calloc((size_t)n * 3 + 1, 8);
    W->acc = calloc((size_t)n * 3 + 1, 8);
    if (with_pairs) {
        W->pstart = malloc(sizeof(int64_t) * (size_t)(n + 1));
        for (int i = 0; i <= n; ++i) W->pstart[i] = W->row_ptr[i];
        W->npairs = W->row_ptr[n];
        W->pairs = calloc((size_t)W->npairs + 1, sizeof(pair_t));
    }
    return 0;
}

static int run_pass1(const orc_params *P, const orc_state *S, work_t *W)
{
    int rc = ORC_OK, n = S->n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        int e = pass1_one(P, S, W, i);
        if (e) {
#pragma omp critical
            rc = e;
        }
    }
    return rc;
}

static int run_pass2(const orc_params *P, const orc_state *S, work_t *W, int do_pred)
{
    int rc = ORC_OK, n = S->n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        int e = pass2_one(P, S, W, i, do_pred);
        if (e) {
#pragma omp critical
            rc = e;
        }
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Public: SPH(2) derivatives of arbitrary fields (ncomp components, each n   */
/* values, component-major).  Outputs for fluid particles, 0 elsewhere:       */
/*   grad_hat[(c*d + K)*n + i]  <d phi_c / d x^_K>^(1)                        */
/*   d2_hat[(c*m + a)*n + i]    second derivatives, order 2-D [xx, zz, xz],   */
/*                              3-D [xx, yy, zz, xy, yz, zx] (cross undoubled) */
/*   lap_phys[c*n + i]          c_trans . D^ phi (Eq. lap_VCT)               */
/* ------------------------------------------------------------------------ */
int orc_sph2_derivatives(const orc_params *P, const orc_bathy *b, orc_state *S, const double *phi,
                         int ncomp, double *grad_hat, double *d2_hat, double *lap_phys)
{
    work_t W;
    memset(&W, 0, sizeof W);
    int n = S->n, d = P->dim;
    stage_geometry(P, b, S, &W);
    int m = W.m;
    alloc_work(&W, n, 1);
    int rc = run_pass1(P, S, &W);
    if (!rc) rc = run_pass2(P, S, &W, 0);
    if (rc) { work_free(&W); return rc; }
    if (grad_hat) memset(grad_hat, 0, sizeof(double) * (size_t)ncomp * d * n);
    if (d2_hat) memset(d2_hat, 0, sizeof(double) * (size_t)ncomp * m * n);
    if (lap_phys) memset(lap_phys, 0, sizeof(double) * (size_t)ncomp * n);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        const pair_t *pp = W.pairs + W.pstart[i];
        int np = (int)(W.pstart[i + 1] - W.pstart[i]);
        double ct[6];
        ctilde(d, W.met + 7 * i, ct);
        for (int c = 0; c < ncomp; ++c) {
            const double *f = phi + (size_t)c * n;
            double g[3] = {0}, bb[6] = {0};
            for (int k = 0; k < np && pp[k].j >= 0; ++k)
                for (int K = 0; K < d; ++K) g[K] += pp[k].V * (f[pp[k].j] - f[i]) * pp[k].gt[K];
            for (int k = 0; k < np && pp[k].j >= 0; ++k) {
                double rg = 0.0;
                for (int K = 0; K < d; ++K) rg += pp[k].r[K] * g[K];
                for (int a = 0; a < m; ++a)
                    bb[a] += pp[k].V * pp[k].F * pp[k].q[a] * ((f[pp[k].j] - f[i]) - rg);
            }
            if (P->operators == 1) {   /* ISPH: 0th-order second derivatives */
                for (int a = 0; a < m; ++a) bb[a] = 0.0;
                for (int k = 0; k < np && pp[k].j >= 0; ++k)
                    for (int a = 0; a < m; ++a) bb[a] += pp[k].V * pp[k].k0[a] * (f[pp[k].j] - f[i]);
            } else {
                double Mc[36];
                memcpy(Mc, W.LU + (size_t)36 * i, sizeof(double) * m * m);
                if (gauss_solve(m, Mc, 1, bb)) continue;
                for (int a = 0; a < m; ++a) bb[a] *= 2.0;   /* D = 2 M^-1 b */
            }
            if (grad_hat)
                for (int K = 0; K < d; ++K) grad_hat[((size_t)c * d + K) * n + i] = g[K];
            if (d2_hat)
                for (int a = 0; a < m; ++a)
                    d2_hat[((size_t)c * m + a) * n + i] = a < d ? bb[a] : 0.5 * bb[a];
            if (lap_phys) {
                double lap = W.met[7 * i + 3] * g[d - 1];
                for (int a = 0; a < m; ++a) lap += ct[a] * bb[a];
                lap_phys[(size_t)c * n + i] = lap;
            }
        }
    }
    work_free(&W);
    return ORC_OK;
}

/* Public: the summation gradient of Eq. (gra_sum) with constant density,
 * <grad^ phi>+_i = sum_j V_j (phi_j + phi_i) grad w_ij over fluid and wall
 * neighbours (wall values from phi), in projected coordinates, for fluid
 * particles (0 elsewhere): out[(c*d + K)*n + i]. */
int orc_summation_gradient(const orc_params *P, const orc_bathy *b, orc_state *S, const double *phi,
                           int ncomp, double *out)
{
    work_t W;
    memset(&W, 0, sizeof W);
    int n = S->n, d = P->dim;
    stage_geometry(P, b, S, &W);
    alloc_work(&W, n, 1);
    int rc = run_pass1(P, S, &W);
    if (!rc) rc = run_pass2(P, S, &W, 0);
    if (rc) { work_free(&W); return rc; }
    memset(out, 0, sizeof(double) * (size_t)ncomp * d * n);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        const pair_t *pp = W.pairs + W.pstart[i];
        int np = (int)(W.pstart[i + 1] - W.pstart[i]);
        for (int c = 0; c < ncomp; ++c) {
            const double *f = phi + (size_t)c * n;
            double g[3] = {0};
            for (int k = 0; k < np && pp[k].j >= 0; ++k)
                for (int K = 0; K < d; ++K) g[K] += pp[k].V * (f[pp[k].j] + f[i]) * pp[k].gw[K];
            for (int K = 0; K < d; ++K) out[((size_t)c * d + K) * n + i] = g[K];
        }
    }
    work_free(&W);
    return ORC_OK;
}

/* Public: the SPH(2) moment matrices M_i = sum_j V_j F_ij q_ij p_ij^T of Eq.
 * (sec_SPH2), row-major m x m per fluid particle (zero elsewhere): M[(i*m + a)*m + c].
 * For conditioning bounds in parity checks. */
int orc_moment_matrices(const orc_params *P, const orc_bathy *b, orc_state *S, double *M)
{
    work_t W;
    memset(&W, 0, sizeof W);
    int n = S->n;
    stage_geometry(P, b, S, &W);
    int m = W.m;
    alloc_work(&W, n, 1);
    int rc = run_pass1(P, S, &W);
    if (!rc) rc = run_pass2(P, S, &W, 0);
    if (!rc) {
        memset(M, 0, sizeof(double) * (size_t)n * m * m);
        for (int i = 0; i < n; ++i)
            if (S->type[i] == ORC_FLUID)
                memcpy(M + (size_t)i * m * m, W.LU + (size_t)36 * i, sizeof(double) * m * m);
    }
    work_free(&W);
    return rc;
}

/* Public: volume smoothing alone (for its conservation pin). */
int orc_volume_smoothing(const orc_params *P, const orc_bathy *b, orc_state *S, int mode)
{
    work_t W;
    memset(&W, 0, sizeof W);
    stage_geometry(P, b, S, &W);
    stage_smoothing(P, S, &W, mode);
    work_free(&W);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Particle regularisation after the position update.  Sec. 4.1 stabilises   */
/* every simulation with optimized particle shifting (shift parameter 0.2),  */
/* dynamic stabilization (allowed overlap 40 % of the particle diameter) and */
/* XSPH on free-surface particles (velocity smoothing 5e-3); it gives the    */
/* parameters only.  Restated here from the cited methods, in projected      */
/* space (where particles are isotropic with spacing d0), with the step's    */
/* neighbour sets and the positions after the update:                        */
/*  DS   (Tsuruta et al.): every pair with |r^_ij| < d_DS = (1 - overlap) d0  */
/*       is pushed apart so that, moving with the corrected velocities for    */
/*       one step, it would be d_DS apart: du^_i = -sum mu_ij (d_DS - |r^_ij|) */
/*       / dt e_ij, e_ij = r^_ij/|r^_ij| (towards j), mu = 1/2 for a fluid j  */
/*       (equal masses, momentum kept), 1 for a wall or virtual j (fixed);    */
/*       the velocity gains J^-1 du^ and the position dt J^-1 du^.            */
/*  XSPH (Monaghan): free-surface particles take                              */
/*       u_i + eps sum_{j fluid} V0 (u_j - u_i) w(|r^_ij|), the DS-corrected   */
/*       velocities on both sides.                                            */
/*  OPS  (Fickian shifting of Lind et al. with the free-surface treatment of  */
/*       Khayyer et al.): dr^_i = -A l |v^_i| dt grad^C_i, grad^C_i =          */
/*       sum_{all j} V0 grad w_ij, v^ = J v the projected velocity after XSPH; */
/*       on free-surface particles only the part tangential to the surface is */
/*       kept, with the normal of Marrone et al., n = -L grad^C / |L grad^C|,  */
/*       L = B^-1, B = sum_{all j} V0 (r^_j - r^_i) (x) grad w_ij (no shift if */
/*       B is singular).                                                      */
/* The projected displacement dr^ goes back to physical space through the     */
/* Jacobian at the new position: dx = dx^, dy = dy^, dz = (dz^ - s_x dx^ -    */
/* s_y dy^)/alpha.  Every particle's correction uses the same inputs (no      */
/* in-place updates), so the result does not depend on the particle order.  */
/* ------------------------------------------------------------------------ */
static void to_phys(int d, const double *met, const double *dh, double *dp)
{
    dp[0] = dh[0];
    if (d == 2) {
        dp[1] = (dh[1] - met[1] * dh[0]) / met[0];
    } else {
        dp[1] = dh[1];
        dp[2] = (dh[2] - met[1] * dh[0] - met[2] * dh[1]) / met[0];
    }
}

static void stage_regularise(const orc_params *P, const orc_bathy *b, orc_state *S, const work_t *W)
{
    int n = S->n, d = P->dim;
    double l = W->l, V0 = W->V0, dt = P->dt;
    double *xh = malloc(sizeof(double) * (size_t)n * d + 8);
    double *met = malloc(sizeof(double) * (size_t)n * 7 + 8);
    double *ud = malloc(sizeof(double) * (size_t)n * 3 + 8);   /* DS-corrected velocity */
    double *dh = calloc((size_t)n * 3 + 1, 8);                 /* projected displacement */
    double *un = malloc(sizeof(double) * (size_t)n * 3 + 8);   /* final velocity */
    for (int i = 0; i < n; ++i) {
        double y = d == 3 ? S->y[i] : 0.0, zh;
        metric_at(P, b, S->x[i], y, S->z[i], &zh, met + 7 * i);
        xh[d * i] = S->x[i];
        if (d == 3) xh[3 * i + 1] = S->y[i];
        xh[d * i + d - 1] = zh;
        for (int c = 0; c < d; ++c) ud[3 * i + c] = vel(S, d, i, c);
    }
    /* dynamic stabilization */
    double dds = (1.0 - P->ds_overlap) * P->d0;
    if (P->ds_overlap > 0.0) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            if (S->type[i] != ORC_FLUID) continue;
            double du[3] = {0.0, 0.0, 0.0};
            for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
                int j = W->col[k];
                double r[3], r2 = 0.0;
                for (int K = 0; K < d; ++K) {
                    r[K] = xh[d * j + K] - xh[d * i + K];
                    r2 += r[K] * r[K];
                }
                double rr = sqrt(r2);
                if (!(rr < dds) || rr == 0.0) continue;
                double mu = S->type[j] == ORC_FLUID ? 0.5 : 1.0;
                double f = mu * (dds - rr) / (dt * rr);
                for (int K = 0; K < d; ++K) du[K] -= f * r[K];
            }
            double dv[3];
            to_phys(d, met + 7 * i, du, dv);
            for (int c = 0; c < d; ++c) {
                ud[3 * i + c] += dv[c];
                dh[3 * i + c] = dt * du[c];
            }
        }
    }
    /* XSPH on free-surface particles, then optimized particle shifting */
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < d; ++c) un[3 * i + c] = ud[3 * i + c];
        if (S->type[i] != ORC_FLUID) continue;
        double gc[3] = {0.0, 0.0, 0.0}, xs[3] = {0.0, 0.0, 0.0}, B[9] = {0.0};
        for (int64_t k = W->row_ptr[i]; k < W->row_ptr[i + 1]; ++k) {
            int j = W->col[k];
            double r[3], r2 = 0.0;
            for (int K = 0; K < d; ++K) {
                r[K] = xh[d * i + K] - xh[d * j + K];   /* r^_i - r^_j */
                r2 += r[K] * r[K];
            }
            double rr = sqrt(r2);
            if (rr == 0.0) continue;
            if (P->xsph_eps > 0.0 && W->fs[i] && S->type[j] == ORC_FLUID) {
                double wv = kern_w(rr, l, d);
                for (int c = 0; c < d; ++c) xs[c] += V0 * (ud[3 * j + c] - ud[3 * i + c]) * wv;
            }
            if (P->ops_shift > 0.0) {
                double dwr = kern_dw(rr, l, d) / rr;
                for (int K = 0; K < d; ++K) gc[K] += V0 * dwr * r[K];
                for (int a = 0; a < d; ++a)
                    for (int c = 0; c < d; ++c) B[a * d + c] -= V0 * dwr * r[a] * r[c];
            }
        }
        if (P->xsph_eps > 0.0 && W->fs[i])
            for (int c = 0; c < d; ++c) un[3 * i + c] = ud[3 * i + c] + P->xsph_eps * xs[c];
        if (P->ops_shift > 0.0) {
            const double *m = met + 7 * i;
            double vh[3];
            vh[0] = un[3 * i];
            if (d == 2) {
                vh[1] = m[1] * un[3 * i] + m[0] * un[3 * i + 1];
            } else {
                vh[1] = un[3 * i + 1];
                vh[2] = m[1] * un[3 * i] + m[2] * un[3 * i + 1] + m[0] * un[3 * i + 2];
            }
            double sp = 0.0;
            for (int K = 0; K < d; ++K) sp += vh[K] * vh[K];
            double D = P->ops_shift * l * sqrt(sp) * dt, s[3];
            for (int K = 0; K < d; ++K) s[K] = -D * gc[K];
            if (W->fs[i]) {
                double Li[9], nv[3], nn = 0.0, sn = 0.0;
                int bad = invert_dxd(d, B, Li);
                for (int a = 0; a < d && !bad; ++a) {
                    nv[a] = 0.0;
                    for (int c = 0; c < d; ++c) nv[a] -= Li[a * d + c] * gc[c];
                    nn += nv[a] * nv[a];
                }
                if (bad || !(nn > 0.0)) {
                    for (int K = 0; K < d; ++K) s[K] = 0.0;
                } else {
                    nn = sqrt(nn);
                    for (int K = 0; K < d; ++K) {
                        nv[K] /= nn;
                        sn += s[K] * nv[K];
                    }
                    for (int K = 0; K < d; ++K) s[K] -= sn * nv[K];
                }
            }
            for (int K = 0; K < d; ++K) dh[3 * i + K] += s[K];
        }
    }
    for (int i = 0; i < n; ++i) {
        if (S->type[i] != ORC_FLUID) continue;
        double dp[3];
        to_phys(d, met + 7 * i, dh + 3 * i, dp);
        S->x[i] += dp[0];
        if (d == 2) {
            S->z[i] += dp[1];
            S->u[i] = un[3 * i]; S->w[i] = un[3 * i + 1];
        } else {
            S->y[i] += dp[1];
            S->z[i] += dp[2];
            S->u[i] = un[3 * i]; S->v[i] = un[3 * i + 1]; S->w[i] = un[3 * i + 2];
        }
    }
    free(xh); free(met); free(ud); free(dh); free(un);
}

/* Public: regularisation alone on a state, with neighbour sets taken at the
 * given positions (for its pins). */
int orc_regularise(const orc_params *P, const orc_bathy *b, orc_state *S, const int32_t *fs)
{
    work_t W;
    memset(&W, 0, sizeof W);
    stage_geometry(P, b, S, &W);
    W.fs = (int32_t *)calloc((size_t)S->n + 1, 4);
    for (int i = 0; i < S->n; ++i) W.fs[i] = fs ? fs[i] : 0;
    stage_regularise(P, b, S, &W);
    work_free(&W);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Public: nsteps of the projection scheme (Sec. 3.3 with the VCT equations). */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_params *P, const orc_bathy *b, orc_state *S, int nsteps, orc_probe *pr,
             int *total_iters)
{
    int n = S->n, d = P->dim, rc = ORC_OK;
    if (total_iters) *total_iters = 0;
    for (int step = 0; step < nsteps && !rc; ++step) {
        work_t W;
        memset(&W, 0, sizeof W);
        stage_geometry(P, b, S, &W);
        if (P->map_kind == ORC_MAP_SIGMA && P->volume_mode == 2)
            stage_smoothing(P, S, &W, P->smoothing_mode);
        alloc_work(&W, n, 1);
        if (P->wall_slip) stage_wall_velocity(P, S, &W);
        rc = run_pass1(P, S, &W);
        if (!rc) rc = run_pass2(P, S, &W, 1);
        if (rc) { work_free(&W); break; }

        /* unknowns: fluid, not free surface */
        char *unk = calloc((size_t)n + 1, 1);
        for (int i = 0; i < n; ++i) unk[i] = S->type[i] == ORC_FLUID && !W.fs[i];
        /* right side of Eq. (VCT_ppe_w): rho/dt tr(J <grad^ (x) v*>) + gamma (rho fac - rho^)/dt^2 */
        double *rhs = calloc((size_t)n + 1, 8), *c0 = calloc((size_t)n + 1, 8);
        double *zero = calloc((size_t)n + 1, 8), *x = calloc((size_t)n + 1, 8);
        double gamma = P->gamma_over_dt * P->dt;
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            if (!unk[i]) continue;
            const pair_t *pp = W.pairs + W.pstart[i];
            int np = (int)(W.pstart[i + 1] - W.pstart[i]);
            double X[9] = {0}; /* X[c][K] = <d v*_c / d x^_K> */
            for (int k = 0; k < np && pp[k].j >= 0; ++k)
                for (int c = 0; c < d; ++c) {
                    /* a wall neighbour carries v_wall + dt f_i: the intermediate velocity
                     * it would have under the acceleration that Eq. (PNC) assumes */
                    double vj = pp[k].tj == ORC_FLUID ? W.vstar[d * pp[k].j + c]
                                                      : wall_vel(&W, pp[k].j, c) + P->dt * W.acc[d * i + c];
                    double vij = vj - W.vstar[d * i + c];
                    for (int K = 0; K < d; ++K) X[c * d + K] += pp[k].V * vij * pp[k].gt[K];
                }
            double Jm[9], div = 0.0;
            jac(d, W.met + 7 * i, Jm);
            for (int I = 0; I < d; ++I)
                for (int K = 0; K < d; ++K) div += Jm[I * d + K] * X[I * d + K];
            double fac = P->volume_mode == 0 ? 1.0 : S->jbar[i] / W.met[7 * i];
            rhs[i] = P->rho / P->dt * div + gamma * (P->rho * fac - W.rho_hat[i]) / (P->dt * P->dt);
        }
        ppe_ctx C = {P, &W, unk, zero};
        /* c0 = op(0): wall (PNC) contributions, independent of p */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) c0[i] = unk[i] ? ppe_op_one(P, &W, i, zero) : 0.0;
        C.c0 = c0;
        double *bl = calloc((size_t)n + 1, 8);
        for (int i = 0; i < n; ++i) bl[i] = unk[i] ? rhs[i] - c0[i] : 0.0;
        for (int i = 0; i < n; ++i) x[i] = unk[i] ? S->p[i] : 0.0;
        int it = 0;
        double res = 0.0;
        int e = bicgstab(&C, bl, x, P->ppe_rtol, P->ppe_max_iter, &it, &res);
        if (total_iters) *total_iters += it;
        if (e) rc = e;
        if (pr && step == nsteps - 1) {
            if (pr->fs) for (int i = 0; i < n; ++i) pr->fs[i] = W.fs[i];
            if (pr->rho_hat) for (int i = 0; i < n; ++i) pr->rho_hat[i] = W.rho_hat[i];
            if (pr->nu) for (int i = 0; i < n; ++i) pr->nu[i] = S->type[i] == ORC_FLUID ? W.nu[i] : 0.0;
            if (pr->lam_min) for (int i = 0; i < n; ++i) pr->lam_min[i] = W.lam[i];
            if (pr->vstar)
                for (int c = 0; c < d; ++c)
                    for (int i = 0; i < n; ++i)
                        pr->vstar[(size_t)c * n + i] = S->type[i] == ORC_FLUID ? W.vstar[d * i + c] : 0.0;
            if (pr->ppe_b) for (int i = 0; i < n; ++i) pr->ppe_b[i] = bl[i];
            if (pr->jbar_used) for (int i = 0; i < n; ++i) pr->jbar_used[i] = S->jbar[i];
            if (pr->vwall)
                for (int c = 0; c < d; ++c)
                    for (int i = 0; i < n; ++i)
                        pr->vwall[(size_t)c * n + i] = S->type[i] == ORC_WALL ? wall_vel(&W, i, c) : 0.0;
            if (pr->x_test && pr->ppe_Ax) {
                double *xt = calloc((size_t)n + 1, 8);
                for (int i = 0; i < n; ++i) xt[i] = unk[i] ? pr->x_test[i] : 0.0;
                ppe_apply(&C, xt, pr->ppe_Ax);
                free(xt);
            }
            pr->n_iter = it;
            pr->resid = res;
        }
        /* corrector + position update (Eqs. VCT_predictor, VCT_update) */
        if (!rc) {
            double *pn = calloc((size_t)n + 1, 8);
            for (int i = 0; i < n; ++i) pn[i] = unk[i] ? x[i] : 0.0;
            double *vn = calloc((size_t)n * 3 + 1, 8);
#pragma omp parallel for schedule(dynamic, 64)
            for (int i = 0; i < n; ++i) {
                if (S->type[i] != ORC_FLUID) continue;
                const pair_t *pp = W.pairs + W.pstart[i];
                int np = (int)(W.pstart[i + 1] - W.pstart[i]);
                double gp[3] = {0};
                for (int k = 0; k < np && pp[k].j >= 0; ++k) {
                    double pij;
                    if (pp[k].tj == ORC_FLUID) pij = pn[pp[k].j] - pn[i];
                    else {
                        double s = 0.0;
                        for (int K = 0; K < d; ++K) s += pp[k].rp[K] * W.acc[d * i + K];
                        pij = P->rho * s;
                    }
                    if (P->operators == 1)   /* summation gradient (Eq. gra_sum), p_j + p_i */
                        for (int K = 0; K < d; ++K) gp[K] += pp[k].V * (pij + 2.0 * pn[i]) * pp[k].gw[K];
                    else
                        for (int K = 0; K < d; ++K) gp[K] += pp[k].V * pij * pp[k].gt[K];
                }
                double Jm[9];
                jac(d, W.met + 7 * i, Jm);
                for (int I = 0; I < d; ++I) {
                    double s = 0.0;
                    for (int K = 0; K < d; ++K) s += Jm[I * d + K] * gp[K];
                    vn[d * i + I] = W.vstar[d * i + I] - P->dt / P->rho * s;
                }
            }
            for (int i = 0; i < n; ++i) {
                if (S->type[i] != ORC_FLUID) continue;
                S->p[i] = pn[i];
                if (d == 2) {
                    S->u[i] = vn[2 * i]; S->w[i] = vn[2 * i + 1];
                    S->x[i] += P->dt * S->u[i];
                    S->z[i] += P->dt * S->w[i];
                } else {
                    S->u[i] = vn[3 * i]; S->v[i] = vn[3 * i + 1]; S->w[i] = vn[3 * i + 2];
                    S->x[i] += P->dt * S->u[i];
                    S->y[i] += P->dt * S->v[i];
                    S->z[i] += P->dt * S->w[i];
                }
            }
            if (P->ops_shift > 0.0 || P->ds_overlap > 0.0 || P->xsph_eps > 0.0)
                stage_regularise(P, b, S, &W);
            for (int i = 0; i < n; ++i)
                if (S->type[i] == ORC_FLUID && !(isfinite(S->x[i]) && isfinite(S->z[i]) && isfinite(S->p[i])))
                    rc = ORC_ERR_NONFINITE;
            free(pn);
            free(vn);
        }
        free(unk); free(rhs); free(c0); free(zero); free(x); free(bl);
        work_free(&W);
    }
    return rc;
}

int orc_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
    return omp_get_max_threads();
#else
    (void)nt;
    return 1;
#endif
}

int orc_abi_version(void) { return 1; }
