// Internal declarations of the VCT + SPH(2) CUDA library (sm_103a).
//
// Data layout in HBM: every per-particle quantity is a separate array in
// cell-sorted order (structure of arrays); multi-component quantities are
// component-major, q[k * cap + i], so one thread per particle reads and
// writes coalesced.  Neighbour lists and pressure-equation coefficients are
// ELL, slot-major, nbr[k * cap + i].
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "vct.h"

namespace vct {

constexpr int FLUID = 0, WALL = 1, VIRTUAL = 2;
// Default bound on the polls of one grid-barrier wait: ~1-2 s on this GPU.
constexpr unsigned long long SPIN_LIMIT_DEFAULT = 40000000ull;
constexpr int MAXG = VCT_MAX_GAUSS;

// Parameters broadcast to every kernel by value (kernel-parameter bank).
struct DevParams {
    int dim, kind, smag, volume_mode;
    int n_gauss, max_nbr, precision, max_iter;
    int nc[3];                // cells per axis (x, y, z); 2-D: y = 1
    int slip;                 // 1: free-slip walls (wall particles carry a mirrored velocity)
    double aspect, rho, nu_k, g, dt, d0, l, inv_l, re, re2, V0, ad;
    double ops_shift, ds_overlap, xsph_eps;   // particle regularisation (0: off)
    int pguess;               // order of the pressure extrapolation of the initial guess
    int operators;            // 0: ISPH(2) (SPH(2) second derivatives, 1st-order pressure
                              // gradient); 1: ISPH (0th-order second derivatives, summation
                              // pressure gradient)
    double gamma, cv, cs, ds, H, H_hat, amin, amax, lam_lo, lam_hi, rtol;
    double inner_floor;       // mixed form: each FP32 BiCGSTAB pass stops at this relative residual
    double box_lo[3], cell_h, inv_cell_h;
    double h0, slope_x, slope_y, cos_amp, cos_len;
    double gamp[MAXG], gcx[MAXG], gcy[MAXG], gwid[MAXG];
    double ginv2[MAXG];       // 1 / width^2 of each bump (the map's per-particle divisions, once)
};

// One buffer set of the cell-sorted particle state.
struct Part {
    double *x, *y, *z;        // physical position
    double *u, *v, *w;        // physical velocity
    double *p, *jbar;
    int32_t *type, *orig;     // orig = caller index
    double *xh, *yh, *zh;     // projected position
    double *J, *sx, *sy, *c0, *c3;  // metric: J = alpha, s = third column of the
                                    // Jacobian, c_trans entries 0 and 3
};

// Slot kk of row i in the pressure-equation ELL arrays.  Slots are kept in
// blocks of EG consecutive slots per row (EG = 4 in 2-D, 8 in 3-D: the width of
// the solver's row groups), blocks of all rows one after the other, so the EG
// lanes of a row group read one contiguous EG x 4-byte segment per block and a
// warp's load covers one 128-byte line.  Storage: roundup(max_nbr, EG) x cap.
template <int EG>
__host__ __device__ __forceinline__ int64_t ell_at(int kk, int64_t i, int64_t cap)
{
    return ((int64_t)(kk / EG) * cap + i) * EG + (kk % EG);
}
__host__ __device__ __forceinline__ int64_t ell_at_dim(int dim, int kk, int64_t i, int64_t cap)
{
    return dim == 2 ? ell_at<4>(kk, i, cap) : ell_at<8>(kk, i, cap);
}
template <int D>
__host__ __device__ constexpr int ell_group() { return D == 2 ? 4 : 8; }

// Scratch of one step.
struct Work {
    int64_t cap;
    int32_t max_nbr;          // ELL slots per particle
    int32_t *key, *cell_count, *cell_start, *cursor, *perm, *scan_tmp;
    int64_t ncell;
    int32_t *nbr_cnt, *nbr;   // ELL neighbour lists, slot-major
    double *L, *gv, *Ct;      // [d*d], [d*d], [d*m] per particle, component-major
    double *rho_hat, *lam, *nu;
    int32_t *fs;
    double *vstar, *acc;      // [d] per particle
    int32_t *pcnt, *pcol;     // pressure-equation coefficients (ELL, slot-blocked: ell_at)
    double *pval, *diag, *bvec, *wallrhs;
    double *pwall;            // [d] per unknown row: rho sum over wall neighbours of a_ij (r_j - r_i),
                              // so that wallrhs = pwall . f_i (Eq. PNC; read by the step's reverse)
    float *pvalf;             // FP32 coefficients of the mixed form
    double *jbar_tmp;
    // Krylov
    double *kx, *kf;          // FP64 iterate and residual
    double *kr, *krh, *kp0, *kp1, *kv0, *kv1, *kt, *ks, *kd;   // inner vectors (FP64 or FP32)
    double *partial, *scal;
    int32_t *kiters;          // per-step iteration counts (device)
    double *kresid;           // per-step relative residuals (device)
    unsigned int *bar;        // grid barrier: [0] count, [1] generation
    int32_t *status;          // [0] code, [1] first particle (sorted index), [2] spin-timeouts
    unsigned long long spin_limit;  // polls before a grid-barrier wait gives up
    long long *counts;        // [0] unknown rows, [1] off-diagonal coefficients (last step)
    // csr export
    int64_t *row_tmp;
    // multigrid preconditioner
    int32_t *cellid;          // level-1 node (cell) of each sorted particle
    float *mg_dsc;            // 1 / diag of each unknown row (0 elsewhere)
    float *mg_pool;           // coarse operators and vectors of all levels
    float *mg_B;              // row-cell operator (3^d entries per row, entry-major), or null
    double *kr0;              // fine residual of the V-cycle (FP32 or FP64 slots)
    double *kq0, *kq1;        // preconditioned directions p^, s^
    double *kz0, *kzb;        // V-cycle: first Jacobi step and prolonged correction
    double *adj;              // adjoint scratch: [3 (m + dim)] per particle
    double *sadj;             // step reverse, cell order: [3 dim + dim^2] per particle (allocated on first use)
    double *sadj_co;          // step reverse, caller order: [dim + 2] per particle
    double *radj;             // regularisation reverse, cell order (rows: regadj_rows) + caller-order
                              // u'_bar, x'_bar [2 dim] (allocated on first use)
    double *rxh, *rmet;       // regularisation: projected position [d] and J, s_x, s_y
    double *rud, *rdh;        //   at the updated positions; corrected velocity [d],
                              //   projected displacement [d]
    double *jratio;           // J / Jbar per particle (sorted order), for the smoothing
    float4 *hatf;             // projected position rounded to FP32 (sorted order; y = 0
                              // in 2-D), the neighbour search's first test, and the
    float4 *hatlo;            // rest, fl32(x - hatf): hi + lo pairs for the mixed form's
    float4 *velhi, *vello;    // pair differences, like the velocity's and
    float4 *vshi, *vslo;      // the intermediate velocity v*'s
    double *vol;              // V_i = V0 J_i / Jbar_i (Sec. 3.6; V0 under Condition A), once
    float *volf;              // per step, and rounded to FP32
    int32_t *urow_flag, *urow_pos, *urow;   // unknown rows (pcnt >= 0) in ascending order,
                                            // urow_pos[n] = their number (large-system solve)
    double *p_last, *p_prev;  // caller order: pressure after the last step and before
    double *p_prev2;          // it, and before that (NaN until set), for the solve's
                              // initial guess
};

// Coarse levels of the aggregation multigrid: level 1 = the cell grid, level
// l+1 = 2 x 2 (x 2) blocks of level l.  Each level stores, in mg_pool, its
// stencil operator A[o * n + I] (S = 3^dim entries per node) at offA and four
// vectors at offv: dinv, b, z, zu (each n floats).
constexpr int MG_MAXL = 24;
struct MG {
    int L;               // coarsest level index (levels 1..L)
    int first_local;     // first level processed by block 0 alone
    int S;               // stencil size, 9 (2-D) or 27 (3-D)
    int coarse_sweeps;   // Jacobi sweeps on the coarsest level
    int presmooth;       // 1: V(1,1); 0: V(0,1), no fine pre-smoothing (on-the-fly form)
    float omega, kappa;  // Jacobi damping and coarse-correction scale (cells to particles)
    float kappa_c;       // coarse-correction scale between the coarse levels
    float omega_c;       // Jacobi damping on the coarse levels (cells and coarser)
    int n[MG_MAXL + 1];
    int dims[MG_MAXL + 1][3];
    int shift[MG_MAXL + 1][3];     // level l -> l+1: factor 2^shift per axis (x, y, z)
    long long offA[MG_MAXL + 1];
    long long offv[MG_MAXL + 1];
    long long soff[MG_MAXL + 1];   // shared-memory offsets (floats) of levels first_local..L
    long long sh_floats;           // shared memory of block 0's levels (floats)
    int fly;                       // 1: V-cycle inputs formed on the fly (small systems)
    int staged;                    // large-system form: rows staged by cp.async
    int gather_l1;                 // large-system form: fine gathers through L1
    int rowcell;                   // large-system form: V(0,1) cycles whose fine post-smoothing
                                   // reads the row-cell operator W.mg_B (0: V(1,1) cycles)
    long long stage_off;           // byte offset of the row-staging area (large systems)
    long long smem_bytes;          // dynamic shared memory of the solver launch
};

// One scenario's pressure solve inside a batched launch (vct_batch_step):
// it owns blocks [b0, b0 + nb) of the cooperative grid.
struct FlyJob {
    Work W;
    MG M;
    int n, maxit;
    double rtol, inner_floor;
    unsigned b0, nb;
};

// One scenario in a batched stage launch (vct_batch_step): each stage of the
// step except the pressure solve runs as one launch over all scenarios, every
// scenario on a contiguous range of the launch's blocks.  The members most
// stages read come first, so that a block copies into shared memory only the
// prefix its stage reads; every member starts on a 16-byte boundary.
struct StageJob {
    int64_t n;
    int64_t reserved;
    alignas(16) Part cur;     // the sorted state the stage reads
    alignas(16) Work W;
    alignas(16) DevParams P;
    alignas(16) Part alt;     // the other buffer set (reorder target)
    alignas(16) MG M;
};

// Stages of a batched step, in step order (BS_MG_COARSEN once per level).
enum BatchStage {
    BS_ZERO, BS_MAP_KEY, BS_CSCAN_BLOCKS, BS_CSCAN_TOPS, BS_CSCAN_ADD, BS_SCATTER,
    BS_CELL_SORT, BS_REORDER,
    BS_NEIGHBOURS, BS_SMOOTHING, BS_JBAR_COPY, BS_WALL_VELOCITY, BS_PASS1, BS_PASS2,
    BS_PASS2_ISPH, BS_RHS, BS_UROW_FLAGS, BS_RSCAN_BLOCKS, BS_RSCAN_TOPS, BS_RSCAN_ADD,
    BS_UROW_SCATTER, BS_MG_DSC, BS_MG_ROWCELL, BS_MG_LEVEL1, BS_MG_COARSEN, BS_MG_COARSEN_SMALL,
    BS_CORRECTOR, BS_CORRECTOR_SUM, BS_REG_GEOM, BS_REG_DS, BS_REG_APPLY,
    BS_COUNT
};

struct Ctx;

// ---- launchers (vct_kernels.cu) ----
// Blocks one scenario takes in batched stage s (0: the scenario skips it);
// rows_list: its solve iterates over the unknown-row list; level: the
// coarsening level of BS_MG_COARSEN.  Exactly the grid of the stage's own
// launcher for that scenario.
int batch_stage_blocks(int s, const DevParams &P, const Work &W, const MG &M, int64_t n,
                       bool rows_list, int level);
// Deepest level BS_MG_COARSEN runs at for any scenario of the batch, plus one.
int batch_coarsen_levels(const MG &M);
// One batched launch of stage s over njobs scenarios: jobs (device), bs
// (device, njobs + 1 ascending block starts, bs[njobs] = total blocks).
void launch_batched(int s, int dim, int precision, const StageJob *jobs, const int *bs, int njobs,
                    int total, int level, cudaStream_t st);
void launch_load(const DevParams &P, Part cur, vct_state s, int64_t n, cudaStream_t st);
void launch_store(const DevParams &P, Part cur, vct_state s, int64_t n, const int32_t *status,
                  cudaStream_t st);
void launch_map_key(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_sort(const DevParams &P, Part cur, Part alt, Work W, int64_t n, cudaStream_t st);
void launch_neighbours(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_smoothing(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_pass1(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_pass2(const DevParams &P, Part cur, Work W, int64_t n, int predictor,
                  cudaStream_t st);
void launch_rhs(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
int launch_krylov(const DevParams &P, Part cur, Work W, int64_t n, int step_slot,
                  int nblocks_coop, cudaStream_t st);
void launch_mg_setup(const DevParams &P, Work W, const MG &M, int64_t n, cudaStream_t st,
                     bool rows_list);
int mg_setup_launches(const MG &M);
// the large-system form's V(0,1) cycles with the row-cell operator
bool mg_rowcell_on(const MG &M);
int launch_krylov_mg(const DevParams &P, Work W, const MG &M, int64_t n, int nblocks_coop,
                     cudaStream_t st);
bool krylov_mg_fly_default(long long rows, int dim);
int krylov_fly_batch_blocks(int precision, int dim, size_t smem, bool expl);
size_t krylov_batch_stage_bytes(int precision, int dim);
// derivative of the SPH(2) second derivatives with respect to the projected positions
// (ppe: the pressure operator's linear part with phi = x and wbar = pbar)
void launch_d2pos(const DevParams &P, Part cur, Work W, int64_t n, bool ppe, const double *phi,
                  const double *wbar, double *xh_bar, cudaStream_t st);
// derivative of the density estimate with respect to the projected positions
void launch_rhopos(const DevParams &P, Part cur, Work W, int64_t n, const double *rho_bar,
                   double *xh_bar, cudaStream_t st);
// derivative of the corrected gradient with respect to the projected positions
void launch_gradpos(const DevParams &P, Part cur, Work W, int64_t n, int ncomp, const double *phi,
                    const double *grad_bar, double *xh_bar, cudaStream_t st);
// adjoint of the last step's pressure solve by the Jacobi-preconditioned BiCGSTAB
// on A^T (products through the transposed-slot table): b_bar = A^-T p_bar (caller order)
int launch_ppe_adjoint(const DevParams &P, Part cur, Work W, int64_t n, const double *p_bar,
                       double *b_bar, cudaStream_t st);
// A <-> A^T in place (build_slots: write the transposed-slot table first, into
// the neighbour-list scratch); the right side p_bar gathered into the solver's
// vectors, and the solution scattered to b_bar (caller order)
void launch_ppe_transpose(const DevParams &P, Work W, int64_t n, bool build_slots, cudaStream_t st);
void launch_adj_gather(Part cur, Work W, int64_t n, const double *p_bar, cudaStream_t st);
void launch_adj_scatter(Part cur, Work W, int64_t n, double *b_bar, cudaStream_t st);
// reverse of one step with respect to the velocities, in three parts around the
// two adjoint solves (scratch W.sadj, W.sadj_co):
//   a: the corrector's adjoint, the pressure adjoint p_bar into W.sadj_co (caller order);
//   b: after b_bar = A^-T p_bar (W.sadj_co + n), the right side's adjoint and the
//      viscous term's lap_bar into W.sadj_co + 2n;
//   c: after the SPH(2) adjoint wrote phi_bar into v_bar_in, v_bar_in += v*_bar.
void launch_stepadj_a(const DevParams &P, Part cur, Work W, int64_t n, const double *v_bar,
                      const double *x_bar, const double *p_bar, cudaStream_t st);
void launch_stepadj_b(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_stepadj_c(const DevParams &P, Part cur, Work W, int64_t n, double *v_bar_in,
                      cudaStream_t st);
// reverse of the particle regularisation for the step's reverse: the rows of
// W.radj per particle, x' saved before the forward regularisation runs, and the
// reverse itself from the step outputs' adjoints (v_bar, x_bar, caller order) to
// u'_bar and x'_bar (caller order) at the corrector's output
int regadj_rows(int dim);
void launch_regadj_save(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_regadj(const DevParams &P, Part cur, Work W, int64_t n, const double *v_bar,
                   const double *x_bar, double *vb_co, double *xb_co, cudaStream_t st);
// adjoint of the ISPH operator set's gradient and Laplacian (the step reverse's
// viscous term under that set); arrays as launch_sph2_adjoint's
void launch_isph_adjoint(const DevParams &P, Part cur, Work W, int64_t n, int ncomp,
                         const double *gbar, const double *lapbar, double *phibar, cudaStream_t st);
int launch_krylov_fly_batch(int precision, int dim, const FlyJob *jobs, int njobs, unsigned nblocks,
                            size_t smem, bool expl, cudaStream_t st);
int krylov_mg_coop_blocks(int precision, int dim, size_t smem, bool fly);
size_t krylov_mg_stage_bytes(int precision, int dim, bool staged);
void launch_corrector(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
bool regularise_on(const DevParams &P);
int launch_regularise(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_sph2_field(const DevParams &P, Part cur, Work W, int64_t n, const double *phi,
                       int ncomp, double *grad, double *d2, double *lap, cudaStream_t st);
void launch_csr_export(const DevParams &P, Part cur, Work W, int64_t n, int64_t *row_ptr,
                       int32_t *col, int64_t col_cap, cudaStream_t st);
int launch_map_adjoint(const DevParams &P, vct_state s, int64_t n, const double *const *mbar_dev,
                       double *partial, int64_t partial_cap, double *out, cudaStream_t st);
// water level at gauges, its squared sum and gradient (returns 1: bad gauge
// count, 2: scratch too small); res: 3 ng + 1 doubles on the device
int launch_gauge_loss(const DevParams &P, vct_state s, int64_t n, const int32_t *fs, int ng,
                      const double *gxy, double *partial, int64_t partial_cap, double *res,
                      double *pos_bar, cudaStream_t st);
// derivative of the per-particle metric with respect to the physical positions
void launch_map_pos_adjoint(const DevParams &P, vct_state s, int64_t n, const double *const *mbar_dev,
                            double *pos_bar, cudaStream_t st);
void launch_sph2_adjoint(const DevParams &P, Part cur, Work W, int64_t n, int ncomp,
                         const double *gbar, const double *d2bar, const double *lapbar,
                         double *phibar, cudaStream_t st);
void launch_probe_out(const DevParams &P, Part cur, Work W, int64_t n, const vct_probe &pr,
                      cudaStream_t st);
void launch_force_fs(Part cur, Work W, int64_t n, const int32_t *fs_in, cudaStream_t st);
// free-slip wall velocities (Sec. 3.5) into the sorted state's wall particles
void launch_wall_velocity(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st);
void launch_probe_ax(const DevParams &P, Part cur, Work W, int64_t n, const double *x_test,
                     double *out, cudaStream_t st);
int krylov_coop_blocks(int precision, int dim);

// Background cell grid of edge re over the projected box of prm (the
// cells of the neighbour search, Sec. 3.4).  Checks, before any integer
// conversion, that re is positive and finite, that the box is finite and
// ordered, and that every axis holds between 1 and `limit` cells and the
// whole grid at most `limit` cells.  VCT_ERR_ARG for a bad radius or box,
// VCT_ERR_CAPACITY for a grid above the limit.
inline vct_status cell_grid(const vct_params *prm, double re, int64_t limit, int nc[3],
                            int64_t *ncell)
{
    if (!(re > 0.0) || !(re < 1.0e300)) return VCT_ERR_ARG;
    double total = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double lo = prm->box_lo[k], hi = prm->box_hi[k];
        if (!(lo > -1.0e300 && hi < 1.0e300 && hi >= lo)) return VCT_ERR_ARG;
        double ext = (prm->dim == 2 && k == 1) ? 1.0 : floor((hi - lo) / re) + 1.0;
        if (!(ext >= 1.0) || ext > (double)limit) return VCT_ERR_CAPACITY;
        total *= ext;
        if (total > (double)limit) return VCT_ERR_CAPACITY;
        nc[k] = (int)ext;
    }
    *ncell = (int64_t)nc[0] * nc[1] * nc[2];
    if (*ncell < 1 || *ncell > limit) return VCT_ERR_CAPACITY;
    return VCT_OK;
}

}  // namespace vct
