/*
 * vct.h -- C ABI of the VCT + SPH(2) free-surface step on one B300 (sm_103a).
 *
 * The method: incompressible SPH with SPH(2) second derivatives, run in a
 * vertically transformed ("projected") coordinate r^ = (x, y, alpha (z + beta))
 * (Sec. 2.1, Eq. VCT) with the E, BF, BFE and sigma maps of Sec. 2.2.  One
 * step is the projection scheme of Sec. 3.3 written with the VCT metric
 * (Eqs. VCT_predictor, VCT_ppe / VCT_ppe_w, VCT_update).
 *
 * Conventions shared by every entry point
 *  - All particle arrays are structure-of-arrays, one value per particle,
 *    indexed by the caller's particle index i in [0, n).  That index is the
 *    particle's id: neighbour lists are sorted by it and outputs are written
 *    at it.  In 2-D the vertical axis is z; y and v are ignored (may be NULL).
 *  - Particle type (int32): 0 fluid, 1 wall (on the wall surface), 2 virtual
 *    (outside the wall; enters only the density and the free-surface test),
 *    Sec. 3.5.
 *  - Pointers are DEVICE pointers unless stated otherwise.  The caller owns
 *    every buffer it passes; the context owns its scratch, allocated once in
 *    vct_init up to `capacity` particles.  No call allocates device memory
 *    after vct_init.
 *  - Work is queued on the context's stream.  Calls that return a status
 *    synchronise that stream once at their end to read the device status
 *    word; nothing else blocks.
 *  - Errors: every call returns a vct_status; no C++ exception crosses the
 *    ABI.  Device-side problems (singular moment matrix, non-finite state,
 *    Krylov not converged, neighbour capacity, spin-wait timeout) are sticky
 *    in the context until the next call; vct_last_error() names the first
 *    offending particle.  After an error the caller's state is left as it was
 *    at the start of the failed call (vct_step writes back only on success).
 *  - Units are the caller's (SI in this project's workloads).
 */
#ifndef VCT_H
#define VCT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VCT_OK = 0,
    VCT_ERR_ARG = 1,        /* invalid argument (NULL, size, dimension, capacity) */
    VCT_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    VCT_ERR_CAPACITY = 3,   /* more neighbours than max_neighbours, or n > capacity */
    VCT_ERR_SINGULAR = 4,   /* B_i or M_i not invertible (isolated particle) */
    VCT_ERR_NONFINITE = 5,  /* NaN/Inf in the updated state */
    VCT_ERR_NOCONV = 6,     /* pressure solve did not reach krylov_rtol in krylov_max_iter */
    VCT_ERR_TIMEOUT = 7     /* a bounded device spin-wait gave up */
} vct_status;

/* Sec. 2.2: E (alpha = aspect, beta = 0), BF (alpha = 1, beta = -h),
 * BFE (alpha = aspect, beta = -h), sigma (alpha = H_hat/(H - h), beta = -h,
 * alpha clamped to [alpha_min, alpha_max] with zero derivatives outside). */
typedef enum { VCT_MAP_E = 0, VCT_MAP_BF = 1, VCT_MAP_BFE = 2, VCT_MAP_SIGMA = 3 } vct_map_kind;

/* FP64: every sum and solve in double.  MIXED: neighbour sums in FP32 with
 * compensated (Kahan) accumulation; in the step's passes 1 and 2, right side
 * corrector, J-bar smoothing and regularisation, the pair offsets r_ij and
 * velocity differences v_ij (v*_ij)
 * come from each particle's value kept as two FP32 numbers (hi + lo), as
 * accurate as the FP64 difference rounded to FP32, and the remainder
 * v_ij - r_ij . <grad v>_i is formed in FP32 from them (sph2_derivatives forms
 * its differences in FP64 and rounds them); inversion of
 * B_i, the SPH(2) solves with M_i and the pressure-equation iterate and
 * residual in FP64. */
typedef enum { VCT_FP64 = 0, VCT_MIXED = 1 } vct_precision;

#define VCT_MAX_GAUSS 32

/* Bottom elevation h(x,y) = h0 + slope_x x + slope_y y + cos_amp cos(2 pi x / cos_len)
 * + sum_g amp_g exp(-((x-cx_g)^2 + (y-cy_g)^2) / (2 width_g^2)).
 * Covers the bottoms of Sec. 4 (flat, linear, cosine, Gaussian bumps).
 * amp/cx/cy/width are HOST arrays of n_gauss <= VCT_MAX_GAUSS entries,
 * copied by vct_init. */
typedef struct {
    double h0, slope_x, slope_y, cos_amp, cos_len;
    int32_t n_gauss;
    int32_t reserved;
    const double *amp, *cx, *cy, *width;
} vct_bathymetry;

typedef struct {
    int32_t dim;            /* 2 (x, z) or 3 (x, y, z) */
    int32_t reserved0;
    double rho;             /* reference density */
    double nu_k;            /* kinematic viscosity */
    double g;               /* gravity magnitude, acting along -z */
    double dt;              /* time step */
    double d0;              /* projected particle spacing; V0 = d0^dim */
    double l_over_d0;       /* smoothing length l = l_over_d0 d0 (1.2, Sec. 3.1) */
    double re_over_l;       /* effective radius r_e = re_over_l l (2.0) */
    double gamma_over_dt;   /* stabilisation gamma = gamma_over_dt dt (100, Sec. 3.3) */
    double cv_over_dt;      /* volume smoothing C_V = cv_over_dt dt (100, Sec. 4.4.2) */
    double cs;              /* Smagorinsky constant (0.2, Sec. 3.4) */
    double ds;              /* reference spacing of the wall damping (0.01 m) */
    double H, H_hat;        /* sigma map: still-water level and projected height */
    double alpha_min, alpha_max; /* sigma map clamp */
    double lam_fs_lo, lam_fs_hi; /* free-surface eigenvalue thresholds (0.2, 0.75) */
    double krylov_rtol;     /* relative residual of the pressure solve */
    int32_t krylov_max_iter;
    int32_t smagorinsky;    /* 1: eddy viscosity on (Sec. 3.4) */
    int32_t precision;      /* vct_precision */
    int32_t volume_mode;    /* 0: Eq. VCT_ppe; 1: Eq. VCT_ppe_w0 (Jbar = J^0); 2: Eq. VCT_ppe_w */
    double box_lo[3], box_hi[3]; /* projected-space box of the cell grid; particles
                                    outside are clamped into the border cells */
    int32_t max_neighbours; /* neighbour-list capacity per particle (0: 64 in 2-D, 160 in 3-D) */
    int32_t preconditioner; /* pressure solve: 0 plain BiCGSTAB; 1 BiCGSTAB preconditioned by an
                               aggregation multigrid V-cycle on the cell grid (Jacobi damping
                               0.85 / 0.7 on the particles and 1.0 / 0.8 on the coarse
                               levels, coarse-correction scale 1.3 / 1.2 in 2-D / 3-D,
                               z-only coarsening while the operator's z coupling dominates,
                               coarsening down to <= 64 / 4 nodes (2-D / 3-D), no sweeps on
                               the coarsest level, small levels in block 0's shared memory:
                               96 KB up to 75k particles in 2-D / 30k in 3-D, 16 KB above, where the solver
                               also stages operator rows with cp.async and gathers through
                               L1).  vct_init reads overrides from the environment:
                               VCT_MG_OMEGA, VCT_MG_KAPPA, VCT_MG_SWEEPS, VCT_MG_SMEM_KB,
                               VCT_MG_FORM (fly | explicit), VCT_MG_STAGE, VCT_GATHER_L1,
                               VCT_MG_PRESMOOTH (0: V(0,1)), VCT_MG_SHIFT (aggregation
                               2^s per axis), VCT_SOLVE_BLOCKS (grid cap), VCT_PGUESS
                               (initial guess: 0 p^N, 1 linear, 2 quadratic extrapolation
                               of the context's last pressures, the default),
                               VCT_MG_MINN (coarsest level size), VCT_MG_OMEGA_C (coarse
                               levels' damping), VCT_MG_KAPPA_C (scale
                               between coarse levels, = kappa), VCT_MG_SMALL (levels up
                               to this size coarsened by one block in the set-up),
                               VCT_INNER_FLOOR (mixed form: relative residual at which
                               each FP32 BiCGSTAB pass hands back to the FP64 residual,
                               1e-4) */
    /* Particle regularisation after the position update (Sec. 4.1 applies all
     * three; 0 switches each off).  It acts in projected space with the
     * step's neighbour lists; pair sums in FP64 (FP64 form) or compensated
     * FP32 on the hi/lo FP32 position differences (mixed form), corrections
     * applied in FP64:
     *   ds_overlap  dynamic stabilization: pairs closer than (1 - ds_overlap) d0
     *               are pushed back to that distance within the step (0.4)
     *   xsph_eps    XSPH velocity smoothing of free-surface particles (5e-3)
     *   ops_shift   optimized particle shifting, dr^ = -A l |v^| dt grad^C,
     *               tangential only at the free surface (0.2)
     * ds_overlap outside [0, 1) or a negative value is VCT_ERR_ARG. */
    double ops_shift, ds_overlap, xsph_eps;
    /* Bounded waits (failure detection): the pressure solve's persistent
     * kernels synchronise their blocks with grid barriers whose waits poll at
     * most spin_limit times (0 = the default, about 1-2 s).  A wait that runs
     * out records VCT_ERR_TIMEOUT, every block leaves at its next barrier, the
     * call returns VCT_ERR_TIMEOUT and the caller's state is left as it was.
     * Negative is VCT_ERR_ARG. */
    int64_t spin_limit;
    /* Operator set (Table tab:case_names): 0 = ISPH(2): SPH(2) second derivatives
     * (Eq. sec_SPH2) in the viscous term and the pressure equation, first-order
     * corrected pressure gradient (Eq. gra_1st); 1 = ISPH: 0th-order second
     * derivatives of Espanol & Revenga (Eq. sec_0th), summation pressure
     * gradient (Eq. gra_sum).  Velocity divergence first-order in both.
     * sph2_derivatives returns the set's second derivatives.  The backward
     * entries differentiate the ISPH(2) set only.  Other values: VCT_ERR_ARG. */
    int32_t operators;
    /* Wall condition for the velocity (Sec. 3.5): 0 = no-slip, wall particles at
     * rest; 1 = free-slip, a wall particle carries (I - 2 n n) v_wall with
     * v_wall the SPH interpolation of its fluid neighbours' velocity and n the
     * outer unit normal in physical space (J^T of the projected normal, which
     * points to the virtual particles outside).  Other values: VCT_ERR_ARG. */
    int32_t wall_slip;
    /* Schedule knobs (chosen per scenario size by the autotuner of the Python
     * package; 0 = the built-in defaults).  They change how the step runs, not
     * what it computes (the same neighbour sets, the same system, the same
     * solution to the solver tolerance):
     *   cell_over_re  edge of the background cells over r_e (>= 1; neighbour
     *                 search visits the 3^dim adjacent cells; the multigrid's
     *                 first coarse level is the cells)
     *   mg_omega      Jacobi damping of the multigrid smoother on the particles
     *   mg_kappa      scale of the coarse-grid correction
     *   solve_form    1: small-system form (V-cycle inputs formed inside the
     *                 products), 2: large-system form (staged rows), 0: by size
     *   mg_cycle      large-system form's multigrid cycle: 1: V(1,1) (a fine
     *                 Jacobi step before and after the coarse correction, each
     *                 through the assembled rows), 2: V(0,1) whose fine step
     *                 reads the row-cell operator (per row, the sums of its
     *                 coefficients over the 3^dim cells around its own: 9 or
     *                 27 values instead of the row), 0: the default, 2
     * cell_over_re in (0, 1), a negative value, a solve_form other than 0-2 or
     * an mg_cycle other than 0-2 is VCT_ERR_ARG. */
    double cell_over_re, mg_omega, mg_kappa;
    int32_t solve_form;
    int32_t mg_cycle;
} vct_params;

/* Particle state, caller order, DEVICE arrays of n entries (host arrays for
 * vct_step_host).  jbar <= 0 means "set Jbar = J at the first step". */
typedef struct {
    int64_t n;
    double *x, *y, *z;      /* physical position */
    double *u, *v, *w;      /* physical velocity */
    double *p;              /* pressure */
    double *jbar;           /* smoothed Jacobian Jbar (Sec. 3.6) */
    const int32_t *type;    /* 0 fluid, 1 wall, 2 virtual */
} vct_state;

typedef struct {
    int64_t steps_done;
    int64_t krylov_iters_total;
    int32_t krylov_iters_max;
    int32_t graph_steps;    /* steps of this call replayed from a captured CUDA graph */
    double last_residual;   /* relative residual of the last pressure solve */
    int64_t ppe_rows;       /* unknowns (fluid, not free surface) of the last step */
    int64_t ppe_nnz;        /* off-diagonal coefficients of the last step's operator */
    int64_t kernel_launches;/* kernels this call launched */
    int32_t solve_form;     /* pressure solver that ran: 0 Jacobi BiCGSTAB, 1 multigrid
                             * small-system form (k_krylov_mg_fly), 2 multigrid
                             * large-system form (k_krylov_mg, or the batched solve
                             * of vct_batch_step in that form) */
    int32_t mg_cycle;       /* its cycle in the large-system form (vct_params.mg_cycle:
                             * 1 V(1,1), 2 V(0,1) through the row-cell operator); 0
                             * in the other forms */
} vct_stats;

/* Stages timed by vct_stage_times, in step order. */
typedef enum {
    VCT_STAGE_LOAD = 0, VCT_STAGE_MAP, VCT_STAGE_SORT, VCT_STAGE_NEIGHBOURS,
    VCT_STAGE_SMOOTHING, VCT_STAGE_PASS1, VCT_STAGE_PASS2, VCT_STAGE_RHS, VCT_STAGE_PRECOND,
    VCT_STAGE_KRYLOV, VCT_STAGE_CORRECTOR, VCT_STAGE_REGULARISE, VCT_STAGE_STORE, VCT_NSTAGES
} vct_stage;

/* Device buffers (caller order) that vct_step_probe fills for its single
 * step; any pointer may be NULL. */
typedef struct {
    int32_t *fs;            /* free-surface flag (1: Dirichlet p = 0) */
    double *rho_hat;        /* <rho^>_i, projected numerical density */
    double *nu;             /* nu_K + nu_E */
    double *lam_min;        /* smallest eigenvalue of B_i over all particle types */
    double *vstar;          /* predictor velocity, dim x n component-major */
    double *ppe_b;          /* right side of A p = b on unknown rows (0 elsewhere) */
    const double *x_test;   /* optional input vector, n entries */
    double *ppe_Ax;         /* A x_test on unknown rows (0 elsewhere) */
    double *jbar_used;      /* Jbar after this step's volume smoothing */
    const int32_t *fs_in;   /* optional INPUT, n entries, caller order: free-surface
                             * flags to use for fluid particles instead of those the
                             * step decides.  A flag is a threshold on a rounded
                             * eigenvalue; within rounding of the threshold two correct
                             * evaluations can differ, and parity checks pass one
                             * side's flags to the other so both solve the same
                             * system.  NULL: the step's own flags. */
    double *vwall;          /* velocity each wall particle carries in the step's sums,
                             * dim x n component-major (free-slip walls; 0 under
                             * no-slip and for other particles) */
} vct_probe;

typedef struct vct_ctx vct_ctx;

/* Create a context: validates parameters, copies the bathymetry, allocates
 * all scratch for up to `capacity` particles on the current CUDA device.
 * stream: a cudaStream_t (NULL = legacy default stream).  (Sec. 2, Sec. 3.)
 * Before anything is allocated, r_e = re_over_l * l_over_d0 * d0 must be
 * positive and finite and the box finite and ordered (else VCT_ERR_ARG), and
 * the cell grid of edge r_e over the box must hold at most 2^30 cells (else
 * VCT_ERR_CAPACITY). */
vct_status vct_init(vct_ctx **ctx, const vct_bathymetry *bathy, vct_map_kind kind,
                    double aspect_ratio, const vct_params *params, int64_t capacity,
                    void *stream);

vct_status vct_set_stream(vct_ctx *ctx, void *stream);

/* Forget the pressures of the context's previous steps (the history the
 * pressure solve's initial guess extrapolates, used when a call continues the
 * previous call's state): the next step starts its solve from the state's own
 * pressure, as a fresh context would.  A run that is replayed from a snapshot
 * (checkpointing for a reverse sweep) calls it at each snapshot, on the
 * forward run and on the replay, so that both compute the same bits.  Queued
 * on the context's stream; allocates nothing. */
vct_status vct_reset_history(vct_ctx *ctx);

/* Neighbour sets S_i = { j != i : |r^_j - r^_i| < r_e } in projected space
 * (Eq. SPH_neighbor_set), squared distance summed in coordinate order without
 * FMA.  Writes CSR over caller indices: row_ptr (n+1 int64, device) and col
 * (device, capacity col_cap) with each row sorted by ascending index; either
 * may be NULL to get only *nnz (host).  VCT_ERR_CAPACITY if col_cap < nnz. */
vct_status vct_build_neighbours(vct_ctx *ctx, const vct_state *state, int64_t *row_ptr,
                                int32_t *col, int64_t col_cap, int64_t *nnz);

/* Allocation-free variant of vct_build_neighbours (the paper has no counterpart:
 * this serves callers that cannot allocate device memory when they need the
 * lists -- an application whose device memory is all handed to its own pool, or
 * a loop that cannot afford cudaMalloc/cudaFree -- and so cannot own a vct_ctx).
 * It takes the map and parameters directly (only dim, d0, l_over_d0, re_over_l,
 * H, H_hat, alpha_min/max and the box are read), the DEVICE state arrays
 * x, (y), z of n particles, and writes the same CSR as vct_build_neighbours:
 * row_ptr (n+1 int64, device, required) and col (device, capacity col_cap,
 * may be NULL to get only *nnz, host).  It allocates nothing: its scratch is a
 * static device array of about 1 MB, held by every GPU that loads the library,
 * which limits it to n <= 16384 particles and a cell grid of at most 32768 cells
 * (VCT_ERR_CAPACITY beyond either, also if col_cap < nnz).  The first call on a
 * device looks up that array's device address (once per device); make that
 * first call before any stream capture.  Work runs on `stream` (a
 * cudaStream_t) and the call synchronises it once.  All calls on a device share
 * the array: calls that overlap on the GPU race and must not be issued.  The
 * cached address assumes the device's primary context is not reset
 * (cudaDeviceReset) between calls.  The radius and box are checked before any
 * work: VCT_ERR_ARG for r_e not positive and finite or a box that is not
 * finite and ordered, VCT_ERR_CAPACITY for a cell grid beyond the limit.  An
 * error the calling thread left pending from earlier CUDA work is neither
 * cleared nor reported as this call's. */
vct_status vct_build_neighbours_noalloc(const vct_bathymetry *bathy, vct_map_kind kind,
                                        double aspect_ratio, const vct_params *params,
                                        const vct_state *state, int64_t *row_ptr, int32_t *col,
                                        int64_t col_cap, int64_t *nnz, void *stream);

/* SPH(2) derivatives of ncomp fields phi (ncomp x n, component-major, all
 * particle types; wall values enter the sums) at the fluid particles:
 *   grad_hat[(c*dim + K)*n + i] = <d phi_c / d x^_K>^(1)           (Eq. gra_1st)
 *   d2_hat[(c*m + a)*n + i]     second projected derivatives, m = 3 in 2-D
 *                               [xx, zz, xz], m = 6 in 3-D [xx, yy, zz, xy, yz, zx]
 *                               (Eq. sec_SPH2, cross derivatives not doubled)
 *   lap_phys[c*n + i]           c_trans . D^ phi, the physical Laplacian (Eq. lap_VCT)
 * Non-fluid entries are 0.  Any output may be NULL.  Sums run over fluid and
 * wall neighbours (virtual particles excluded), in the context's precision. */
vct_status sph2_derivatives(vct_ctx *ctx, const vct_state *state, const double *phi,
                            int32_t ncomp, double *grad_hat, double *d2_hat, double *lap_phys);

/* Adjoint of sph2_derivatives with respect to the fields (same state, same
 * layouts): given the adjoints of the outputs grad_hat_bar (ncomp x dim x n),
 * d2_hat_bar (ncomp x m x n), lap_phys_bar (ncomp x n) -- any may be NULL for
 * zero -- writes phi_bar (ncomp x n) = J^T (output adjoints), J the Jacobian of
 * the linear map phi -> (grad_hat, d2_hat, lap_phys) at the current positions.
 * Transpose of the SPH(2) operator (Eq. sec_SPH2) including the adjoint of the
 * per-particle solve with M_i^T; computed as a gather over the symmetric
 * neighbour relation, deterministic.  Virtual particles get 0. */
vct_status sph2_derivatives_backward(vct_ctx *ctx, const vct_state *state, int32_t ncomp,
                                     const double *grad_hat_bar, const double *d2_hat_bar,
                                     const double *lap_phys_bar, double *phi_bar);

/* Derivative of the corrected gradient of sph2_derivatives (grad_hat =
 * L_i sum_j V_j (phi_j - phi_i) grad w_ij, Eq. gra_1st) with respect to the
 * projected particle positions, through the kernel's first and second
 * derivatives, for the current state with its neighbour sets and particle
 * volumes held fixed: given grad_hat_bar (ncomp x dim x n, caller order) and
 * the fields phi (ncomp x n), writes xh_bar (dim x n, caller order) = the
 * gradient of sum grad_hat_bar . grad_hat with respect to r^ (x, [y], z^).
 * ncomp 1..3.  FP64; a gather over the symmetric neighbour relation,
 * deterministic; virtual particles get 0.  Overwrites the context's pass-1
 * scratch (rebuilt by the next step). */
vct_status sph2_gradient_backward_positions(vct_ctx *ctx, const vct_state *state,
                                            const double *phi, int32_t ncomp,
                                            const double *grad_hat_bar, double *xh_bar);

/* Derivative of the SPH(2) second derivatives of sph2_derivatives (d2_hat, from
 * D = 2 M_i^-1 b_i, Eq. sec_SPH2, cross terms halved) with respect to the
 * projected particle positions, through the kernel's first and second
 * derivatives, the corrected gradient, C_i, F_ij, q_ij and p_ij, for the current
 * state with its neighbour sets and particle volumes held fixed: given one field
 * phi (n, caller order) and d2_hat_bar (m x n, caller order; m = 3 / 6), writes
 * xh_bar (dim x n, caller order) = the gradient of sum d2_hat_bar . d2_hat with
 * respect to r^.  FP64; deterministic; virtual particles get 0.  Keeps its
 * per-particle factors (2 d^2 + 2 d m + 2 d + 2 m doubles) in the context's
 * pressure-coefficient storage: VCT_ERR_CAPACITY if max_neighbours leaves too
 * few slots there; the next step rebuilds that storage. */
vct_status sph2_d2_backward_positions(vct_ctx *ctx, const vct_state *state, const double *phi,
                                      const double *d2_hat_bar, double *xh_bar);

/* Derivative of the pressure operator's linear part (Eqs. VCT_ppe, lap_VCT:
 * (A x)_i = c0_i <dx/dz^>_i + c~_i . D_i on the unknown rows, D the SPH(2)
 * second derivatives of x; x = 0 on free-surface particles, wall neighbours in
 * the right side) with respect to the projected positions of the current
 * state: given x and pbar (n, caller order; entries off the unknown rows are
 * ignored), writes xh_bar (dim x n) = the gradient of pbar . (A x) with respect
 * to r^, through the same chain as sph2_d2_backward_positions, with neighbour
 * sets, free-surface flags, volumes and the metric terms c0, c~ held fixed
 * (exact for maps with a constant metric).  With vct_ppe_adjoint's b_bar as
 * pbar and the solution p as x it is the pressure solve's position term
 * -b_bar^T (dA/dr^) p with the sign reversed.  FP64; the same scratch rule and
 * VCT_ERR_CAPACITY as sph2_d2_backward_positions. */
vct_status vct_ppe_backward_positions(vct_ctx *ctx, const vct_state *state, const double *x,
                                      const double *p_bar, double *xh_bar);

/* Derivative of the density estimate rho^_i = rho sum_j V0 w_ij (self term
 * included; every neighbour type; the <rho^> of the pressure equation's
 * stabilisation term) with respect to the projected positions of the current
 * state, neighbour sets fixed: given rho_bar (n, caller order; used on fluid
 * particles), writes xh_bar (dim x n, caller order) = the gradient of
 * sum_i rho_bar_i rho^_i with respect to r^.  FP64; deterministic. */
vct_status vct_rho_backward_positions(vct_ctx *ctx, const vct_state *state, const double *rho_bar,
                                      double *xh_bar);

/* Derivative through the map with respect to the bathymetry parameters
 * theta = [h0, slope_x, slope_y, cos_amp, cos_len, amp[G], cx[G], cy[G], width[G]]
 * (G = n_gauss; 5 + 4G entries): given per-particle adjoints (DEVICE arrays of n,
 * caller order, any may be NULL for zero) of the projected height z^ =
 * alpha (z + beta), J = alpha, the Jacobian column s_x, s_y and the c_trans
 * entries c0 and c3 (Sec. 2, Eqs. VCT, jacobi, lap_VCT), writes theta_bar (HOST,
 * 5 + 4G doubles) = sum_i sum_q mbar_q,i dm_q,i / dtheta at the state's
 * physical positions.  Exact derivatives (forward-mode dual arithmetic, one
 * parameter per pass), summed over particles in a fixed order.  The sigma
 * clamp is respected: where alpha is clamped its derivatives are zero. */
vct_status vct_map_backward(vct_ctx *ctx, const vct_state *state, const double *zh_bar,
                            const double *J_bar, const double *sx_bar, const double *sy_bar,
                            const double *c0_bar, const double *c3_bar, double *theta_bar);

/* Derivative through the map with respect to the particles' physical positions
 * (the metric under moving particles): given the same per-particle adjoints as
 * vct_map_backward (DEVICE arrays of n, caller order, any may be NULL for
 * zero) of z^, J, s_x, s_y, c0 and c3, writes pos_bar (DEVICE, dim x n,
 * component-major: x, z in 2-D; x, y, z in 3-D) with
 * pos_bar[k*n + i] = sum_q mbar_q,i dm_q,i / dx_k,i -- each particle's metric
 * depends on its own position only (Sec. 2: alpha, beta and their derivatives
 * at (x, y); z^ = alpha (z + beta)).  The identity parts x^ = x, y^ = y of the
 * projected position are not included.  Exact derivatives (forward-mode dual
 * arithmetic, one coordinate per pass; third derivatives of the bathymetry
 * enter through c0); where the sigma clamp holds alpha its derivatives are 0.
 * FP64, deterministic. */
vct_status vct_map_backward_positions(vct_ctx *ctx, const vct_state *state, const double *zh_bar,
                                      const double *J_bar, const double *sx_bar,
                                      const double *sy_bar, const double *c0_bar,
                                      const double *c3_bar, double *pos_bar);

/* Water level at wave gauges and the squared-level loss of the adjoint workload
 * (the paper's experiments record water levels at fixed gauges, Sec. 4.4.2).
 * At gauge g, eta_g = sum_i w_ig z_i / sum_i w_ig - H over the free-surface
 * fluid particles (fs[i] == 1; fs DEVICE int32, caller order, e.g. the flags
 * vct_step_probe exports; they are held fixed), w_ig = the cubic spline shape
 * of the horizontal distance to the gauge over l (support 2 l); eta_g = 0 if no
 * surface particle lies within 2 l.  gauges (HOST): n_gauges x positions in
 * 2-D, n_gauges (x, y) pairs in 3-D; 1 <= n_gauges <= 16.  Writes loss (HOST)
 * = sum_g eta_g^2, eta (HOST, n_gauges, may be NULL) and pos_bar (DEVICE,
 * dim x n component-major: x, z in 2-D; x, y, z in 3-D; may be NULL) = the
 * loss's gradient with respect to the physical positions.  FP64; sums in a
 * fixed order.  VCT_ERR_ARG for a bad count or non-finite gauge position. */
vct_status vct_gauge_loss(vct_ctx *ctx, const vct_state *state, const int32_t *fs, int32_t n_gauges,
                          const double *gauges, double *loss, double *eta, double *pos_bar);

/* Advance the state by nsteps steps of Sec. 3.3 with the VCT equations:
 * map + cell sort, neighbours, Jbar smoothing (sigma, volume_mode 2),
 * corrected gradients, free surface, eddy viscosity, SPH(2) predictor,
 * pressure equation with wall Neumann extrapolation (Eq. PNC), BiCGSTAB,
 * corrector and position update, then the particle regularisation of
 * vct_params when on.  Device arrays, updated in place on success; on an
 * error the state is left as it was and the steps after the failing one do
 * no work.  out (host, may be NULL) receives solve statistics.  The steps
 * are replayed from CUDA graphs, one step each, captured on the first call for
 * each particle count and sorted-buffer parity and kept by the context; they
 * run on a stream the context creates for them, ordered after the load and
 * before the write-back on the context's stream, with results identical to
 * direct launches.  Not with stage profiling on, nor with the environment
 * variable VCT_STEP_NOGRAPH set; if a capture fails, the context launches
 * directly from then on; stats.graph_steps counts the replayed steps. */
vct_status vct_step(vct_ctx *ctx, vct_state *state, int32_t nsteps, vct_stats *out);

/* Adjoint of the pressure solve of the context's last step (Sec. 3.3, Eqs.
 * VCT_ppe and PNC give the system A p = b on the unknown rows, the fluid
 * particles off the free surface).  For p = A^-1 b and a gradient p_bar of a
 * loss with respect to p, writes b_bar = A^-T p_bar, the gradient with respect
 * to b; the gradient with respect to A's coefficients is then -b_bar p^T on A's
 * pattern.  The operator is the one the forward solve used (FP32 coefficients
 * in the mixed form).  A's pattern is symmetric, so A^T is formed in place of A
 * (each pair of coefficients swapped) and solved by the context's own solver
 * (its form for A, with a multigrid hierarchy built for A^T), then A is
 * restored; without multigrid, or if that solve does not converge, the call
 * solves again by Jacobi-preconditioned BiCGSTAB in FP64 on A^T's products; to
 * the context's krylov_rtol relative to |p_bar|, at most krylov_max_iter
 * iterations per attempt (VCT_ERR_NOCONV otherwise).
 * p_bar, b_bar: device arrays of n doubles in caller order, n the particle
 * count of that step; entries of rows that are not unknowns are ignored in
 * p_bar and written as 0 in b_bar.  Returns VCT_ERR_ARG if the context holds
 * no pressure system (no step yet, or a call since then that sorted the
 * particles again: vct_build_neighbours, sph2_derivatives).  Overwrites the
 * context's neighbour lists, solver vectors and multigrid hierarchy, which the
 * next step rebuilds.  out (host, may be NULL) receives the iteration count and
 * residual. */
vct_status vct_ppe_adjoint(vct_ctx *ctx, const double *p_bar, double *b_bar, vct_stats *out);

/* Reverse of one time step with respect to the fluid velocities (Sec. 3.3:
 * predictor Eq. VCT_predictor with the viscous term of Eq. lap_VCT, the
 * pressure equation Eqs. VCT_ppe and PNC, corrector and update Eq. VCT_update),
 * with the positions held at the start of the step.  At fixed positions and
 * without the eddy viscosity the step is affine in the velocities v^N
 * (neighbour sets, free-surface flags, volumes, metric, moment matrices and
 * the pressure operator all follow from the positions), so the result is the
 * exact gradient, to the transposed solve's tolerance, of the loss
 *   l = v_bar . v^(N+1) + x_bar . x^(N+1) + p_bar . p^(N+1)
 * with respect to v^N; the positions' own gradient (x^(N+1) = x^N + dt v^(N+1)
 * passes x_bar on, the geometry's dependence on x^N) is not part of it.
 * state: device SoA in caller order at the start of the step (read only; the
 * step is not advanced).  With the Smagorinsky model (Sec. 3.4) the step is not
 * affine in v (nu_E grows with the strain rate): the result is then the
 * gradient at v^N (the chain through nu_E, its gradient term and the eddy
 * viscosity's Laplacian factor; nu_E is not differentiable where the strain
 * rate vanishes, and its share is taken as 0 there).
 * v_bar, x_bar: device, dim x n doubles, component-major
 * (u, [v], w / x, [y], z), caller order; p_bar: device, n doubles; each may be
 * NULL (zero); entries of non-fluid particles are ignored, and p_bar's off the
 * unknown rows (the fluid particles off the free surface).  v_bar_in: device,
 * dim x n doubles, written with dl/dv^N (0 for non-fluid particles).  Runs the
 * step's assembly at the state's positions (map, sort, neighbours, smoothing,
 * pass 1, pass 2, right side, multigrid setup), then the corrector's adjoint,
 * the transposed pressure solve (as vct_ppe_adjoint: out receives its
 * iteration count and residual), the right side's and the wall terms'
 * adjoints, the SPH(2) derivative operator's adjoint for the viscous term, and
 * with free-slip walls (Sec. 3.5) the adjoint of the wall particles' reflected
 * Shepard velocities; under the ISPH operator set (vct_params.operators = 1)
 * the adjoints of its summation pressure gradient and 0th-order second
 * derivatives; with the particle regularisation on (Sec. 4.1: dynamic
 * stabilization, XSPH, optimized shifting, all acting on the corrector's
 * positions x' and velocities u'), its reverse first: the call then runs the
 * step forward up to and through the regularisation (solve, corrector), takes
 * the regularisation's reverse at x', u' (its pair terms' position derivatives
 * through w' and w'', the metric at x' through duals), and clears the context's
 * pressure history (as vct_reset_history), which that forward run wrote.  The
 * dynamic stabilization switches on below a pair distance and the shift
 * scales with |v|: the gradient is that of the branch the step took.  FP64
 * arithmetic in the reverse; the operators in the context's precision.
 * VCT_ERR_ARG if v_bar_in is NULL.
 * Allocates (7 dim + 3 dim^2 + 3) doubles per particle of capacity on the
 * first call (with the regularisation on, (10 dim + dim^2 + 13) more);
 * afterwards the context holds this step's pressure system (as after
 * vct_step, for vct_ppe_adjoint). */
vct_status vct_step_backward_velocity(vct_ctx *ctx, const vct_state *state, const double *v_bar,
                                      const double *x_bar, const double *p_bar, double *v_bar_in,
                                      vct_stats *out);

/* Ensemble: advance n_scen independent scenarios (one context and one device
 * state each, uneven particle counts allowed) by nsteps steps in one call,
 * with no host synchronisation until the end, where each scenario's status is
 * read once.  When every scenario uses the multigrid solver with the same
 * dimension and precision, the scenarios run side by side (to the solver the
 * batch counts as one system: above 75k particles in total in 2-D, 30k in 3-D,
 * or with any large scenario, every solve uses the large-system form): each
 * stage of the step is ONE launch over all scenarios (every scenario on the
 * blocks its own launch of the stage would take, with its own parameters and
 * buffers), and one cooperative launch solves all pressure systems at once,
 * each on a share of the grid in proportion to its particles, all on a
 * stream the FIRST context keeps for it (each scenario's load and store run
 * on a stream of its own, created on first use and kept by its context).
 * Every stage runs the same device code as the scenario's own launch of it
 * (compiled into another kernel, so multiply-add fusion may differ in the last
 * bit); results agree with vct_step to the solver tolerance (the solves'
 * partial sums are grouped differently), and repeat bit for bit.
 * The batch's launches are counted in the first scenario's
 * stats.kernel_launches (the others count their load and store).  In this
 * form, steps run in pairs from a CUDA graph: the first call for a batch
 * captures two steps and instantiates them once; that call's and later
 * calls' pairs (same contexts, particle counts and buffer parity) are one
 * graph launch each, an odd last step runs from direct launches.  A changed
 * batch is captured anew (the first context keeps one graph).  Not with
 * stage profiling on (the first context's stage times are then the batch's),
 * nor with the environment variable VCT_BATCH_NOGRAPH set; if a capture
 * fails, the first context uses direct launches from then on.  Graph and
 * direct launches give identical results; stats.graph_steps counts the
 * replayed steps.
 * Otherwise, or with the environment variable VCT_BATCH_SERIAL set, all
 * kernels are queued back to back on the first context's stream and each
 * result is bit-identical to vct_step on its own.  The call returns when all
 * work is done.  out (host, may be NULL) receives n_scen stats.  Returns the
 * first failing status; scenarios that failed keep their state, the others
 * are written back. */
vct_status vct_batch_step(vct_ctx *const *ctxs, vct_state *const *states, int32_t n_scen,
                          int32_t nsteps, vct_stats *out);

/* Same as vct_step with HOST arrays: copies in, steps, copies back. */
vct_status vct_step_host(vct_ctx *ctx, vct_state *host_state, int32_t nsteps, vct_stats *out);

/* One step like vct_step that also writes the intermediate fields named in
 * probe (device buffers, caller order). */
vct_status vct_step_probe(vct_ctx *ctx, vct_state *state, const vct_probe *probe,
                          vct_stats *out);

/* Profiling: when on, every stage of every step (up to 512 steps per call) is
 * bracketed by CUDA events on the context's stream; vct_stage_times adds the
 * elapsed device milliseconds per stage and the number of bracketed launches
 * (host arrays of VCT_NSTAGES).  Turning profiling on resets the totals.  Off
 * by default; when off no event is recorded.  In vct_batch_step side by side,
 * the first context's stage times are those of the batched launches of all
 * scenarios (on its batch stream), and no step is replayed from the graph. */
vct_status vct_set_profiling(vct_ctx *ctx, int32_t on);
vct_status vct_stage_times(vct_ctx *ctx, double *ms, int64_t *launches);

/* First failing particle of the last error (caller index, -1 if none). */
vct_status vct_last_error(vct_ctx *ctx, int64_t *particle);

const char *vct_strerror(vct_status status);

void vct_destroy(vct_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VCT_H */
