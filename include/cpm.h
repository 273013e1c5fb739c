/*
 * cpm.h -- C ABI of the GB300 (sm_103a) closest-point multigrid library.
 *
 * Solves the shifted surface Poisson equation (c - Lap_S) u = f on a closed
 * curve or surface S (Chen & Macdonald, "The Closest Point Method and
 * multigrid solvers for elliptic equations on surfaces", Sec. 2.1, Eq. 2.1)
 * by the closest point method on a narrow band of a uniform Cartesian grid.
 *
 * The discrete system (Sec. 2.3 Eq. 2.10, Sec. 3.1, Remark 3.2) is
 *
 *     A u = f,   A = diag(c) - M,   M = diag(L) + (L - diag L) E,
 *
 * where L is the 2d+1-point Laplacian and E the degree-3 tensor-product
 * barycentric Lagrange interpolation at each grid node's closest point
 * (Sec. 3.1, Eq. 3.1).  The solver is the closest-point V-cycle of
 * Algorithm 4.1 (Sec. 4) with weighted Jacobi smoothing (Eq. 4.1, Sec. 4.4),
 * closest-point restriction and prolongation (Sec. 4.3) and a direct solve on
 * the coarsest level, inside an outer defect-correction loop.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Status codes only; nothing throws across the ABI.  cpm_last_error()
 *   returns a message for the last failing call of the calling thread.
 * - Vectors are caller-owned DEVICE pointers of the stated length, in the
 *   library's band order (bricks of 4x4x4 grid nodes in Morton order, nodes
 *   inside a brick x-fastest); cpm_band_export gives the grid coordinates
 *   of that order.  FP64 vectors are double*, FP32 vectors float*.
 * - Handles own every device allocation they make; *_destroy frees them.
 * - Calls are asynchronous on the given stream unless stated otherwise.
 *   Passing 0 selects the legacy default stream.
 * - Handles are not thread safe: one thread (or stream) at a time per handle.
 */
#ifndef CPM_H
#define CPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cpm_stream; /* a cudaStream_t */

typedef enum cpm_status {
  CPM_OK = 0,
  CPM_ERR_ARG = 1,          /* invalid argument, size or descriptor          */
  CPM_ERR_OOM = 2,          /* device allocation failed                       */
  CPM_ERR_CUDA = 3,         /* a CUDA runtime call failed                     */
  CPM_ERR_REACH = 4,        /* band too wide for the surface: cp undefined on
                               the ghost ring, or a stencil leaves the band  */
  CPM_ERR_DIVERGED = 5,     /* residual grew 1e3x or became non-finite        */
  CPM_ERR_NOT_CONVERGED = 6,/* max_iter reached above tolerance               */
  CPM_ERR_TIMEOUT = 7,      /* a bounded device wait gave up                  */
  CPM_ERR_CHECKED = 8,      /* a device-side bounds / consistency check failed */
  CPM_ERR_SINGULAR = 9      /* coarsest-level matrix is singular              */
} cpm_status;

const char* cpm_status_str(cpm_status s);
/* Message of the calling thread's last failing call ("" if none). */
const char* cpm_last_error(void);

/* ---------------------------------------------------------------- geometry */

typedef enum cpm_surface_kind {
  CPM_CIRCLE = 0,    /* d = 2, param[0] = radius R (centre at the origin)     */
  CPM_SPHERE = 1,    /* d = 3, param[0] = radius R                             */
  CPM_TORUS = 2,     /* d = 3, about the z axis: param[0] = R, param[1] = r    */
  CPM_ELLIPSOID = 3, /* d = 3, semi-axes param[0..2]                           */
  CPM_DZIUK = 4      /* d = 3, the level set (x1 - x3^2)^2 + x2^2 + x3^2 = 1 of
                        Sec. 4.5.5; cp by Newton's method on the Lagrange
                        conditions (30 steps from the node); reach 0.0957, so
                        bands need dx <= 1/64 on the [-2, 2] grid           */
} cpm_surface_kind;

/* A closed surface with a closed-form or Newton closest point (Sec. 2.1). */
typedef struct cpm_surface {
  int32_t kind;      /* cpm_surface_kind */
  int32_t pad_;
  double param[8];
} cpm_surface;

/* Uniform grid x_i = lo + i dx, i = 0..n-1 on every axis (Sec. 3.1).
 * n = 0 selects n = round(-2 lo / dx) + 1 (a grid symmetric about 0).
 * lambda2 = 0 selects the tube radius^2 / dx^2 that makes the band contain
 * every interpolation stencil and its difference stencils:
 * (d-1)(p+1)^2/4 + (1+(p+1)/2)^2 with p = 3 (13 for d = 2, 17 for d = 3). */
typedef struct cpm_grid {
  double lo;
  double dx;
  int64_t n;
  double lambda2;
} cpm_grid;

/* ---------------------------------------------------------------- band */

typedef struct cpm_band_s* cpm_band;

/*
 * Build the band B = {x : |x - cp(x)|^2 <= lambda2 dx^2} (Sec. 3.1, the tube
 * whose sizes match Table 4.1), its ghost ring G (Laplacian neighbours of B
 * outside B) and the cubic stencil records of B+ = B with G, on the device.
 * Membership is decided in FP64 with a fixed operation order (no fused
 * multiply-add), so it is reproducible bit for bit.
 * Errors: CPM_ERR_ARG for dx <= 0, an unknown kind or non-positive radii;
 * CPM_ERR_REACH if cp is undefined on B+ or a stencil leaves B.
 * Synchronous (returns after the band is built).
 */
cpm_status cpm_build_band(const cpm_surface* surface, const cpm_grid* grid,
                          cpm_stream stream, cpm_band* out);

/* |B| and |G|.  Synchronous, host outputs. */
cpm_status cpm_band_info(cpm_band band, int64_t* n_band, int64_t* n_ghost);

/*
 * Copy out, for the n_band + n_ghost points of B+ in band order (B first,
 * then G): grid coordinates ijk (int32 x d per point, may be NULL), closest
 * points cp (double x d per point, may be NULL) and cubic stencil base nodes
 * (int32 x d per point: floor((cp - lo)/dx) - 1, may be NULL).
 * All outputs are HOST pointers.  Synchronous.
 */
cpm_status cpm_band_export(cpm_band band, int32_t* ijk, double* cp, int32_t* stencil_base);

/*
 * The sizes Table 4.1 reports for a band, counted on the device: counts[0] =
 * |B|, counts[1] = nnz(L) of the 2d+1-point Laplacian restricted to B
 * (out-of-band neighbours dropped), counts[2] = nnz(E_3) = |B| 4^d, counts[3]
 * = nnz(M) of M = E_1 L - gamma (I - E_3) (Eq. 3.3): the cubic stencil pattern
 * plus one diagonal entry for every node outside its own stencil.  counts:
 * HOST array of 4 int64.  Synchronous.
 */
cpm_status cpm_band_counts(cpm_band band, int64_t* counts, cpm_stream stream);

cpm_status cpm_band_destroy(cpm_band band);

/* ---------------------------------------------------------------- hierarchy */

typedef enum cpm_smoother {
  CPM_SMOOTH_JACOBI = 0, /* weighted Jacobi on A (Eq. 4.1, Sec. 4.4)            */
  CPM_SMOOTH_RM = 1,     /* Ruuth-Merriman: Jacobi on cI - L, then u := E u
                            (Eq. 4.2, Sec. 4.2)                                 */
  CPM_SMOOTH_RBGS = 2    /* Gauss-Seidel on A in red-black order (the
                            alternative named in Sec. 4.4): the weighted Jacobi
                            update of the red nodes (even i+j+k), then that of
                            the black nodes from a fresh extension.  The
                            interpolation stencils couple nodes of one colour,
                            so this is not an exact Gauss-Seidel sweep; on the
                            closest-point operators it does not make the
                            defect correction converge (measured contraction
                            above 0.5 per cycle, often above 1)               */
} cpm_smoother;

typedef enum cpm_prec { CPM_F64 = 0, CPM_F32 = 1 } cpm_prec;

typedef struct cpm_mg_opts {
  double coarsest_dx;   /* spacing of the coarsest level.  0: coarsen while
                           (sqrt(lambda2)+1)*dx < reach and |B| > 64, so that cp
                           is unique on B+ of every level; then, only while the
                           coarsest level is larger than coarse_dense_max, add
                           levels whose band half-width sqrt(lambda2)*dx stays
                           below the reach and whose band builds (cp defined on
                           B+, every stencil inside the band).  > 0: levels
                           down to that spacing, each with
                           sqrt(lambda2)*dx < reach (CPM_ERR_REACH otherwise)  */
  int32_t nu1, nu2;     /* pre / post smoothing sweeps (0: 3 and 3)             */
  double omega;         /* Jacobi weight (0: 0.8)                               */
  int32_t smoother;     /* cpm_smoother                                         */
  int32_t transfer_deg; /* restriction / prolongation interpolation degree:
                           1 (linear, Sec. 4.5) or 3 (cubic) (0: 1)            */
  double c;             /* constant shift c > 0 (used when c_device is NULL)    */
  const double* c_device; /* optional per-point c on the finest band (device,
                             length n_band); coarse levels take c(cp) by
                             linear interpolation from the finest band          */
  int32_t residual_mode;  /* residual restricted by the Jacobi V-cycle:
                             0: f - A (E u) (Sec. 4.4), 1: f - A u              */
  int32_t coarse_sweeps;  /* coarsest level: 0 = direct solve by an explicit
                             inverse, FP64 (Gauss-Jordan) up to coarse_f64_max
                             points (FP32 V-cycles multiply by its FP32
                             rounding when it has at most 8192), FP32
                             (library LU at setup, two FP64
                             refinement steps in FP64 V-cycles) up to
                             coarse_dense_max, else restarted GMRES(30)
                             (coarse_gmres restarts);
                             > 0 = that many Jacobi sweeps                      */
  int32_t coarse_f64_max;   /* 0: 16384 (the FP64 inverse costs 8 n^2 bytes)   */
  int32_t coarse_dense_max; /* 0: 40000 (the FP32 inverse costs 4 n^2 bytes);
                               at most 65536                                    */
  int32_t op_form;          /* discrete operator M on every level:
                               CPM_OP_MBR (0): diag(L) + (L - diag L) E, cubic E
                               in both terms (Eq. 2.10, Remark 3.2);
                               CPM_OP_PAPER (1): the paper's scheme
                               E_1 L_B - gamma (I - E_3) with L_B the
                               band-restricted Laplacian (Sec. 3.1 Eq. 3.3,
                               Theorem 3.3);
                               CPM_OP_VARDIFF (2): variable diffusion
                               -div_S(a grad_S u) + c u = f (Sec. 4.5.6):
                               E_1 L~ - diag(gamma a)(I - E_3) with
                               L~ = sum over axes of D^b diag(A^f a) D^f on B
                               and a from a_device (smoothing on A only)       */
  int32_t cycle;            /* coarse-grid corrections per level: 1 V-cycle
                               (Algorithm 4.1), 2 W-cycle (the remark at
                               Algorithm 4.1; the second from the first's
                               result) (0: 1)                                   */
  const double* a_device;   /* CPM_OP_VARDIFF: the diffusion coefficient a(cp(x))
                               > 0 on the finest band (device, length n_band);
                               coarse levels take its restriction, like c      */
  int32_t relative;         /* CPM_OP_MBR, Jacobi: 1 = the V-cycles evaluate
                               their residuals and Jacobi updates in the
                               relative form of cpm_residual (extension of
                               u - u_ref per tile, differences formed from
                               exact inputs), which lowers the FP32 rounding
                               floor of the FP32 V-cycle; 0 = the direct form  */
  int32_t coarse_gmres;     /* restarts of the GMRES(30) coarsest solve used
                               above coarse_dense_max (0: 3): right-
                               preconditioned by omega / diag(A), classical
                               Gram-Schmidt twice, fixed step counts, all on
                               the device                                      */
  int32_t ext_variant;      /* FP32 extension work decomposition of every level
                               (see cpm_hier_ext_tuning): 0 = chosen per level
                               by timing when the hierarchy is built; 1, 2, 3 =
                               variant 0, 1, 2 everywhere                       */
  int32_t outer_f64;        /* CPM_OP_MBR: arithmetic of the outer residual
                               (cpm_residual, cpm_solve, cpm_solve_batch):
                               0 = FP32 pairs (about 48 significand bits, see
                               cpm_residual), 1 = FP64.  Other forms: ignored
                               (their residual is FP64, direct form)            */
} cpm_mg_opts;

typedef enum cpm_op_form { CPM_OP_MBR = 0, CPM_OP_PAPER = 1, CPM_OP_VARDIFF = 2 } cpm_op_form;

typedef struct cpm_hier_s* cpm_hier;

/*
 * Build levels dx, 2dx, .., coarsest_dx (each with its own band, Sec. 4.3),
 * the restriction and prolongation records, diag(A) on every level and the
 * inverse of the coarsest-level matrix (FP64, for the direct solve of
 * Algorithm 4.1 step 2).  The finest band is copied; `finest` may be
 * destroyed afterwards.  Synchronous.
 * Errors: CPM_ERR_ARG (bad options), CPM_ERR_REACH, CPM_ERR_SINGULAR.
 */
cpm_status cpm_build_hierarchy(cpm_band finest, const cpm_mg_opts* opts,
                               cpm_stream stream, cpm_hier* out);

/* Number of levels and |B| of level l (host outputs, synchronous). */
cpm_status cpm_hier_info(cpm_hier h, int32_t* n_levels, int32_t level, int64_t* n_band);

/*
 * The work decomposition of level `level`'s FP32 extension, chosen when the
 * hierarchy was built by timing each candidate on that level (three launches
 * over B+ after a warm-up): 0 one CTA per extension tile and one thread per
 * point, 1 persistent CTAs that stage the next tile while evaluating the
 * current one, 2 one thread per chunk of points that share a stencil base.
 * variant: host int32 (may be NULL); ms: host array of 3 doubles, the measured
 * milliseconds of each candidate (may be NULL).  No counterpart in the paper.
 */
cpm_status cpm_hier_ext_tuning(cpm_hier h, int32_t level, int32_t* variant, double* ms);

/*
 * Mu = M u on level `level` (0 = finest).  CPM_OP_MBR: w = E u on B+, then
 * (Mu)_i = sum_{k in N(i)} (w_k - w_i)/dx^2 + gamma (w_i - u_i),
 * gamma = 2d/dx^2 (Sec. 2.3 Eq. 2.10).  CPM_OP_PAPER: v = L_B u on B, w = E_3 u
 * on B, (Mu)_i = (E_1 v)_i - gamma (u_i - w_i) (Sec. 3.1 Eq. 3.3).
 * u, Mu: device vectors of length |B_level|, type per prec.
 */
cpm_status cpm_apply(cpm_hier h, int32_t level, int32_t prec, const void* u, void* Mu,
                     cpm_stream stream);

/*
 * Closest-point extension w = E u on level `level` (Sec. 3.1 Eq. 3.1 with
 * cubic tensor-product weights; the re-extension step of Eq. 4.2b): for every
 * point x_i of B (and of the ghost ring G when with_ghost != 0), w_i is the
 * degree-3 interpolant of u at cp(x_i) from the 4^d stencil nodes (all in B).
 * u: device vector of length |B_level|; w: length |B_level| (+ |G_level| when
 * with_ghost), B entries first.  Type per prec.
 */
cpm_status cpm_extend(cpm_hier h, int32_t level, int32_t prec, const void* u, void* w,
                      int32_t with_ghost, cpm_stream stream);

/*
 * `sweeps` smoothing steps of the hierarchy's smoother on level `level` for
 * A u = f, in place on u (Eq. 4.1 or Eq. 4.2).  f, u: device, |B_level|.
 */
cpm_status cpm_smooth(cpm_hier h, int32_t level, int32_t prec, const void* f, void* u,
                      int32_t sweeps, cpm_stream stream);

/*
 * One V-cycle of Algorithm 4.1 from the finest level: u := V(u, f).
 * prec = CPM_F64 runs every level in FP64; CPM_F32 runs them in FP32 with
 * the coarsest solve in FP64.  f, u: device vectors of length |B_0|.
 */
cpm_status cpm_vcycle(cpm_hier h, int32_t prec, const void* f, void* u, cpm_stream stream);

/* ------------------------------------------------------- learned smoother */

/*
 * A per-band-point network that replaces the first pre-smoothing Jacobi sweep
 * (Eq. 4.1) on the finest level of FP32 V-cycles; weighted Jacobi is its
 * fallback and judge (cpm_solve_opts.learned).  The paper has no learned
 * component.  Features of band point i (31): the residual on the 3x3x3 grid
 * neighbourhood of x_i (0 off the band) divided by its max |r| = s_i,
 * (x_i - cp(x_i))/dx (3), dx^2 M_ii (1).  Network 31 -> 64 -> 64 -> 1 with
 * ReLU, BF16 weights and features, FP32 accumulation on the tensor cores;
 * correction du_i = s_i dx^2 y_i.  Parameters: CPM_MLP_NPARAMS floats, W1
 * (32 x 64, row 31 unused), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1),
 * matrices row-major [input][output].
 */
#define CPM_MLP_NPARAMS 6337
typedef struct cpm_mlp_s* cpm_mlp;

/* Seeded random initialisation (He-scaled normal weights, zero biases). */
cpm_status cpm_mlp_create(uint64_t seed, cpm_mlp* out);
/* Copy parameters from / to HOST memory (n must be CPM_MLP_NPARAMS). */
cpm_status cpm_mlp_set_params(cpm_mlp m, const float* params, int32_t n);
cpm_status cpm_mlp_get_params(cpm_mlp m, float* params, int32_t n);
cpm_status cpm_mlp_destroy(cpm_mlp m);

/* Use m (NULL: none) as the learned smoother of the finest level of h. */
cpm_status cpm_hier_set_smoother(cpm_hier h, cpm_mlp m);

/* du = network correction for the FP32 residual r on the finest level
 * (device vectors of length |B_0|).  Needs cpm_hier_set_smoother first. */
cpm_status cpm_mlp_correction(cpm_hier h, const float* r, float* du, cpm_stream stream);

/*
 * Training loss L = ||r - A du||^2 / ||r||^2 of one FP32 residual field r on
 * the finest level of h (A applied in FP32) and its gradient with respect to
 * the parameters (analytic backward pass; A^T by a transposed neighbour
 * gather and a transposed extension scatter).  loss and grad are HOST outputs
 * (grad: CPM_MLP_NPARAMS floats, may be NULL).  Synchronous.
 */
cpm_status cpm_mlp_loss_grad(cpm_hier h, const float* r, double* loss, float* grad,
                             cpm_stream stream);

/* One Adam step (lr; beta1 0.9, beta2 0.999) on the loss above.  loss: host
 * output (may be NULL; reading it synchronises). */
cpm_status cpm_mlp_train_step(cpm_hier h, const float* r, float lr, double* loss, cpm_stream stream);

/*
 * A training set for cpm_mlp_train: n_fields residual fields, field k living
 * on the finest level of hier[k] (hierarchies may repeat).  r[k]: FP64 DEVICE
 * vector of |B_0| of hier[k] (caller-owned, read only).  Each field is scaled
 * by 1 / max_i |r_i| and cast to FP32 inside the library before training.
 */
typedef struct cpm_train_set {
  int32_t n_fields;
  const cpm_hier* hier;
  const double* const* r;
} cpm_train_set;

typedef struct cpm_train_opts {
  int32_t steps;     /* Adam steps in all (0: 400)                             */
  float lr;          /* learning rate of the first step (0: 2e-3)              */
  float lr_final;    /* learning rate of the last step; linear in between
                        (0: equal to lr, a constant rate)                      */
  int32_t reset;     /* 1: clear the Adam moments and step count first        */
} cpm_train_opts;

typedef struct cpm_train_report {
  int32_t steps;     /* Adam steps taken                                       */
  int32_t n_fields;
  double loss_first; /* mean loss over the fields before the first step       */
  double loss_last;  /* mean loss over the fields after the last step         */
  double seconds;    /* wall time of the call                                 */
} cpm_train_report;

/*
 * Train m on a set of residual fields of the method's own V-cycles (the
 * learned smoother has no counterpart in the paper).  The library scales each
 * FP64 field by 1 / max|r| into FP32, makes m the learned smoother of every
 * hierarchy in the set (as cpm_hier_set_smoother), then runs opts->steps Adam
 * steps of cpm_mlp_train_step, cycling over the fields with
 * max(1, steps / n_fields) consecutive steps per field, at a learning rate
 * falling linearly from opts->lr to opts->lr_final.  report (may be NULL):
 * mean loss over the fields before and after.  Synchronous.
 * Errors: CPM_ERR_ARG (NULL or empty set, a field of a 2-D hierarchy,
 * non-finite or zero field).
 */
cpm_status cpm_mlp_train(cpm_mlp m, const cpm_train_set* set, const cpm_train_opts* opts,
                         cpm_train_report* report, cpm_stream stream);

/*
 * Write the network (parameters, Adam moments and step count) to a file at
 * path: the 8 bytes "CPMMLP01", int32 CPM_MLP_NPARAMS, int64 step, then
 * params, m and v as CPM_MLP_NPARAMS little-endian floats each.  Synchronous.
 */
cpm_status cpm_mlp_save(cpm_mlp m, const char* path);

/* Create a network from a file written by cpm_mlp_save (CPM_ERR_ARG if the
 * file is missing, short or of another format).  Synchronous. */
cpm_status cpm_mlp_load(const char* path, cpm_mlp* out);


typedef enum cpm_solve_mode {
  CPM_SOLVE_F64 = 0,   /* FP64 V-cycles in FP64 defect correction            */
  CPM_SOLVE_MIXED = 1  /* FP32 V-cycle preconditioning an FP64 outer loop:
                          r = f - A u in FP64, d = V32(r / s), u += s d      */
} cpm_solve_mode;

typedef struct cpm_solve_opts {
  double tol;          /* stop when ||f - A u||_inf <= tol ||f||_inf (0: 1e-10) */
  int32_t max_iter;    /* outer iterations (0: 100)                           */
  int32_t mode;        /* cpm_solve_mode                                      */
  int32_t use_graph;   /* capture the V-cycle in a CUDA graph (default 1 when
                          opts is NULL; 0 = plain launches)                   */
  int32_t zero_init;   /* 1: start from u = 0 (ignore u on entry)             */
  int32_t inner_cycles;/* MIXED: FP32 V-cycles per outer iteration, each after
                          the first starting from the previous correction
                          (an FP32 inner defect correction; 0: 1)             */
  int32_t learned;     /* MIXED: 1 = use the smoother set by
                          cpm_hier_set_smoother, judged against Jacobi: the
                          first outer iteration runs plain Jacobi V-cycles and
                          gives the reference reduction factor; an iteration
                          with the network whose reduction factor exceeds
                          1.25 x the reference switches the network off for
                          the rest of the solve                             */
  int32_t fmg;         /* 1: the first outer iteration's correction is full
                          multigrid (remark at Algorithm 4.1): the residual is
                          restricted to every level, the coarsest level solved,
                          and on each finer level the prolonged coarse
                          solution starts one cycle of that level; later
                          iterations use cycles from zero.  Plain launches for
                          that iteration; not in batches                    */
} cpm_solve_opts;

#define CPM_MAX_HISTORY 256
typedef struct cpm_solve_report {
  int32_t iters;               /* outer iterations performed                  */
  int32_t converged;           /* 1 if the tolerance was reached              */
  double rel_residual;         /* final ||f - A u||_inf / ||f||_inf            */
  double history[CPM_MAX_HISTORY]; /* relative residual before each iteration  */
  double seconds;              /* wall time of the solve (host clock)         */
  int32_t learned_iters;       /* outer iterations that used the network      */
  int32_t fallback;            /* 1 if the judge switched the network off     */
  double jacobi_factor;        /* reference reduction factor (Jacobi)         */
  double learned_factor;       /* mean reduction factor with the network      */
  double learned_worst;        /* largest reduction factor with the network   */
  int32_t f64_checks;          /* outer residuals in FP32 pairs checked in FP64
                                  (see cpm_solve)                             */
  double pair_floor;           /* last estimate of the pair residual's rounding
                                  error relative to ||f||_inf (0: FP64 only)  */
} cpm_solve_report;

/*
 * Solve A u = f on the finest level.  f, u: FP64 device vectors of length
 * |B_0|; u holds the initial guess unless zero_init.  The solution accumulator
 * is FP64 in both modes; the outer residual is evaluated as cpm_residual
 * (FP32 pairs unless outer_f64).  With pairs, the residual also yields an
 * estimate of its rounding error (4 x 2^-48 max|u - u_ref| 6d / dx^2, about
 * ten times the measured error).  A pair residual that meets the tolerance
 * only within that estimate is checked pointwise: the points whose |r_i| lies
 * within the estimate of the tolerance (at most 65536; more fall back to the
 * next check) are evaluated in FP64, and the solve has converged if none
 * exceeds the tolerance (rel_residual is then their largest |r_i|).  A pair
 * residual that has reached its estimate, has stopped falling (at most halved
 * by an outer iteration) or failed the pointwise check is replaced by the
 * full FP64 evaluation of the same iterate, and if that misses the tolerance
 * the rest of the solve uses FP64 residuals.  Synchronous (reads the
 * residual norms once per outer iteration).  report may be NULL.
 * Errors: CPM_ERR_ARG (NULL arguments, bad options, a NaN or infinity in f),
 * CPM_ERR_NOT_CONVERGED, CPM_ERR_DIVERGED (u holds the last iterate).
 */
cpm_status cpm_solve(cpm_hier h, const double* f, double* u, const cpm_solve_opts* opts,
                     cpm_solve_report* report, cpm_stream stream);

/*
 * r = f - A u on the finest level (the outer residual of cpm_solve,
 * difference form of M, Eq. 2.10), FP64 inputs and output.  Evaluated in
 * relative form: the extension of each tile works on u - u_ref (u_ref = u at
 * one band node of the tile) and the stencil combines reference differences
 * and extension differences formed from exact inputs, so the rounding error
 * scales with local differences of u rather than |u|/dx^2 (the plain form has
 * a relative floor near 1e-10 at dx = 1/512).  With outer_f64 = 0 (CPM_OP_MBR,
 * the default) the reference is rounded to float, u - u_ref is formed in FP64
 * and split into a pair of floats, and the extension and the stencil sums
 * run in FP32-pair arithmetic (exact products by fused multiply-add, TwoSum
 * for the leading parts: about 48 significand bits) on the FP32 pipe; the
 * term u_ref - u, the scaling by 1/dx^2 and the last sums are FP64.  Its
 * relative floor grows like 1/dx, about 4e-12 at dx = 1/512 on the unit sphere
 * against 1e-12 for the FP64 form.  Other operator forms evaluate r in FP64,
 * direct form.  f, u, r: FP64 device vectors of length |B_0|.
 * cpm_residual_norms uses the same evaluation.
 */
cpm_status cpm_residual(cpm_hier h, const double* f, const double* u, double* r, cpm_stream stream);

/* ---------------------------------------------------------------- batches */

typedef struct cpm_batch_s* cpm_batch;

#define CPM_BATCH_MAX_SYSTEMS 4096

/*
 * A batch of independent systems (c - Delta_S) u = f (the problem of Sec. 2.1
 * posed on several surfaces and with several right-hand sides, band sizes
 * uneven): n_hier hierarchies, each with n_rhs right-hand sides; system
 * s = i * n_rhs + k uses hierarchy i (n_hier * n_rhs <= CPM_BATCH_MAX_SYSTEMS).
 * Every system gets its own workspace (work vectors of every level, about
 * 130 bytes per finest band point); the hierarchies' static data is shared,
 * not owned by the batch, and must outlive it.  tune_cache: optional path of a
 * text file ("<batch key> <K>" per line) in which the autotuner keeps the
 * concurrency it chose for a batch of this shape (NULL: no file).  No
 * counterpart in the paper, which solves one system at a time.  Synchronous.
 */
cpm_status cpm_build_batch(const cpm_hier* hiers, int32_t n_hier, int32_t n_rhs,
                           const char* tune_cache, cpm_batch* out);

/*
 * Solve every system of the batch with the outer loop of cpm_solve (FP64
 * defect correction or FP32 V-cycles in FP64 iterative refinement; the
 * learned smoother is not used in batches: CPM_ERR_ARG if opts->learned).
 * f[s], u[s]: host arrays of n_hier * n_rhs device pointers to FP64 vectors of
 * length |B_0| of system s's hierarchy (caller-owned); u[s] is the initial
 * guess unless opts->zero_init.  Each outer iteration of all active systems is
 * one launch of a CUDA graph.  Systems of the same hierarchy form lockstep
 * groups (up to 16): one stream issues every V-cycle step for each member in
 * turn and the coarsest direct solve reads the dense inverse once for up to 4
 * members.  The groups run on K concurrent branches (largest first, each to
 * the least loaded branch); the autotuner picks K: the first outer iterations
 * try K = 1, 2, 4, ..., min(32, groups), each a real iteration, and keep the
 * fastest (stored in the tune cache; read from it when present).  Each
 * system's arithmetic is that of cpm_solve, bit for bit.  After each
 * launch the host reads every system's residual norm.  A system's result is
 * its first iterate with ||f - A u||_inf / ||f||_inf <= tol (the same iterate
 * cpm_solve returns); its workspace may keep iterating inside the graph until
 * the graph is re-captured over the remaining systems (when they are at most
 * half of it).  reports: n_hier * n_rhs entries or NULL (seconds = wall time
 * of the whole batch).  Returns CPM_ERR_NOT_CONVERGED / CPM_ERR_DIVERGED if
 * any system did (its last iterate is then in u[s]).  Synchronous.
 */
cpm_status cpm_solve_batch(cpm_batch b, const double* const* f, double* const* u,
                           const cpm_solve_opts* opts, cpm_solve_report* reports, cpm_stream stream);

/* Concurrency chosen by the autotuner (0 before the first solve) and the
 * measured device time of one outer iteration (ms) for each K tried, scaled
 * to the whole batch by the band points its graph covered (systems converge
 * while the candidates are tried) (tune_ms[q] for K = 2^q, q < 8; 0 where not
 * tried).  Host outputs, either may be NULL. */
cpm_status cpm_batch_info(cpm_batch b, int32_t* concurrency, double* tune_ms);

/* Free the workspaces and streams of the batch (not its hierarchies). */
cpm_status cpm_batch_destroy(cpm_batch b);

/*
 * Relative residual ||f - A u||_inf / ||f||_inf and ||f - A u||_2 on the
 * finest level in FP64 (host outputs).  Synchronous.
 */
cpm_status cpm_residual_norms(cpm_hier h, const double* f, const double* u, double* rel_inf,
                              double* abs_l2, cpm_stream stream);

/*
 * Allocation-free form of cpm_residual_norms (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory when they need a residual:
 * loops with hard latency budgets that forbid allocator calls, and frameworks
 * that hand out all device memory from their own pool.  It computes
 * r = f - A u on the finest level in FP64 in the direct form (w = E u, then
 * the stencil on w and u; unlike cpm_residual_norms, which uses the relative
 * form described at cpm_residual).  Its rounding floor
 * is that of the direct form, about 6 eps |u| / dx^2 in absolute terms; on the
 * levels it accepts (at most 1048576 band + ghost points, dx >= 1/128 for the
 * unit sphere) that is below 1e-12 |M u| for smooth u, so near a converged
 * solution the max |r_i| of the two entry points may differ by up to about
 * 1e-12 max |f_i|.  It writes
 * norms[0] = max_i |r_i|
 * and norms[1] = sum_i r_i^2 to the DEVICE pointer `norms` (2 doubles,
 * asynchronously on `stream`; nothing is copied to the host).  f, u: FP64
 * device vectors of length |B_0|.
 *
 * It calls no cudaMalloc / cudaFree or allocating library routine.  Its
 * scratch (E u on B+ and block partial norms) is one file-scope device array
 * of CPM_NOALLOC_MAX_POINTS doubles plus 8192 doubles (about 8.1 MB), held on
 * every GPU that loads the library until the process exits.  The first call
 * on a device (with that device current) looks up the array's device address;
 * the address is cached with the id of the CUDA context that was current, so
 * after cudaDeviceReset (a new context) the next call looks it up again.
 * Every call shares the one array and overwrites it: calls whose kernels
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Nothing in the scratch needs to start at zero.
 * Errors: CPM_ERR_ARG if |B_0| + |G_0| > CPM_NOALLOC_MAX_POINTS (use
 * cpm_residual_norms then) or on NULL arguments.
 */
#define CPM_NOALLOC_MAX_POINTS 1048576
cpm_status cpm_residual_norms_noalloc(cpm_hier h, const double* f, const double* u, double* norms,
                                      cpm_stream stream);

/*
 * Number of kernels this library has launched in the process so far (kernels
 * inside replayed CUDA graphs included).  Host counter, no device work.
 */
int64_t cpm_kernel_launches(void);

cpm_status cpm_hier_destroy(cpm_hier h);

#ifdef __cplusplus
}
#endif

#endif /* CPM_H */
