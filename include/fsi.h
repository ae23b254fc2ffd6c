/*
 * fsi.h -- C ABI of the GB300 monolithic fluid-structure Newton-Krylov-Schwarz solver.
 *
 * The solver advances the monolithically coupled ALE fluid-structure system of
 * Kong, Kheyfets, Finol & Cai (arXiv 1810.04289) by one backward-Euler step per
 * fsi_step call:
 *   - ALE map x = X + d_m and harmonic mesh motion (Sec. 2.1, Eq. 1);
 *   - St. Venant-Kirchhoff wall, total Lagrangian (Sec. 2.1, Eq. 2);
 *   - incompressible Navier-Stokes on the moving fluid domain (Sec. 2.1, Eq. 3),
 *     stabilised P1-P1 (Sec. 2.2), strong interface coupling with one set of
 *     unknowns per interface node (Sec. 2.2, Eq. 6-7);
 *   - backward Euler in time, F(y) = 0 per step (Sec. 2.2, Eq. 9-10);
 *   - inexact Newton with backtracking (Sec. 3, Eq. 11-12), right-preconditioned
 *     GMRES with a restricted additive Schwarz preconditioner whose subdomain
 *     solver is a block incomplete LU factorisation, ILU(k) with level of fill
 *     k = 0..3 (Sec. 3, Eq. 13-16; Sec. 4.3).
 *
 * Unknowns: 7 per mesh node, node-major: y[i*7 + c], c = 0..6 =
 * [u_x, u_y, u_z, p, d_x, d_y, d_z] (fluid velocity, pressure, displacement; on
 * wall-only nodes the u and p slots are constrained to zero). Units: cm, g, s.
 *
 * Conventions shared by every call:
 *   - Nothing throws across the ABI. Every call returns an fsi_status;
 *     fsi_last_error() gives a message for the last failure on that context.
 *   - Pointers documented as "device" must be CUDA device (or managed) memory
 *     of the current device; pointers documented as "host" are host memory.
 *     The caller owns every pointer it passes; the context keeps none of them
 *     beyond the call (mesh arrays are copied by fsi_create).
 *   - All GPU work of a context is ordered on the CUDA stream given to
 *     fsi_create (NULL = the legacy default stream). Calls return after the
 *     work they need to report a result is complete on that stream.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef FSI_GB300_H
#define FSI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsi_ctx fsi_ctx;

typedef enum {
  FSI_OK = 0,
  FSI_ERR_ARG = 1,              /* invalid argument (null pointer, size, option) */
  FSI_ERR_MESH = 2,             /* invalid mesh (index out of range, degenerate tet) */
  FSI_ERR_CUDA = 3,             /* a CUDA runtime call failed */
  FSI_ERR_NOMEM = 4,            /* device or host allocation failed */
  FSI_ERR_ZERO_PIVOT = 5,       /* singular 7x7 pivot block in the ILU factorisation */
  FSI_ERR_LINEAR_DIVERGED = 6,  /* GMRES reached its iteration limit above tolerance */
  FSI_ERR_DIVERGED = 7,         /* Newton reached its iteration limit above tolerance */
  FSI_ERR_LINESEARCH = 8,       /* backtracking found no sufficient decrease */
  FSI_ERR_TIMEOUT = 9,          /* a bounded device-side wait gave up */
  FSI_ERR_NONFINITE = 10        /* NaN or Inf in the residual */
} fsi_status;

/* Node tag bits (fsi_mesh.node_tag). FLUID: belongs to a fluid tet; WALL: to a
 * wall tet; INTERFACE: vertex of the wet interface (a fluid-tet face shared with
 * a wall tet, Sec. 4.8, Algorithm 1); INLET / OUTLET: fluid node on an inflow /
 * outflow cap; WALL_END: wall node on a cap (clamped, Eq. 2); OUTER: outer wall
 * surface (zero traction). */
enum {
  FSI_TAG_FLUID = 1, FSI_TAG_WALL = 2, FSI_TAG_INTERFACE = 4, FSI_TAG_INLET = 8,
  FSI_TAG_OUTLET = 16, FSI_TAG_WALL_END = 32, FSI_TAG_OUTER = 64
};

/* The mesh: host arrays, copied at fsi_create.
 *   X            [n_nodes*3]  reference coordinates (cm), node-major
 *   tets         [n_tets*4]   vertex ids, positively oriented
 *   tet_domain   [n_tets]     0 = fluid (lumen), 1 = wall
 *   node_tag     [n_nodes]    FSI_TAG_* bits
 *   node_problem [n_nodes]    problem id of each node for batched meshes of
 *                             independent vessels (non-decreasing: each
 *                             problem's nodes stored one after another;
 *                             otherwise FSI_ERR_MESH), or NULL for one problem */
typedef struct {
  int64_t n_nodes, n_tets;
  const double *X;
  const int32_t *tets;
  const uint8_t *tet_domain;
  const uint32_t *node_tag;
  const int32_t *node_problem;
} fsi_mesh;

/* Materials (Sec. 2.1): blood density rho_f (g/cm^3) and dynamic viscosity
 * mu_f (P); wall density rho_s, Young's modulus E_s (dyn/cm^2), Poisson ratio
 * nu_s, damping eta_s (g/(cm^3 s)). */
typedef struct {
  double rho_f, mu_f, rho_s, E_s, nu_s, eta_s;
} fsi_material;

/* Inflow boundary of one problem (Eq. 3, u_f = v_f^d on the inlet):
 * u = U(t) (1 - r^2/R^2)_+ n, U(t) = peak (1 + amp sin(2 pi freq t + phase)),
 * r = distance from the line through `center` along `normal` (the unit normal
 * pointing into the lumen), R = radius. rigid_wall != 0 clamps every wall node
 * (d = 0), which reduces the problem to flow in a rigid vessel. */
typedef struct {
  double center[3], normal[3], radius;
  double peak, amp, freq, phase;
  int32_t rigid_wall;
} fsi_bc;

/* Solver options (Sec. 4: defaults Newton rtol 1e-6, GMRES rtol 1e-3,
 * overlap 1). precision 0 = FP64 throughout; 1 = mixed: Jacobian, ILU factors,
 * preconditioner apply and matrix values in FP32, residual, Krylov basis,
 * Arnoldi, least squares and Newton update in FP64. Start from
 * fsi_default_options. In fsi_create, zero or negative dt, tolerances, iteration
 * counts, restart and n_subdomains, and negative overlap / ilu_level, take the
 * defaults; precision, jac_lag (>= 1), ilu_level and overlap are used as given. */
typedef struct {
  double dt;              /* time step (s) */
  double newton_rtol;     /* stop when ||F|| <= newton_rtol ||F(y^(0))|| */
  double newton_atol;     /* or when ||F|| <= newton_atol */
  double gmres_rtol;      /* GMRES stop: ||J dy + F|| <= gmres_rtol ||F|| */
  int32_t newton_maxit;
  int32_t gmres_restart;  /* Krylov dimension per cycle (<= 64) */
  int32_t gmres_maxit;    /* total GMRES iterations per linear solve */
  int32_t n_subdomains;   /* Schwarz subdomains (Sec. 3) */
  int32_t overlap;        /* overlap delta in node layers (Sec. 3) */
  int32_t precision;      /* 0 FP64, 1 mixed FP32/FP64 */
  int32_t jac_lag;        /* reuse the Jacobian for this many Newton iterations (Eq. 12), >= 1 */
  int32_t ilu_level;      /* level of fill k of the subdomain block ILU(k), 0..3 (Sec. 4.3) */
  int32_t threads_per_row;/* BSR SpMV mapping: 32 = one warp per block row, 16 = two rows per warp */
  int32_t ordering;       /* node order inside each subdomain (Sec. 4.5): 0 natural
                             (global node order), 1 RCM, 2 RCM with lumen nodes
                             before interface and wall nodes, 3 nested dissection
                             (coordinate bisection, up to 3 levels, RCM inside each
                             part; the parts of one level are solved side by side) */
  int32_t factor_mode;    /* ILU factorisation kernel: 0 automatic (4 when the
                             subdomains are dissected, ordering 3, and its rows fit in
                             shared memory, else 3); rows in order with 1 pivots and
                             update sources prefetched into shared memory, 2 sources
                             only, 3 neither (the row alone in shared memory); 4 the
                             parts of each dissection level factored side by side. A
                             forced mode whose footprint does not fit is FSI_ERR_ARG.
                             All modes give bitwise identical factors. */
  int32_t verbose;        /* print per-iteration norms to stderr */
  int32_t fault_test;     /* tests only: 1 = the preconditioner apply's copy engine
                             issues nothing, so the apply's bounded wait runs out and
                             the call returns FSI_ERR_TIMEOUT; 2 = Gram-Schmidt orth 0
                             forms every new vector's norm from the updated vector (its
                             fallback path); 0 otherwise */
  int32_t apply_mode;     /* preconditioner apply kernel: 0 automatic (the streamed
                             apply when its shared-memory footprint fits, else the
                             level-scheduled one); 1 streamed (FSI_ERR_ARG if it does
                             not fit); 2 level-scheduled. Same arithmetic, same result
                             up to the order of the row sums. */
  int32_t stage_blocks;   /* streamed apply: factor blocks per ring stage, 0 = automatic
                             (sized from the shared memory left at ceil(n_subdomains / 152),
                             at most 8, CTAs per SM) */
  int32_t stages;         /* streamed apply: ring stages in flight per warp, 2..8,
                             0 = automatic (2) */
  int32_t orth;           /* Arnoldi orthogonalisation, FP64 (Sec. 4: classical
                             Gram-Schmidt twice): 0 the new vector's norm taken from the
                             second pass (dots; update; dots with ||w||^2; update and
                             scaling in one sweep by 1/sqrt(||w||^2 - ||h||^2), or the
                             vector's own norm where that subtraction would lose two bits
                             or more); 1 a second pass only where the first removed more
                             than 1 - 1/sqrt(2) of the vector's norm (selective
                             reorthogonalisation); 2 dots, update, dots, update, norm,
                             scaling as separate sweeps */
  int32_t jac_chunk;      /* tets per chunk of the Jacobian assembly's element buffer,
                             0 = automatic (as many as the factors' storage, which the
                             buffer shares, holds). Any chunking gives bitwise the same
                             matrix. */
} fsi_options;

typedef struct {
  int32_t iterations;     /* GMRES iterations */
  int32_t converged;      /* 1 if the tolerance was met */
  double rnorm0, rnorm;   /* initial and final true residual norms ||b - J x|| */
} fsi_solve_stats;

typedef struct {
  int32_t newton_iterations;
  int32_t linear_iterations;   /* total GMRES iterations over the step */
  int32_t jacobian_evaluations;
  int32_t residual_evaluations;
  int32_t converged;
  double fnorm0, fnorm;        /* ||F|| at the first and last Newton iterate */
  /* device time per phase (ms), in the paper's timing categories (Table 7),
   * and how many times each phase ran; t_total is the device time of the step.
   * The GMRES restart cycles run as captured CUDA graphs: their whole time
   * (preconditioner applies, SpMVs, orthogonalisation) is t_krylov, and
   * t_pcapply / t_spmv / t_orth only count work outside the graphs. */
  double t_funceval, t_jaceval, t_pcsetup, t_pcapply, t_spmv, t_orth, t_total, t_krylov;
  int32_t n_funceval, n_jaceval, n_pcsetup, n_pcapply, n_spmv, n_orth;
  int64_t kernel_launches;     /* CUDA kernels launched by the step */
} fsi_step_stats;

typedef struct {
  int64_t n_nodes, n_tets, n_unknowns, nnzb;
  int64_t n_fluid_tets, n_wall_tets;
  int32_t n_problems, n_subdomains;
  int64_t factor_blocks;       /* 7x7 blocks held by all subdomain factors */
  int64_t factor_rows;         /* block rows of all overlapped subdomains */
  int32_t max_levels;          /* deepest level schedule over the subdomains */
  int64_t device_bytes;        /* device memory held by the context */
  int64_t n_wss_faces;         /* inner-wall faces (fluid tet against wall tet) */
  int32_t nd_depth;            /* deepest nested dissection of a subdomain (ordering 3), else 0 */
  int32_t apply_kernel;        /* preconditioner apply in use: 1 streamed, 2 level-scheduled */
} fsi_info;

/* Defaults: dt 1e-3, newton_rtol 1e-6, newton_atol 1e-10, gmres_rtol 1e-3,
 * newton_maxit 20, gmres_restart 30, gmres_maxit 1000, n_subdomains 64,
 * overlap 1, precision 0, jac_lag 1, ilu_level 1 (the paper's default subdomain
 * solver, Sec. 4), threads_per_row 32, ordering 1 (RCM, the paper's default,
 * Sec. 4.5). A negative ilu_level or overlap in the
 * caller's options also selects the default. */
void fsi_default_options(fsi_options *opts);

/* Build a solver context for `mesh` (the discrete problem of Sec. 2.2, Eq. 6-7:
 * one block of 7 unknowns per mesh node, strong coupling at the interface
 * nodes; its Schwarz subdomains Omega_i and overlaps Omega_i^delta of Sec. 3,
 * Eq. 14). bc: array of n_problems inflow boundaries (n_problems >= 1;
 * node_problem picks one per node). Performs all symbolic work on the host
 * (block-sparse pattern, assembly gather lists, subdomain partition, overlap,
 * subdomain ordering, ILU(k) pattern, level schedules), copies the mesh to the
 * device and allocates every device buffer the solver needs. The state is zero
 * until fsi_set_state. `cuda_stream` is a cudaStream_t. Host pointers inside
 * mesh / mat / bc are read during the call only.
 * Errors: FSI_ERR_ARG, FSI_ERR_MESH, FSI_ERR_NOMEM, FSI_ERR_CUDA; *out is NULL
 * on failure. */
fsi_status fsi_create(const fsi_mesh *mesh, const fsi_material *mat, const fsi_bc *bc,
                      int32_t n_problems, const fsi_options *opts, void *cuda_stream,
                      fsi_ctx **out);

/* Release every device and host resource of the context. NULL is accepted. */
fsi_status fsi_destroy(fsi_ctx *ctx);

/* Set the time level: y_n (the last accepted state), y_{n-1}, y_{n-2} and the
 * time t_n. Device pointers, [n_nodes*7] FP64 each. y_nm1 / y_nm2 may be NULL
 * (taken equal to y_n). The next fsi_step solves for t_n + dt. */
fsi_status fsi_set_state(fsi_ctx *ctx, const double *y_n, const double *y_nm1,
                         const double *y_nm2, double t);

/* Copy the current state y_n (device, [n_nodes*7]) and time; either may be NULL. */
fsi_status fsi_get_state(fsi_ctx *ctx, double *y_n, double *t);

/* F(y) for the step that ends at t_n + dt, with y_{n-1}, y_{n-2} taken from
 * the context state (Eq. 9-10). y, F: device, [n_nodes*7] FP64. Constraint
 * rows (Dirichlet caps, inlet profile, kinematic interface rows, the unused u/p
 * slots of wall-only nodes) hold (value - prescribed). */
fsi_status fsi_residual(fsi_ctx *ctx, const double *y, double *F);

/* Assemble the exact Jacobian J = dF/dy at y (device, [n_nodes*7]) into the
 * context's block-sparse (7x7 BSR) matrix, in FP64 or, in mixed precision, in
 * FP32: the Jacobian of Eq. 12 formed analytically (exact derivatives of every
 * term, stabilisation parameters included; Sec. 3). The matrix is owned by the
 * context. Marks the preconditioner stale; it is rebuilt by the next linear
 * solve. Errors: FSI_ERR_ARG (null pointer), FSI_ERR_CUDA. */
fsi_status fsi_jacobian(fsi_ctx *ctx, const double *y);

/* Copy the assembled Jacobian out. Host pointers, any may be NULL:
 * row_ptr [n_nodes+1], col [nnzb] (sorted block columns), vals [nnzb*49]
 * (row-major 7x7 blocks, converted to FP64). */
fsi_status fsi_jacobian_export(fsi_ctx *ctx, int32_t *row_ptr, int32_t *col, double *vals);

/* y = J x with the assembled Jacobian. Device pointers, [n_nodes*7] FP64. */
fsi_status fsi_spmv(fsi_ctx *ctx, const double *x, double *y);

/* z = B^{-1} r, the restricted additive Schwarz preconditioner of Eq. 16 built
 * from the assembled Jacobian (built first if stale). Device pointers, FP64. */
fsi_status fsi_pc_apply(fsi_ctx *ctx, const double *r, double *z);

/* Solve J x = rhs, the Newton correction system of Eq. 12-13, with
 * right-preconditioned restarted (flexible) GMRES and the restricted additive
 * Schwarz preconditioner of Eq. 14-16 (built first if stale), to the context's
 * gmres_rtol on the true residual. Device pointers, [n_nodes*7]; rhs is read,
 * x is the output (initial guess 0). stats (host, may be NULL) gets the
 * iteration count and residual norms. Returns FSI_ERR_LINEAR_DIVERGED (x still
 * holds the last iterate) if gmres_maxit is reached; FSI_ERR_ARG if no Jacobian
 * was assembled; FSI_ERR_ZERO_PIVOT if a subdomain factor has a singular pivot
 * block; FSI_ERR_TIMEOUT if a bounded device wait gave up. */
fsi_status fsi_linear_solve(fsi_ctx *ctx, const double *rhs, double *x, fsi_solve_stats *stats);

/* One backward-Euler step (Eq. 9-10: the fully implicit system F(y) = 0 at
 * t_n + dt): inexact Newton with backtracking from y^(0) = y_n (Sec. 3, Eq.
 * 11-12; the Jacobian is rebuilt every jac_lag iterations), each correction from
 * fsi_linear_solve's GMRES, to the Newton tolerance; then the time levels shift
 * (y_{n-2} <- y_{n-1} <- y_n <- y, t <- t + dt). stats (host, may be NULL) gets
 * the iteration counts and, when given, per-phase device times. Errors:
 * FSI_ERR_DIVERGED (newton_maxit reached), FSI_ERR_LINESEARCH,
 * FSI_ERR_NONFINITE, FSI_ERR_ZERO_PIVOT, FSI_ERR_TIMEOUT, FSI_ERR_CUDA; on any
 * failure the state is left at the previous time level. */
fsi_status fsi_step(fsi_ctx *ctx, fsi_step_stats *stats);

/* Wall shear stress on the inner wall of every problem (the WSS and SAWSS
 * formulas of the paper's results section, with sigma_f of Eq. 3): on each face
 * shared by a fluid tet and a wall tet, WSS = sigma n - (sigma n . n) n with
 * sigma = -p I + 2 mu_f eps(u) of the P1 fluid tet on the current configuration
 * x = X + d, p at the face centroid and n the unit normal out of the fluid;
 * SAWSS of a problem = sum of |WSS| x face area / sum of face areas.
 * y: device [n_nodes*7] FP64 state. wss: device [n_wss_faces*3] FP64 output, or
 * NULL. sawss: host [n_problems] output, or NULL (when given, the call waits for
 * the stream). Faces are ordered as fsi_wss_faces lists them. */
fsi_status fsi_wss(fsi_ctx *ctx, const double *y, double *wss, double *sawss);

/* The inner-wall faces used by fsi_wss, in its order (by problem, then fluid
 * tet in input order, then face): n_faces gets their count; tet_face (host
 * [n_faces*2], may be NULL) gets, per face, the input index of its fluid tet and
 * the local index (0..3) of that tet's vertex opposite the face. */
fsi_status fsi_wss_faces(const fsi_ctx *ctx, int64_t *n_faces, int32_t *tet_face);

fsi_status fsi_get_info(const fsi_ctx *ctx, fsi_info *info);

/* Allocation-free variant of fsi_residual (the paper has no counterpart; this
 * is an interface convenience). For callers that must not have the library
 * allocate device memory, e.g. code that fixed its device-memory footprint in
 * advance or that runs while device allocation is not allowed: it computes the
 * same F(y) as fsi_residual (same arguments, device pointers [n_nodes*7] FP64)
 * and allocates nothing itself, because its assembly scratch (28 FP64 values
 * per tet) is one fixed device array built into the library, sized for at most
 * 32,768 tets (7.3 MB per device). Larger meshes get FSI_ERR_ARG with a
 * message. The first call on a device looks up that array's device address
 * (once per device, with the device current); under CUDA's lazy module loading
 * that first lookup is also when the driver loads the library's device code and
 * commits the array's memory on that device, so a caller that must not see any
 * allocation during its run makes one warm-up call per device beforehand (and
 * before any stream capture). From then on every GPU that has done so holds the
 * array until the process exits. All calls share the one array: calls that
 * overlap on the GPU (other streams, other contexts, other host threads) race
 * and must be serialised by the caller. */
fsi_status fsi_residual_noalloc(fsi_ctx *ctx, const double *y, double *F);

/* Message of the last failure on the context (static string if ctx is NULL). */
const char *fsi_last_error(const fsi_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FSI_GB300_H */
