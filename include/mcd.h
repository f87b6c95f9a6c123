/*
 * mcd.h - C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of the mesh-constrained discrete point (MCD) method, arXiv 2404.17542:
 * DP masking and arrangement, chi=1 quadratic MLS stencil weights, and the
 * Bi-CGSTAB pressure-Poisson solve they drive.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Mesh / DP indexing: one DP per background-mesh cell (Sec. 2.2); cell and
 *    DP index k = i + n[0] * (j + n[1] * l).  N = n[0] * n[1] (* n[2]).
 *  - Positions are SoA float64, `dim` rows of N (x then y then z).
 *  - mask is int8 per DP: -1 inner, 0 void, >= 1 boundary id (Sec. 2.2, Eq. (1)).
 *    Whether boundary id b is a Dirichlet or a Neumann boundary is given by
 *    mcd_mls_params.bc_kind[b].
 *  - Every pointer argument named *_dev is DEVICE memory owned by the caller
 *    (e.g. a torch tensor); the library never frees it.  Pointers without the
 *    suffix are host memory.  Opaque handles (mcd_stencils, mcd_net, ...) own
 *    their device buffers and are released by their *_destroy call.
 *  - Work is enqueued on `stream` (NULL = legacy default stream).  Only calls
 *    whose description says "synchronises" wait for the stream.
 *  - Errors are reported only by the returned mcd_status; mcd_last_error()
 *    gives a message for the calling thread.  Nothing falls back to the CPU.
 */
#ifndef MCD_H
#define MCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mcd_stream_t; /* the same type as cudaStream_t */

typedef enum {
    MCD_OK = 0,
    MCD_EINVAL = 1,      /* bad argument (NULL, size, unsupported combination) */
    MCD_ENOMEM = 2,      /* device allocation failed */
    MCD_ECUDA = 3,       /* a CUDA runtime call failed */
    MCD_ESINGULAR = 4,   /* an MLS moment matrix is not positive definite */
    MCD_ENOCONV = 5,     /* the solve hit max_iter before reaching tol */
    MCD_EBREAKDOWN = 6,  /* Bi-CGSTAB broke down and restarting did not help */
    MCD_ENONFINITE = 7,  /* NaN or Inf in an input or a residual */
    MCD_ETIMEOUT = 8,    /* a bounded device wait gave up */
    MCD_ENOTSUP = 9      /* feature not built (e.g. 3D arrangement) */
} mcd_status;

enum { MCD_FP64 = 0, MCD_MIXED = 1 };          /* arithmetic of a solve */
enum { MCD_DT_F64 = 0, MCD_DT_F32 = 1 };       /* element type of a vector */
enum { MCD_W_GAUSS = 0, MCD_W_COS2 = 1, MCD_W_LSMPS = 2 };   /* MLS weight function */
enum { MCD_BC_DIRICHLET = 0, MCD_BC_NEUMANN = 1 };

/* Uniform Cartesian background mesh of width l0 (Sec. 2.1-2.2).  dim is 2 or
 * 3; n[2] = 1 and periodic[2] = 0 when dim = 2. */
typedef struct {
    int dim;
    int n[3];
    double l0;
    double origin[3];
    int periodic[3];
} mcd_mesh;

/* -------------------------------------------------------------------------
 * MLS stencil weights (Sec. 3.2, Eqs. (12)-(17))
 * ---------------------------------------------------------------------- */

/* weight_kind  MCD_W_COS2: w = cos^2(pi r / (2 r_e)) for r <= r_e, else 0
 *              (Eq. (17); the paper uses r_e = 2.5 l0);
 *              MCD_W_GAUSS: w = exp(-(r / r_e)^2), no cut-off;
 *              MCD_W_LSMPS: w = (1 - r / r_e)^2 for r < r_e, else 0 (the
 *              least-squares MPS weight the paper pairs with its expanded
 *              9x9 stencil, r_e = 3.5 l0, Sec. 4.1).
 * r_s          scaling length of X = (x - x_c) / r_s (Eq. (12); paper: l0).
 * precision    MCD_FP64 keeps FP64 rows only; MCD_MIXED also keeps an FP32
 *              copy of the rows for the inner solve of a mixed solve.
 * want_derivs  1: also keep the per-component derivative weights (gradient
 *              and Hessian, needed by the projection driver); 0: rows only.
 * bc_kind[b]   MCD_BC_DIRICHLET or MCD_BC_NEUMANN for boundary id b. */
typedef struct {
    int weight_kind;
    double r_e;
    double r_s;
    int precision;
    int want_derivs;
    uint8_t bc_kind[128];
    int support;   /* support radius R: the fit uses the (2R+1)^dim cells
                      around the DP's cell; 0 or 1: 3x3 (3x3x3), the MCD
                      stencil; 4 (2D only): the expanded 9x9 stencil of
                      Sec. 4.1; other values: MCD_EINVAL */
} mcd_mls_params;

typedef struct mcd_stencils mcd_stencils;  /* opaque; owns its device arrays */

/* mcd_build_stencils - chi=1 quadratic MLS weights of every DP and the rows
 * of the pressure-Poisson system (Sec. 3.2, Eqs. (12)-(17); Sec. 3.3, Eq. (21)).
 *
 * For DP i the fit uses the DPs of the 3x3 (3x3x3) cells around cell i, or
 * of the 9x9 cells with prm->support = 4 (2D; every slot-major array below
 * then has S = 81 slots, slot s = (di + 4) + 9 (dj + 4); periodic axes need
 * n >= 9).
 *  inner DP:     Lambda_c = inner and Dirichlet neighbours (values),
 *                Lambda^N_c = Neumann neighbours (normal-derivative data),
 *                basis (X, Y, X^2/2, XY, Y^2/2) (3D: 9 terms);
 *                row = MLS Laplacian; the Neumann data terms move to the RHS.
 *  Neumann DP:   linear fit over all non-void neighbours; row = n . grad,
 *                scaled so its diagonal is -1/r_s^2 (right-hand side scaled
 *                alike).
 *  Dirichlet DP, void DP: identity row.
 * Arguments
 *  mesh        host; periodic axes use the minimum image.
 *  pos_dev     device float64 [dim][N] DP positions.
 *  mask_dev    device int8 [N].
 *  normal_dev  device float64 [dim][N] unit normals of Neumann DPs (others
 *              ignored); may be NULL when no bc_kind entry is Neumann.
 *  prm         host parameters (above).
 *  st          in/out: *st == NULL allocates a new handle; an existing
 *              handle of the same mesh size and options is refilled.
 * A DP whose moment matrix is not positive definite is recorded on the
 * device; mcd_stencils_check() reports it (MCD_ESINGULAR) and
 * mcd_solve_pressure() refuses to run on such a handle.  Asynchronous. */
mcd_status mcd_build_stencils(const mcd_mesh *mesh, const double *pos_dev,
                              const int8_t *mask_dev, const double *normal_dev,
                              const mcd_mls_params *prm, mcd_stencils **st,
                              mcd_stream_t stream);

/* Synchronises `stream`; MCD_ESINGULAR (and *first_bad_dp >= 0) if a moment
 * matrix failed, MCD_OK (and -1) otherwise.  first_bad_dp may be NULL. */
mcd_status mcd_stencils_check(const mcd_stencils *st, int64_t *first_bad_dp,
                              mcd_stream_t stream);

void mcd_stencils_destroy(mcd_stencils *st);

/* Device arrays of a handle, for parity tests and drivers (read-only).
 *  MCD_ARR_ROW64   float64 [S][N] PPE rows (slot-major, S = (2 support + 1)^dim)
 *  MCD_ARR_ROW32   float32 [S][N] (MCD_MIXED only), difference form: slots
 *                  other than the centre C = S/2 hold the rounded FP64
 *                  weights, slot C the row sum (0 for MLS rows, whose sum
 *                  vanishes because chi = 1 MLS reproduces constants; 1 for
 *                  identity rows); (A x)_i = row[C] x_i + sum_{s != C}
 *                  row[s] (x_{j_s} - x_i)
 *  MCD_ARR_QL64    float64 [S][N] Neumann-data weights of the PPE rows
 *  MCD_ARR_D64     float64 [nb][S][N] value weights of each derivative
 *                  (nb = 5 in 2D: d/dx, d/dy, d2/dx2, d2/dxdy, d2/dy2;
 *                  9 in 3D: x, y, z, xx, yy, zz, xy, yz, xz); want_derivs only
 *  MCD_ARR_QD64    float64 [nb][S][N] Neumann-data weights of each derivative
 *  MCD_ARR_RSCALE  float64 [N] right-hand-side factor of boundary rows
 *  MCD_ARR_KIND    int8 [N]: 0 void, 1 inner, 2 Dirichlet, 3 Neumann
 * *count receives the number of elements (may be NULL). */
enum {
    MCD_ARR_ROW64 = 0, MCD_ARR_ROW32 = 1, MCD_ARR_QL64 = 2, MCD_ARR_D64 = 3,
    MCD_ARR_QD64 = 4, MCD_ARR_RSCALE = 5, MCD_ARR_KIND = 6
};
mcd_status mcd_stencils_array(const mcd_stencils *st, int which,
                              const void **dev_ptr, int64_t *count);

/* Copy array `which` (as above) into caller device memory dst_dev, which
 * must hold *count elements of the array's type.  Asynchronous. */
mcd_status mcd_stencils_copy(const mcd_stencils *st, int which, void *dst_dev,
                             mcd_stream_t stream);

/* mcd_apply_laplacian - y = A x with the PPE rows of `st` (the matrix-free
 * stencil SpMV of Eq. (21)).  dtype MCD_DT_F64 uses the FP64 rows and FP64
 * vectors; MCD_DT_F32 the FP32 rows (MCD_MIXED handles) and FP32 vectors.
 * x_dev, y_dev: device [N], must not alias.  Asynchronous. */
mcd_status mcd_apply_laplacian(const mcd_stencils *st, const void *x_dev,
                               void *y_dev, int dtype, mcd_stream_t stream);

/* mcd_assemble_rhs - right-hand side b of the PPE system (Eq. (21), (23)):
 * inner DP b = rhs - sum(QL * bnd over Neumann neighbours); Dirichlet DP
 * b = bnd; Neumann DP b = rscale * bnd; void DP b = 0.  rhs_dev, bnd_dev,
 * b_dev: device float64 [N].  Asynchronous. */
mcd_status mcd_assemble_rhs(const mcd_stencils *st, const double *rhs_dev,
                            const double *bnd_dev, double *b_dev,
                            mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Pressure solve (Sec. 3.3: Bi-CGSTAB on the MLS PPE)
 * ---------------------------------------------------------------------- */
typedef struct mcd_net mcd_net;   /* learned warm start, declared below */

/* tol          stop when ||b - A p||_2 <= tol ||b||_2 (FP64 residual).
 * max_iter     cap on Krylov iterations (all refinements together).
 * mode         MCD_FP64: plain FP64 Bi-CGSTAB (restarted from the true
 *              residual if the recursive one converged early);
 *              MCD_MIXED: FP32 Bi-CGSTAB on the FP32 rows whose iterate is
 *              folded into an FP64 solution, with reliable updates: the
 *              FP32 recursive residual is replaced by the FP64 residual
 *              b - A64 x (iterative refinement on an FP64 residual that
 *              keeps the Krylov direction); needs an MCD_MIXED handle.
 * inner_tol    (MIXED) reliable-update factor in (0, 1): an FP64 residual
 *              is taken once the FP32 residual has fallen by this factor
 *              since the last one (0.3 is the tested choice).  A recursion
 *              whose residual grows 100-fold since the last update while
 *              residuals are replaced has diverged: its correction is dropped
 *              and the solve continues on the restarting schedule; one that
 *              grows 1e4-fold while restarting ends the FP32 solve, which
 *              finishes in FP64 from the last folded iterate.
 * max_refine   cap on FP64 restarts (FP64 mode).
 * net          NULL, or a network whose correction is added to the guess
 *              before the Krylov solve (mcd_net_warm_start; 2D only).
 * check_every  Krylov iterations between host convergence checks (0: auto).
 * update_restart (MIXED) 1: restart the FP32 recurrence (fresh shadow
 *              residual, p = r) at every reliable update; 0 (adaptive):
 *              residual replacement, the recurrence continues with p, v and
 *              the shadow residual kept and beta recomputed from the replaced
 *              residual (restarts still follow the first update, an ||s||
 *              stop or a breakdown), until a cycle diverges; from then on
 *              the solve restarts at every update, as with 1.
 * barriers     grid barriers per Bi-CGSTAB iteration of the persistent solve:
 *              0 (default) or 2: two, the x, r update fused into the next
 *              p, v = A p phase, beta from the recurrence r^.s - omega r^.t;
 *              1: one where it applies (MCD_MIXED on a non-periodic 2D 3x3
 *              mesh with n_x a multiple of 4 and at least 40 x 20 cells),
 *              else two: each phase finishes iteration k and forms
 *              p', v' = A p', q' = A v', u' = A r' of k+1, and one reduction
 *              gives alpha, omega and beta, the last two as polynomials in
 *              alpha of its dot products (slower than two barriers on this
 *              GPU: more work per phase); 3: textbook.
 * net_dprev    with net: device float64 [N] or NULL, in and out: the
 *              increment the warm start reads (the pressure of the last
 *              step minus the one before); after a converged solve it
 *              holds this solve's increment, p(out) - p(in), for the next.
 * precond      NULL, or a network used as the preconditioner of the
 *              iterative refinement (MCD_MIXED, one- or two-barrier
 *              persistent schedule): every FP64 true-residual update that does not
 *              meet tol and restarts the FP32 recursion (the first update, a
 *              cycle dropped after diverging, an ||s|| stop or a breakdown;
 *              every update with update_restart = 1) begins a refinement
 *              cycle whose d0 is the network's correction of that residual
 *              (features without an increment: channel 6 is 0), added along
 *              its residual-minimising step before the recursion restarts.
 *              The residual never grows; a correction that cuts it by less
 *              than 10 % ends the network's part in that solve, which goes
 *              on plain (mcd_solve_info.net_corrections counts the
 *              applications). */
typedef struct {
    double tol;
    int max_iter;
    int mode;
    double inner_tol;
    int max_refine;
    const mcd_net *net;
    int check_every;
    int update_restart;
    double *net_dprev;
    int barriers;
    const mcd_net *precond;
} mcd_solve_params;

typedef struct {
    int iters;          /* Krylov iterations done */
    int refinements;    /* FP64 true-residual updates (reliable updates) */
    int restarts;       /* Bi-CGSTAB restarts after a rho breakdown */
    double rel_res;     /* final ||b - A p|| / ||b|| in FP64 */
    double b_norm;      /* ||b||_2 */
    int64_t unknowns;   /* non-void DPs of the system (DP unknowns solved) */
    double rel_res_guess;  /* with a net: ||b - A p|| / ||b|| of the guess, else -1 */
    double rel_res_start;  /* with a net: the same after the warm start, else -1 */
    int fallback;       /* MIXED: nonzero if the FP32 recursion failed and FP64
                           finished; why: 1 a restarted cycle diverged, 2 breakdown
                           restarts exhausted, 3 r^.v breakdown (alpha), 4 t = 0,
                           5 a non-finite dot, 6 max_iter, 7 other */
    int net_corrections;   /* with precond: network corrections applied */
    int discarded;      /* MIXED: FP32 cycles whose residual grew 100-fold; their
                           correction was dropped and the recursion restarted */
} mcd_solve_info;

/* mcd_solve_pressure - solve A p = b (b from mcd_assemble_rhs(rhs, bnd)).
 * p_dev: device float64 [N]; in: initial guess (with a net, the point the
 * warm start corrects), out: solution.  Dirichlet entries of the guess are
 * replaced by their values.  info: host, may be NULL.  Synchronises `stream`.
 * Returns MCD_ENOCONV if max_iter is reached (p holds the last iterate),
 * MCD_ENONFINITE if b or a residual is not finite, MCD_ESINGULAR if the
 * handle recorded a singular stencil. */
mcd_status mcd_solve_pressure(const mcd_stencils *st, const double *rhs_dev,
                              const double *bnd_dev, double *p_dev,
                              const mcd_solve_params *prm, mcd_solve_info *info,
                              mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Fractional-step driver (Sec. 3.3, Eqs. (20)-(22)), 2D
 * ---------------------------------------------------------------------- */

/* mcd_flow_predict - intermediate velocity and PPE source of one step with
 * the DPs held in place.  For every inner DP
 *   u* = F_MOC + nu dt lap u                                      (Eq. (20))
 * where F_MOC = u + d.grad u + 1/2 d^T H d, d = -u dt, is the second-order
 * Taylor value at the departure point, built like Eq. (19) from the MLS
 * derivative weights (Eq. (14)); then src = (1/dt) div u* (Eq. (21)).
 * Non-inner DPs: u* = (ubc, vbc) (0 at void DPs), src = 0.
 *  vel         stencil handle built with want_derivs = 1; its boundary ids
 *              should all be Dirichlet (velocity values are prescribed there).
 *  u, v, ubc, vbc   device float64 [N] (current and boundary velocity).
 *  us, vs, src      device float64 [N] outputs; us/vs must not alias u/v.
 * Asynchronous.  MCD_ENOTSUP for 3D meshes. */
mcd_status mcd_flow_predict(const mcd_stencils *vel, const double *u_dev,
                            const double *v_dev, const double *ubc_dev,
                            const double *vbc_dev, double nu, double dt,
                            double *us_dev, double *vs_dev, double *src_dev,
                            mcd_stream_t stream);

/* mcd_flow_project - u = u* - dt grad P at inner DPs (Eq. (22)); grad P is
 * the MLS gradient of the pressure stencils `pst` (want_derivs = 1), with
 * the Neumann-data terms of Eq. (15) taken from bnd (the same array passed
 * to mcd_solve_pressure).  Non-inner DPs: (ubc, vbc), 0 at void DPs.
 * All arrays device float64 [N].  Asynchronous. */
mcd_status mcd_flow_project(const mcd_stencils *pst, const double *P_dev,
                            const double *bnd_dev, const double *us_dev,
                            const double *vs_dev, const double *ubc_dev,
                            const double *vbc_dev, double dt, double *u_dev,
                            double *v_dev, mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Moving-boundary DP update (Sec. 2.2-2.4)
 * ---------------------------------------------------------------------- */

/* A rigid body (2D) at the new time: boundary id (>= 2; id 1 is the domain
 * wall), centre c, translational velocity and acceleration (the paper's
 * V_trans and dV_trans/dt, Eqs. (24)-(29)), posture angle theta, angular
 * velocity omega and acceleration omega_dot.
 *  sdf_dev == NULL: a circle of `radius` about c (analytic SDF).
 *  sdf_dev != NULL: a body given by SDF samples (Sec. 2.5), device float64
 *    [sdf_n[1]][sdf_n[0]], psi > 0 in the fluid, at
 *    sdf_origin + (i, j) sdf_h in the body's local frame; a world point x
 *    has local coordinates R(-theta) (x - c).  psi and grad psi at a point
 *    come from the chi = 1 quadratic MLS fit centred at the nearest grid
 *    point over its 3x3 grid support (cos^2 weight, r_e = 2.5 sdf_h,
 *    r_s = sdf_h), evaluated at the point; outside the box of grid points
 *    1 .. n - 2 psi is +inf, so the grid has to cover the DP band around
 *    the body.  The array must stay valid until the call's kernels finish.
 * Fields left zero give a circle without rotation. */
#define MCD_MAX_BODIES 64   /* bodies per call of the functions below */
typedef struct {
    int id;
    double c[3];
    double radius;
    double vel[3];
    double acc[3];
    double theta;
    double omega;
    double omega_dot;
    const double *sdf_dev;
    int sdf_n[2];
    double sdf_origin[2];
    double sdf_h;
} mcd_body;

/* mcd_update_dps - one DP update for the body positions of the new step.
 *  bodies[0 .. nbodies-1], 1 <= nbodies <= MCD_MAX_BODIES, distinct ids in
 *  2..127, disjoint circles.  At every point the SDF psi is that of the body
 *  with the smallest |psi| (Sec. 2.5; the first in the list on a tie),
 *  psi = sqrt(dx*dx + dy*dy) - R with every operation rounded separately.
 *  1. mask_prev <- mask.
 *  2. Role reassignment (Sec. 2.4) of every non-wall cell whose centroid is
 *     within `band` of the boundary (|psi(centroid)| < band; band <= 0: every
 *     cell): count the cell vertices with psi >= 0, evaluated for the
 *     vertex's nearest body as dx*dx + dy*dy >= R*R with every operation
 *     rounded separately, and map 0/1 -> void, 2/3 -> the id of the body
 *     nearest the centroid, 4 -> inner (Eq. (1)).  Cells with a face on the
 *     domain wall keep their mask.
 *  3. DPs of band cells that became void go to their cell centroid.
 *  4. n_relax Jacobi sweeps over the non-void band DPs: spring relaxation
 *     x* = x - kappa l0 sum_j (1 - r_ij/l0^SPG) x~_ij (Eqs. (5)-(8)), body DPs
 *     relocated onto the circle whose id they carry (Eq. (9)), inner DPs
 *     moved by beta psi d^ of the body nearest x* when alpha > 0 (Sec. 4.7,
 *     Eqs. (45)-(46), r_e = 5 l0), clamp into the cell.
 * pos_dev (float64 [2][N]) and mask_dev (int8 [N]) are updated in place;
 * mask_prev_dev (int8 [N]) receives the old mask.  2D only (MCD_ENOTSUP
 * otherwise); a bad body list gives MCD_EINVAL.  Asynchronous.
 * The Jacobi sweeps use one scratch buffer per device inside the library
 * (grown with cudaMalloc/cudaFree when a larger mesh comes): calls whose
 * work may overlap on the GPU (on two streams, or from two threads) race on
 * it and must be serialised by the caller. */
mcd_status mcd_update_dps(const mcd_mesh *mesh, const mcd_body *bodies,
                          int nbodies, double *pos_dev, int8_t *mask_dev,
                          int8_t *mask_prev_dev, double kappa, int n_relax,
                          double band, double alpha, mcd_stream_t stream);

/* Largest mesh (in DPs) that mcd_update_dps_static accepts. */
#define MCD_NOALLOC_MAX_DPS (1 << 20)

/* mcd_update_dps_static - mcd_update_dps without any GPU memory allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate while they step (a framework whose caching allocator has
 * already reserved the device's memory, a time-stepping loop that cannot
 * take the device synchronisation and latency cudaMalloc/cudaFree may bring,
 * or code that forbids allocation after start-up).  Arguments, results and
 * error codes are those of mcd_update_dps.  Differences:
 *  - the Jacobi scratch is a fixed device array of 2 * MCD_NOALLOC_MAX_DPS
 *    doubles (16 MiB) inside the library, reserved on every GPU that loads
 *    the library until the process exits; meshes with more than
 *    MCD_NOALLOC_MAX_DPS cells are rejected with MCD_EINVAL;
 *  - the first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress, with that device current) and keeps it; make
 *    that first call before any stream capture, and do not reset the device
 *    (cudaDeviceReset) after it in a process that goes on calling this
 *    entry point (the kept address would no longer be valid);
 *  - all calls share the one array: calls whose work may overlap on the GPU
 *    (for instance on two streams) race and must be serialised by the
 *    caller.  Each call overwrites the scratch it reads, so nothing needs
 *    clearing between calls. */
mcd_status mcd_update_dps_static(const mcd_mesh *mesh, const mcd_body *bodies,
                                 int nbodies, double *pos_dev, int8_t *mask_dev,
                                 int8_t *mask_prev_dev, double kappa, int n_relax,
                                 double band, double alpha, mcd_stream_t stream);

/* mcd_bodies_boundary - boundary data of the DPs of every body (mask == id
 * of bodies[b], 1 <= nbodies <= MCD_MAX_BODIES, distinct ids in 2..127):
 *  normal_dev  float64 [2][N]: unit normal grad psi / |grad psi| of the
 *              DP's body (Sec. 2.5; (x - c)/|x - c| for a circle); 0 at
 *              every other DP;
 *  neumann_dev float64 [N] or NULL: the pressure Neumann datum of Eq. (23),
 *              dP/dn = -(dV/dt) . n with the rigid-body
 *              dV/dt = acc + omega_dot x r + omega x (omega x r), r = x - c
 *              (Eqs. (26)-(29)); 0 at every other DP.
 * 2D only.  Asynchronous. */
mcd_status mcd_bodies_boundary(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                               const double *pos_dev, const int8_t *mask_dev,
                               double *normal_dev, double *neumann_dev,
                               mcd_stream_t stream);

/* mcd_bodies_velocity - the boundary velocity of every DP (the velocity
 * boundary data of mcd_flow_predict / mcd_flow_project): a DP at x with the
 * id of bodies[b] takes V = vel + omega x (x - c) (Eqs. (24)-(25)), every
 * other DP (domain walls included) 0.  pos_dev float64 [2][N]; ubc_dev,
 * vbc_dev float64 [N].  2D only.  Asynchronous. */
mcd_status mcd_bodies_velocity(const mcd_mesh *mesh, const mcd_body *bodies, int nbodies,
                               const double *pos_dev, const int8_t *mask_dev, double *ubc_dev,
                               double *vbc_dev, mcd_stream_t stream);

/* mcd_body_boundary - mcd_bodies_boundary for the single body *body. */
mcd_status mcd_body_boundary(const mcd_mesh *mesh, const mcd_body *body,
                             const double *pos_dev, const int8_t *mask_dev,
                             double *normal_dev, double *neumann_dev,
                             mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * ALE step and fluid force (Sec. 3.3, Eq. (19), Appendix A; Sec. 3.4)
 * ---------------------------------------------------------------------- */

/* mcd_ale_interpolate - the step-k velocity (u_dev, v_dev, float64 [N]) at
 * the step-(k+1) DP positions (Eq. (19) with p = 2):
 *   u~ = u + dx u_x + dy u_y + (dx^2 u_xx + 2 dx dy u_xy + dy^2 u_yy) / 2
 * with the derivatives of the step-k chi=1 quadratic MLS fit (vel_k: a 2D
 * 3x3 handle built with want_derivs = 1 on pos_k_dev / mask_k_dev, every
 * boundary a Dirichlet boundary), (dx, dy) = x^{k+1} - x_src^k:
 *  - DP inner at k and k+1: src = the DP itself (Eq. (A.1));
 *  - DP inner at k+1 only (role changed): src = the DP at the centre of its
 *    support shifted by (sign n_x, sign n_y) cells, n the outward normal of
 *    the body of bodies_k nearest its step-k position (Eq. (A.2)); if src is
 *    not inner at step k the DP keeps its step-k value and *fallbacks_dev
 *    (int32 device counter, may be NULL) is incremented;
 *  - DPs not inner at k+1 keep their step-k values.
 * pos_* float64 [2][N]; mask_* int8 [N]; the outputs must not alias the
 * inputs.  MCD_ENOTSUP for other stencil shapes.  Asynchronous. */
mcd_status mcd_ale_interpolate(const mcd_stencils *vel_k, const mcd_body *bodies_k, int nbodies,
                               const double *pos_k_dev, const double *pos_k1_dev,
                               const int8_t *mask_k_dev, const int8_t *mask_k1_dev,
                               const double *u_dev, const double *v_dev,
                               double *u_out_dev, double *v_out_dev, int *fallbacks_dev,
                               mcd_stream_t stream);

/* mcd_fluid_force - force of the fluid on the DPs with mask == body_id
 * (Eq. (30)): F = sum_i t_i dGamma_i, t = (-P I + mu (grad u + grad u^T)) . n
 * with n = normal_dev (float64 [2][N], outward from the body).  P and
 * grad u at a boundary DP come from the chi=1 quadratic fit of the DP at
 * the centre of its support shifted by (sign n_x, sign n_y) cells (Sec.
 * 3.4); the pressure fit includes the Neumann data bnd_dev (the boundary
 * data given to the solve; required when pres has Neumann ids).  dGamma_i
 * (Eq. (31)) is half the sum of the distances to the nearest DP of the same
 * id on each side of the tangent (-n_y, n_x) within the 5x5 cells around
 * it.  pres / vel: 2D 3x3 handles with want_derivs = 1 on the same cloud.
 * out_host[4] = {F_x, F_y, sum dGamma, DPs skipped because their shifted
 * centre is not an inner DP}.  Synchronises the stream. */
mcd_status mcd_fluid_force(const mcd_stencils *pres, const mcd_stencils *vel, int body_id,
                           const double *pos_dev, const int8_t *mask_dev, const double *normal_dev,
                           const double *P_dev, const double *bnd_dev, const double *u_dev,
                           const double *v_dev, double mu, double *out_host, mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * The moving-boundary fractional step (Sec. 3.3), one call per time step
 * ---------------------------------------------------------------------- */
typedef struct mcd_flow mcd_flow;   /* opaque: stencils and work arrays of a run */

/* nu           kinematic viscosity (the force uses mu = nu: unit density).
 * weight_kind, r_e   MLS weight of the velocity and pressure stencils (r_e
 *              0: l0); r_s = l0; 3x3 stencils.
 * precision    pressure stencils: MCD_FP64 or MCD_MIXED (needed by MIXED
 *              solves).
 * kappa, n_relax, band, alpha   the DP update of every step (as in
 *              mcd_update_dps; band <= 0: 5 l0, the band of Sec. 2.4).
 * ale_pressure 1: the PPE's initial guess is the step-k pressure carried to
 *              the new DP positions by the same ALE interpolation as the
 *              velocity (Eq. (19) and Appendix A: the role-changed DPs get
 *              the shifted-support value of Eq. (A.2)); 0: the step-k
 *              pressure as it is.
 * forces       1: compute the fluid force on every body (Eqs. (30)-(31)). */
typedef struct {
    double nu;
    int weight_kind;
    double r_e;
    int precision;
    double kappa;
    int n_relax;
    double band;
    double alpha;
    int ale_pressure;
    int forces;
} mcd_flow_params;

typedef struct {
    mcd_solve_info solve;      /* the step's PPE solve */
    int ale_fallbacks;         /* velocity ALE: role-changed DPs without an inner
                                  shifted centre (they keep u^k; Appendix A) */
    int ale_fallbacks_p;       /* the same for the pressure guess */
    int nbodies;
    double force[MCD_MAX_BODIES][2];   /* F of body b (order of the body list) */
    double perimeter[MCD_MAX_BODIES];  /* sum of dGamma of its DPs (Eq. (31)) */
    int skipped[MCD_MAX_BODIES];       /* its DPs whose shifted centre is not inner */
} mcd_flow_info;

/* mcd_flow_create - state of a moving-boundary run on the 2D mesh `mesh`
 * (3x3 stencils): arranges the DPs of pos_dev (float64 [2][N], in/out) and
 * mask_dev (int8 [N], in/out; walls already marked) for `bodies` over the
 * whole mesh (mcd_update_dps with band 0) and builds the velocity stencils
 * the first step's ALE interpolation reads.  The body ids and their order
 * are fixed for the run (1..MCD_MAX_BODIES bodies; their pressure boundary is
 * Neumann, every other boundary id Dirichlet).  Allocates about 20 N doubles
 * plus two stencil handles.  Asynchronous; *out receives the handle. */
mcd_status mcd_flow_create(const mcd_mesh *mesh, const mcd_flow_params *prm, const mcd_body *bodies,
                           int nbodies, double *pos_dev, int8_t *mask_dev, mcd_flow **out,
                           mcd_stream_t stream);
void mcd_flow_destroy(mcd_flow *f);

/* mcd_flow_restart - continue a run from a saved cloud (checkpoint / resume,
 * or repeating steps from a snapshot): rebuilds the velocity stencils of
 * pos_dev / mask_dev, the step-k weights the next step's ALE interpolation
 * reads.  The caller restores its own u, v, P with the cloud.
 * Asynchronous. */
mcd_status mcd_flow_restart(mcd_flow *f, const double *pos_dev, const int8_t *mask_dev, mcd_stream_t stream);

/* mcd_flow_step - one fractional step from t_k to t_{k+1} = t_k + dt in the
 * order of Sec. 3.3:
 *  1. every body's dV/dt = (vel^{k+1} - vel^k) / dt and
 *     d omega/dt = (omega^{k+1} - omega^k) / dt (Eq. (29)); the acc and
 *     omega_dot fields of the lists are not read;
 *  2. DP update to bodies_k1 (mcd_update_dps with the run's parameters);
 *  3. u~ = u^k(x^{k+1}) (mcd_ale_interpolate with the step-k velocity
 *     stencils and bodies_k; with ale_pressure also the PPE's guess);
 *  4. velocity stencils of the new cloud, the bodies' normals and Neumann
 *     data dP/dn = -dV/dt . n (Eq. (23)), pressure stencils;
 *  5. boundary velocities V + omega x r on the body DPs, 0 on the walls
 *     (Eqs. (24)-(25)); u* and src = (1/dt) div u* (Eqs. (20)-(21));
 *  6. the PPE (mcd_solve_pressure with `solve`, walls P = 0) and
 *     u^{k+1} = u* - dt grad P (Eq. (22));
 *  7. (forces = 1) the force on every body (Eqs. (30)-(31)).
 * bodies_k, bodies_k1: the bodies at t_k and t_{k+1} (positions, posture,
 * velocities vel and omega), the ids of mcd_flow_create in the same order.
 * pos_dev, mask_dev: the cloud of the last step (in), of this step (out);
 * u_dev, v_dev, P_dev: float64 [N] fields of step k in, k+1 out (P_dev is
 * also the solve's warm start).  info: host, may be NULL.  Synchronises the
 * stream.  A failed solve returns its status before the projection (the
 * cloud and the stencils are already those of step k+1). */
mcd_status mcd_flow_step(mcd_flow *f, const mcd_body *bodies_k, const mcd_body *bodies_k1, int nbodies,
                         double dt, const mcd_solve_params *solve, double *pos_dev, int8_t *mask_dev,
                         double *u_dev, double *v_dev, double *P_dev, mcd_flow_info *info,
                         mcd_stream_t stream);

/* The stencil handles of the run's current cloud (owned by the run; valid
 * until its next step or mcd_flow_destroy), e.g. for mcd_net_features on
 * the pressure system of the last step.  NULL for an unknown `which`. */
enum { MCD_FLOW_VELOCITY = 0, MCD_FLOW_PRESSURE = 1 };
const mcd_stencils *mcd_flow_stencils(const mcd_flow *f, int which);

/* Copy an array of the last step into dst_dev (device float64; [N], or
 * [2][N] for the normals): MCD_FLOW_B the assembled PPE right-hand side,
 * MCD_FLOW_GUESS the solve's initial guess, MCD_FLOW_BND the boundary data
 * (Neumann data on the bodies), MCD_FLOW_SRC (1/dt) div u*, MCD_FLOW_NORMAL
 * the body normals.  Asynchronous. */
enum { MCD_FLOW_B = 0, MCD_FLOW_GUESS = 1, MCD_FLOW_BND = 2, MCD_FLOW_SRC = 3, MCD_FLOW_NORMAL = 4 };
mcd_status mcd_flow_copy(const mcd_flow *f, int which, double *dst_dev, mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Batched systems (an addition: the paper solves one system at a time)
 *
 * `count` independent 2D systems (Sec. 2.2 meshes, Dirichlet boundary ids
 * only) built and solved together.  They are stored back to back: system i
 * owns DPs [off_i, off_i + N_i) (off_i = mcd_batch_offset(bt, i)) of every
 * per-DP device array (mask, rhs, bnd, p: [total N]); its positions are the
 * [2][N_i] block starting at element 2 off_i of pos.  In mcd_mls_params the
 * radii r_e and r_s are multiples of each system's own l0.
 * ---------------------------------------------------------------------- */
typedef struct mcd_batch mcd_batch;

/* Tiling of the batched solve: tiles of 32 x (8 rows) DPs per CTA step, and
 * CTAs per SM of the persistent launch (0: as many as fit, at most 4; the
 * FP32 kernels with 1 or 2 rows and the FP64 kernel with 1 row are built to
 * fit 4). */
typedef struct {
    int rows;          /* 1, 2 or 4 */
    int ctas_per_sm;   /* 0 .. 4 */
} mcd_batch_tuning;

typedef struct {
    int status;        /* MCD_OK, MCD_ENOCONV, MCD_EBREAKDOWN or MCD_ENONFINITE */
    int iters;         /* Bi-CGSTAB iterations of this system */
    int updates;       /* true-residual updates after the first */
    double rel_res;    /* ||b - A p|| / ||b|| (FP64) at the last update */
    int fallback;      /* MIXED: 1 if the FP32 recursion failed and FP64 finished */
    int discarded;     /* MIXED: cycles dropped after diverging (see mcd_solve_params) */
} mcd_batch_result;

/* meshes: host [count], each 2D.  Returns MCD_ENOTSUP for a 3D mesh or a
 * Neumann boundary id.  Allocates the stencil arrays of all systems. */
mcd_status mcd_batch_create(const mcd_mesh *meshes, int count, const mcd_mls_params *prm,
                            mcd_batch **bt);
void mcd_batch_destroy(mcd_batch *bt);

/* DP offset of system i (i = count gives the total), or -1. */
int64_t mcd_batch_offset(const mcd_batch *bt, int i);

/* MLS stencils of every system (one launch; same rules as
 * mcd_build_stencils).  Asynchronous. */
mcd_status mcd_batch_build(mcd_batch *bt, const double *pos_dev, const int8_t *mask_dev,
                           mcd_stream_t stream);

/* MCD_ESINGULAR (and the first failing DP, batch-global index) if a moment
 * matrix was singular in the last build.  Synchronises the stream. */
mcd_status mcd_batch_check(const mcd_batch *bt, int64_t *first_bad_dp, mcd_stream_t stream);

/* mcd_batch_solve - solve every system A_i p_i = b_i (b from rhs / bnd as in
 * mcd_assemble_rhs) in one persistent cooperative launch: Bi-CGSTAB in
 * lockstep sweeps with per-system scalars and convergence, the work of the
 * systems still running spread over all CTAs each sweep.  prm: tol (per
 * system, ||b_i - A_i p_i|| <= tol ||b_i||), max_iter (per system), mode
 * (MCD_MIXED: FP32 recursion with FP64 true-residual updates, inner_tol and
 * update_restart as in mcd_solve_pressure -- per system -- and systems whose
 * FP32 recursion fails finished by a second launch in FP64 from their last
 * folded iterate; MCD_FP64), net: NULL or the learned warm start, applied
 * to each system's guess (features without an increment) before the solve.
 * p_dev: initial guess
 * in, solutions out.  use_graph: capture the launches in a CUDA graph on the
 * first call and replay it while the arguments and tuning stay the same.
 * results: host [count] or NULL.  Synchronises the stream.  Returns MCD_OK
 * if every system converged, else the first failure status. */
mcd_status mcd_batch_solve(mcd_batch *bt, const double *rhs_dev, const double *bnd_dev,
                           double *p_dev, const mcd_solve_params *prm, int use_graph,
                           mcd_batch_result *results, mcd_stream_t stream);

/* System i of the batch as a stencil handle over the batch's arrays (owned
 * by the batch; valid after mcd_batch_build until mcd_batch_destroy), e.g.
 * for mcd_net_features or mcd_apply_laplacian on that system; NULL for a
 * bad index. */
const mcd_stencils *mcd_batch_stencils(const mcd_batch *bt, int i);

mcd_status mcd_batch_set_tuning(mcd_batch *bt, const mcd_batch_tuning *t);
mcd_status mcd_batch_get_tuning(const mcd_batch *bt, mcd_batch_tuning *t);

/* mcd_batch_autotune - time `sweeps` sweeps of the solve for every tiling
 * (rows 1, 2, 4 x 1 .. 4 CTAs per SM within the kernel's occupancy) and keep
 * the fastest per sweep.  A budget longer than the solve times whole solves,
 * which is what the choice should rest on: the per-sweep cost of a tiling
 * changes as small systems converge and large ones run alone.
 * cache_path (may be NULL): a text file of
 * "<device, sizes and mode key> | rows ctas_per_sm ms" lines; a matching
 * line is used without timing, a new result is appended.  p_dev is
 * overwritten (it is the iterate of the trial solves).  best_ms_per_sweep:
 * host, may be NULL.  Synchronises the device. */
mcd_status mcd_batch_autotune(mcd_batch *bt, const double *rhs_dev, const double *bnd_dev,
                              double *p_dev, const mcd_solve_params *prm, int sweeps,
                              const char *cache_path, double *best_ms_per_sweep,
                              mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Learned warm start (an addition: the paper has no network)
 *
 * A stack of `layers` 3x3 convolutions on the 2D background-mesh grid (zero
 * padding, stride 1, cross-correlation), `width` channels, ReLU between
 * layers, one output channel.  bf16 weights and activations on the tensor
 * cores, FP32 accumulation, FP32 master parameters and Adam moments.
 *
 * Parameters (host float32, flat): for each layer W[o][c][dj][di]
 * (o output, c input channel, dj/di the row/column tap 0..2; input cell
 * (i + di - 1, j + dj - 1) feeds output cell (i, j)), then b[o].
 *
 * Features (device bf16 [N][8], cell index k = i + n0 j, raw uint16 bits):
 * 0 r / s_r, with r = b - A p the residual of the guess and s_r its rms over
 * non-void DPs; 1, 2, 3 one-hot role (inner, boundary, void); 4, 5 the DP
 * offset (x - x_cell) / l0; 6 dprev / s_d, dprev the last pressure increment
 * and s_d its rms (0 without one); 7 zero.  Channels 0, 4, 5, 6 are 0 at
 * void DPs.  The network output y is a correction in units of
 * s_out = s_d if s_d > 0, else s_r l0^2.
 * ---------------------------------------------------------------------- */
enum { MCD_NET_PARAMS = 0, MCD_NET_GRADS = 1, MCD_NET_ADAM_M = 2, MCD_NET_ADAM_V = 3 };

/* Number of parameters, or -1 for an unsupported shape (supported: c_in in
 * [1, 8], width 32, layers in [2, 8]). */
int64_t mcd_net_param_count(int c_in, int width, int layers);

/* mcd_net_create - network with the given host parameters (copied); Adam
 * moments zero.  Returns MCD_ENOTSUP for an unsupported shape, MCD_EINVAL if
 * n_params does not match.  Synchronises the device. */
mcd_status mcd_net_create(int c_in, int width, int layers, const float *params,
                          int64_t n_params, mcd_net **net);
void mcd_net_destroy(mcd_net *net);

/* Copy the FP32 parameters (MCD_NET_PARAMS), the gradients of the last
 * training step (MCD_NET_GRADS) or an Adam moment to host_out [count];
 * count must equal the parameter count.  Synchronises the device.  Returns
 * MCD_ETIMEOUT if a tensor-core convolution of this network ever gave up
 * waiting for its MMAs (bounded wait; its outputs were not written). */
mcd_status mcd_net_read(const mcd_net *net, int which, float *host_out, int64_t count);

/* mcd_net_features - features of the system of `st` at the guess p:
 * r = b - A p (b the assembled right-hand side, mcd_assemble_rhs), written
 * to x_dev (bf16 [N][8], layout above).  dprev_dev: device float64 [N] or
 * NULL.  With p_true_dev (device float64 [N], the converged solution) also
 * the training target (p_true - p) / s_out and weight 1 on unknown DPs
 * (inner and Neumann; 0 and 0 elsewhere) into target_dev / weight_dev
 * (device float32 [N]).  2D stencil handles only (else MCD_ENOTSUP).
 * Asynchronous; uses the network's scratch (one call at a time per net). */
mcd_status mcd_net_features(mcd_net *net, const mcd_stencils *st, const double *b_dev,
                            const double *p_dev, const double *dprev_dev,
                            const double *p_true_dev, uint16_t *x_dev, float *target_dev,
                            float *weight_dev, mcd_stream_t stream);

/* mcd_net_forward - y_dev (device float32 [nx*ny]) = network(x_dev) with
 * x_dev the bf16 features [nx*ny][8].  Asynchronous. */
mcd_status mcd_net_forward(mcd_net *net, const uint16_t *x_dev, int nx, int ny,
                           float *y_dev, mcd_stream_t stream);

/* mcd_net_train_step - one Adam step (lr, beta = 0.9 / 0.999, eps = 1e-8)
 * on the loss sum_k w_k (y_k - target_k)^2 / sum_k w_k of one sample
 * (x_dev bf16 [nx*ny][8]; target_dev, weight_dev float32 [nx*ny]).
 * loss_dev: device float64 [1] receiving the loss before the step, or NULL.
 * Asynchronous. */
mcd_status mcd_net_train_step(mcd_net *net, const uint16_t *x_dev, const float *target_dev,
                              const float *weight_dev, int nx, int ny, float lr,
                              double *loss_dev, mcd_stream_t stream);

/* mcd_net_warm_start - p <- p + s e, e = y s_out on unknown DPs (0 elsewhere),
 * y = network(features of (b, p, dprev)), s = <r, A e> / <A e, A e> the step
 * that minimises ||b - A (p + s e)||_2 (0 if A e = 0): the residual never
 * grows.  b_dev: assembled right-hand side; p_dev updated in place.
 * stats: host double [3] or NULL; when given (synchronises the stream) it
 * receives ||r|| / ||b|| before and after and the step s. */
mcd_status mcd_net_warm_start(mcd_net *net, const mcd_stencils *st, const double *b_dev,
                              const double *dprev_dev, double *p_dev, double *stats,
                              mcd_stream_t stream);

/* -------------------------------------------------------------------------
 * Instrumentation (metrics and tracing; not part of the method)
 * ---------------------------------------------------------------------- */
enum {
    MCD_K_BICG_A = 0,    /* p update + v = A p + r^.v          */
    MCD_K_BICG_B = 1,    /* s = r - alpha v + t = A s + dots    */
    MCD_K_BICG_C = 2,    /* x, r update + dots                  */
    MCD_K_RESIDUAL = 3,  /* FP64 residual b - A x               */
    MCD_K_BUILD = 4,     /* MLS stencil build                   */
    MCD_K_UPDATE = 5,    /* remask + relaxation sweeps          */
    MCD_K_OTHER = 6,     /* everything else                     */
    MCD_K_SOLVE = 7,     /* persistent cooperative Bi-CGSTAB     */
    MCD_K_CNN = 8,       /* network: convolutions, features, training */
    MCD_K_BATCH = 9,     /* batched solve (persistent launch or graph replay) */
    MCD_K_COUNT = 10
};

/* When sample_every > 0, every sample_every-th launch of each kernel class
 * is bracketed by CUDA events recorded on the stream it is launched on
 * (0 disables).  Resets the accumulated samples.  Not thread-safe with
 * concurrent solves. */
mcd_status mcd_timing_enable(int sample_every);

/* Synchronises the recorded events of kernel class `kernel` and returns the
 * number of sampled launches and their summed device time in ms. */
mcd_status mcd_timing_read(int kernel, int64_t *sampled, double *total_ms);

/* Phase trace of the persistent solver: when enabled (on = 1), thread 0 of
 * block 0 records %globaltimer stamps (ns) for the first 64 iterations of
 * each launch: host_out[8*it + slot].  Three-barrier schedule: slot 0
 * iteration start, 1 phase A done, 2 A reduced, 3 B done, 4 B reduced, 5 C
 * done, 6 C reduced; two-barrier schedule: 0 start, 1 phase CA done, 2 CA
 * reduced, 3 B done, 4 B reduced.  For iteration 10 and block b < 2048:
 * host_out[512 + b] = end of its first phase, host_out[2560 + b] = its SM
 * id, host_out[4608 + b] = its start of the iteration.  Stages of the grid
 * barriers with epoch e < 256 of a launch (the barriers of its first ~120
 * iterations), host_out[6656 + 8*e + k]: block 0 entering (k = 0), its
 * partial sums published (1), every block's partials seen and added (2, 3),
 * the scalars updated (4), the other blocks released (5); the latest
 * arrival of any block (6) and the latest wake-up of a released block (7),
 * both maxima over the launches since tracing was enabled.  mcd_trace_read
 * synchronises the device and copies the 8704 values. */
mcd_status mcd_trace_enable(int on);
mcd_status mcd_trace_read(unsigned long long *host_out);

/* Self-test of the bounded device wait that the grid barriers of the
 * persistent solvers use (failure detection without a GPU fault).  One
 * thread polls a device word for the value 1, at most `polls` times: the
 * first 256 back to back, then 64 ns apart.  With set_flag = 0 nothing sets
 * the word, so the wait gives up.  The call then returns MCD_ETIMEOUT, and
 * the context stays usable.  With set_flag = 1 the word holds 1 and the
 * call returns MCD_OK.  polls must be in [1, 2^20], about a second at
 * most; otherwise MCD_EINVAL.  The call allocates and frees 8 bytes of
 * device memory and synchronises `stream`. */
mcd_status mcd_selftest_bounded_wait(int set_flag, int64_t polls, mcd_stream_t stream);

/* Staging of the persistent solve's operands (a measurement switch, not
 * part of the method): on = 1 (the default) lets the two-barrier FP32 solve
 * of 2D 3x3 stencils on non-periodic meshes stage each tile's rows and
 * vectors in shared memory with TMA copies, two tiles in flight per block;
 * on = 0 makes it load them directly.  Results are the same either way (the
 * same arithmetic in the same order).  Process-wide; affects later solves. */
mcd_status mcd_solver_set_staging(int on);

/* Number of kernels this library has launched since it was loaded. */
int64_t mcd_launch_count(void);

/* Message of the last error on the calling thread (never NULL). */
const char *mcd_last_error(void);

/* Library version string. */
const char *mcd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MCD_H */
