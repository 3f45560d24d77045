/*
 * pd.h -- C ABI of the GB300 projective-dynamics library (libpdgb300.so).
 *
 * The library time-steps a tetrahedral mesh whose elements carry their own
 * strain and volume stiffness, with the domain-decomposed projective
 * dynamics of "Volumetric Homogenization for Knitwear Simulation"
 * (arXiv 2405.12484), Sec. 7:
 *   - implicit Euler, inertial target y = x* + dt v* + dt^2 g   (Sec. 7, eq. for a)
 *   - PD local step: per tet F = Ds Dm^-1, SVD, rotation target R(F) and
 *     volume target V(F)                                        (Sec. 7.1, Eq. pd_local, Eq. vol_pre)
 *   - PD global step K x = b                                     (Sec. 7.1, K and b)
 *     solved by the domain-decomposed subspace solve: per-domain internal
 *     solves, boundary modes Psi = -Kii^-1 Kib, and the reduced (interface)
 *     system                                                     (Sec. 7.2, Eq. cms_boundary,
 *                                                                 Eq. global_subspace, Eq. dd)
 *   - the elasticity of Eq. energy with per-element gamma_s, gamma_v >= 0
 *                                                                (Sec. 6, Eq. energy, Eq. elasticity_fit)
 *
 * Conventions shared by every entry point
 *   - Status: every function returns pd_status (0 = PD_OK, < 0 = error).
 *     No function aborts, prints, or traps the device.  pd_last_error()
 *     returns a text description of the most recent error of the calling
 *     thread.
 *   - Memory: arguments marked [host] are read or written on the host
 *     before the call returns.  Arguments marked [device] are CUDA device
 *     pointers on the current device, accessed in stream order on the
 *     mesh's stream; the caller keeps them alive until that work is done.
 *     The caller owns every buffer it passes; the library owns everything
 *     it derives (matrices, factors, orderings, scratch).
 *   - Vertex arrays are n_v x 3 float (x, y, z per vertex, row-major) in the
 *     caller's vertex order.  Pinned-vertex arrays list the pinned vertices
 *     in increasing vertex id.
 *   - Calls on one mesh are stream-ordered and asynchronous; a device-side
 *     error (non-finite state, failed factorisation) is reported by the next
 *     pd_sync().
 *   - A mesh object is not thread-safe: one host thread at a time.
 */
#ifndef PD_GB300_H
#define PD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pd_status;

enum {
    PD_OK = 0,
    PD_ERR_INVALID_ARG = -1,      /* null pointer, size out of range, bad option */
    PD_ERR_BAD_MESH = -2,         /* index out of range, repeated corner, rest volume <= 0, isolated vertex */
    PD_ERR_BAD_MATERIAL = -3,     /* gamma < 0 or non-finite (Sec. 6: gamma >= 0) */
    PD_ERR_NOT_PREFACTORED = -4,  /* pd_step before pd_prefactor, or after pd_set_materials */
    PD_ERR_NOT_SPD = -5,          /* a Cholesky pivot was <= 0 during pd_prefactor */
    PD_ERR_NO_MEMORY = -6,        /* device or host allocation failed */
    PD_ERR_NONFINITE = -7,        /* NaN/Inf found in the state (device flag) */
    PD_ERR_TIMEOUT = -8,          /* a bounded wait expired */
    PD_ERR_CUDA = -9,             /* any other CUDA runtime error */
    PD_ERR_UNSUPPORTED = -10      /* option not available in this build */
};

/* Arithmetic of the per-iteration dense products of the subspace solve. */
enum {
    PD_PREC_FP32 = 0,   /* FP32 storage, FP32 accumulation */
    PD_PREC_BF16 = 1,   /* BF16 storage, FP32 accumulation (FP64-residual refinement advised) */
    PD_PREC_TF32 = 2    /* TF32-rounded storage, FP32 accumulation */
};

/* pd_solver_opts.flags */
enum {
    /* Solve each PD iteration's global step for the correction: r = b - K x_k
     * with FP64 accumulation, x_{k+1} = x_k + S(r) where S is the subspace
     * solve in the chosen precision.  Equal to x_{k+1} = S(b) in exact
     * arithmetic; with low-precision matrices the error only scales the small
     * correction, so PD's own iterations act as iterative refinement. */
    PD_SOLVE_CORRECTION = 1,
    /* Solve the interface system with one dense S^-1 even when the mesh has
     * enough domains for the two-level interface solve (groups of domains
     * condensed onto a top-level interface first; chosen automatically). */
    PD_SOLVE_SINGLE_LEVEL = 2,
    /* Run the whole subspace solve as one cooperative persistent launch that
     * streams every factor through shared memory with bulk asynchronous copies
     * (phases separated by bounded grid-wide counters).  Same results up to
     * FP32 summation order; off by default (the separate launches are faster
     * on the meshes measured so far). */
    PD_SOLVE_STREAMING = 4,
    /* The paper's own global step (Sec. 7.2 and its solver set-up): per domain
     * only the `modes` fixed-interface normal modes of K_ii with the smallest
     * eigenvalues (besides the exact boundary modes), then `jacobi_sweeps`
     * full-space Jacobi sweeps with Chebyshev weights.  Approximate: the error
     * falls with the sweeps.  Not with PD_SOLVE_STREAMING. */
    PD_SOLVE_MODAL = 8
};

typedef struct pd_solver_opts {
    int32_t precision;     /* PD_PREC_*; default PD_PREC_FP32 */
    int32_t refine_steps;  /* 0..2 extra refinement steps per PD iteration with an FP64 residual r = b - K x */
    int32_t use_graphs;    /* 1: replay each frame as a captured CUDA graph (default), 0: plain launches */
    int32_t flags;         /* PD_SOLVE_* bits; 0 = direct solve x = S(b) */
    int32_t modes;         /* PD_SOLVE_MODAL: normal modes per domain (1..64; 0 = 20) */
    int32_t jacobi_sweeps; /* PD_SOLVE_MODAL: Chebyshev-Jacobi sweeps after the subspace solve (0..1000) */
    double jacobi_rho;     /* PD_SOLVE_MODAL: spectral radius of I - D^-1 K for the Chebyshev
                              weights (0 < rho < 1), or <= 0: estimated by power iteration */
} pd_solver_opts;

typedef struct pd_mesh pd_mesh;   /* opaque, library-owned */

typedef struct pd_mesh_info {
    int32_t n_vertices, n_tets, n_domains, n_pinned;
    int32_t n_interface;           /* vertices shared by two or more domains (not pinned) */
    int32_t n_internal;            /* sum over domains of internal (non-interface, non-pinned) vertices */
    int32_t max_domain_internal;   /* largest per-domain internal vertex count */
    int32_t max_domain_boundary;   /* largest per-domain boundary-mode count */
    int64_t device_bytes;          /* device memory held by the mesh */
    double prefactor_seconds;      /* wall time of the last pd_prefactor */
    int32_t launches_per_iter;     /* kernels launched per PD iteration (after pd_prefactor) */
    int32_t launches_per_frame;    /* kernels launched per frame besides the iterations (pin copy, inertia, velocity) */
    int64_t phase_bytes[24];       /* algorithmic bytes moved by one launch of each phase (pd_phase_name order) */
    int32_t n_groups;              /* domain groups of the two-level interface solve (0 = single level) */
    int32_t n_top_interface;       /* interface vertices shared by two or more groups */
    int32_t two_level;             /* 1 when the last pd_prefactor built the two-level interface solve */
    int32_t phase_launches[24];    /* launches of each phase per PD iteration (per frame for the phases
                                      outside the loop); phase_bytes and pd_phase_times are per launch */
} pd_mesh_info;

/*
 * pd_create_mesh -- build a mesh object from rest geometry (Sec. 4: tet mesh;
 * Sec. 7.2: element-based partition into domains).
 *   rest_xyz    [host]  n_v x 3 double rest positions.
 *   tets        [host]  n_t x 4 int32 vertex ids (any orientation; the rest
 *                       volume |det Dm|/6 must be > 0).
 *   vertex_mass [host]  n_v double lumped masses, or NULL: then
 *                       m_v = sum over incident tets of density * V_e / 4.
 *   tet_domain  [host]  n_t int32 domain ids in [0, n_domains), or NULL:
 *                       then tets are split into n_domains slabs along the
 *                       longest axis of the rest bounding box.
 *   pinned      [host]  n_v uint8, nonzero = Dirichlet vertex, or NULL.
 *   cuda_stream         cudaStream_t used for all work on this mesh (NULL =
 *                       legacy default stream).
 *   out         [host]  receives the new mesh.
 * Vertices touching tets of two or more domains become interface vertices;
 * the others are internal to their domain.  Errors: INVALID_ARG, BAD_MESH,
 * NO_MEMORY, CUDA.  On error *out is NULL and nothing is leaked.
 */
pd_status pd_create_mesh(const double* rest_xyz, int32_t n_v, const int32_t* tets, int32_t n_t,
                         const double* vertex_mass, double density, const int32_t* tet_domain,
                         int32_t n_domains, const uint8_t* pinned, void* cuda_stream, pd_mesh** out);

/* Release every resource of the mesh (synchronises its stream first).  NULL is ignored. */
void pd_destroy_mesh(pd_mesh* mesh);

/*
 * pd_set_materials -- per-element parameters gamma_s (strain) and gamma_v
 * (volume) of Eq. energy (Sec. 6); n_t floats each, in the caller's tet
 * order; host or device pointers (detected).  Values must be finite and
 * >= 0 (Sec. 6, constraint of Eq. elasticity_fit), else BAD_MATERIAL and
 * nothing changes.  Invalidates the prefactorisation.
 */
pd_status pd_set_materials(pd_mesh* mesh, const float* gamma_s, const float* gamma_v);

/*
 * pd_prefactor -- assemble K = M/dt^2 + sum_e V_e (gs+gv) B^T (D^T:D) B
 * (Sec. 7.1) and precompute the subspace solve on the device in FP64
 * (Sec. 7.2): per domain the Cholesky factor of K_ii, K_ii^-1 and the
 * boundary modes Psi = -K_ii^-1 K_ib (Eq. cms_boundary); the reduced
 * interface matrix S = K_BB + sum_d K_bi Psi and its inverse; then the
 * per-iteration copies in the requested precision.
 *   dt    time step (> 0).
 *   opts  [host] or NULL for defaults.
 * Synchronous.  Errors: NOT_SPD, NO_MEMORY, INVALID_ARG, UNSUPPORTED, CUDA.
 */
pd_status pd_prefactor(pd_mesh* mesh, double dt, const pd_solver_opts* opts);

/* Set / read positions and velocities (n_v x 3 float each, [device]; either may be NULL to skip). */
pd_status pd_set_state(pd_mesh* mesh, const float* x, const float* v);
pd_status pd_get_state(pd_mesh* mesh, float* x, float* v);

/*
 * pd_step -- one implicit-Euler frame (Sec. 7): y = x* + dt v* + dt^2 g,
 * x^0 = y, then n_iter PD iterations (local step, RHS assembly, subspace
 * global solve), then v = (x - x*)/dt.
 *   pin_targets [device] n_pinned x 3 float positions of the pinned
 *               vertices at the end of the frame, or NULL to hold them.
 *   gravity     [host]   3 floats (m/s^2), or NULL for (0, 0, -9.81).
 *   n_iter      PD iterations (1..1000).
 *   x_out       [device] n_v x 3 float, receives the new positions, or NULL.
 * Asynchronous on the mesh stream.  Errors: NOT_PREFACTORED, INVALID_ARG, CUDA.
 */
pd_status pd_step(pd_mesh* mesh, const float* pin_targets, const float* gravity, int32_t n_iter,
                  float* x_out);

/* Wait for the mesh stream; report and clear device-side error flags (NONFINITE, NOT_SPD). */
pd_status pd_sync(pd_mesh* mesh);

/* Sizes and memory of the mesh ([host] out). */
pd_status pd_get_info(pd_mesh* mesh, pd_mesh_info* out);

/* Text for a status code (static storage). */
const char* pd_status_string(pd_status status);

/* Description of the last error on the calling thread (static thread-local storage). */
const char* pd_last_error(void);

/* ---- Diagnostics: single phases of the step, for parity checks ---- */

/*
 * pd_project -- the local-step projections alone (Sec. 7.1, Eq. pd_local,
 * Eq. vol_pre) on n deformation gradients.
 *   F      [device] n x 9 float, row-major 3x3.
 *   R, V   [device] n x 9 float outputs (either may be NULL): nearest
 *          rotation and nearest unit-determinant matrix with every target
 *          singular value >= 0.01.
 *   sigma  [device] n x 3 float signed singular values (descending
 *          magnitude, last one carries sign(det F)), or NULL.
 *   stream cudaStream_t.
 */
pd_status pd_project(const float* F, int32_t n, float* R, float* V, float* sigma, void* stream);

/*
 * pd_local_rhs -- local step plus RHS assembly at positions x with inertial
 * target y (both [device] n_v x 3): b = (M/dt^2) y + sum_e V_e B^T D^T :
 * (gs R + gv V) - K_fp x_p for free vertices (Sec. 7.1, b); rows of pinned
 * vertices are set to 0.  b [device] n_v x 3.  Requires pd_prefactor.
 */
pd_status pd_local_rhs(pd_mesh* mesh, const float* x, const float* y, float* b);

/*
 * pd_solve -- the subspace global solve alone (Sec. 7.2): x_f = K_ff^-1 r_f
 * for the free vertices; rows of pinned vertices of x are set to 0.
 * r, x [device] n_v x 3 (may not alias).  Requires pd_prefactor.
 */
pd_status pd_solve(pd_mesh* mesh, const float* r, float* x);

/*
 * pd_phase_times -- mean device time per launch (ms) of each kernel class
 * during the last frame replayed with timing enabled (see
 * pd_enable_timing); out[k] for k < n_out, in the order named by
 * pd_phase_name(k).  Returns the number of phases in *n_phases.
 */
pd_status pd_enable_timing(pd_mesh* mesh, int32_t enable);
/*
 * pd_set_timing_iteration -- restrict the events of the kernel classes that
 * run inside the PD iteration loop (local step, solve phases, residual) to
 * iteration `iteration` of every frame (0-based; -1, the default: every
 * iteration).  One event pair per frame instead of one per iteration keeps
 * the timing's own cost out of the frame time; pd_phase_times then averages
 * the sampled launches.  Kernels outside the loop (inertia, velocity) are
 * timed in every frame.  Errors: INVALID_ARG (iteration < -1).
 */
pd_status pd_set_timing_iteration(pd_mesh* mesh, int32_t iteration);
pd_status pd_phase_times(pd_mesh* mesh, float* out, int32_t n_out, int32_t* n_phases);
const char* pd_phase_name(int32_t k);

/*
 * pd_test_offset_phase_counter -- testing hook for failure detection (no
 * counterpart in the paper).  Adds `delta` to the completion counter of
 * phase `phase` of the streaming solve (PD_SOLVE_STREAMING), so that the
 * next solve's wait on that phase can never be satisfied: the wait runs out
 * after its iteration limit, the launch finishes without a fault, and the
 * next pd_sync returns PD_ERR_TIMEOUT (and clears the counters, leaving the
 * mesh usable).  Errors: INVALID_ARG (no streaming plan, phase out of range).
 */
pd_status pd_test_offset_phase_counter(pd_mesh* mesh, int32_t phase, int32_t delta);

/*
 * Test hook for the bounded waits of the tile-streaming products (failure
 * detection without a fault): the next tile stream to start (block 0, first
 * stage) expects `bytes` more than its bulk copy delivers, so the consumers'
 * wait for that stage runs out after 1 s; the launch drains its copies and
 * ends, and the next pd_sync returns PD_ERR_TIMEOUT (the flags are cleared,
 * the mesh stays usable; the state of that frame is not meaningful).
 * bytes: a non-negative multiple of 16 (0 cancels).  Synchronous.
 * Errors: INVALID_ARG (no tiled products: streaming solve, or bad bytes).
 */
pd_status pd_test_inflate_copy(pd_mesh* mesh, int32_t bytes);

/* ---- Differentiation: equilibrium steps and the adjoint step (Sec. 6.1) ---- */

typedef struct pd_adjoint pd_adjoint;   /* opaque workspace: CG vectors and the adjoint states */

/*
 * pd_adjoint_create -- workspace for pd_equilibrium_step / pd_adjoint_step on
 * one mesh.  cg_iters (1..500): preconditioned-CG iterations per linear
 * solve with the true Hessian H = M/dt^2 + sum_e d^2E_e/dx^2 (Sec. 6.1,
 * Eq. adjoint_state_solve); the preconditioner is the mesh's subspace solve
 * of the PD matrix K.  The workspace holds lambda_{n+1}, lambda_{n+2}
 * (zero after creation and after pd_adjoint_reset).
 */
pd_status pd_adjoint_create(pd_mesh* mesh, int32_t cg_iters, pd_adjoint** out);
void pd_adjoint_destroy(pd_adjoint* adj);
pd_status pd_adjoint_reset(pd_adjoint* adj);

/*
 * pd_equilibrium_step -- one time step solved to equilibrium (Eq. g):
 * n_pd_iter PD iterations as pd_step, then n_newton (0..50) Newton steps
 * H dx = -g(x), g = (M/dt^2)(x - y) + grad E(x), with g evaluated in FP64
 * at the workspace's FP64 state (see pd_adjoint_get_state64) and dx by FP32
 * PCG.  Same arguments as pd_step; the mesh state (x, v) advances.
 * Asynchronous.
 */
pd_status pd_equilibrium_step(pd_mesh* mesh, pd_adjoint* adj, const float* pin_targets, const float* gravity,
                              int32_t n_pd_iter, int32_t n_newton, float* x_out);

/*
 * pd_adjoint_step -- one backward step of the adjoint recurrence for a loss
 * L(x_1..x_N) over equilibrium steps (Sec. 6.1, Eq. adjoint_state and
 * Eq. adjoint_state_solve, chained in time because x_n enters the inertial
 * targets of steps n+1 and n+2):
 *   H(x_n) lambda_n = dL/dx_n + (M/dt^2)(2 lambda_{n+1} - lambda_{n+2}),
 *   dL/dgamma^s_e -= V_e <F_e - R(F_e), sum_c lambda_c (outer) g_c>,
 *   dL/dgamma^v_e -= V_e <F_e - V(F_e), sum_c lambda_c (outer) g_c>.
 * Call for n = N, N-1, ..., 1 after pd_adjoint_reset.
 *   x_n          [device] n_v x 3 equilibrium positions of step n.
 *   dL_dx        [device] n_v x 3 partial derivative of L with respect to x_n
 *                (rows of pinned vertices are ignored).
 *   dL_dgamma_s, dL_dgamma_v [device] n_t floats, caller's tet order,
 *                accumulated (the caller zeroes them before step N).
 * Asynchronous.  Errors: INVALID_ARG, NOT_PREFACTORED, CUDA.
 */
pd_status pd_adjoint_step(pd_mesh* mesh, pd_adjoint* adj, const float* x_n, const float* dL_dx,
                          float* dL_dgamma_s, float* dL_dgamma_v);

/*
 * pd_adjoint_step64 -- pd_adjoint_step at an FP64 state x_n ([device]
 * n_v x 3 double, caller's vertex order), as pd_adjoint_get_state64 gives
 * it after the equilibrium step n.  Both entry points form every per-tet
 * term in FP64 (F, its SVD, R(F), V(F), the stress derivative and
 * V_e <F - P(F), Lambda_e>) and refine the FP32 PCG solution of the adjoint
 * state once with an FP64 residual rhs - H(x_n) lambda_n: at strains of
 * 1e-3 the FP32 rounding of F - R(F) alone would cost 1e-4 relative in the
 * gradient.  pd_adjoint_step rounds nothing further but starts from its
 * FP32 x_n.  Asynchronous.  Errors: INVALID_ARG, NOT_PREFACTORED, CUDA.
 */
pd_status pd_adjoint_step64(pd_mesh* mesh, pd_adjoint* adj, const double* x_n, const float* dL_dx,
                            float* dL_dgamma_s, float* dL_dgamma_v);

/*
 * FP64 state of the equilibrium steps.  pd_equilibrium_step keeps the
 * mesh's positions and velocities in FP64 inside the workspace: its Newton
 * steps evaluate the residual g of Eq. g in FP64 at that state and add FP32
 * PCG corrections to it (iterative refinement), so the equilibrium is met
 * to FP64 accuracy; the mesh's FP32 state is its rounding.  The FP64 state
 * follows the FP32 one whenever that changed by other means (pd_set_state,
 * pd_step).  get: [device] n_v x 3 double out (either may be NULL);
 * set: [device] n_v x 3 double in, also sets the mesh's FP32 state (a
 * checkpoint restored this way continues bitwise as the original run).
 * Asynchronous.  Errors: INVALID_ARG, CUDA.
 */
pd_status pd_adjoint_get_state64(pd_adjoint* adj, double* x, double* v);
pd_status pd_adjoint_set_state64(pd_adjoint* adj, const double* x, const double* v);

/* Diagnostics: H(x) v with v = 0 on pinned vertices (rows of pinned vertices
 * of Hv are 0), and the equilibrium residual g(x) of Eq. g for the step that
 * started at (x_prev, v_prev).  All [device] n_v x 3.  Synchronous. */
pd_status pd_hessian_vec(pd_mesh* mesh, const float* x, const float* v, float* Hv);
pd_status pd_residual(pd_mesh* mesh, const float* x, const float* x_prev, const float* v_prev,
                      const float* gravity, float* g);

/* ---- Material fitting: adjoint Gauss-Newton (Sec. 6.2) and its loop (Sec. 6.3) ----
 *
 * One sample pose is fitted at a time.  It starts from a known state
 * (x_prev, v_prev), so its inertial target y is known and the equilibrium
 * constraint of Eq. g is g(x, gamma) = (M/dt^2)(x - y) + grad E(x; gamma) = 0
 * (what pd_equilibrium_step solves).  Its loss is the misfit
 * eps = sum over free vertices of ||x - xhat||^2, so G = d^2 eps/dx^2 = 2 I.
 *
 * Parameter vectors hold 2 n_t floats, gamma = [gamma_s | gamma_v]: gamma_s
 * of every tet, then gamma_v of every tet, in the caller's tet order (the
 * 2 n_E material vector of Sec. 6).  Activity masks are 2 n_t uint8 in the
 * same layout: nonzero = the parameter takes part, zero = pivoted (removed
 * from the Gauss-Newton solve, Sec. 6.3).
 */

/*
 * pd_pose_misfit -- eps and d eps/dx = 2 (x - xhat) (0 on pinned vertices).
 *   x, target [device] n_v x 3.   dL_dx [device] n_v x 3 out, or NULL.
 *   loss      [device] one double out.
 * Asynchronous.  Errors: INVALID_ARG.
 */
pd_status pd_pose_misfit(pd_mesh* mesh, const float* x, const float* target, float* dL_dx, double* loss);

/*
 * pd_pose_misfit_accumulate -- as pd_pose_misfit, but *loss += eps: the
 * trajectory loss L = sum_n sum_free ||x_n - xhat_n||^2 of the adjoint
 * gradient (Sec. 6.1, the pose-matching objective over a sequence of
 * poses) summed on the device over the steps.  Asynchronous.  Errors: INVALID_ARG.
 */
pd_status pd_pose_misfit_accumulate(pd_mesh* mesh, const float* x, const float* target, float* dL_dx,
                                    double* loss);

/*
 * pd_tied_gradient -- the gradient for one stiffness parameter per element
 * with the volume weight tied to it (gamma_s = theta, gamma_v = ratio theta;
 * Sec. 6's per-element gamma with a fixed volume-to-strain ratio):
 * dL/dtheta = scale (dL/dgamma_s + ratio dL/dgamma_v), evaluated in FP64.
 *   dL_dgamma_s, dL_dgamma_v [device] n_t floats (as pd_adjoint_step gives them).
 *   scale     [device] one double (e.g. the incoming gradient of a composite
 *             loss), or NULL for 1.
 *   dL_dtheta [device] n_t floats out.
 * Asynchronous on the mesh stream.  Errors: INVALID_ARG.
 */
pd_status pd_tied_gradient(pd_mesh* mesh, const float* dL_dgamma_s, const float* dL_dgamma_v, double ratio,
                           const double* scale, float* dL_dtheta);

/*
 * pd_gn_product -- P v, P = J^T G J with J = dx/dgamma = -H^-1 B
 * (Eq. pxpgamma; H = dg/dx, B = dg/dgamma) and G = g_scale I: the matrix of
 * Eq. gn, applied through the eliminated block system of Eq. agn:
 * mu = H^-1 B v, nu = H^-1 G mu, P v = B^T nu, the two solves by
 * preconditioned CG with the workspace's cg_iters (the rows of each solve
 * are scaled to unit norm first, so that no FP32 vector underflows).
 *   x      [device] n_v x 3 equilibrium positions of the pose.
 *   v, Pv  [device] 2 n_t.  active [device] 2 n_t or NULL (all active):
 *          inactive entries of v are ignored and those of Pv are 0.
 * Asynchronous.  Errors: INVALID_ARG, NOT_PREFACTORED, CUDA.
 */
pd_status pd_gn_product(pd_mesh* mesh, pd_adjoint* adj, const float* x, const float* v, const uint8_t* active,
                        float g_scale, float* Pv);

/*
 * pd_gn_direction -- the Gauss-Newton direction of Eq. gn with the
 * Levenberg-Marquardt shift, (P + kappa I) d = -grad on the active
 * parameters and d = 0 on the rest, by outer_iters CG iterations over the
 * parameters (one pd_gn_product each).  kappa = kappa_rel g^T P g / g^T g
 * with g = grad on the active set (the curvature along the gradient),
 * evaluated on the device in the first iteration.
 *   x         [device] n_v x 3 equilibrium positions.
 *   grad      [device] 2 n_t, d eps/d gamma (pd_adjoint_step gives it).
 *   active    [device] 2 n_t or NULL.
 *   d         [device] 2 n_t out.   kappa_out [device] one double, or NULL.
 * Asynchronous.  Errors: INVALID_ARG (outer_iters outside 1..1000,
 * kappa_rel < 0 or not finite), NOT_PREFACTORED, CUDA.
 */
pd_status pd_gn_direction(pd_mesh* mesh, pd_adjoint* adj, const float* x, const float* grad, const uint8_t* active,
                          double kappa_rel, float g_scale, int32_t outer_iters, float* d, double* kappa_out);

typedef struct pd_fit_opts {
    int32_t n_gd;          /* gradient-descent iterations first (Sec. 6.3 uses 10-15) */
    int32_t n_gn;          /* Gauss-Newton iterations after them (20-30) */
    float gd_step;         /* initial GD step (0.01): the GD direction -grad is scaled so that
                              max_j |d_j| / gamma_j = 1, so a step moves no parameter by more
                              than that fraction of its value */
    float gn_step;         /* initial GN step (1.0) */
    double kappa_rel;      /* Levenberg-Marquardt shift, relative as in pd_gn_direction */
    float floor;           /* value given to a parameter pushed below zero (1e-3) */
    int32_t max_halvings;  /* step halvings of one line search (12) */
    int32_t max_pivots;    /* pivots added in one iteration (8) */
    int32_t n_pd_iter;     /* PD iterations of each equilibrium solve */
    int32_t n_newton;      /* Newton steps after them (Sec. 8: three to five) */
    int32_t outer_iters;   /* CG iterations of each Gauss-Newton direction */
    double dt;             /* time step (> 0) */
    const pd_solver_opts* solver;  /* pd_prefactor options after each material change (NULL = defaults) */
} pd_fit_opts;

typedef struct pd_fit_report {
    int32_t iterations;    /* iterations whose line search lowered the loss */
    int32_t trials;        /* equilibrium solves of the line searches */
    int32_t clamped;       /* parameters cached as clamped at the end */
    int32_t pivots;        /* parameters pivoted at the end */
    double loss0, loss;    /* pose loss before and after */
    double seconds;        /* wall time */
} pd_fit_report;

/*
 * pd_fit_pose -- the two-stage fitting loop of Sec. 6.3 on one pose: n_gd
 * gradient-descent iterations, then n_gn Gauss-Newton iterations.  Each
 * iteration: gradient by the adjoint (pd_adjoint_step); direction; a cached
 * (clamped) parameter may not decrease (its component is zeroed); a
 * Gauss-Newton direction that is then not a descent direction pivots the
 * cached parameter at the floor whose tentative value gamma_j + d_j is most
 * negative and is recomputed without it (at most max_pivots times); line
 * search from the initial step, halving until the loss decreases; a
 * negative component of the accepted step is set to the floor and cached.
 * Every trial re-assembles and re-factors the PD matrix (pd_set_materials,
 * pd_prefactor) and solves the pose to equilibrium (pd_set_state(x_prev,
 * v_prev), pd_equilibrium_step).  The loop stops early when a line search
 * fails.  On return the mesh holds the fitted materials, prefactored.
 *   x_prev, v_prev [device] n_v x 3 state the pose starts from.
 *   pin_targets    [device] n_pinned x 3, or NULL.   gravity [host] 3 floats or NULL.
 *   target         [device] n_v x 3 pose to match.
 *   gamma          [device] 2 n_t, in: initial materials, out: fitted.
 *   losses         [host] n_gd + n_gn + 1 doubles, or NULL: the loss before the
 *                  loop and after each iteration (repeated after an early stop).
 *   report         [host] or NULL.
 * Synchronous.  Errors: INVALID_ARG, BAD_MATERIAL, NOT_SPD, NONFINITE, CUDA.
 */
pd_status pd_fit_pose(pd_mesh* mesh, pd_adjoint* adj, const pd_fit_opts* opts, const float* x_prev,
                      const float* v_prev, const float* pin_targets, const float* gravity, const float* target,
                      float* gamma, double* losses, pd_fit_report* report);

/*
 * pd_harmonic_basis -- harmonic material basis (Sec. 6, Harmonic
 * Initialization): the r lowest eigenpairs of the graph Laplacian L = D - A
 * of the tets' face adjacency (two tets are adjacent when they share a face),
 * by Chebyshev-filtered subspace iteration in FP64 on the device (block of
 * r + 8 vectors; the polynomial degree adapts to the ratio of the block's
 * largest Ritz value to the bound 2 max-degree of lambda_max; until every
 * residual |L h - lambda h| <= 1e-9 times that bound).
 *   r          1 .. min(56, n_t).
 *   H          [device] n_t x r float, column-major in the caller's tet order
 *              (column k = h_{k+1}, n_t contiguous floats); orthonormal; the
 *              entry of largest magnitude of each column is positive, so h_1
 *              is the constant 1/sqrt(n_t) on a connected mesh.
 *   lambda     [host] r doubles, ascending, or NULL.
 *   iterations [host] filter iterations used, or NULL.
 * Synchronous.  Errors: INVALID_ARG, NOT_SPD (the block lost rank), TIMEOUT
 * (not converged in 500 iterations), CUDA.
 */
pd_status pd_harmonic_basis(pd_mesh* mesh, int32_t r, float* H, double* lambda, int32_t* iterations);

/*
 * pd_fit_pose_reduced -- Gauss-Newton iterations of one pose in the reduced
 * coordinates q of gamma = diag(H, H) q (Eq. q2gamma): q starts as
 * diag(H, H)^T gamma; each iteration forms P_q = D^T P D (2 r products
 * pd_gn_product) and grad_q = D^T grad, solves (P_q + kappa I) d_q = -grad_q
 * (kappa relative as in pd_gn_direction; the 2r x 2r system is solved on
 * the host), and line-searches q + alpha d_q from gn_step with halving; a
 * trial whose gamma has a component below `floor` is rejected (gamma stays
 * in the span of H).  Uses n_gn, gn_step, kappa_rel, floor, max_halvings,
 * n_pd_iter, n_newton, dt, solver of opts (n_gd, max_pivots, outer_iters,
 * gd_step are not used).
 *   H       [device] n_t x r, as written by pd_harmonic_basis (any
 *           orthonormal columns work).
 *   gamma   [device] 2 n_t, in: the guess, out: D q.
 *   other arguments as pd_fit_pose.
 * Synchronous.  Errors: INVALID_ARG, BAD_MATERIAL (the projected guess has a
 * component below the floor), NOT_SPD, NONFINITE, CUDA.
 */
pd_status pd_fit_pose_reduced(pd_mesh* mesh, pd_adjoint* adj, const pd_fit_opts* opts, const float* H, int32_t r,
                              const float* x_prev, const float* v_prev, const float* pin_targets, const float* gravity,
                              const float* target, float* gamma, double* losses, pd_fit_report* report);

/* ---- Serving: many garment simulations resident on one GPU ---- */

typedef struct pd_server pd_server;   /* opaque */
typedef int64_t pd_request_id;

enum { PD_REQ_QUEUED = 0, PD_REQ_ACTIVE = 1, PD_REQ_DONE = 2, PD_REQ_FAILED = 3 };

/* One simulation request.  Arrays are [host] and copied by pd_submit. */
typedef struct pd_request {
    const double* rest_xyz;  int32_t n_v;        /* as pd_create_mesh */
    const int32_t* tets;     int32_t n_t;
    const int32_t* tet_domain; int32_t n_domains;
    const uint8_t* pinned;                      /* or NULL */
    const float* gamma_s;    const float* gamma_v;   /* per tet, >= 0 (Sec. 6) */
    double density, dt;
    int32_t n_frames;                           /* frames to advance, >= 1 */
    float gravity[3];
    /* pinned targets at time t: rest + drive_amp * sin(2 pi drive_freq t) along drive_axis (0, 1, 2) */
    float drive_amp, drive_freq;
    int32_t drive_axis;
} pd_request;

/*
 * pd_server_create -- a serving loop with continuous batching.
 * hbm_budget_bytes caps the device memory of resident requests (their steady
 * footprint plus the transient FP64 prefactorisation of the one being
 * admitted); max_slots caps how many are resident; n_iter is the PD
 * iteration count of every frame.  Admission threads of the server build
 * and prefactor queued requests, each on its own stream of the device's
 * lowest priority, while the resident ones keep advancing; the first of them
 * also frees the meshes of retired requests.  Requests are prefactored in
 * FP32, with the two-level interface solve where pd_prefactor chooses it and
 * every row of its row-form blocks fits one bulk-copy stage (else one
 * level).  The frames run on a stream of
 * the server's own at the device's highest priority (ahead of admission work
 * whenever an SM frees up).  Requests and results are host arrays, so the
 * frames need no ordering with the caller's work; if cuda_stream is not
 * NULL, every pd_server_tick is still ordered after the work queued on it
 * before the call (NULL, the legacy default stream, is not waited on).
 */
pd_status pd_server_create(int64_t hbm_budget_bytes, int32_t max_slots, int32_t n_iter, void* cuda_stream,
                           pd_server** out);
/* Stops the admission thread and releases every request and resource. */
void pd_server_destroy(pd_server* server);

/* Queue a request (host copy of its arrays); returns its id.  Admission runs in the background. */
pd_status pd_submit(pd_server* server, const pd_request* request, pd_request_id* id);

/*
 * pd_server_tick -- retire requests that finished (their meshes are freed by
 * the admission thread), let the requests it has prepared join the batch,
 * then advance every resident request by one frame in shared batched launches
 * (one captured CUDA graph per set of resident requests; the local steps,
 * assemblies and subspace solves of all requests run in the same kernels).
 * Admission (in arrival order, while slots and the budget allow) happens
 * meanwhile on the admission thread: a request that does not fit the budget
 * even with nothing resident is marked PD_REQ_FAILED and leaves the queue; one
 * that must wait for resident requests to retire keeps its first memory
 * estimate and is not rebuilt.  When nothing is resident but requests are
 * being prepared, the tick waits up to 5 ms for the first of them.
 * Synchronous; *frame_ms receives the GPU time of the batched frame.
 * Errors: TIMEOUT (a bounded wait of the batched products ran out), CUDA,
 * NO_MEMORY, UNSUPPORTED.
 */
pd_status pd_server_tick(pd_server* server, int32_t* n_active, float* frame_ms);

/*
 * pd_server_run -- pd_server_tick until no request is queued, being
 * prepared or resident, at most max_ticks (>= 1) ticks; *ticks (or NULL)
 * receives the ticks run.  Synchronous.  Errors: INVALID_ARG; TIMEOUT when
 * max_ticks ticks ran and requests are still outstanding; and those of
 * pd_server_tick (the loop stops at the first).
 */
pd_status pd_server_run(pd_server* server, int32_t max_ticks, int32_t* ticks);

pd_status pd_poll(pd_server* server, pd_request_id id, int32_t* state, int32_t* frames_done);
/* Final positions (n_v x 3, [host]) and per-frame latencies (n_frames floats, [host], ms) of a finished
 * request: the wall time from the end of its admission (first frame) or of its previous frame to the end of
 * the frame, so it includes every wait of the request (admissions of others, graph rebuilds, the tick cadence). */
pd_status pd_fetch(pd_server* server, pd_request_id id, float* x_out, float* frame_ms);
pd_status pd_release(pd_server* server, pd_request_id id);
/* Requests waiting for admission (not yet prepared), resident requests (prepared or running), their
 * estimated device bytes, and the largest admission-time estimate (resident + new request + its
 * prefactorisation workspace) seen so far. */
pd_status pd_server_stats(pd_server* server, int32_t* n_queued, int32_t* n_active, int64_t* used_bytes,
                          int64_t* peak_bytes);

/*
 * pd_solve_noalloc -- the same solve as pd_solve (same kernels, same
 * result), for callers that must not allocate device memory during the
 * call: a host that hands every library a fixed memory pool at start-up and
 * forbids cudaMalloc/cudaFree afterwards, or code running where an
 * allocation would stall the device.  The paper has no counterpart; this is
 * a deployment variant of the pd_solve diagnostic.
 *   r, x  [device] n_v x 3 (may not alias), caller-owned as in pd_solve.
 * Every temporary comes from one file-scope device array of 16 MiB
 * (16777216 bytes) that each GPU loading this library holds until the
 * process exits; a mesh whose temporaries exceed it is rejected with
 * PD_ERR_UNSUPPORTED (pd_last_error gives the bytes needed).  The array's
 * device address is looked up (cudaGetSymbolAddress) once per device by
 * pd_prefactor, which is also when the CUDA runtime, loading modules lazily,
 * takes the 16 MiB from that device; after pd_prefactor, pd_solve_noalloc
 * takes no device memory.  (Only a call on a device where no pd_prefactor
 * ran makes the lookup itself; such a call must come before any stream
 * capture.)  All calls share the one array, which
 * keeps the last call's contents (the solution buffer is cleared on entry):
 * calls that overlap on the GPU -- from two host threads, or on two meshes
 * with different streams -- race and must be serialised by the caller.
 * Synchronous.  Errors: INVALID_ARG, NOT_PREFACTORED, UNSUPPORTED, CUDA.
 */
pd_status pd_solve_noalloc(pd_mesh* mesh, const float* r, float* x);

#ifdef __cplusplus
}
#endif

#endif /* PD_GB300_H */
