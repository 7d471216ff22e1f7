/*
 * pp.h -- C ABI of libpp, a single-GPU (sm_103a) implementation of the fully
 * discrete periodic shooting and periodic adjoint method of Zahr, Persson and
 * Wilkening, "A fully discrete adjoint method for optimization of flow problems
 * on deforming domains with time-periodicity constraints".
 *
 * Conventions common to every call
 * --------------------------------
 * - Every function returns PP_OK (0) or a negative status code; the message of
 *   the last failure is available from pp_last_error().  No call aborts, traps
 *   or exits the process.
 * - Arrays documented as DEVICE are CUDA device pointers (e.g. torch
 *   data_ptr()) on the context's device; the caller owns them and the library
 *   never frees them.  Arrays documented as HOST are ordinary host memory.
 *   All floating point arrays are IEEE double (FP64).
 * - State layout ("u layout"): u[(e*4 + a)*Np + i] for element e, conservative
 *   variable a in (rho, rho*u, rho*v, rho*E) and node i; N_u = Ne*4*Np with
 *   Np = (p+1)(p+2)/2.  Nodes are equispaced on the reference triangle
 *   (0,0),(1,0),(0,1), ordered j-major: for j = 0..p, i = 0..p-j, node
 *   (i/p, j/p); element vertex k maps to the k-th corner.
 * - Work is issued on the context's stream; calls that return host values
 *   synchronize that stream before returning.
 * - Each Arnoldi step of the linear solves is one cooperative launch whose CTAs
 *   wait on one another at grid barriers (one CTA per SM, all resident; the
 *   barrier words belong to the context).  Two contexts solving at the same time
 *   on one device compete for the SMs; a barrier wait is bounded (about one
 *   second), after which the call fails with PP_ECUDA instead of hanging.
 * - Nondimensionalization: chord 1, leading edge at the origin, free stream
 *   rho = 1, velocity (1, 0), p = 1/(gamma Mach^2), viscosity 1/Re.
 */
#ifndef PP_H
#define PP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PP_OK 0
#define PP_EINVAL -1      /* invalid argument (sizes, null pointers, bad mesh) */
#define PP_ENOMEM -2      /* device allocation failed */
#define PP_ENOCONV -3     /* an iteration hit its cap before its tolerance */
#define PP_ENAN -4        /* a non-finite value appeared in a norm */
#define PP_EBREAKDOWN -5  /* Krylov breakdown with a nonzero residual */
#define PP_ECUDA -6       /* a CUDA runtime call failed */
#define PP_ESTATE -7      /* call needs a linearization that is not set */

/* arithmetic of the stage linear solves */
#define PP_PREC_FP64 0   /* FP64 block Jacobians, preconditioner and Krylov vectors throughout */
#define PP_PREC_MIXED 1  /* FP32 copies of the block Jacobians and FP32 block-Jacobi inverses: the
                            primal Newton steps are solved by FP32 GMRES (the Newton residual stays
                            FP64); tangent / adjoint stage solves are FP64 flexible GMRES on the exact
                            FP64 operator, preconditioned by a short FP32 GMRES */

/* motion parametrizations (mu) -- Sec. 6.1 single-Fourier-mode motion */
#define PP_KIN_HEAVE_PITCH 0 /* mu = (h0, theta0, phi): h = h0 sin(wt), theta = theta0 sin(wt + phi) */
#define PP_KIN_FOURIER6 1    /* mu = (a1, b1, a2, al1, be1, al2): h = a1 sin wt + b1 cos wt + a2 sin 2wt,
                                theta = al1 sin wt + be1 cos wt + al2 sin 2wt;  w = 2 pi / T */
#define PP_KIN_SPLINE8 2     /* Sec. 6.2, Eq. mirror: mu = (h0, h1, h2, h3, th0, th1, th2, th3), the knots at
                                t = 0, T/8, T/4, 3T/8; h and theta are the periodic cubic splines through the
                                8 equally spaced knots (f0, f1, f2, f3, -f0, -f1, -f2, -f3), so that
                                f(t + T/2) = -f(t) */

typedef struct pp_ctx pp_ctx;
typedef struct pp_mesh pp_mesh;

typedef struct pp_config {
  int p;              /* polynomial degree, 1..4 */
  double gamma;       /* ratio of specific heats (1.4) */
  double Pr;          /* Prandtl number (0.72) */
  double Mach;        /* free-stream Mach number (0.2) */
  double Re;          /* Reynolds number based on chord (1000) */
  double T;           /* period of the motion (5) */
  int kin;            /* PP_KIN_* */
  int device;         /* CUDA device ordinal */
  void* stream;       /* cudaStream_t to issue work on; NULL = the library's own non-blocking
                         stream, which does not wait for work on other streams (including the
                         legacy default stream): device inputs must be complete before a call */
  /* primal stage solves (Newton with GMRES, block-Jacobi preconditioned) */
  double newton_tol;  /* stop when ||dk||_2 <= newton_tol * max(1, ||u_i||_2) */
  int newton_maxit;
  double gmres_rtol;  /* relative tolerance of the Newton-step GMRES */
  int gmres_restart;
  int gmres_maxit;    /* cap on GMRES iterations per linear solve */
  /* tangent and adjoint stage solves (linear, must be tight for exact sensitivities) */
  double lin_rtol;
  /* shooting (Algorithm primal) */
  double nk_gmres_rtol; /* relative tolerance of the shooting GMRES, ||(Phi-I)du - R|| <= rtol ||R|| */
  int nk_restart;
  int nk_max_newton;
  int nk_max_krylov;    /* cap on tangent sweeps per Newton step */
  /* periodic adjoint (Algorithm dual) */
  double adj_tol;     /* absolute tolerance on ||lambda^(0)(x) - x||_2 */
  int adj_restart;
  int adj_maxit;
  /* precision of the stage linear solves (PP_PREC_*) */
  int precision;
  int inner_maxit;    /* PP_PREC_MIXED: FP32 GMRES iterations per preconditioner application */
  double inner_rtol;  /* PP_PREC_MIXED: relative tolerance of that inner solve */
  /* 0: the primal sweep keeps the stage linearization of the whole period in HBM.
     K > 0: it keeps the state and Newton predictor every K steps and one K-step segment
     of stage data; tangent / adjoint sweeps recompute each segment from its checkpoint
     (identical iterates, so identical results) -- memory ~ Nt/K states + 3K stages. */
  int checkpoint_stride;
  /* pp_shoot_nk: m >= 0 steps of Algorithm fixedpt (u0 <- u^(Nt)(u0)) before the Newton
     iterations, the nonlinear preconditioning of Sec. 6.1 (0: none) */
  int nk_fixed_point_pre;
} pp_config;

/* Fills *cfg with the paper's case (Sec. 6.1: gamma 1.4, Pr 0.72, Mach 0.2,
   Re 1000, T = 5, p = 3) and default tolerances. */
void pp_config_default(pp_config* cfg);

/* Creates a context on cfg->device.  The context owns all device workspace,
   including the stored linearization of a period (allocated by the first sweep):
   per stage the stage state, the element block Jacobians, the explicit inverses of
   the stage diagonal blocks and, while 8 GB of device memory stay free, the stage
   operator with the block-Jacobi preconditioner folded in (normal and transposed)
   and transposed Jacobian copies.  About 420 MB per stage for 2048 elements at p = 3
   in FP64; with checkpoint_stride K only one K-step segment of stages is kept.
   One process uses one CUDA device: every context of the process must name the same
   cfg->device (the kernels' launch set-up is cached per process).
   Errors: PP_EINVAL (p out of range, null pointers, a second device), PP_ECUDA. */
int pp_create(const pp_config* cfg, pp_ctx** out);
int pp_destroy(pp_ctx* ctx);
const char* pp_last_error(const pp_ctx* ctx);
const char* pp_version(void);

/* Mesh of straight-sided triangles in the reference configuration (Eq. defmap
   maps it rigidly to the physical domain).  HOST arrays, copied:
   verts [nv][2] coordinates; tris [nt][3] counter-clockwise vertex indices;
   ftag [nt][3] tag of local face f = edge (v_f, v_(f+1)%3): 0 interior,
   1 wall (no-slip airfoil), 2 far field.
   Errors: PP_EINVAL if an index is out of range, an element is inverted or a
   tag contradicts the connectivity (a shared edge must be tagged 0). */
int pp_mesh_create(pp_ctx* ctx, const double* verts, int nv, const int32_t* tris, const int32_t* ftag,
                   int nt, pp_mesh** out);
int pp_mesh_destroy(pp_mesh* mesh);

/* Seeded O-grid around a symmetric 12%-thick 4-digit airfoil (closed trailing edge), the
   synthetic stand-in for the paper's flapping-airfoil mesh (Sec. 6.1; the paper's mesh is
   not published): n_theta wall points equally spaced in arc length counter-clockwise from
   the trailing edge, far-field circle of radius r_far about (0.5, 0), n_r + 1 rings with
   geometric stretching q = 1 + 4/n_r, interior vertices jittered by up to 10% of the
   distance to their nearest grid neighbour with the counter-based SplitMix64 generator
   (output c of seed s: state s + (c + 1) 0x9E3779B97F4A7C15, then the published finalizer;
   u = -1 + 2 (x >> 11) 2^-53), each quad split into two counter-clockwise triangles.
   Vertex (k, j) (wall index k, ring j) has index k (n_r + 1) + j; nv = n_theta (n_r + 1),
   nt = 2 n_theta n_r.  pp_ogrid_generate is host code (no GPU, no context): verts HOST
   [nv][2], tris and ftag HOST [nt][3] (any may be NULL; tags as in pp_mesh_create), nv and nt
   receive the sizes.  pp_mesh_ogrid generates the mesh and creates it on ctx's device.
   Errors: PP_EINVAL (n_theta < 3, n_r < 1, r_far <= 1), and those of pp_mesh_create. */
int pp_ogrid_generate(int n_theta, int n_r, double r_far, uint64_t seed, double* verts, int32_t* tris,
                      int32_t* ftag, int* nv, int* nt);
int pp_mesh_ogrid(pp_ctx* ctx, int n_theta, int n_r, double r_far, uint64_t seed, pp_mesh** out);
/* ne, np (nodes per element) and nu = ne*4*np; any output may be NULL. */
int pp_mesh_info(const pp_mesh* mesh, int* ne, int* np, int64_t* nu);

/* The prescribed motion that enters the rigid map (Eq. defmap): out[0..2] = (theta, theta',
   h') at time t for the kinematics mode kin (PP_KIN_*, Sec. 6.1 single Fourier mode or the
   Sec. 6.2 mirrored splines), then out[3 + 3 j .. 5 + 3 j] = d(theta, theta', h') / d mu_j
   for j < n_mu -- the quantities every sweep and gradient takes from the same code.  Host
   code (no GPU, no context).  mu: HOST [n_mu], n_mu the mode's parameter count (3, 6, 8);
   out: HOST [3 + 3 n_mu].  Errors: PP_EINVAL (unknown mode, wrong n_mu, T <= 0, NULL). */
int pp_motion_eval(int kin, double T, const double* mu, int n_mu, double t, double* out);

/* Semi-discrete residual r(u, mu, t) of M du/dt = r (Eq. semidisc; ALE DG of
   Sec. 6).  u, r: DEVICE [N_u].  mu: HOST [n_mu]. */
int pp_residual(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u,
                double* r);

/* Element block Jacobian dr/du at (u, mu, t): DEVICE blocks [Ne][4][nb][nb]
   with nb = 4*Np, slot 0 = d r_e / d u_e, slot 1+f = d r_e / d u_(neighbour
   across face f) (zero for boundary faces).  Each block is stored COLUMN-major:
   blocks[((e*4 + slot)*nb + col)*nb + row], row/col index (a*Np + i). */
int pp_jacobian_blocks(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t,
                       const double* u, double* blocks);

/* Instantaneous power P^h and x-force F_x^h the fluid exerts on the airfoil
   (Eq. qoi, instantaneous form).  u: DEVICE; out: HOST [2]. */
int pp_qoi_rate(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u,
                double* out);

/* Same result as pp_qoi_rate, but this call allocates no memory: it never calls
   cudaMalloc, cudaFree or an allocating library routine.  It is for callers that may
   not allocate, for example code under an allocator that forbids outside allocations,
   or code that must not allocate after start-up.  (The paper has no counterpart; this
   is a service entry point of the library.)
   - Scratch: one static device array of 1 MiB + 33 KiB per device that loads the library,
     kept until the process exits.  Meshes of more than 65536 elements are rejected with
     PP_EINVAL.
   - First call: the first call on a device looks up the array's device address
     (cudaGetSymbolAddress) with that device current, under a lock, and caches it for the
     life of the process.  Make this first call before any stream capture.  A
     cudaDeviceReset of the device invalidates the cached address (as it invalidates every
     context of this library on that device): do not call this function on that device
     after a reset.
   - Concurrency: every call shares the one array.  Calls that overlap on the GPU, e.g.
     on different streams or from different contexts on the same device, race.  The
     finishing counter is cleared at the start of each call; other contents are
     overwritten.
   - Arguments: as pp_qoi_rate.  u: DEVICE; out: HOST [2] = (P^h, F_x^h). */
int pp_qoi_rate_noalloc(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t, const double* u,
                        double* out);

/* Primal sweep u^(Nt)(u0; mu) over one period (Eq. dirk2) with Nt equal DIRK3
   steps of dt = T/Nt (T from the config).  u0: DEVICE [N_u].  u_traj: DEVICE
   [(Nt+1)][N_u] or NULL.  u_final: DEVICE [N_u] or NULL.  qoi: HOST [4] or NULL:
   (W, J_x, J_E = -W/T, J_T = -J_x/T), W and J_x the solver-consistent
   discrete work and x-impulse (Eqs. qoi, qoi-disc).
   The call stores the linearization (stage states, block Jacobians, block-Jacobi
   inverses, folded stage operators; or state checkpoints, see checkpoint_stride)
   used by pp_tangent_matvec, pp_adjoint_sweep and pp_periodic_adjoint.
   Errors: PP_ENOCONV (stage Newton cap), PP_ENAN, PP_ENOMEM (storage), PP_ECUDA
   (including an expired wait in the shared-memory pipeline of the block-row kernels). */
int pp_primal_period(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                     double* u_traj, double* u_final, double* qoi);

/* out = (I - du^(Nt)/du0) v about the last primal sweep, by one tangent sweep
   (Eqs. dirk-sens-mvp and jac-prim-matvec; the sign is that of I - Phi).
   v, out: DEVICE [N_u] (may alias).  Errors: PP_ESTATE if no sweep is stored. */
int pp_tangent_matvec(pp_ctx* ctx, const double* v, double* out);

/* Backward adjoint sweep lambda^(0)(lambda_Nt) about the last primal sweep
   (Eq. uns-disc-adj-dirk2).  weights: HOST [2] weights (w_W, w_x) of
   F = w_W W + w_x J_x, or NULL for the adjoint sensitivity sweep without QoI
   terms (Eq. uns-disc-adj-dirk-sens-mvp).  lam_Nt, lam0: DEVICE [N_u] (may
   alias).  dFdmu: HOST [n_mu] or NULL: with weights, the reconstruction
   dF/dmu = dF/dmu|explicit + sum_n dt sum_i kappa_i^T dr/dmu
   (Eq. funcl-grad-nosens-dirk) evaluated with this sweep's multipliers. */
int pp_adjoint_sweep(pp_ctx* ctx, const double* lam_Nt, const double* weights, double* lam0, double* dFdmu);

/* Steady flow with the airfoil frozen at its t = 0 pose and the mesh at rest: the
   paper's "steady-state flow" initial guess for shooting (Sec. 6.1).  Pseudo-transient
   continuation from the free stream until ||r(u)||_2 <= tol ||r(u_inf)||_2.
   u: DEVICE [N_u] output.  steps, rel_res: HOST or NULL.  Errors: PP_ENOCONV. */
int pp_steady_state(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double tol, int maxit, double* u,
                    int* steps, double* rel_res);

typedef struct pp_shoot_stats {
  int cold_start;            /* 0 caller's guess, 1 free stream (steady state stalled), 2 steady state */
  int newton_iters;          /* shooting Newton iterations taken */
  int krylov_iters;          /* tangent sweeps (GMRES matvecs) in total */
  int primal_sweeps;
  int stage_newton_iters;    /* summed over all primal stage solves */
  double residual[64];       /* ||u^(Nt)(u0) - u0||_2 per Newton iterate */
  double seconds;
} pp_shoot_stats;

/* Newton-Krylov shooting (Algorithm primal): solves u^(Nt)(u0; mu) = u0 to
   ||u^(Nt)(u0) - u0||_2 <= tol.  u0_guess: DEVICE [N_u] or NULL (NULL = the
   steady flow of pp_steady_state, or the free stream if that stalls; see
   stats->cold_start).  u0_out: DEVICE [N_u] (may alias u0_guess).  qoi: HOST [4] or NULL
   (as in pp_primal_period, at the returned u0).  On return the stored
   linearization is that of the returned u0.  stats: HOST or NULL.
   Errors: PP_ENOCONV (u0_out then holds the last iterate). */
int pp_shoot_nk(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess, int Nt,
                double tol, double* u0_out, double* qoi, pp_shoot_stats* stats);

/* Fixed-point iteration for the periodic initial condition (Algorithm fixedpt): u0 <-
   u^(Nt)(u0) from u0_guess until ||u^(Nt)(u0) - u0||_2 <= tol (Eq. fixedpt); converges when
   the period map is a contraction (all Floquet multipliers inside the unit circle), at the
   rate of the largest multiplier.  u0_guess, u0_out: DEVICE [N_u] (may alias).  qoi: HOST [4]
   or NULL, as in pp_primal_period at the returned u0, whose linearization is stored on
   return.  stats: HOST or NULL (newton_iters = fixed-point iterations, residual history,
   primal_sweeps).  Errors: PP_ENOCONV after maxit iterations (u0_out holds the last iterate),
   PP_ENAN. */
int pp_shoot_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0_guess,
                         int Nt, double tol, int maxit, double* u0_out, double* qoi, pp_shoot_stats* stats);

typedef struct pp_adj_stats {
  int krylov_iters;      /* adjoint sensitivity sweeps in the GMRES */
  double residual;       /* final ||lambda^(0)(lambda_Nt) - lambda_Nt||_2 */
  double seconds;
} pp_adj_stats;

/* Gradient on the manifold of periodic solutions (Algorithms dual and grad).
   If u0 (DEVICE [N_u]) is non-NULL a primal sweep from u0 first sets the
   linearization (u0 should be periodic, e.g. from pp_shoot_nk); if NULL the
   stored linearization is used.  weights: HOST [2] as in pp_adjoint_sweep.
   F: HOST [1] or NULL; dFdmu: HOST [n_mu]; lam_Nt: DEVICE [N_u] or NULL (the
   periodic adjoint final condition).  Tolerance adj_tol from the config. */
int pp_periodic_adjoint(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                        const double* weights, double* F, double* dFdmu, double* lam_Nt, pp_adj_stats* stats);

/* The periodic adjoint problems of n_qoi QoIs (1..4) about one periodic orbit, solved
   together by one restarted block GMRES: the operator Phi^T - I of Algorithm dual does not
   depend on the QoI (Sec. 4), so the right-hand sides -d_q share one block Krylov space and
   each block step applies it to n_qoi vectors.  Then for each QoI the gradient of Algorithm
   grad.  weights: HOST [n_qoi][2], the (w_W, w_x) of each QoI (e.g. (1, 0) and (0, 1) for W
   and J_x).  F: HOST [n_qoi] or NULL; dFdmu: HOST [n_qoi][n_mu]; lam_Nt: DEVICE
   [n_qoi][N_u] or NULL; u0 as in pp_periodic_adjoint.  Tolerance adj_tol on each QoI's
   ||lambda^(0)(x) - x||_2; block steps per restart: 64 / n_qoi - 1, limited by adj_restart
   (adj_restart + 1 >= the basis size).  stats->krylov_iters counts all adjoint sweeps,
   stats->residual is the largest final residual.  Errors: PP_ENOCONV, PP_EINVAL,
   PP_ESTATE, PP_ENOMEM. */
int pp_periodic_adjoint_multi(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0, int Nt,
                              int n_qoi, const double* weights, double* F, double* dFdmu, double* lam_Nt,
                              pp_adj_stats* stats);

/* Batched forms of pp_shoot_nk and pp_periodic_adjoint for n_batch parameter vectors (a
   batch of mu for the derivative of a batched QoI, e.g. through an autograd function).
   mu: HOST [n_batch][n_mu].  Device arrays hold one N_u block per batch entry:
   u0_guess (or NULL), u0_out, u0, lam_Nt (or NULL): DEVICE [n_batch][N_u].  qoi: HOST
   [n_batch][4] or NULL; stats: HOST [n_batch] or NULL; status: HOST [n_batch] or NULL
   (per-entry status of the shooting); weights: HOST [n_batch][2] (one QoI weighting per
   entry); F: HOST [n_batch] or NULL; dFdmu: HOST [n_batch][n_mu].
   The entries run one after the other on the context's stream and reuse its stored
   linearization: each mu needs its own linearization of the whole period (about 126 GB at
   2048 elements, p = 3, 100 steps), so the batch does not fit in device memory at once.
   pp_shoot_nk_batched returns PP_ENOCONV if an entry did not converge (the others still
   run; see status); any other error stops the batch.  On return the stored linearization
   is that of the last entry. */
int pp_shoot_nk_batched(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, int n_batch,
                        const double* u0_guess, int Nt, double tol, double* u0_out, double* qoi, pp_shoot_stats* stats,
                        int* status);
int pp_periodic_adjoint_batched(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, int n_batch,
                                const double* u0, int Nt, const double* weights, double* F, double* dFdmu,
                                double* lam_Nt, pp_adj_stats* stats);

/* Floquet multipliers of the periodic orbit (Sec. 3.3, Eq. stab-def): m steps of Arnoldi
   on Phi = du^(Nt)/du0 about the stored linearization (call pp_shoot_nk first, so that it
   is the periodic orbit's), Phi applied by tangent sweeps (Eq. dirk-sens-mvp), with full
   classical Gram-Schmidt reorthogonalization; the Ritz values of the m x m Hessenberg
   matrix (Francis double-shift QR) approximate the largest-modulus multipliers first.  The
   orbit is stable when every multiplier lies inside the unit circle.  wr, wi: HOST [m],
   real and imaginary parts sorted by modulus, largest first.  hlast: HOST [1] or NULL,
   h_(m+1,m) (0: the Krylov space is invariant and the values are exact).  Allocates an
   (m+1) x N_u device basis for the call.  Errors: PP_ESTATE (no sweep stored), PP_EINVAL
   (m outside [1, N_u]), PP_ENOMEM, PP_ENOCONV (QR iteration cap). */
int pp_floquet(pp_ctx* ctx, int m, double* wr, double* wi, double* hlast);

/* The periodic adjoint condition solved by fixed-point iteration (the dual fixed point of
   Sec. 6.2 on Eq. fixedpt-dual): lambda_Nt <- lambda^(0)(lambda_Nt) from 0 until
   ||lambda^(0)(lambda_Nt) - lambda_Nt||_2 <= tol, then the gradient of Algorithm grad with
   the converged multipliers.  Arguments as pp_periodic_adjoint, plus tol and maxit;
   stats->krylov_iters counts the adjoint sweeps of the iteration.  Errors: PP_ENOCONV,
   PP_ENAN, PP_ESTATE. */
int pp_periodic_adjoint_fixed_point(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, const double* u0,
                                    int Nt, const double* weights, double tol, int maxit, double* F, double* dFdmu,
                                    double* lam_Nt, pp_adj_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* PP_H */
