/*
 * seird.h -- C ABI of the GB300 backward-Euler Newton-Krylov-Schwarz step for
 * the five-compartment SEIRD reaction-diffusion model (arXiv 2208.01839).
 *
 * The method (all references are to the paper):
 *   - PDE: Eq. seird1-5 with N = s+e+i+r+d (Eq. N), vector form Eq.
 *     vec_component1/2, homogeneous Neumann (no-flux) boundary.
 *   - Time discretisation: backward Euler, Eq. timediscrete.
 *   - Space: P1 triangles, weak form Eq. weakform.  Consistent mass, exact
 *     diffusion integral (mean_T(N) |T| grad u . grad phi), reaction term by
 *     Radon's degree-5 seven-point rule (or the three-vertex rule).
 *   - Nonlinear solve: Newton with the exact Jacobian and backtracking on
 *     ||F||_2 (Section 2.2 names Newton as the coupled alternative to its
 *     Picard iteration; both converge to the root of Eq. weakform), or the
 *     coupled Picard iteration of Eq. weak_vec_implicit (options.nonlinear).
 *   - Linear solve: right-preconditioned restarted (F)GMRES with classical
 *     Gram-Schmidt and one re-orthogonalisation (CGS2), or a single pass
 *     (options.gmres_one_pass); stopping rules of Section 3.2 (rtol, atol,
 *     dtol against ||b||_2).
 *   - Preconditioner: restricted additive Schwarz (Eq. RAS) with overlapping
 *     subdomains and block-ILU(k) subdomain solves (options.ilu_fill), plus (optionally) the
 *     additive coarse correction M_2^{-1} = M_RAS^{-1} + Z A_c^{-1} Z^T
 *     (Section 3.1) with Z the per-subdomain, per-compartment constant space.
 *
 * Layouts.  A state is node-major: u[node*5 + c], c = 0..4 = s, e, i, r, d,
 * float64, in the caller's node numbering.  Internally the library renumbers
 * nodes by (subdomain, caller index); every entry point below that takes or
 * returns a state uses the caller's numbering.  Block-sparse matrices are
 * 5x5-block BSR: row_ptr int32[n_rows+1], col int32[nnzb] (sorted within each
 * block row), val float64[nnzb][5][5] row-major inside a block.
 *
 * Ownership.  seird_create copies everything it needs (mesh, parameters,
 * optional fields and partition) to the device; the caller keeps ownership of
 * its arrays.  Pointers passed with on_device = 1 are device pointers that the
 * call reads or writes on the context's stream and never retains; with
 * on_device = 0 they are host pointers and the call returns after the copy.
 *
 * Errors.  Every int-returning call returns SEIRD_OK (0) or a negative
 * SEIRD_E* code; seird_last_error() gives a message.  The library never traps
 * or aborts, never waits without bound, and leaves the state at u^n when a
 * step fails.  No C++ exception crosses this interface: a failed host
 * allocation returns SEIRD_ENOMEM like a failed device one.  A context is
 * used by one host thread at a time.
 */
#ifndef SEIRD_H
#define SEIRD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEIRD_OK 0
#define SEIRD_EINVAL (-1)           /* bad argument or mesh */
#define SEIRD_ENOMEM (-2)           /* device or host allocation failed */
#define SEIRD_ECUDA (-3)            /* a CUDA runtime call failed */
#define SEIRD_ENEWTON_DIVERGED (-4) /* line search could not decrease ||F|| */
#define SEIRD_ENEWTON_MAXIT (-5)    /* Newton iteration limit reached */
#define SEIRD_EGMRES (-6)           /* GMRES diverged (dtol) or hit its limit */
#define SEIRD_ENONFINITE (-7)       /* non-finite value, or N <= 0 where 1/N is needed */
#define SEIRD_ETIMEOUT (-8)         /* a bounded device wait gave up */
#define SEIRD_ESINGULAR (-9)        /* a 5x5 pivot block is singular */

/* Mesh (Section 2.2: P1 triangles).  Host arrays. */
typedef struct {
  int64_t n_nodes;
  int64_t n_tris;
  const double* xy;    /* [n_nodes][2] */
  const int32_t* tri;  /* [n_tris][3], counter-clockwise, 0-based */
} seird_mesh;

/* Rates of Eq. seird1-5 and the diffusion coefficients of Eq. vec_component1. */
typedef struct {
  double A;        /* Allee parameter in (1 - A/N) */
  double beta_i;   /* transmission by infected */
  double beta_e;   /* transmission by exposed */
  double sigma;    /* exposed -> infected */
  double gamma_e;  /* exposed -> recovered */
  double gamma_r;  /* infected -> recovered */
  double gamma_d;  /* infected -> deceased */
  double alpha;    /* births (the paper uses 0) */
  double mu;       /* natural deaths (the paper uses 0) */
  double nu[4];    /* nubar_S, nubar_E, nubar_I, nubar_R ; nubar_D = 0 */
  const double* beta_field; /* optional host [n_nodes] P1 multiplier of beta_i and beta_e
                               (Eq. beta_ie/beta_x frozen in time); NULL means 1 */
} seird_params;

/* Solver options.  seird_default_options() fills the values quoted per field. */
typedef struct {
  double dt;              /* time step (1.0) */
  double newton_rtol;     /* stop when ||F|| <= rtol ||F(u^n)|| + atol (1e-8) */
  double newton_atol;     /* (0) */
  int32_t newton_maxit;   /* (20) */
  int32_t ls_maxit;       /* backtracking halvings (10) */
  int32_t gmres_restart;  /* Krylov vectors per cycle, <= 64 (30) */
  int32_t gmres_maxit;    /* total iterations per linear solve (200, Section 3.2) */
  double gmres_rtol;      /* (1e-5, Section 3.2) */
  double gmres_atol;      /* (1e-50, Section 3.2) */
  double gmres_dtol;      /* (1e5, Section 3.2) */
  int32_t n_subdomains;   /* RAS subdomains when owner == NULL (4) */
  int32_t overlap;        /* graph layers of overlap (1; Section 3.2 uses a minimal one) */
  int32_t coarse;         /* 0: one-level RAS; 1: additive constant coarse space (M_RAS^{-1} + Q);
                             2: multiplicative two-grid of Eq. RAS_2L (RAS, coarse correction,
                             RAS, each on the residual left by the previous step); 3: coarse
                             correction, then RAS on the residual it leaves (Q + M_RAS^{-1}(I - J Q),
                             the two-grid without the pre-smoother) (0) */
  int32_t precision;      /* 0: FP64 throughout; 1: FP32 matrix copy and FP32 subdomain
                             factors inside the FP64 outer FGMRES (0) */
  int32_t quadrature;     /* 0: degree-5 seven-point rule; 1: three-vertex rule (0) */
  int32_t pc_lag;         /* rebuild the preconditioner every pc_lag Newton iterations
                             (the first iteration of every step always rebuilds) (1) */
  const int32_t* owner;   /* optional host [n_nodes]: subdomain of each node, values
                             0..n_subdomains-1 all used; NULL: seeded recursive
                             coordinate bisection into n_subdomains parts */
  uint64_t seed;          /* seed of the bisection's uneven split fractions (0) */
  void* stream;           /* cudaStream_t the context runs on; NULL: a private stream */
  int32_t timing;         /* 1: time every kernel class with CUDA events on the stream and
                             report it in seird_stats.kernel_ms (0) */
  int32_t gmres_forcing;  /* 0: every linear solve to gmres_rtol (Section 3.2); 1: inexact Newton
                             with Eisenstat-Walker forcing terms (choice 2, gamma 0.9, alpha 2,
                             first term 0.1, at most 0.5); once the term comes within 10x of what
                             reaching the Newton target needs, the solve aims at 0.2x that (0) */
  int32_t nonlinear;      /* 0: Newton (exact Jacobian, backtracking line search); 1: the Picard
                             iteration of Eq. weak_vec_implicit, all five compartments coupled:
                             the coefficients nu(u) and B(u) of Eq. vec_component1/2 frozen at the
                             previous iterate, full steps, no line search.  Both iterations have
                             the root of Eq. weakform as fixed point (0) */
  int32_t gmres_one_pass; /* 0: classical Gram-Schmidt with one re-orthogonalisation (CGS2); 1: one
                             classical Gram-Schmidt pass, never refined (PETSc's GMRES default, which
                             Section 3.2's solver configuration leaves in place); half the FMAs (0) */
  double picard_tol;      /* Picard only: stop when eps = ||u^{k+1} - u^k|| / ||u^n|| (Eq. picardtol)
                             is <= picard_tol; 0 stops on the residual test of newton_rtol and
                             newton_atol instead.  newton_maxit bounds the iterations (0) */
  int32_t pc_keep_steps;  /* Newton: a preconditioner may serve the first iterations of up to
                             pc_keep_steps later time steps before it is rebuilt (0: rebuilt at the
                             start of every step).  A linear solve that stops unconverged with a
                             carried-over preconditioner is repeated once with a fresh one (0) */
  int32_t coarse_group;   /* coarse space: one unit per group of this many consecutive subdomains
                             (Z's column (g, c) = indicator of the nodes the group owns in compartment c).
                             0 chooses 1 unless 5 x units would exceed 8192 or units 1160 (the sizes of
                             the explicit coarse inverse), else the smallest group that fits (0) */
  int32_t predictor;      /* Newton's first iterate: 0 u^n (Section 2.2); p = 1-6 the polynomial
                             extrapolation of degree p (or lower while fewer earlier steps are known)
                             through u^n and the p previous states, one step ahead:
                             sum_k (-1)^k C(p+1, k+1) u^{n-k}, e.g. 2 u^n - u^{n-1} (p = 1),
                             4 u^n - 6 u^{n-1} + 4 u^{n-2} - u^{n-3} (p = 3); used when it is
                             admissible and lowers ||F||.  The stopping test stays relative to
                             ||F(u^n)|| either way.  Each degree keeps one more state (5n doubles) (0) */
  int32_t autotune;       /* 1: at the first linear solve, time the candidate launch shapes of the SpMV
                             (128/256/512 threads per CTA), of the Gram-Schmidt kernels (2/3/4/6 CTAs
                             per SM, 128- or 256-entry tiles) and of the subdomain solves (1-4 blocks of
                             solution entries loaded per batch, 7 or 3 consumer warps per CTA, a factor
                             ring of two stages or one) on the context's own vectors and factors
                             and keep the fastest; the choice is reported by seird_get_info.  The
                             Gram-Schmidt shape sets the order of its sums, so results are reproducible
                             for a given choice, not across choices; the other choices leave every sum
                             unchanged.  0: fixed shapes (256 threads, 3 CTAs per SM, 256, 2 blocks) (0) */
  int32_t graph;          /* 1: each GMRES restart cycle runs as one replay of a CUDA graph captured at
                             the first solve: iteration j is a conditional node that the Givens kernel
                             of iteration j - 1 arms while the residual estimate is above the
                             tolerance, so the host reads the outcome once per cycle instead of once
                             per iteration.  Same kernels and arithmetic as 0 (results identical).
                             Needs a driver with conditional graph nodes (CUDA 12.4+); ignored while
                             timing = 1 and in the adjoint's transposed solves (0) */
  double forcing_first;   /* gmres_forcing = 1: the forcing term of each step's first Newton iteration
                             (0 means 0.1, the usual Eisenstat-Walker start).  A Newton iteration that
                             starts close to the root (a good predictor) can afford a smaller one, so
                             that the next iteration already reaches the Newton target (0) */
  int32_t ilu_fill;       /* subdomain factors: block ILU(k) with k = ilu_fill levels of fill, 0-8
                             (Saad, Iterative Methods for Sparse Linear Systems, Section 10.3.3).  Entry
                             (i, j) of a subdomain's factors is kept when lev(i, j) <= k, where
                             lev(i, j) = 0 on the pattern of R_p J R_p^T and every elimination step
                             through a pivot row m < min(i, j) offers lev(i, m) + lev(m, j) + 1.  The
                             factors agree with R_p J R_p^T on every kept entry; 0 is ILU(0), PETSc's
                             default subdomain solver.  More fill costs memory and solve time per
                             application and buys fewer GMRES iterations where diffusion dominates (0) */
} seird_options;

/* Kernel classes of seird_stats.kernel_ms / kernel_calls. */
enum {
  SEIRD_K_RESIDUAL = 0,     /* residual assembly (element + gather + norm) */
  SEIRD_K_JACOBIAN = 1,     /* Jacobian assembly (records + block gather) */
  SEIRD_K_ILU_FACTOR = 2,   /* subdomain block-ILU(k) factorisation */
  SEIRD_K_COARSE_SETUP = 3, /* Z^T J Z and its banded block LU */
  SEIRD_K_SPMV = 4,         /* BSR SpMV */
  SEIRD_K_ILU_SOLVE = 5,    /* subdomain triangular solves (RAS apply) */
  SEIRD_K_COARSE_APPLY = 6, /* Z^T r, banded solve, Z y */
  SEIRD_K_KRYLOV = 7,       /* CGS2, norms and vector updates */
  SEIRD_K_COUNT = 8
};

/* Per-step statistics (the paper's iteration counts and setup/solve split,
 * Table PC_2000_600cores and Fig. setup_hypre). */
typedef struct {
  int32_t newton_its;
  int32_t gmres_its;      /* summed over the step's linear solves */
  int32_t ls_halvings;
  int32_t pc_setups;
  double res0;            /* ||F(u^n)||_2 */
  double res_final;       /* ||F(u^{n+1})||_2 */
  double eps_update;      /* last ||u^{k+1}-u^k|| / ||u^n|| (Eq. picardtol) */
  double ms_assemble;     /* residual + Jacobian assembly */
  double ms_setup;        /* preconditioner setup (subdomain factors, coarse) */
  double ms_solve;        /* GMRES */
  double ms_total;
  double kernel_ms[8];    /* device time per kernel class (options.timing = 1) */
  int32_t kernel_calls[8];
  double alg_bytes[8];    /* algorithmic bytes per kernel class in this step (always counted): what
                             each launch must move at least, every array it needs read or written
                             once at the precision it runs in, summed over the step's launches;
                             scratch kept between a class's own kernels is not counted */
} seird_stats;

/* Sizes of a created context. */
typedef struct {
  int64_t n_nodes, n_tris, nnzb;
  int32_t n_subdomains;
  int64_t subdomain_rows;      /* sum over subdomains of overlapped node counts */
  int64_t subdomain_blocks;    /* sum over subdomains of factor blocks (the local pattern and its fill) */
  int32_t max_levels;          /* deepest level schedule of the subdomain factors */
  int32_t coarse_band;         /* half bandwidth (in coarse units) of the coarse matrix */
  int64_t device_bytes;        /* device memory held by the context */
  int32_t coarse_units;        /* units of the coarse space (groups of options.coarse_group subdomains) */
  int32_t spmv_threads;        /* launch shapes in use (options.autotune): SpMV threads per CTA, */
  int32_t cgs_ctas;            /* Gram-Schmidt CTAs, */
  int32_t cgs_tile;            /* Gram-Schmidt tile entries (0: 256 up to depth 27, then 128) */
  int32_t ilu_batch;           /* subdomain solves: blocks whose solution entries a row loads before
                                  their FMAs (1-4), */
  int32_t ilu_warps;           /* consumer warps per subdomain CTA (7, or 3 in CTAs of 128 threads), */
  int32_t ilu_ring;            /* and factor blocks in the shared-memory ring (236: two stages, 118: one) */
} seird_info;

typedef struct seird_ctx seird_ctx;

/* Fills *opt with the defaults listed above. */
void seird_default_options(seird_options* opt);

/* Builds a context: validates the mesh (indices in range, positive areas),
 * partitions and renumbers nodes, builds the BSR pattern, element maps,
 * overlapping subdomains (Eq. RAS), ILU(k) patterns and level schedules and the coarse
 * pattern, and uploads everything.  The state is set to zero at t = 0.
 * Returns SEIRD_EINVAL for a bad mesh/option, SEIRD_ENOMEM, SEIRD_ECUDA. */
int seird_create(const seird_mesh* mesh, const seird_params* params, const seird_options* opt,
                 seird_ctx** out);

/* Ensemble of n_samples independent problems on one mesh (parameter sweeps and
 * sampling of the rates the paper calibrates, Section 4.2): sample k uses the
 * rates params[k]; params[0].beta_field, if any, is shared by every sample.
 * The samples form one block-diagonal system over n_samples x n_nodes nodes:
 * the mesh is partitioned once (options.owner or the seeded bisection into
 * options.n_subdomains parts) and every sample gets its own copy of those
 * subdomains, so every kernel launch of a step covers all samples, and no
 * subdomain, coarse unknown or matrix block couples two samples.  States are
 * [n_samples][n_nodes][5]; Newton and GMRES test the norms over all samples,
 * and each sample's state is the root of its own system.  An ensemble's rates
 * are fixed (seird_set_params and seird_set_beta_schedule return
 * SEIRD_EINVAL); seird_adjoint gives every sample's gradient. */
int seird_create_ensemble(const seird_mesh* mesh, int32_t n_samples, const seird_params* params,
                          const seird_options* opt, seird_ctx** out);

/* Releases every resource of the context (NULL is ignored). */
void seird_destroy(seird_ctx* ctx);

/* Message of the last error on this context (or of the last failed create
 * when ctx is NULL).  Valid until the next call on the context. */
const char* seird_last_error(const seird_ctx* ctx);

/* Sets the state u^n (caller numbering, [n_nodes][5] float64) and time t.  A new
 * state drops the step history the predictor and the residual reuse; setting the
 * state the context already holds, bit for bit and at its own time (a caller that
 * passes each step's result through its own memory), keeps it. */
int seird_set_state(seird_ctx* ctx, const double* u, int on_device, double t);

/* Copies the current state out (caller numbering) and its time (t may be NULL). */
int seird_get_state(const seird_ctx* ctx, double* u, int on_device, double* t);

/* One backward-Euler step (Eq. timediscrete): u^{n+1} = root of Eq. weakform
 * by Newton-Krylov-Schwarz from the guess u^n; t += dt.  stats may be NULL.
 * On failure the state stays u^n and the code says why. */
int seird_step(seird_ctx* ctx, seird_stats* stats);

/* n_steps steps; per_step may be NULL or point to n_steps records.  Stops at
 * the first failing step and returns its code. */
int seird_run(seird_ctx* ctx, int32_t n_steps, seird_stats* per_step);

/* Sizes of the context. */
int seird_get_info(const seird_ctx* ctx, seird_info* info);

/* Replaces the rates (and, if params->beta_field is not NULL, the transmission
 * field; a NULL field keeps the current one).  The mesh, partition and state are
 * kept.  Host pointers, copied. */
int seird_set_params(seird_ctx* ctx, const seird_params* params);

/* ---- sigmoid transmission schedule (Section 4.2, Eq. beta_ie and Eq. beta_x) --
 *   beta_I(x, t) = beta_E(x, t) = beta(t) beta(x),
 *   beta(t) = b0 - b1 / (1 + exp(t_mid - t)),
 *   beta(x) = beta_central + (beta_eastern - beta_central) / (1 + exp(-k_eastern (x - x_eastern)))
 *                          + (beta_western - beta_central) / (1 + exp( k_western (x - x_western))),
 * with x the first mesh coordinate.  The step from t to t + dt uses beta(t + dt)
 * (backward Euler takes the rates at the end of the step); beta(x) is evaluated
 * at the nodes and interpolated linearly on every triangle, like
 * params.beta_field, which it replaces while the schedule is on.  The paper's
 * values: b0 = 0.101, b1 = 0.05, t_mid = 130 (days), k_eastern = 5,
 * k_western = 10 (per unit of x); the regional betas and boundaries are fitted
 * to case data the paper does not print. */
typedef struct {
  double b0, b1, t_mid;
  double beta_central, beta_eastern, beta_western;
  double x_eastern, x_western;
  double k_eastern, k_western;
} seird_beta_schedule;

/* Turns the schedule on (sched copied) or off (sched == NULL: params.beta_i,
 * beta_e and the transmission field apply again).  The component entry points
 * (seird_eval_residual and the rest) use the rates of the step that ends at the
 * context's time + dt.  seird_adjoint rejects a context whose schedule is on
 * (SEIRD_EINVAL): its gradients are taken with respect to constant rates. */
int seird_set_beta_schedule(seird_ctx* ctx, const seird_beta_schedule* sched);

/* ---- discrete adjoint -------------------------------------------------------
 * Misfit of observed infected (I) and deceased (D) densities,
 *   j = sum_{k in obs_steps} sum_{i in obs_nodes} (u^k_{i,I} - I_hat)^2 + (u^k_{i,D} - D_hat)^2,
 * over a run of n_steps backward-Euler steps from the context's current state
 * u^0.  Gradient parameters (the rates the paper calibrates, Section 4.2):
 *   grad[0..9] = dj/d(beta_i, beta_e, sigma, gamma_e, gamma_r, gamma_d,
 *                     nubar_S, nubar_E, nubar_I, nubar_R)
 * and grad_field[j] = dj/db_j for the per-node transmission multiplier b
 * (1 when the context has no field).  Host arrays. */
typedef struct {
  int32_t n_steps;            /* steps of the forward run */
  int32_t checkpoint_every;   /* states kept every k steps; the reverse sweep recomputes
                                 each segment from its checkpoint (1 keeps every state) */
  int32_t n_obs_nodes;
  const int32_t* obs_nodes;   /* [n_obs_nodes] caller numbering */
  int32_t n_obs_steps;
  const int32_t* obs_steps;   /* [n_obs_steps] step indices in 1..n_steps, increasing */
  const double* I_hat;        /* [n_obs_steps][n_obs_nodes] */
  const double* D_hat;        /* [n_obs_steps][n_obs_nodes] */
  double lin_rtol;            /* relative tolerance of the transposed linear solves (0: 1e-10) */
} seird_misfit;

/* Runs the forward steps (Newton to options.newton_rtol), then the reverse
 * sweep J_k^T lambda_k = -dj/du^k + M lambda_{k+1} (Jacobian of step k, M the
 * consistent mass), each solved by the same right-preconditioned FGMRES with
 * RAS and coarse correction built from J_k^T, and accumulates
 * dj/dp = sum_k lambda_k^T dF^k/dp.  Outputs: *misfit, grad [10], grad_field
 * [n_nodes] (nullable, caller numbering).  On an ensemble the observation
 * nodes are ensemble nodes (sample k's node i is k * n_nodes + i), the misfit
 * sums over the samples and grad is [n_samples][10], each sample's gradient
 * with respect to its own rates.  The state and time are restored to u^0 on
 * return; during the call every step builds its own preconditioner and
 * starts Newton from u^n (pc_keep_steps and predictor are ignored), so
 * recomputed segments repeat the forward states exactly.  FP64 contexts only (options.precision = 0), else SEIRD_EINVAL. */
int seird_adjoint(seird_ctx* ctx, const seird_misfit* spec, double* misfit, double* grad, double* grad_field);

/* ---- component entry points (kernel-level parity and measurement) ---- */

/* F(u; u_prev) of Eq. weakform (caller numbering, [n_nodes][5]).  All three
 * pointers are device pointers when on_device = 1, host pointers otherwise. */
int seird_eval_residual(seird_ctx* ctx, const double* u, const double* u_prev, double* F, int on_device);

/* Assembles, at u, the matrix of the context's nonlinear iteration into its BSR
 * matrix: the exact Jacobian dF/du (options.nonlinear = 0) or the Picard matrix
 * of Eq. weak_vec_implicit, M + dt (nu(u) grad, grad) - dt (B(u) ., .)
 * (options.nonlinear = 1). */
int seird_eval_jacobian(seird_ctx* ctx, const double* u, int on_device);

/* Copies the context's Jacobian out in caller numbering as host BSR arrays
 * (row_ptr [n_nodes+1], col [nnzb] sorted, val [nnzb][25]). */
int seird_get_jacobian(const seird_ctx* ctx, int32_t* row_ptr, int32_t* col, double* val);

/* y = J x with the context's Jacobian (caller numbering). */
int seird_apply_jacobian(seird_ctx* ctx, const double* x, double* y, int on_device);

/* Builds the preconditioner (subdomain block-ILU(k) factors and, if enabled,
 * the coarse matrix Z^T J Z and its factors) from the context's Jacobian. */
int seird_precond_setup(seird_ctx* ctx);

/* z = M^{-1} r with the last preconditioner built (caller numbering). */
int seird_precond_apply(seird_ctx* ctx, const double* r, double* z, int on_device);

/* Pins launch shapes (each 0 keeps the current one): SpMV threads per CTA (128, 256,
 * 512), Gram-Schmidt CTAs (1 .. 64 x SMs) and tile entries (128, 256), and the
 * subdomain solves' dependency-load batch (1-4 blocks), consumer warps (7 or 3)
 * and factor-ring size (236 or 118 blocks; 118 only when every stage fits it).  The autotuner
 * (options.autotune) does not change shapes pinned this way, so the shapes one
 * run reported by seird_get_info reproduce its sums in another run (the
 * Gram-Schmidt shape sets the order of its sums; the other shapes do not change
 * any result).  SEIRD_EINVAL for a value outside these candidates. */
int seird_set_launch_shapes(seird_ctx* ctx, int32_t spmv_threads, int32_t cgs_ctas, int32_t cgs_tile,
                            int32_t ilu_batch, int32_t ilu_warps, int32_t ilu_ring);

/* Failure detection of the bounded device waits (the library never waits
 * without bound).  The subdomain solves of the RAS apply stream each stage's
 * factor blocks through shared memory, and every wait for a stage's data or
 * for ring space polls an mbarrier at most `polls` times (default 2^20) before
 * it gives up; the CTA then stops at the same stage in all its warps, lets
 * every copy it issued land (that wait keeps its fixed bound) and sets the
 * context's error word, and the call returns SEIRD_ETIMEOUT (the step leaves
 * the state at u^n).  polls = 0 restores the default; polls < 0 makes every
 * such wait give up at once, which exercises this path without a fault. */
int seird_set_wait_limit(seird_ctx* ctx, int32_t polls);

/* Solves J x = b with the preconditioned (F)GMRES of the step (x starts at 0),
 * using the context's Jacobian and last preconditioner.  its may be NULL. */
int seird_linear_solve(seird_ctx* ctx, const double* b, double* x, int on_device, int32_t* its);

/* y = A x for a 5x5-block BSR matrix with n_rows block rows; every pointer is a
 * device pointer; stream is a cudaStream_t (NULL: legacy default stream).
 * x has 5 entries per block column, y 5 per block row.  Returns SEIRD_EINVAL
 * for n_rows < 0 or a NULL pointer with n_rows > 0, SEIRD_ECUDA if the launch fails. */
int seird_bsr_spmv(int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val,
                   const double* x, double* y, void* stream);

/* The same product with float32 block values (x and y stay float64): the
 * matrix copy of the mixed-precision path. */
int seird_bsr_spmv_f32val(int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const float* val,
                          const double* x, double* y, void* stream);

/* Number of kernels the library has launched in this process so far. */
int64_t seird_launch_count(void);

/* Host-only check of the set-up the kernels rely on (no device call, no
 * context): builds the partition, the BSR pattern, the overlapping
 * subdomains, the ILU(k) patterns, level schedules and solve plans for `mesh` under
 * `opt` (NULL: defaults) and verifies their invariants: owned ranges tile the
 * nodes, rows sorted with their diagonal, a structurally symmetric pattern,
 * each node's element gather list naming its triangle corners in order and
 * each block's naming the corner pairs that reach it, coarse units tiling the
 * nodes, the J Z segments of the two-grid lying in their row and in one unit,
 * the coarse segment sums visiting every block once, every subdomain's factor
 * pattern symmetric with its diagonal and each block naming its J block (or
 * none, for fill), every owned node in its subdomain, every sweep a permutation of the
 * subdomain's rows, every stage within the shared-memory rings, every
 * dependency of a row in an earlier stage, and the row records numbering the
 * solution entries by sweep position with each owned row written once.
 * stats (nullable) [8]: n_nodes, n_tris, nnzb, subdomains, subdomain rows,
 * forward stages, backward stages, violations.  Returns SEIRD_OK, SEIRD_EINVAL
 * with the first violation in seird_last_error(NULL), or the set-up's own
 * error for a bad mesh or partition. */
int seird_setup_check(const seird_mesh* mesh, const seird_options* opt, int64_t* stats);

/* ---- allocation-free residual --------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot call cudaMalloc: code running inside a framework that owns all device
 * memory through its own arena, or inside a loop that must not allocate
 * (allocation can block, fail or synchronise).  Such a caller cannot create a
 * context, because seird_create allocates.  This entry point evaluates the
 * same residual as seird_eval_residual, by the same two-phase element/gather
 * computation, on a mesh held entirely in caller-owned device memory, and
 * allocates nothing: its scratch is one fixed file-scope device
 * array of SEIRD_NOALLOC_MAX_TRIS element vectors (15 doubles each) and
 * SEIRD_NOALLOC_MAX_NODES node terms (8 doubles each), about 12 MB, which
 * every GPU that loads the library keeps until the process exits.
 *
 * Arguments (all pointers are device pointers except params):
 *   xy [n_nodes][2], tri [n_tris][3] (counter-clockwise), and the node
 *   incidence in CSR form: inc_ptr [n_nodes+1], inc [3*n_tris] holding
 *   3*t + a for every triangle t and corner a, grouped by node and ascending
 *   in t within a node (the summation order of each F entry);
 *   params: host struct; params->beta_field is ignored, beta_field_dev is the
 *   optional device [n_nodes] transmission multiplier (NULL means 1);
 *   u, u_prev, F: [n_nodes][5] in the mesh's numbering; norm2 (nullable):
 *   receives ||F||_2^2.  quadrature as in seird_options.
 * Limits: n_tris <= SEIRD_NOALLOC_MAX_TRIS and n_nodes <= SEIRD_NOALLOC_MAX_NODES,
 * else SEIRD_EINVAL with a message in seird_last_error(NULL).
 * Behaviour: runs on `stream` on the current device (every pointer must be
 * memory of that device) and synchronises the stream before returning, then
 * returns SEIRD_ENONFINITE if N <= 0 at a quadrature point.  The first call
 * on a device looks up the scratch array's device address and uploads the
 * quadrature tables (a one-time set-up per device, with that device current,
 * ending in a device synchronisation).  Every call shares the one scratch array, whose contents
 * are left over from the last call; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the caller. */
#define SEIRD_NOALLOC_MAX_TRIS 65536
#define SEIRD_NOALLOC_MAX_NODES 65536
int seird_residual_noalloc(int64_t n_nodes, int64_t n_tris, const double* xy, const int32_t* tri,
                           const int32_t* inc_ptr, const int32_t* inc, const seird_params* params,
                           const double* beta_field_dev, double dt, int32_t quadrature, const double* u,
                           const double* u_prev, double* F, double* norm2, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SEIRD_H */
