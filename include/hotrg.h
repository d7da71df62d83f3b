/*
 * hotrg.h -- C ABI of the GB300 HOTRG library (forward coarse-graining and
 * its reverse-mode backward, "differentiable TRG").
 *
 * What is computed (paper: "Automatic Differentiation for Second
 * Renormalization of Tensor Networks"):
 *
 *   - SM Sec. A: the partition function of a 2D lattice model is the trace
 *     of a square network of identical rank-4 tensors T0[l][r][u][d].
 *   - SM Sec. B, HOTRG step equation: one coarse-graining step merges two
 *     vertically adjacent tensors,
 *        T'[a][b][y][y'] = sum T[x1][x1'][y][j] T[x2][x2'][j][y']
 *                              w[x1][x2][a] w[x1'][x2'][b],
 *     with the isometry w taken from the local higher-order SVD of the
 *     merged pair, i.e. the leading D' = min(X*X, d_cut) eigenvectors of the
 *     Gram matrix G[(x1 x2)][(x1'' x2'')] of that pair (eigenvalues
 *     descending; each eigenvector sign-fixed so that its largest-magnitude
 *     component is positive).  Steps alternate direction (main text
 *     Fig. 1a): before every step after the first the tensor is re-oriented
 *     T[l][r][u][d] -> T[u][d][l][r].
 *   - Normalisation: after step k the new tensor is divided by its
 *     Frobenius norm c_k (computed in FP64).  With N = 2^n_steps sites,
 *        ln Z / N = sum_k ln(c_k) / 2^k + ln|sum_{x,y} T_n[x][x][y][y]| / 2^n.
 *   - Backward: SM Sec. B second-renormalization recursion = SM Sec. E
 *     chain rule through the Jacobian of each step; main-text Eq. (1) for
 *     the adjoint of w.  hotrg_backward returns d(ln Z / N)/d T0 (per site)
 *     and, for Ising inputs, d(ln Z / N)/d beta.
 *
 * Layouts: every tensor is row-major T[l][r][u][d] (d fastest), float64.
 *
 * Ownership: the caller owns every buffer it passes.  A plan owns all device
 * memory it needs (checkpoints, eigenvectors, workspaces); it is sized at
 * hotrg_plan_create and nothing is allocated inside forward or backward.
 *
 * Threading: a plan is bound to one CUDA stream and is not thread-safe.
 *
 * Errors: every call returns a hotrg_status; no C++ exception crosses this
 * boundary.  After any error the plan stays usable (a new forward must be run
 * before a backward).  hotrg_last_error() gives a one-line description of the
 * last error seen on a plan.
 */
#ifndef HOTRG_H
#define HOTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HOTRG_OK = 0,
  HOTRG_EINVAL = 1,       /* bad argument (sizes, NULL, non-finite input)         */
  HOTRG_ENOMEM = 2,       /* device allocation failed at plan creation             */
  HOTRG_ECUDA = 3,        /* a CUDA runtime/driver/cuSOLVER call failed            */
  HOTRG_ENOTCONV = 4,     /* the eigensolver reported non-convergence              */
  HOTRG_ENONFINITE = 5,   /* a norm or the final trace was zero, NaN or infinite   */
  HOTRG_ETIMEOUT = 6,     /* a bounded device-side wait gave up (error word set)   */
  HOTRG_ESTATE = 7,       /* call out of order (backward before a forward)         */
  HOTRG_EUNSUPPORTED = 8, /* option not available on this device or build          */
  HOTRG_EPENDING = 9      /* server: the request has not finished yet              */
} hotrg_status;

typedef enum {
  HOTRG_FP64 = 0,    /* every contraction in FP64 (CUDA cores)                         */
  HOTRG_BF16X3 = 1,  /* contractions as split-BF16 tensor-core products: hi*hi + hi*lo
                        + lo*hi, FP32 accumulation                                     */
  HOTRG_BF16X6 = 2   /* three-plane split (hi, mid, lo): all products with plane-sum
                        <= 2 (6 products), FP32 accumulation over K-chunks, chunks
                        summed in compensated (double-float) precision                */
} hotrg_precision;

typedef struct {
  int d0;               /* bond dimension of T0 (all four legs)                          */
  int d_cut;            /* truncation: kept eigenvectors per step, D' = min(X*X, d_cut)   */
  int n_steps;          /* number of coarse-graining steps (first one vertical)           */
  int precision;        /* hotrg_precision for steps >= split_from_step                   */
  int split_from_step;  /* 1-based; steps before it always run in FP64                   */
  int want_grad;        /* 1: keep what hotrg_backward needs (eigenvectors per step)      */
  int fixed_w_grad;     /* 1: backward holds every w fixed (SM Sec. E view of w as
                           independent parameters); 0: full derivative through the eigh  */
  double eigh_broadening; /* eta_rel in F = d / (d^2 + eta_rel * lam_1^2); <= 0 -> 1e-12 */
  int gram_split_from_step; /* 1-based; the Gram matrix of split steps before it is formed
                               in FP64 (the eigensolve is the step most sensitive to
                               rounding); <= split_from_step: same as the contractions   */
  int hi_precision_steps;   /* with HOTRG_BF16X6: the first hi_precision_steps split steps use
                               four bf16 planes (10 products, ~32 significant bits) instead of
                               three; these steps weigh most in ln Z / N (weight 2^-k)     */
  int eigh_mode;            /* plans without gradients: 0 = cuSOLVER partial eigensolve of the
                               D'+1 largest pairs; 1 = randomized subspace eigensolver (block
                               power iteration on eigh_block vectors with FP64 Householder QR,
                               then FP64 Rayleigh-Ritz; the products G Q run on the
                               four-plane tensor-core GEMM on split steps, in FP64
                               otherwise; used where 4 D' < X^2).  Plans with full
                               gradients always take all eigenpairs; fixed_w_grad plans
                               (whose backward needs only the kept ones) and forward-only
                               plans follow eigh_mode.  w_rule 1 ignores it.              */
  int eigh_power_iters;     /* power iterations of eigh_mode 1 (<= 0: 4)                   */
  int eigh_block;           /* vectors in the block of eigh_mode 1 (<= 0: 4 D'; at least
                               D' + 1)                                                     */
  int epilogue_split;       /* three-plane split steps: 1 = the stage-1 and stage-2 GEMMs
                               write their outputs as bf16 planes from the epilogue where
                               the layout allows it; 0 = through an FP32 buffer and a
                               separate split kernel (bit-identical results)               */
  long long split_chunk_elems; /* split steps: elements per bf16 plane of the y-chunked
                               stage buffers (the D^5 intermediates; <= 0: 2^30).  Smaller
                               values make the plan smaller and the stage GEMMs shorter;
                               results do not depend on it.                               */
  int w_given;              /* 1 = the isometries are parameters (differentiable-TRG sweeps,
                               main text after Eq. (1)): the forward uses the ones loaded
                               with hotrg_set_isometries or left by hotrg_mera_update and
                               forms no Gram and no eigensolve.  Needs want_grad = 1 and
                               fixed_w_grad = 1.                                          */
  double eigh_residual_tol; /* eigh_mode 1: accuracy guard of the subspace eigensolver.  After
                               the subspace solve of step k the kept Ritz pairs are checked on
                               the device, r_k = max_a ||G v_a - theta_a v_a||_2 / theta_1.
                               Where 2^-k r_k exceeds this bound (<= 0: 1e-9; an error at step
                               k enters ln Z / N with weight 2^-k) the step gets up to four more
                               power iterations, each checked again, and if it still fails the
                               exact partial eigensolver (cuSOLVER syevdx).  Reading the check
                               costs one host synchronisation per subspace step.  Must be
                               finite and >= 0.                                           */
  int stage2_n_group;       /* tile order of the O(D^7) stage-2 GEMM: its persistent CTAs walk
                               the output in groups of this many 128-wide N-tiles (all M-tiles
                               of a group before the next), so that one stripe of the B
                               operand stays in L2 while A streams; 0 = the default (16);
                               a value >= the N-tile count = plain N-fastest order.  Results
                               do not depend on it.                                        */
  int stage2_pair;          /* stage-2 GEMM of the three-plane steps on CTA pairs (tcgen05
                               cta_group::2: 256-row tiles, each CTA of a cluster of two loads
                               its 128 rows of U and half of the 128-row tile of the other
                               operand); 0 = the default (one CTA per tile, measured
                               faster), > 0 = on.  Results are bit-identical either way.   */
  int gemm_sm_reserve;      /* SMs the persistent tensor-core contraction GEMMs leave free
                               (0..64, default 0): with several plans running concurrently on
                               their own streams, the latency-bound eigensolver kernels of one
                               solve then run beside the other's contractions instead of
                               waiting for whole GEMMs.  Results do not depend on it.      */
  int eigh_warm_start;      /* eigh_mode 1: > 0 = start the subspace block of step k from the
                               kept eigenvectors of step k - 2 (the same leg bases near the
                               fixed point of the flow) and run this many power iterations
                               there instead of eigh_power_iters; the accuracy guard still
                               checks every step.  0 = off (default), at most 16.          */
  int scheme;               /* 0 = scheme (a) of main text Fig. 1a (default): steps alternate
                               direction and the last tensor is traced as a torus.
                               1 = scheme (b) of Fig. 1b: vertical merges only (the MPO
                               product rho(2 tau) = rho(tau) rho(tau) for a density matrix,
                               SM Sec. F): no re-orientation, the vertical (physical) legs keep
                               dimension d0 and the horizontal bond grows to D' = min(X^2,
                               d_cut); T0 is the cell tensor of a translation-invariant chain.
                               The remaining one-dimensional structure is contracted exactly:
                               the free energy of the depth-n chain is evaluated as
                               Tr[rho rho] of two copies of it on the infinite chain,
                                 lnz = sum_k ln c_k / 2^k + ln lambda_max(A_n) / 2^(n+1),
                                 (A V)[x1][x2] = sum_{y,j} T~_n[x1][x1'][y][j] V[x1'][x2']
                                                 T~_n[x2][x2'][j][y],
                               lambda_max the dominant eigenvalue of that cell transfer
                               operator (FP64 power iteration; HOTRG_ENOTCONV if it has no
                               simple positive dominant eigenvalue).  lnz is ln Z per copy of
                               T0 in the 2^(n+1)-deep network: ln Tr rho(2^(n+1) tau) per cell
                               is 2^(n+1) lnz.  d_cut <= 4096.                             */
  int chain_steps;          /* scheme 1: 1 = also evaluate lnz of every depth k < n during the
                               forward (hotrg_chain_lnz_steps: the whole cooling curve, beta_k
                               = 2^(k+1) tau, from one forward); 0 = the last depth only.  */
  int w_rule;               /* which environment gives the isometry (SM Sec. B, "local HOSVD"):
                               0 = the Gram matrix of the merged pair along its left bond
                               (x1 x2), always (default); 1 = Xie2012's rule: the HOSVD along
                               the left and along the right bond (x1' x2'), the side whose
                               discarded eigenvalues sum to less gives w (both Gram matrices
                               have the same trace; relative differences up to 1e-12 count as a
                               tie, which takes the left side).  The backward differentiates
                               through the side taken (discontinuous where the two are equal).
                               w_rule 1 doubles the Gram and eigensolve work, uses the exact
                               eigensolvers (eigh_mode is ignored) and needs w_given = 0.  */
} hotrg_config;

typedef struct hotrg_plan_s* hotrg_plan;

/* Fill a config with defaults: FP64, split_from_step = 1, want_grad = 1,
 * fixed_w_grad = 0, eigh_broadening = 1e-12, gram_split_from_step = 0,
 * hi_precision_steps = 2, eigh_mode = 0, eigh_power_iters = 4, eigh_block = 0,
 * epilogue_split = 1, split_chunk_elems = 0, w_given = 0, eigh_residual_tol = 0,
 * stage2_n_group = 0, stage2_pair = 0, gemm_sm_reserve = 0, eigh_warm_start = 0,
 * scheme = 0, chain_steps = 0, w_rule = 0.
 * d0, d_cut, n_steps as given. */
void hotrg_config_default(hotrg_config* cfg, int d0, int d_cut, int n_steps);

/* Differentiable TRG (main text: SRG as backpropagation, Eq. (1) E_w = wbar / N_i,
 * and the MERA update of w from the SVD of E_w).  All buffers below are the
 * isometries of every step, concatenated over k = 1..n_steps; step k holds
 * X'_k x X_k^2 doubles, row a = the a-th kept vector over (x1 x2), x1 major
 * (X, X' from hotrg_step_dims).  Host buffers, caller-owned; the calls
 * synchronise the plan's stream.
 *
 * hotrg_isometries: the isometries of the last forward (gradient plans) or
 *   the ones loaded / updated (w_given plans).
 * hotrg_set_isometries: load them into a w_given plan (entries must be finite;
 *   they are used as given, orthonormal or not).
 * hotrg_isometry_adjoints: d(ln Z/N)/d w_k of the last backward (gradient
 *   plans): with fixed_w_grad = 1 this is the environment of w_k, E_w = wbar.
 * hotrg_mera_update(plan, k): after a backward of a w_given plan, replace w_k
 *   by the isometry maximising Tr(E_w^T w): E_w = U S V^T (cuSOLVER gesvd,
 *   FP64), w_k = U V^T.  The next forward sees the new w_k.
 * HOTRG_ESTATE when called out of order (no forward / backward yet, or a plan
 * without w_given). */
/* hotrg_plan_set_given_steps(plan, k0) (w_given plans): the following
 * forwards use the stored isometries of steps 1..k0 and take those of later
 * steps from the Gram matrix as HOTRG does (stored, so that a later call with
 * a larger k0 uses them as parameters); 0 <= k0 <= n_steps, default n_steps.
 * A forward needs defined isometries for steps 1..min(k0, steps run): loaded
 * with hotrg_set_isometries or formed by an earlier forward.  This grows a
 * network one layer at a time (scheme (b) cooling with differentiable-TRG
 * optimisation of the newest layers). */
hotrg_status hotrg_plan_set_given_steps(hotrg_plan plan, int k0);
hotrg_status hotrg_isometries(hotrg_plan plan, double* w);
hotrg_status hotrg_set_isometries(hotrg_plan plan, const double* w);
hotrg_status hotrg_isometry_adjoints(hotrg_plan plan, double* wbar);
hotrg_status hotrg_mera_update(hotrg_plan plan, int step);

/* Quasi-Newton optimisation of one layer's isometry (SM Sec. D): w_k = exp(B)
 * truncated to D' columns, B antisymmetric N x N (N = X_k^2), updated by
 * L-BFGS to maximise ln Z / N with every other isometry fixed.  The run starts
 * at the layer's current isometry: w_k(B) = Q exp(B) E with Q the complete
 * Householder QR factor of w_k (columns sign-fixed so that Q E = w_k), E the
 * first D' columns of the identity, B = 0 (the paper's exp(B) is Q = I).  The
 * gradient comes from the plan's fixed-w backward (main-text Eq. (1)) through
 * the adjoint Frechet derivative of the matrix exponential (the upper-right
 * block of exp([[B^T, C], [0, B^T]]), C = Q^T wbar E^T); every matrix
 * exponential is scaling and squaring of a degree-16 Taylor polynomial on the
 * FP64 GEMM.  L-BFGS: two-loop recursion with `history` pairs and
 * H_0 = (s^T y / y^T y) I, the first step along the gradient scaled to length
 * step0 (radians of rotation), backtracking from the full step until the
 * Armijo condition with constant c1 holds (at most max_backtracks halvings;
 * a failed search ends the run), pairs with s^T y <= 0 not stored.  Cost
 * O(N^3) = O(D^6) per evaluation (the paper's figure for this optimiser).
 *
 * hotrg_lbfgs_create: for a w_given plan (want_grad = fixed_w_grad = 1) that
 *   has run a forward (its site tensor is reused); allocates the optimiser's
 *   device memory (about (2 history + 20) N^2 doubles for the largest N).
 * hotrg_lbfgs_layer: n_iter iterations on layer `step` (1 <= step <= the
 *   steps the plan runs, with that step's isometry given); f_hist (host,
 *   n_iter + 1 doubles, may be NULL) receives ln Z / N at the start and after
 *   each accepted iteration, n_accepted / n_evals (may be NULL) the accepted
 *   iterations and forward evaluations.  The plan keeps the last accepted
 *   isometry.  Synchronises the plan's stream.
 * hotrg_lbfgs_destroy: frees it (before its plan). */
typedef struct hotrg_lbfgs_s* hotrg_lbfgs;
hotrg_status hotrg_lbfgs_create(hotrg_plan plan, int history, hotrg_lbfgs* out);
hotrg_status hotrg_lbfgs_layer(hotrg_lbfgs opt, int step, int n_iter, double step0, double c1,
                               int max_backtracks, double* f_hist, int* n_accepted,
                               int* n_evals);
void hotrg_lbfgs_destroy(hotrg_lbfgs opt);

/* sizeof(hotrg_config) as compiled into the library, so that a binding can
 * check that its copy of the struct matches. */
size_t hotrg_config_sizeof(void);

/* Device bytes a plan with this config would allocate (for admission control). */
hotrg_status hotrg_plan_workspace_bytes(const hotrg_config* cfg, size_t* bytes);

/* Create a plan on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream).  All device memory is allocated here. */
hotrg_status hotrg_plan_create(const hotrg_config* cfg, void* cuda_stream, hotrg_plan* out);
void hotrg_plan_destroy(hotrg_plan plan);

/* Forward from a caller tensor.  T0_host: d0^4 float64, host memory, layout
 * [l][r][u][d].  Outputs (host, may be NULL): lnz_per_site (1 value),
 * log_norms (n_steps values ln c_k), trace_sign (+1/-1 sign of the final
 * trace).  Blocks until the results are on the host. */
hotrg_status hotrg_forward_tensor(hotrg_plan plan, const double* T0_host,
                                  double* lnz_per_site, double* log_norms, int* trace_sign);

/* Forward for the square-lattice Ising model H = -J sum s_i s_j - h sum s_i
 * (s = +-1), one tensor per spin, T0 built on the device from the Boltzmann
 * weights (SM Sec. A): T0 = sum_s e^{beta h s} W[s][l] W[s][r] W[s][u] W[s][d],
 * W[s][0] = sqrt(cosh beta J), W[s][1] = s sqrt(sinh beta J).  Needs
 * beta*J >= 0 and d0 == 2.  Outputs as hotrg_forward_tensor. */
hotrg_status hotrg_forward_ising(hotrg_plan plan, double beta, double J, double h,
                                 double* lnz_per_site, double* log_norms, int* trace_sign);

/* Forward for the quantum XY chain H = J sum_i (S^x_i S^x_{i+1} + S^y_i S^y_{i+1})
 * (main text, "Infinite quantum XY chain"; needs scheme = 1 and d0 == 4).  T0 is
 * built on the device: the second-order Trotter MPO of rho(tau) (SM Sec. F),
 * rho(tau) = e^{-tau/2 H_o} e^{-tau H_e} e^{-tau/2 H_o}, one tensor per
 * two-site cell (u, d = the cell's two spins, 4 states; l, r = the operator-SVD
 * index of the bond between cells, 4 values).  After n steps the output is
 * lnz (see scheme) at beta = 2^(n+1) tau; ln Z per site = 2^n lnz, the free
 * energy per site f = -2^n lnz / beta.  tau > 0.  Outputs (host, may be NULL)
 * as hotrg_forward_tensor. */
hotrg_status hotrg_forward_xy(hotrg_plan plan, double tau, double J, double* lnz_per_copy,
                              double* log_norms);

/* Grouped forward (the solve server's grouped launch of same-shape steps of
 * different requests).  A group holds the batched operand buffers of one
 * problem shape for up to max_count plans; hotrg_forward_group_* runs the
 * forwards of `count` plans created with that config (any depths set with
 * hotrg_plan_set_steps) in lockstep: one host thread per plan issues the
 * plan's work on the plan's own stream (plans on different streams overlap
 * their eigensolves); per step each plan forms its own isometry (Gram matrix
 * and eigensolve) and, on split steps whose free leg fits one chunk, prepares
 * its operands in the group's buffers; the three contractions of all plans are
 * then ONE tensor-core launch per stage on the group's stream (each problem's
 * operand rows at its own offset of the group's buffers, ordered after every
 * plan's preparation by events), after which each plan normalises on its own
 * stream; other steps run plan by plan.  The call synchronises all streams.  Every plan ends as after its
 * own forward (results bit-identical; hotrg_backward, diagnostics and the
 * outputs work per plan).  T0_host: count * d0^4 float64 (plan i's tensor at
 * i * d0^4); beta, J, h: count values; lnz (host, may be NULL): count values.
 * Scheme 0, w_given 0 and w_rule 0 only.  Device errors of a grouped launch
 * are reported by every plan of the call.  hotrg_group_launches: grouped
 * launches issued so far. */
typedef struct hotrg_group_s* hotrg_group;
hotrg_status hotrg_group_create(const hotrg_config* cfg, int max_count, void* cuda_stream,
                                hotrg_group* out);
hotrg_status hotrg_forward_group_tensor(hotrg_group group, hotrg_plan* plans, int count,
                                        const double* T0_host, double* lnz_per_site);
hotrg_status hotrg_forward_group_ising(hotrg_group group, hotrg_plan* plans, int count,
                                       const double* beta, const double* J, const double* h,
                                       double* lnz_per_site);
unsigned long long hotrg_group_launches(hotrg_group group);
/* Device bytes hotrg_group_create would allocate (for admission control). */
hotrg_status hotrg_group_workspace_bytes(const hotrg_config* cfg, int max_count, size_t* bytes);
void hotrg_group_destroy(hotrg_group group);

/* w_rule 1: the side (0 = left, 1 = right) each step of the last forward took
 * its isometry from (host array of the steps run; all 0 for w_rule 0). */
hotrg_status hotrg_isometry_sides(hotrg_plan plan, int* side);

/* Scheme 1: lnz of every depth k = 1..n of the last forward (host array of
 * the steps run); entries before the last are NaN unless chain_steps = 1. */
hotrg_status hotrg_chain_lnz_steps(hotrg_plan plan, double* lnz_steps);

/* Device-resident forward: T0_dev is a device pointer (d0^4 float64); results
 * are written to the device buffer out_dev = [lnz_per_site, trace_sign,
 * ln c_1 .. ln c_n] (n_steps + 2 doubles).  Enqueued on the plan's stream;
 * returns without synchronising, except that with eigh_mode 1 each step's
 * eigensolver accuracy check is read on the host (see eigh_residual_tol).
 * Device-side failures (eigensolver, non-finite norm, timeouts) are reported
 * by hotrg_sync. */
hotrg_status hotrg_forward_device(hotrg_plan plan, const double* T0_dev, double* out_dev);

/* Backward after a forward (needs want_grad = 1).  dlnz_dT0_host: d0^4
 * float64 (host), d(ln Z / N)/d T0.  dlnz_dbeta_host: may be NULL; if not,
 * the last forward must have been hotrg_forward_ising, and it receives
 * d(ln Z / N)/d beta (the internal energy per site is its negative). */
hotrg_status hotrg_backward(hotrg_plan plan, double* dlnz_dT0_host, double* dlnz_dbeta_host);

/* Device-resident backward: writes d(ln Z/N)/d T0 (d0^4 float64) to grad_dev. */
hotrg_status hotrg_backward_device(hotrg_plan plan, double* grad_dev);

/* Run only the first n_steps (1 <= n_steps <= the plan's n_steps) in the
 * following forwards and backwards: the result is that of a plan created with
 * n_steps (bit for bit: every step depends only on the steps before it), so one
 * plan serves requests of any depth up to its own.  Output arrays
 * (log_norms, out_dev) then hold n_steps + 2 / n_steps values; the per-step
 * diagnostics keep the plan's length, with entries past n_steps stale. */
hotrg_status hotrg_plan_set_steps(hotrg_plan plan, int n_steps);

/* Bind the plan to another CUDA stream (NULL = legacy default stream): waits
 * for the plan's work on its current stream, then enqueues everything on the
 * new one. */
hotrg_status hotrg_plan_set_stream(hotrg_plan plan, void* cuda_stream);

/* Wait for the plan's stream and report any device-side failure. */
hotrg_status hotrg_sync(hotrg_plan plan);

/* Per-step diagnostics of the last forward (host arrays of n_steps, may be
 * NULL): trunc_err = sum of discarded eigenvalues / sum of all; cut_gap =
 * (lam_D' - lam_D'+1) / lam_1 (0 where nothing is cut); step_is_split = 1
 * where the step ran in the split tensor-core precision. */
hotrg_status hotrg_diagnostics(hotrg_plan plan, double* trunc_err, double* cut_gap,
                               int* step_is_split);

/* Eigensolver diagnostics of the last forward (host arrays of n_steps, may be
 * NULL): residual = the guard's max_a ||G v_a - theta_a v_a||_2 / theta_1 of
 * the kept Ritz pairs where the subspace eigensolver ran (NaN elsewhere and
 * where the exact solver finished the step); extra_iters = power iterations
 * the guard added to the step; exact_step = 1 where the step was finished by
 * the exact partial eigensolver; guard_steps = steps on which the guard fired
 * over the plan's lifetime. */
hotrg_status hotrg_eigh_diagnostics(hotrg_plan plan, double* residual, int* extra_iters,
                                    int* exact_step, long long* guard_steps);

/* Per-step bond dimensions of a plan: X (merged legs), Y (other legs), X' (kept). */
hotrg_status hotrg_step_dims(hotrg_plan plan, int step, int* X, int* Y, int* Xp);

const char* hotrg_status_string(hotrg_status s);
const char* hotrg_last_error(hotrg_plan plan);

/* Device capability check: HOTRG_OK if the current device can run the split
 * tensor-core path (compute capability 10.3). */
hotrg_status hotrg_device_supports_split(void);

/* ---- Solve server (continuous batching) -------------------------------------
 * Ising solves (forward, optionally backward) submitted at any time are run by
 * max_slots concurrent slots, each a host worker thread with its own CUDA
 * stream on the device current at hotrg_server_create, so requests that arrive
 * while others are on the GPU start as soon as a slot and device memory are
 * free and their kernels overlap on the device.  Every live plan is charged
 * its hotrg_plan_workspace_bytes against hbm_budget_bytes; built plans stay in
 * one pool shared by all slots for reuse by later requests of the same D_cut,
 * precision and gradient need (plans are built for 40 steps, or the request's
 * depth if larger or if a 40-step plan would not fit the budget, and run each
 * request's own depth); idle ones are freed, coldest first, when a new plan
 * would not fit, and a slot waits for a running request's plan when all
 * pooled plans are in use.  A request whose plan alone exceeds the budget
 * finishes with status HOTRG_ENOMEM.  Under backlog (every other slot busy),
 * forward-only split-precision requests with D_cut <= 32 that are queued
 * together (up to 4 of one D_cut, precision and split step) are taken by one
 * slot and run as one grouped forward
 * (hotrg_forward_group_ising: their contractions one tensor-core launch per
 * stage; each result bit-identical to the request's own solve).  Requests without gradients use the
 * randomized subspace eigensolver (eigh_mode 1, 2 power iterations).  Times are seconds since the server was
 * created.  Submit, poll, wait, drain and stats are thread-safe. */
typedef struct hotrg_server_s* hotrg_server;
typedef struct {
  double beta, J, h;        /* Ising parameters (beta * J >= 0)                     */
  int d_cut, n_steps;       /* truncation and number of steps                       */
  int want_grad;            /* 1: also run the backward and return d(lnZ/N)/d beta  */
  int precision;            /* hotrg_precision of the split steps                   */
  int split_from_step;      /* as in hotrg_config                                   */
} hotrg_request;
typedef struct {
  uint64_t ticket;
  int status;               /* hotrg_status of the solve                            */
  int slot;                 /* slot that ran it                                     */
  double lnz_per_site, dlnz_dbeta;
  double t_submit, t_start, t_finish;
} hotrg_result;
typedef struct {
  uint64_t submitted, completed, failed, plans_created, plans_evicted;
  size_t bytes_in_use, peak_bytes;
  int queue_depth, busy_slots;
  uint64_t admission_waits;  /* requests that waited for device memory before their plan */
  uint64_t grouped;          /* requests run in a grouped forward with others */
  uint64_t groups;           /* grouped forwards run */
} hotrg_server_stats;
hotrg_status hotrg_server_create(size_t hbm_budget_bytes, int max_slots, hotrg_server* out);
hotrg_status hotrg_server_submit(hotrg_server server, const hotrg_request* req, uint64_t* ticket);
/* HOTRG_EPENDING until the request has finished; then the result (kept until destroy). */
hotrg_status hotrg_server_poll(hotrg_server server, uint64_t ticket, hotrg_result* out);
hotrg_status hotrg_server_wait(hotrg_server server, uint64_t ticket, hotrg_result* out);
/* Block until the queue is empty and no slot is running. */
hotrg_status hotrg_server_drain(hotrg_server server);
hotrg_status hotrg_server_get_stats(hotrg_server server, hotrg_server_stats* out);
/* Finishes every queued request, then frees all plans and joins the slots. */
void hotrg_server_destroy(hotrg_server server);

/* Per-stage timing.  hotrg_profile_enable(plan, 1) creates a pool of CUDA
 * events (outside any forward/backward) and from then on brackets every stage
 * launch with events on the plan's stream; 0 turns it off.
 * hotrg_profile_read synchronises the stream and returns, per slot, the summed
 * milliseconds and the number of bracketed launches since the last read (both
 * arrays hold HOTRG_PROFILE_SLOTS entries; counts may be NULL), then resets.
 * Slots: 0 Gram, 1 eigensolve (+ sort/sign fix), 2 stage-1 contraction,
 * 3 stage-2 contraction (the O(D^7) GEMM), 4 stage-3 contraction, 5 norm,
 * 6 operand preparation (bf16 split), 7 backward contractions, 8 backward
 * eigensolve adjoint, 9 backward Gram adjoint, 10 stage-2 contraction of the
 * four-plane steps; inside slot 1, for the subspace eigensolver: 11 products
 * G Q (with the split of G), 12 QR, 13 Rayleigh-Ritz, 14 the residual check of
 * the kept Ritz pairs; slot + 16 = the same
 * stage run by the FP64 GEMM instead of the tensor-core GEMM. */
#define HOTRG_PROFILE_SLOTS 32
hotrg_status hotrg_profile_enable(hotrg_plan plan, int enable);
hotrg_status hotrg_profile_read(hotrg_plan plan, double* ms, int* counts);

/* Number of kernels this library has launched in this process (all plans). */
unsigned long long hotrg_kernel_launches(void);

/* Failure-detection hooks (tests of the error paths without a GPU fault).
 * hotrg_debug_inject(what, arg), process-wide until reset with what = 0:
 *   1 = the arg-th device allocation after this call fails (-> HOTRG_ENOMEM),
 *   2 = the eigensolver of step arg reports failure (-> HOTRG_ENOTCONV),
 *   3 = a NaN is written into the new tensor of step arg (-> HOTRG_ENONFINITE).
 * hotrg_check_bounded_wait(timeout_ms) runs a one-thread kernel that waits on an
 * mbarrier nothing arrives at, with the given limit instead of the library's
 * 2 s; it returns HOTRG_ETIMEOUT when the bounded wait gave up and reported it
 * (the expected outcome), leaving the device usable. */
hotrg_status hotrg_debug_inject(int what, int arg);
hotrg_status hotrg_check_bounded_wait(double timeout_ms);

/* Kernel checks (used by the test-suite; not part of the HOTRG path).
 * C = A B^T for row-major float64 host matrices A (M x K), B (N x K), C (M x N),
 * computed on the device by the split-BF16 tensor-core GEMM (planes = 2 or 3
 * bf16 planes per operand, FP32 accumulation in chunks of kchunk * 64 along K,
 * 0 = a single chunk; K must be a multiple of 8) or by the FP64 GEMM.  They
 * allocate and free temporary device memory and synchronise the device. */
hotrg_status hotrg_gemm_split_check(int M, int N, int K, int planes, int kchunk, int cta_pair,
                                    const double* A, const double* B, double* C);
                                    /* planes: 2, 3 or 4; cta_pair = 1: three planes with
                                       N > 64 run on CTA pairs (256-row tiles) */
hotrg_status hotrg_gemm_f64_check(int M, int N, int K, const double* A, const double* B, double* C);

/* Allocation-free variant of hotrg_gemm_split_check (the paper has no
 * counterpart; this is a library facility).  For callers that may not call
 * cudaMalloc: their device memory is owned by another allocator (a
 * framework's caching allocator or a fixed arena), or they run latency-bound
 * loops where an allocation would synchronise the device or could fail
 * mid-request.  The caller passes device buffers: A_dev (M x K), B_dev
 * (N x K), C_dev (M x N), row-major float64; C = A B^T as in
 * hotrg_gemm_split_check.  Scratch (the bf16 operand planes and an error
 * word) lives in a static device array of 8 MiB that every GPU loading this
 * library holds until process exit; sizes with
 * 256 + 2 * planes * (roundup64(M*K) + roundup64(N*K)) > 8 MiB are rejected
 * with HOTRG_EINVAL.  Nothing is allocated: no cudaMalloc, no cudaFree.
 * The operand planes are prepared exactly as hotrg_gemm_split_check prepares
 * them, so C is the same as that entry point's C.
 * The first call on a device does a one-time set-up: it looks up the array's
 * device address and the device's attributes (once per device, with that
 * device current); make that first call before any stream capture.  Work is
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream); the
 * call then reads the error word back and synchronises `stream`, so it
 * returns with C complete.  All calls share the one array and each call
 * overwrites the previous call's contents, so calls that overlap on the GPU
 * (other threads, other streams) race. */
hotrg_status hotrg_gemm_split_noalloc(int M, int N, int K, int planes, int kchunk,
                                      const double* A_dev, const double* B_dev, double* C_dev,
                                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HOTRG_H */
