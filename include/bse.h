/*
 * bse.h - C ABI of the GB300 double-grid BSE Haydock library.
 *
 * The library computes the macroscopic dielectric function of the
 * Bethe-Salpeter equation in the Tamm-Dancoff approximation (Sec. 2,
 * Eqs. bse1, epsmacro) with the Lanczos-Haydock recursion (Eqs. ai, bi, ci)
 * and its continued fraction (Eq. fraccont).  Every Lanczos step applies the
 * dense-mesh Hamiltonian H = diag(Delta E) + K^i, with K^i interpolated on
 * the fly from the coarse-mesh kernel K_c (Sec. 4, Eqs. interpmatmul,
 * matmul1-matmul3: restrict -> K_c apply -> prolong), optionally with the
 * near-diagonal treatment of the small-q divergence ("Method 3", Sec. 4,
 * Eq. diverg).
 *
 * Conventions shared by every call
 *   - All functions are extern "C", thread-compatible (one context per host
 *     thread), and return an int status: 0 = BSE_OK, < 0 an error, > 0 a
 *     warning.  bse_last_error(ctx) returns a message for the last failure.
 *   - "host" pointers are read or written during the call only.  "device"
 *     pointers are CUDA global-memory addresses on the context's device
 *     (e.g. torch tensor data_ptr()); the caller keeps them alive for the
 *     call.  Handles own their device memory and free it in bse_free_*.
 *   - Complex numbers are interleaved (re, im) pairs: double2 for complex128,
 *     float2 for complex64.
 *   - Meshes (Sec. 3): coarse k~_(i) = i / n, i in [0, n)^3, coarse index
 *     ic = (i1 n + i2) n + i3.  Dense k = (i + j / n_div) / n, j in
 *     [0, n_div)^3, dense index coarse-major kd = ic * n_div^3 + js,
 *     js = (j1 n_div + j2) n_div + j3.  Transition index tr = v * nc + c.
 *     A vector of the transition space has N = t * N_k entries, t = nv * nc,
 *     element kd * t + tr.
 *   - There is no CPU fallback: without a CUDA device every call that needs
 *     one returns BSE_ERR_CUDA.
 */
#ifndef BSE_H
#define BSE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
#define BSE_OK                0
#define BSE_ERR_ARG          -1   /* bad size, pointer, flag or non-finite input  */
#define BSE_ERR_OOM          -2   /* device allocation failed                    */
#define BSE_ERR_CUDA         -3   /* CUDA runtime error (message has the detail) */
#define BSE_ERR_TIMEOUT      -4   /* a bounded device wait gave up               */
#define BSE_ERR_UNSUPPORTED  -5   /* combination not built (e.g. size limits)    */
#define BSE_WARN_BREAKDOWN    1   /* some chain stopped early: b_{i+1} ~ 0       */

/* -------------------------------------------------------------- precisions */
#define BSE_PREC_F64   0   /* complex128 storage / FP64 arithmetic                  */
#define BSE_PREC_F32   1   /* complex64 storage / FP32 arithmetic                   */
#define BSE_PREC_BF16  2   /* K_c as separate BF16 real and imaginary planes,
                              applied on the tensor cores with FP32 accumulation   */

/* ----------------------------------------------------------------- schemes */
#define BSE_SCHEME_M1   0  /* Method 1: interpolation everywhere (Sec. 4)           */
#define BSE_SCHEME_M3   1  /* Method 3: M1 plus divergence treatment on near pairs  */
#define BSE_SCHEME_M2   2  /* Method 2: the coefficients of Eq. diverg interpolated
                              for every pair and divided by the dense q; the whole
                              H is stored (complex128, N <= 16384)                 */
#define BSE_NB1        16  /* OR-flag: one-neighbour weights (Eq. eqRL, f = 1 on
                              the nearest coarse corner) instead of trilinear 8NB   */
#define BSE_NF_CUDA_CORES 32 /* OR-flag: apply the M3 near field on the CUDA cores
                              even where the tensor-core kernel applies (FP32
                              vectors, t <= 16, n_div <= 4); same result to
                              TF32 rounding of the head blocks and y1, z        */

/* ------------------------------------------------------------ Haydock flags */
#define BSE_REORTH_CGS2   1  /* full reorthogonalisation, classical Gram-Schmidt x2 */
#define BSE_USE_GRAPH     2  /* run the step loop as a CUDA graph; the instantiated
                                graph is kept in the handle (or, for a batch, in
                                the context) and replayed by the next run with
                                the same chains, steps and flags                    */
#define BSE_PROFILE       4  /* time the kernel classes with events (see
                                bse_last_kernel_times)                              */
#define BSE_STOP_CONVERGED 8 /* stop each chain once its spectrum has converged by
                                the rule set with bse_set_stop_rule (Sec. 5.1)      */

/* Synthetic model crystal (stand-in for the ab initio inputs of Sec. 2,
 * Eqs. bse2-bse3b).  All arrays are host, row-major, complex interleaved:
 *   offsets [nv][nc]          real, eV
 *   gen_v   [3][2][nv][nv]    Hermitian gauge generators (axis, kind sin / 1-cos)
 *   gen_c   [3][2][nc][nc]
 *   mu      [7][26][nv][nc]   exchange form-factor coefficients per k-harmonic
 *                             (1, cos 2pi k1, sin 2pi k1, cos k2, sin k2, cos k3,
 *                             sin k3) and non-zero G in {-1,0,1}^3 (lexicographic)
 *   dip     [7][3][nv][nc]    dipole coefficients per harmonic and direction
 * Band gauge U_b(k) = expm(i sum_a [sin(2 pi k_a) gen[a][0] + (1 - cos 2 pi k_a) gen[a][1]]);
 * overlaps d = U(k~)^H U(k) (Eq. completeness); kernel on a grid of N_g points
 *   K = (e_k / N_g) [ 2 sum_{G!=0} (4 pi / |G|^2) conj(M_vc(k,G)) M_v'c'(k',G)
 *                     - (1 / eps_inf) O^v_vv'(k,k') O^c_cc'(k,k') h(k - k') ],
 * M = U_v^H mu U_c, O^v = U_v(k)^T conj(U_v(k')), O^c = U_c(k)^H U_c(k'),
 * h(q) = sum_G exp(-|G|^2) 4 pi / (|q + G|^2 + kappa^2) over direct_shells G
 * (27 or the G = 0 shell only), q the minimum image (ties averaged), or
 * h = h0 when h_const.  Delta E_vc(k) = e_gap + band_width sum_i (1 - cos 2 pi k_i)
 * + offsets[v][c].  Dipoles P_vc = [U_v^T pi(k) conj(U_c)]_vc.                  */
typedef struct bse_model {
    int nv, nc;
    double eps_inf, kappa, e_k, e_gap, band_width;
    int direct_shells;        /* 27 or 1 */
    int h_const;              /* 0 / 1   */
    double h0;
    int exchange_on;          /* 0 / 1   */
    const double* offsets;
    const double* gen_v;
    const double* gen_c;
    const double* mu;
    const double* dip;
} bse_model;

typedef struct bse_ctx bse_ctx;
typedef struct bse_coarse bse_coarse;
typedef struct bse_interp bse_interp;

/* Library version (major * 10000 + minor * 100 + patch). */
int bse_version(void);

/* Create a context on `device`.  `cuda_stream` is a cudaStream_t (e.g. a
 * torch.cuda.Stream's cuda_stream); every kernel and copy of the context is
 * issued on it.  NULL makes the context create (and later destroy) a blocking
 * stream of its own, ordered with the legacy default stream.  Returns
 * BSE_ERR_CUDA when no device is present. */
int bse_ctx_create(bse_ctx** out, int device, void* cuda_stream);
void bse_ctx_destroy(bse_ctx* ctx);
const char* bse_last_error(const bse_ctx* ctx);

/* Coarse-mesh BSE data (Sec. 3-4): builds on the device the band gauge at the
 * n^3 coarse points, the coarse kernel K_c (Eq. bse2 with the model of
 * bse_model, dimension N_c = t n^3, Hermitian) stored in `kc_prec`
 * (BSE_PREC_F64 complex128, BSE_PREC_F32 complex64, BSE_PREC_BF16 planes),
 * and the head factors of Eq. diverg (the G = 0 direct term,
 * A_c = alpha O^v (x) O^c with alpha = -(e_k / n^3) 4 pi / eps_inf).
 * `user_kc` (nullable) is a device complex128 [N_c][N_c] row-major K_c
 * (Sec. 4: the coarse BSE matrix elements computed elsewhere, e.g. from ab
 * initio wavefunctions) that replaces the model's kernel; it is read during
 * the call only and converted to `kc_prec`.  The model still supplies the
 * band gauge (overlaps d and the Method-3 head factors) and the sizes; with a
 * user K_c, Method 3 takes c = K_c - A_c h_head(q_c) for the remainder.  A
 * non-finite user K_c entry is stored as it is and propagates.
 * Errors: BSE_ERR_ARG (nv, nc outside 1..8, n < 1, non-finite model numbers,
 * direct_shells not 1 or 27), BSE_ERR_OOM, BSE_ERR_CUDA. */
int bse_build_coarse(bse_ctx* ctx, const bse_model* model, int n_coarse, int kc_prec,
                     const void* user_kc, bse_coarse** out);
/* Copy K_c to host as complex128 [N_c][N_c] (converted from its storage). */
int bse_coarse_get_kc(bse_ctx* ctx, const bse_coarse* coarse, double* host_kc);
void bse_free_coarse(bse_coarse* coarse);

/* Dense-mesh inputs supplied by the caller instead of the model (all host,
 * complex numbers interleaved, dense points in the coarse-major order above,
 * N = t N_k):
 *   dE  [N]                 real, Delta E_vck = e_ck - e_vk (Eq. bse1), eV
 *   P   [3][N]              complex128, dipoles P^alpha_vck (Eq. epsmacro)
 *   Dv  [N_k][8][nv][nv]    complex128, Dv[kd][l][n'][v] = d_{v k}^{n' k~_l}, the
 *   Dc  [N_k][8][nc][nc]    overlaps of Eq. completeness with the 8 coarse corners
 *                           k~_l = k~(i + (l1, l2, l3)), l = 4 l1 + 2 l2 + l3
 *                           (corners of zero weight are not read)
 * Any pointer may be NULL: that table then comes from the model.  Read during
 * bse_interp_setup only.  Non-finite entries are rejected (BSE_ERR_ARG). */
typedef struct bse_dense_inputs {
    const double* dE;
    const double* P;
    const double* Dv;
    const double* Dc;
} bse_dense_inputs;

/* Interpolation set-up for one dense mesh refining `coarse` by n_div per
 * axis (Sec. 3): dense Delta E (exact on the dense mesh), dipoles P^alpha,
 * band overlaps d for every (dense k, coarse corner) with a non-zero weight
 * (Eq. completeness, v-c mixing neglected as in Sec. 5.1), trilinear or
 * one-neighbour weights (Eqs. interpwfn, eqRL), and for BSE_SCHEME_M3 the
 * near-pair tables: pairs with ||k - k'|| <= width_w * d, d one coarse
 * spacing, tested on the integer dense offset delta as
 * |delta|^2 <= floor(width_w^2 n_div^2 + 1e-9).
 * `vec_prec` (F64 or F32) is the precision of the Lanczos vectors and of the
 * restrict / prolong / near-field arithmetic; the Lanczos reductions sum
 * across warps and blocks in FP64 in every mode (with F32 vectors each
 * thread first sums its few products in FP32, and the ||w||^2 of the Lanczos
 * update is also summed over a warp's 32 threads in FP32).  The coarse
 * handle must outlive the interp handle.
 * With BF16 K_c the set-up autotunes the tensor-core apply: it times its
 * pipeline depths (4, 5, 6 stages) and chunk lengths (8 to 64 k-blocks) on
 * this K_c and keeps the fastest (cached per shape for the process;
 * bse_interp_kc_plan reports the choice).
 * BSE_SCHEME_M2 (Sec. 4, Method 2) builds the dense interpolated Hamiltonian
 *   H = diag(Delta E) + (1/N_div)[(F A F^H) h_head(q_dense) + F (K_c - A h_head(q_coarse)) F^H]
 * for every pair (no width; F of Eq. interpwfn, A the head for every coarse pair)
 * once, stored as complex128 [N][N], and every H application is a dense
 * product with it: complex128 K_c and vectors, N <= 16384 (else
 * BSE_ERR_UNSUPPORTED), the Yukawa direct term (h_const = 0).
 * `dense` (nullable) replaces the model's dense tables (bse_dense_inputs).
 * Errors: BSE_ERR_ARG (n_div < 1; M3 with width_w >= n / 2, where the near
 * region would wrap around the zone; bad flags; non-finite dense inputs),
 * BSE_ERR_OOM, BSE_ERR_CUDA. */
int bse_interp_setup(bse_ctx* ctx, const bse_coarse* coarse, int n_div, int scheme,
                     double width_w, int vec_prec, const bse_dense_inputs* dense, bse_interp** out);
void bse_free_interp(bse_interp* interp);

/* Sizes of an interp handle: info[0] = N (dense dimension), [1] = N_k,
 * [2] = N_c (coarse dimension), [3] = t, [4] = n, [5] = n_div,
 * [6] = number of near offsets (M3, else 0), [7] = vec_prec. */
int bse_interp_info(const bse_interp* interp, long long* info);

/* Launch shape the set-up's autotuner chose for the tensor-core K_c apply
 * (BF16 K_c only; Eq. matmul2): plan[0] = pipeline stages (TMA ring depth),
 * plan[1] = k-blocks of 64 columns per work chunk, plan[2] = CTAs.
 * Host array `plan` [3], written on success.  Errors: BSE_ERR_ARG (NULL),
 * BSE_ERR_UNSUPPORTED (K_c not BF16). */
int bse_interp_kc_plan(const bse_interp* interp, int* plan);

/* Dipole start vectors P(e) = sum_alpha e_alpha P^alpha for `npol`
 * directions (host [npol][3]) into device `p_out` [npol][N] in the interp's
 * vector precision, and their squared norms (FP64) into host `pnorm2` [npol]. */
int bse_dipoles(bse_ctx* ctx, bse_interp* interp, int npol, const double* pol_dirs,
                void* p_out, double* pnorm2);

/* One application y = H x of the interpolated dense Hamiltonian
 * (Eqs. interpmatmul, matmul1-3, plus the M3 near-field when set up) to
 * `nvec` (1..4) device vectors x [nvec][N] -> y [nvec][N] in the interp's
 * vector precision.  Uses the handle's scratch; calls on the same handle
 * must not overlap. */
int bse_apply_h(bse_ctx* ctx, bse_interp* interp, int nvec, const void* x, void* y);

/* Same result as bse_apply_h, but allocates no device memory: the per-call
 * scratch comes from one static device array of 32 MiB inside the library
 * (held by a device from the time the library's device module is loaded on
 * it, at the latest the first bse_ctx_create on that device, until the
 * process exits), not from the handle.  The paper has no counterpart; this
 * exists for callers that must not call cudaMalloc once their work has
 * started, such as a host framework that owns all device memory through its
 * own pool, or a loop where cudaMalloc's implicit device synchronisation is
 * not allowed.  bse_ctx_create looks up the array's device address
 * (cudaGetSymbolAddress, with that device current), which also loads the
 * module under lazy loading; create the context before any stream capture.
 * All calls share the array and it keeps the
 * previous call's contents (what must start at zero is cleared each call):
 * calls that overlap on the GPU race.  Sizes whose scratch does not fit
 * (nvec vectors of Q and R, for M3 the per-corner pieces, for BF16 the
 * operand and tile partials) return BSE_ERR_UNSUPPORTED with the byte count
 * in bse_last_error.  Other errors as bse_apply_h. */
int bse_apply_h_noalloc(bse_ctx* ctx, bse_interp* interp, int nvec, const void* x, void* y);

/* Stopping rule for BSE_STOP_CONVERGED runs (Sec. 5.1: the chains were
 * stopped once the whole dielectric spectrum changed by less than 1 % in its
 * real and in its imaginary part).  Every `check_every` steps each chain
 * evaluates eps(omega) on the device (Eq. fraccont, FP64, the steps done so
 * far) with eps = 1 - (s_eps / N_k) ||P||^2 g_1(omega + i eta) on the `nw`
 * frequencies `omega` (host, copied), and stops at the first check where
 *   max_w |Re eps - Re eps_prev| <= tol max_w |Re eps|   and
 *   max_w |Im eps - Im eps_prev| <= tol max_w |Im eps|,
 * eps_prev being the previous check's spectrum (so no chain stops before
 * 2 check_every steps).  steps_done then reports the steps run.  Such a chain
 * is not a breakdown: it does not raise BSE_WARN_BREAKDOWN.  A single system
 * run with this flag is issued check by check and ends as soon as every chain
 * has stopped (BSE_USE_GRAPH is then not used); in a batch the stopped chains
 * skip their work inside the one graph.  The rule stays set on the context.
 * Errors: BSE_ERR_ARG (tol <= 0, check_every < 1, eta <= 0, nw < 1,
 * non-finite numbers), BSE_ERR_OOM, BSE_ERR_CUDA. */
int bse_set_stop_rule(bse_ctx* ctx, double tol, int check_every, double s_eps, double eta, int nw,
                      const double* omega);

/* Haydock recursion (Eqs. ai, bi, ci) for `nsys` systems sharing the context.
 * System s runs npol[s] (1..4) chains starting from P(e) for the directions
 * pol_dirs (host, 3 doubles per chain, systems in order).  nsteps Lanczos
 * steps per chain.  Outputs (host, chains in order):
 *   a          [chains][nsteps]       a_1 .. a_m
 *   b          [chains][nsteps + 1]   b_1 = 0, b_2 .. b_{m+1}
 *   pnorm2     [chains]               ||P||^2
 *   steps_done [chains]               m, or fewer after a breakdown
 * With BSE_USE_GRAPH and nsys > 1 the whole batch is captured as one CUDA
 * graph (each system's loop on its own branch, longest systems spread over up
 * to 8 concurrent branches) and launched once; the results equal the
 * systems run one by one.  Each handle may appear once (it owns the scratch).
 * flags: BSE_REORTH_CGS2, BSE_USE_GRAPH, BSE_PROFILE, BSE_STOP_CONVERGED.  A
 * chain whose b_{i+1} < 1e-12 max|a| stops there (BSE_WARN_BREAKDOWN).
 * Device waits are bounded; a wait that gives up returns BSE_ERR_TIMEOUT.
 * No device memory is allocated after the first run of a handle with a given
 * number of steps (the per-run buffers live in the handle). */
int bse_haydock_run(bse_ctx* ctx, bse_interp* const* sys, int nsys, const int* npol,
                    const double* pol_dirs, int nsteps, int flags, double* a, double* b,
                    double* pnorm2, int* steps_done);

/* Testing aid for the failure path: the clock-cycle budget of the bounded
 * mbarrier waits in the pipeline of the tensor-core K_c apply (`cycles` = 0
 * restores the default, about 2 s).  A budget too short for a normal launch
 * makes its first wait give up: the kernel raises its status bit, drains its
 * copies and MMAs under the default budget, frees its tensor memory and
 * returns, and the call returns BSE_ERR_TIMEOUT with the status word cleared,
 * so the context stays usable.  Errors: BSE_ERR_ARG (cycles < 0). */
int bse_ctx_set_wait_limit(bse_ctx* ctx, long long cycles);

/* Kernel-class device times of the last BSE_PROFILE run, averaged per
 * launch, in ms: [0] restrict, [1] K_c apply, [2] prolong+diagonal,
 * [3] M3 near field, [4] Lanczos vector updates; counts[] launches. */
int bse_last_kernel_times(const bse_ctx* ctx, double* ms_per_launch, long long* counts);

/* Continued fraction (Eq. fraccont) on the device, FP64, bottom-up,
 * truncated after steps_done[c] levels:
 *   eps_c(w) = 1 - prefactor * pnorm2[c] * g_1(w + i eta)
 * a [nchains][nsteps], b [nchains][nsteps + 1] as returned by
 * bse_haydock_run; omega [nw]; eps out [nchains][nw] complex128.  All host. */
int bse_spectrum(bse_ctx* ctx, int nchains, int nsteps, const int* steps_done,
                 const double* a, const double* b, const double* pnorm2, double prefactor,
                 double eta, int nw, const double* omega, double* eps);

/* ------------------------------------------------------------------------
 * Learned near-diagonal residual.  Not in the paper: a small network
 * predicts N_k (K_explicit - K_M1) for dense pairs closer than a radius, and
 * its evaluation, as a Hermitian translation-invariant stencil, is added to
 * the M1 Hamiltonian in place of the Method-3 treatment.  M1 without it stays
 * the fallback and the reference its error is judged against.
 *
 * Network: d_in -> 128 -> 128 -> 128 -> 2, exact-erf GELU, BF16 weights,
 * FP32 activations and accumulation, FP32 master weights and Adam state.
 * Parameters (FP32, d_in = 6 + 2 t for a system with t transitions):
 * W1 [128][d_in], b1 [128], W2 [128][128], b2, W3 [128][128], b3,
 * W4 [2][128], b4 [2].  Inputs per (k, k', vc, v'c'): q (3, minimum image of
 * k - k' on orthonormal axes), |q|, onehot(vc) [t], onehot(v'c') [t],
 * dE_vc(k), dE_v'c'(k').  Device buffers X [batch][d_in], Y and out
 * [batch][2] are FP32.                                                       */
typedef struct bse_mlp bse_mlp;

/* Number of FP32 parameters for input size d_in. */
int bse_mlp_param_count(int d_in);
/* Network with host initial parameters init_params [bse_mlp_param_count]
 * (the caller draws them), able to process batches up to max_batch. */
int bse_mlp_create(bse_ctx* ctx, int d_in, int max_batch, const float* init_params, bse_mlp** out);
void bse_mlp_free(bse_mlp* mlp);
/* Copy the FP32 master parameters to host. */
int bse_mlp_get_params(bse_ctx* ctx, const bse_mlp* mlp, float* host_params);
/* Inference with the BF16 weights: out [batch][2] (device). */
int bse_mlp_forward(bse_ctx* ctx, bse_mlp* mlp, int batch, const float* X, float* out);
/* Gradients of the loss mean_b sum_{re,im} (out - Y)^2 with respect to the
 * parameters (host, FP32, parameter layout) and the loss; no update. */
int bse_mlp_gradients(bse_ctx* ctx, bse_mlp* mlp, int batch, const float* X, const float* Y,
                      float* grad_host, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on that
 * loss with learning rate lr; *loss gets the loss before the step. */
int bse_mlp_train_step(bse_ctx* ctx, bse_mlp* mlp, int batch, const float* X, const float* Y, float lr,
                       double* loss);
/* Training data from the method: for nblocks sampled dense pairs
 * (host_kd[i], host_kd2[i]) of `interp` (complex128 or complex64 K_c,
 * t <= 24), all t x t entries: features X [nblocks t^2][6 + 2t] and targets
 * Y = N_k (K_explicit - K_M1) [nblocks t^2][2] (device), row order
 * (pair, vc, v'c').  K_explicit is the model kernel on the dense mesh in FP64
 * (Eqs. bse2-bse3b with the model); K_M1 = (1/N_div) F K_c F^H (Eq. interp1). */
int bse_pairs_generate(bse_ctx* ctx, const bse_interp* interp, int nblocks, const int* host_kd,
                       const int* host_kd2, float* X, float* Y);
/* Evaluate `mlp` once over every dense offset delta with |delta| < radius
 * (dense steps) and every band pair, with each dE input at its average over
 * the dense mesh, symmetrise it to a Hermitian stencil T(delta) =
 * [out(delta) + out(-delta)^H] / (2 N_k), and add (T * psi)(k) =
 * sum_delta T(delta) psi(k - delta) (periodic convolution, computed with
 * separable DFTs) to every H application of `interp` (an M1 handle).
 * mlp = NULL switches the correction off.  Requires 1 <= radius <= L/2,
 * L = n n_div. */
int bse_interp_set_learned(bse_ctx* ctx, bse_interp* interp, bse_mlp* mlp, int radius);

#ifdef __cplusplus
}
#endif

#endif /* BSE_H */
