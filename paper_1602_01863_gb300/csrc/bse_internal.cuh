// Internal declarations of the GB300 double-grid BSE Haydock library.
//
// Data layout on the device (all row-major, complex interleaved):
//   coarse  Uv [nkc][nv][nv], Uc [nkc][nc][nc]      band gauge at coarse points (FP64)
//           K_c: complex128 / complex64 [Nc][Nc], or BF16 planes Kr, Ki [Nc][ldk]
//   dense   dE [N] (vector precision), P^alpha [3][N] (FP64)
//           Dv [nk][8][nv][nv], Dc [nk][8][nc][nc]  overlaps d per corner (Eq. completeness)
//   M3      near-pair contribution lists per sub-cell position, head factors
//           Hv [nkc][nrel][nv][nv] = alpha O^v, Hc [nkc][nrel][nc][nc] = O^c, hc [nrel]
//   vectors [chain][N]; coarse vectors [chain][Nc]; per-(dense k, corner)
//           restricted pieces X and near-field results Unf [chain][nk][8][t].
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <vector>

#include "bse.h"

#define BSE_MAX_BANDS 8
#define BSE_MAX_T (BSE_MAX_BANDS * BSE_MAX_BANDS)
#define BSE_MAX_CHAINS 4
#define BSE_VEC_THREADS 256
#define BSE_MAX_VEC_BLOCKS 1024

// ------------------------------------------------------------ complex math
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ inline double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 conjg(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline float2 conjg(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

template <typename T> struct Cx;
template <> struct Cx<double> { using V = double2; };
template <> struct Cx<float> { using V = float2; };

template <typename V> __host__ __device__ inline V czero();
template <> __host__ __device__ inline double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __host__ __device__ inline float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename V> __host__ __device__ inline V from_d2(double2 a);
template <> __host__ __device__ inline double2 from_d2<double2>(double2 a) { return a; }
template <> __host__ __device__ inline float2 from_d2<float2>(double2 a) {
    return make_float2((float)a.x, (float)a.y);
}
__host__ __device__ inline double2 to_d2(double2 a) { return a; }
__host__ __device__ inline double2 to_d2(float2 a) { return make_double2(a.x, a.y); }

// --------------------------------------------------------- grid utilities
struct Int3 { int a, b, c; };

__host__ __device__ inline int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
__host__ __device__ inline int floordiv(int a, int n) { return (a - imod(a, n)) / n; }
__host__ __device__ inline Int3 unflat3(int idx, int n) { return Int3{idx / (n * n), (idx / n) % n, idx % n}; }
__host__ __device__ inline int flat3(int a, int b, int c, int n) {
    return (imod(a, n) * n + imod(b, n)) * n + imod(c, n);
}

// Interpolation prefactor f(k, k~^{lmn}) for sub-cell position js and corner l
// (l = l1*4 + l2*2 + l3): trilinear f^l_j = (1 - j/n_div | j/n_div) per axis
// (Sec. 3, Eq. interpwfn), or the one-neighbour scheme (Eq. eqRL: f = 1 on
// the nearest corner, j/n_div = 1/2 going to l = 0).
// Trilinear weight f^l_j = prod_a (l_a ? j_a / n_div : 1 - j_a / n_div) as an
// integer numerator over n_div^3 (exact for n_div <= 16); one-neighbour
// weights (nb1) are 0 or 1 with denominator 1.
__host__ __device__ inline int interp_num(int js, int l, int nd, int nb1) {
    const int j1 = js / (nd * nd), j2 = (js / nd) % nd, j3 = js % nd;
    const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
    if (nb1) return ((2 * j1 > nd) == l1 && (2 * j2 > nd) == l2 && (2 * j3 > nd) == l3) ? 1 : 0;
    return (l1 ? j1 : nd - j1) * (l2 ? j2 : nd - j2) * (l3 ? j3 : nd - j3);
}
// whether f^l_j != 0 (integer test, no division)
__host__ __device__ inline bool interp_active(int js, int l, int nd, int nb1) { return interp_num(js, l, nd, nb1) != 0; }
__host__ __device__ inline double interp_weight(int js, int l, int nd, int nb1) {
    const int num = interp_num(js, l, nd, nb1);
    return nb1 ? (double)num : (double)num / (double)(nd * nd * nd);
}
// the same weight in FP32 (one correctly rounded division)
__host__ __device__ inline float interp_weight_f(int js, int l, int nd, int nb1) {
    const int num = interp_num(js, l, nd, nb1);
    return nb1 ? (float)num : (float)num / (float)(nd * nd * nd);
}
template <typename T>
__host__ __device__ inline T interp_weight_as(int js, int l, int nd, int nb1) {
    if constexpr (sizeof(T) == sizeof(float)) return interp_weight_f(js, l, nd, nb1);
    else return interp_weight(js, l, nd, nb1);
}

// ------------------------------------------------------------------ handles
enum KernelClass { KC_RESTRICT = 0, KC_KCAPPLY = 1, KC_PROLONG = 2, KC_NEAR = 3, KC_LANCZOS = 4, KC_COUNT = 5 };

struct bse_ctx {
    long long serial = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;          // created by the context (caller passed NULL)
    std::string err;
    int* d_status = nullptr;          // device status word: bit value 1 / 2 = a bounded wait gave up in the K_c apply / near field
    double kt_ms[KC_COUNT] = {0, 0, 0, 0, 0};
    long long kt_n[KC_COUNT] = {0, 0, 0, 0, 0};
    int sm_count = 0;
    long long wait_cycles = 0;        // bounded-wait budget of the K_c apply pipeline (0: default)
    // stopping rule of BSE_STOP_CONVERGED runs (bse_set_stop_rule)
    int stop_set = 0, stop_every = 0, stop_nw = 0;
    double stop_tol = 0, stop_seps = 0, stop_eta = 0;
    double* d_stop_omega = nullptr;  // [stop_nw]
    // grow-only scratch of bse_spectrum (no allocation once large enough)
    void* cf_buf = nullptr;
    size_t cf_bytes = 0;
    // batched runs: side streams, events and the cached graph of the last batch
    cudaStream_t side[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t side_join[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t side_fork = nullptr;
    cudaGraphExec_t batch_graph = nullptr;
    std::vector<long long> batch_key;   // serials of the systems, npol, steps, flags
    // Concurrent K_c apply beside the near field: one auxiliary stream and a
    // fork / join event pair per lane (0: the context stream, 1 + k: batch side
    // stream k); `lane` is the lane whose stream ctx->stream currently is.
    cudaStream_t aux[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t aux_fork[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t aux_join[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int lane = 0;
    int prio_least = 0, prio_greatest = 0;   // stream priority range of the device
};

struct bse_coarse {
    int n = 0, nv = 0, nc = 0, t = 0, nkc = 0, Nc = 0;
    int kc_prec = 0, ldk = 0;
    double eps_inf = 0, kappa = 0, e_k = 0, e_gap = 0, band_width = 0, h0 = 0, alpha = 0;
    int direct_shells = 27, h_const = 0, exchange_on = 1;
    // model parameters on the device (FP64)
    double* d_offsets = nullptr;
    double2 *d_gen_v = nullptr, *d_gen_c = nullptr, *d_mu = nullptr, *d_dip = nullptr;
    double2 *d_Uv = nullptr, *d_Uc = nullptr;     // coarse band gauge
    void* d_kc = nullptr;                         // K_c storage
    __nv_bfloat16 *d_kr = nullptr, *d_ki = nullptr; // BF16 planes (inside d_kc)
};

struct NearEntry { int co; int js_src; int l_src; int near_idx; };   // co packed 3 x 4 bits (+8 bias)

struct bse_interp {
    const bse_coarse* co = nullptr;
    int n = 0, nd = 0, Ndiv = 0, nk = 0, N = 0, t = 0, nv = 0, nc = 0;
    int scheme = 0, nb1 = 0, vec_prec = 0;
    double width = 0;
    // Method 2: the dense interpolated Hamiltonian, complex128 [N][N]
    void* d_H2 = nullptr;
    // dense tables
    void* d_dE = nullptr;            // T [N]
    void* d_Dv = nullptr;            // V [nk][8][nv*nv]
    void* d_Dc = nullptr;            // V [nk][8][nc*nc]
    double2* d_P = nullptr;          // [3][N]
    // M3 tables
    int n_near = 0, smin = 0, ns1 = 0, nslot = 0, rmin = 0, nr1 = 0, nrel = 0;
    NearEntry* d_list = nullptr;
    int* d_list_start = nullptr;     // [Ndiv][nslot + 1]
    // cell-batched near field: active (js, corner) pairs and per-(js, slot)
    // contribution lists (source pair index | near-offset index << 16)
    int npairs = 0;
    int* d_pairs = nullptr;          // [npairs]  js | corner << 16
    int* d_clist = nullptr;
    int* d_cstart = nullptr;         // [Ndiv][nslot + 1]
    size_t cell_smem = 0;            // dynamic shared memory of the cell kernel (0: not usable)
    int nf_tc = 0;                   // the tensor-core near field serves this handle
    int nf_tc_tpad = 0;              // FP16 pieces per (dense k, corner): t rounded up to a multiple of 4
    float nf_tc_sb = 1.f;            // stage-2 operand scale (power of two)
    double dbound = 0;               // bound of ||d_v||_F ||d_c||_F over the non-zero-weight pieces
    float* d_xscale = nullptr;       // [4] FP16 piece scales of unit-norm vectors (Haydock loop)
    float* d_xscale_gen = nullptr;   // [4] piece scales computed from the input norms (bse_apply_h)
    int nf_tc_nsl = 0;               // slots that reach the cell
    int nf_tc_nkg = 0;               // their stage-1 K-blocks
    int nf_tc_nrows = 0;             // their source rows (all slots)
    void* d_tc_rows = nullptr;       // [K-blocks][32] source rows: js | corner << 8, 0xFFFF none (ushort)
    int4* d_tc_slots = nullptr;      // per slot {slot, first K-block, K-blocks, rows}
    void* d_tc_kinfo = nullptr;      // [K-blocks] slot of each K-block (uchar)
    unsigned char* d_tc_simg = nullptr;   // near pattern images, 8 KB per K-block
    unsigned char* d_tc_aimg = nullptr;   // head images, 4 KB per (coarse point, relative offset)
    int nf_force_cuda_cores = 0;     // BSE_NF_CUDA_CORES: keep the CUDA-core near-field kernels
    void* d_hd = nullptr;            // T [n_near]   h_head at dense near offsets
    void* d_Hv = nullptr;            // V [nkc][nrel][nv*nv]
    void* d_Hc = nullptr;            // V [nkc][nrel][nc*nc]
    void* d_hc = nullptr;            // T [nrel]
    // scratch (BSE_MAX_CHAINS chains)
    void* d_Q = nullptr;             // V [4][Nc]  restricted coarse vectors
    void* d_R = nullptr;             // V [4][Nc]  K_c Q
    void* d_X = nullptr;             // V [4][nk][8][t]
    void* d_U = nullptr;             // V [4][nk][8][t]
    __nv_bfloat16* d_Bop = nullptr;  // [16][ldk] split-BF16 operand of the tensor-core apply
    float* d_part = nullptr;         // chunk partials + counters of the tensor-core apply
    int tc_ctas = 0, tc_kblocks = 0; // tensor-core schedule: CTAs, k-blocks per chunk
    int tc_stages = 0;               // and pipeline depth (autotuned)
    void* tc_state = nullptr;        // tensor maps + schedule tables (bse_tc.cu)
    void* d_vec[3] = {nullptr, nullptr, nullptr};   // V [4][N]: psi_A, psi_B, w
    double2* d_part_dot = nullptr;   // [4][BSE_MAX_VEC_BLOCKS] FP64 block partials
    double* d_part_nrm = nullptr;    // [4][BSE_MAX_VEC_BLOCKS]
    // Haydock state (device)
    double* d_a = nullptr;           // [4][m]
    double* d_aim = nullptr;         // [4][m]
    double* d_b = nullptr;           // [4][m + 1]
    int* d_stop = nullptr;           // [4]  0 = running, else steps done
    int m_alloc = 0;
    void* d_basis = nullptr;         // V [4][m + 1][N] when reorthogonalising
    int basis_m = 0;
    double2* d_cgs_part = nullptr;   // [4][(m+1)][nblk]
    double2* d_cgs_h = nullptr;      // [4][m + 1]
    // learned near-diagonal residual (M1 + periodic convolution with the stencil)
    int learned = 0, learned_radius = 0;
    float2* d_lker = nullptr;        // DFT of the stencil [t][t][L^3]
    float2* d_lgrid = nullptr;       // 2 x [4][t][L^3] work grids
    float2* d_tw_fwd = nullptr;      // [2 L] twiddles (forward, inverse)
    float2* d_tw_inv = nullptr;
    // per-run buffers (kept: no allocation inside a run once they exist)
    double* d_dirs = nullptr;        // [4][3] polarisation directions
    double* d_pn2 = nullptr;         // [4]    ||P||^2
    int* d_lz_ctr = nullptr;         // finished-block counter of k_lanczos_axpy4_ab (zero between launches)
    double2* d_eps_prev = nullptr;   // [4][eps_nw] spectrum at the previous convergence check
    double* d_conv_part = nullptr;   // [4][eps_nblk][4] block maxima of a convergence check
    int eps_nw = 0;
    // cached graph of the step loop (BSE_USE_GRAPH) and what it was captured for
    cudaGraphExec_t graph = nullptr;
    long long graph_key[6] = {0, 0, 0, 0, 0, 0};   // context serial, chains, steps, flags, state serial, wait limit
    long long serial = 0;            // unique per handle (the batch graph key)
    long long state_serial = 0;      // bumped whenever buffers a captured graph uses are replaced
};

// Unique serial numbers for handles and contexts (graph cache keys).
long long bse_next_serial();
// Looks up the device address of the no-allocation scratch array on the
// context's device (bse_noalloc.cu), at context creation.
int bse_noalloc_prepare(bse_ctx* ctx);

// ----------------------------------------------------------------- helpers
#define BSE_CUDA_TRY(ctx, call)                                                       \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return BSE_ERR_CUDA;                                                      \
        }                                                                             \
    } while (0)

int bse_alloc(bse_ctx* ctx, void** p, size_t bytes, const char* what);

// Status word bits raised by bounded device waits: 1 = tensor-core K_c apply,
// 2 = tensor-core near field.
inline const char* bse_timeout_message(int status) {
    if (status & 2) return "a bounded device wait in the tensor-core near field gave up";
    return "a bounded device wait in the tensor-core K_c apply gave up";
}

// setup kernels (bse_setup.cu)
int bse_setup_coarse_device(bse_ctx* ctx, bse_coarse* c, const void* user_kc);
int bse_setup_interp_device(bse_ctx* ctx, bse_interp* s, const bse_dense_inputs* dense);

// hot path (bse_apply.cu)
int bse_apply_once(bse_ctx* ctx, bse_interp* s, int nvec, const void* x, void* y, bool profile);
int bse_run_chains(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, int nsteps,
                   int flags, double* a, double* b, double* pnorm2, int* steps_done);
void bse_release_run_state(bse_interp* s);
void bse_invalidate_graph(bse_interp* s);   // a cached step-loop graph no longer matches the handle
void bse_release_ctx_state(bse_ctx* ctx);
int bse_prepare_aux(bse_ctx* ctx);          // auxiliary streams of the concurrent K_c apply
int bse_run_batch(bse_ctx* ctx, bse_interp* const* sys, int nsys, const int* npol, const double* pol_dirs, int m,
                  int flags, double* a, double* b, double* pnorm2, int* steps_done);
int bse_make_dipoles(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, void* p_out,
                     double* pnorm2);
int bse_cf_device(bse_ctx* ctx, int nchains, int nsteps, const int* steps_done, const double* a,
                  const double* b, const double* pnorm2, double prefactor, double eta, int nw,
                  const double* omega, double* eps);

// tensor-core K_c apply (bse_tc.cu)
int bse_tc_prepare(bse_ctx* ctx, bse_interp* s);
// prio: launch with scheduling priority prio_value (used when the apply runs
// beside the near field on an auxiliary stream).
int bse_tc_apply(bse_ctx* ctx, bse_interp* s, int nchains, cudaStream_t stream, bool prio, int prio_value);
void bse_tc_release(bse_interp* s);

// Per-call scratch of one H application, supplied by the caller instead of the
// handle (used by the no-allocation entry point, bse_noalloc.cu).
struct ApplyScratch {
    void* Q;                 // V [nvec][Nc]       (complex128 / complex64 paths)
    void* R;                 // V [nvec][Nc]
    void* X;                 // V [nvec][nk][8][t] (M3 only)
    void* U;                 // V [nvec][nk][8][t] (M3 only)
    double2* dot;            // [nvec][BSE_MAX_VEC_BLOCKS]
    __nv_bfloat16* bop;      // [16][ldk]          (BF16 path only)
    float* part;             // tile partials      (BF16 path only)
};
int bse_launch_near_field(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, const float* xscale, void* U);
int bse_apply_learned(bse_ctx* ctx, const bse_interp* s, int nchains, const void* psi, void* w, double2* dot);
int bse_near_tc_prepare(bse_ctx* ctx, bse_interp* s, const std::vector<std::vector<NearEntry>>& per_slot);
int bse_near_tc_launch(bse_ctx* ctx, const bse_interp* s, int nchains, const void* Xh, const float* xscale, void* U,
                       bool prio = false, int prio_value = 0);
float bse_near_tc_xscale(const bse_interp* s, double norm);
size_t bse_tc_part_bytes(const bse_interp* s);
int bse_tc_apply_scratch(bse_ctx* ctx, const bse_interp* s, int nchains, __nv_bfloat16* bop, float* part, void* R);
int bse_apply_scratch(bse_ctx* ctx, const bse_interp* s, int nvec, const void* x, void* y, const ApplyScratch& sc);
