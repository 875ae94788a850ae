// Learned near-diagonal residual: MLP training / inference kernels, pair-data
// generation from the method itself, and the learned correction applied as a
// periodic convolution on the dense mesh.
//
// Network (not in the paper): x -> 128 -> 128 -> 128 -> 2 with exact-erf GELU,
// BF16 weights, FP32 activations and accumulation, FP32 master weights and
// Adam state.  Parameter layout (FP32 master, gradients, Adam moments, and the
// BF16 weight copy share it): W1 [w][d_in], b1 [w], W2 [w][w], b2 [w],
// W3 [w][w], b3 [w], W4 [2][w], b4 [2].
//
// Inputs per (dense k, dense k', vc, v'c'): q (3, minimum image of k - k',
// orthonormal axes), |q|, onehot(vc) [t], onehot(v'c') [t], dE_vc(k),
// dE_v'c'(k').  Target: N_k (K_explicit - K_M1) (Re, Im).
#include <cmath>
#include <type_traits>
#include <vector>

#include "bse_dmat.cuh"
#include "bse_internal.cuh"

namespace {

constexpr int W = 128;
constexpr int TPB = 256;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// z = in W^T + b (and h = gelu(z) when ACT): 32 rows per block, W^T staged in
// shared memory as BF16, FP32 accumulation.
template <bool ACT>
__global__ void __launch_bounds__(TPB) k_lin_fwd(const float* __restrict__ in, int K, const __nv_bfloat16* __restrict__ Wt,
                                                 const float* __restrict__ bias, int N, int B, float* __restrict__ z,
                                                 float* __restrict__ h) {
    extern __shared__ unsigned char sm[];
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(sm);        // [K][N]
    float* Xs = reinterpret_cast<float*>(Ws + ((K * N + 7) / 8) * 8); // [32][K]
    const int r0 = blockIdx.x * 32;
    for (int i = threadIdx.x; i < K * N; i += TPB) {
        const int n = i / K, k = i % K;
        Ws[k * N + n] = Wt[(size_t)n * K + k];
    }
    for (int i = threadIdx.x; i < 32 * K; i += TPB) {
        const int r = i / K, k = i % K;
        Xs[i] = (r0 + r < B) ? in[(size_t)(r0 + r) * K + k] : 0.f;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 32 * N; o += TPB) {
        const int r = o / N, n = o % N;
        if (r0 + r >= B) continue;
        float acc = bias[n];
        for (int k = 0; k < K; ++k) acc = fmaf(Xs[r * K + k], __bfloat162float(Ws[k * N + n]), acc);
        z[(size_t)(r0 + r) * N + n] = acc;
        if (ACT) h[(size_t)(r0 + r) * N + n] = gelu_f(acc);
    }
}

// dzprev[b][k] = (sum_n dz[b][n] W[n][k]) * gelu'(zprev[b][k])
__global__ void __launch_bounds__(TPB) k_lin_bwd_data(const float* __restrict__ dz, int N, const __nv_bfloat16* __restrict__ Wt,
                                                      int K, int B, const float* __restrict__ zprev, float* __restrict__ dzprev) {
    const long long i = (long long)blockIdx.x * TPB + threadIdx.x;
    if (i >= (long long)B * K) return;
    const int b = (int)(i / K), k = (int)(i % K);
    float acc = 0.f;
    for (int n = 0; n < N; ++n) acc = fmaf(dz[(size_t)b * N + n], __bfloat162float(Wt[(size_t)n * K + k]), acc);
    dzprev[i] = acc * gelu_grad_f(zprev[i]);
}

// dW[n][k] = sum_b dz[b][n] in[b][k] (k < K), db[n] = sum_b dz[b][n] (k == K);
// one thread per output, batch summed in order.
__global__ void __launch_bounds__(TPB) k_lin_bwd_weight(const float* __restrict__ dz, int N, const float* __restrict__ in,
                                                        int K, int B, float* __restrict__ dW, float* __restrict__ db) {
    const int i = blockIdx.x * TPB + threadIdx.x;
    if (i >= N * (K + 1)) return;
    const int n = i / (K + 1), k = i % (K + 1);
    float acc = 0.f;
    if (k < K)
        for (int b = 0; b < B; ++b) acc = fmaf(dz[(size_t)b * N + n], in[(size_t)b * K + k], acc);
    else
        for (int b = 0; b < B; ++b) acc += dz[(size_t)b * N + n];
    if (k < K) dW[(size_t)n * K + k] = acc;
    else db[n] = acc;
}

// dout = 2 (out - y) / B, block partial sums of the squared error
__global__ void __launch_bounds__(TPB) k_mse(const float* __restrict__ out, const float* __restrict__ y, int n, float inv_b,
                                             float* __restrict__ dout, double* __restrict__ part) {
    __shared__ double sh[TPB];
    double s = 0.0;
    for (int i = blockIdx.x * TPB + threadIdx.x; i < n; i += gridDim.x * TPB) {
        const float d = out[i] - y[i];
        dout[i] = 2.f * d * inv_b;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = TPB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam on the FP32 master copy; BF16 weight copy refreshed (biases stay FP32).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    wbf[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, int n, __nv_bfloat16* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace

// ------------------------------------------------------------------ handle
struct bse_mlp {
    int d_in = 0, nparams = 0, max_batch = 0, step = 0;
    float* d_p = nullptr;                // master FP32
    float* d_g = nullptr;                // gradients
    float* d_m = nullptr;
    float* d_v = nullptr;
    __nv_bfloat16* d_w = nullptr;        // BF16 copy
    float* d_z[4] = {nullptr, nullptr, nullptr, nullptr};   // pre-activations [B][N_i]
    float* d_h[3] = {nullptr, nullptr, nullptr};            // activations
    float* d_dz[4] = {nullptr, nullptr, nullptr, nullptr};  // gradients of z
    double* d_part = nullptr;
};

namespace {

struct Layout {
    size_t off_w[4], off_b[4];
    int in_dim[4], out_dim[4];
};

Layout layout(int d_in) {
    Layout L;
    const int dims[5] = {d_in, W, W, W, 2};
    size_t o = 0;
    for (int i = 0; i < 4; ++i) {
        L.in_dim[i] = dims[i];
        L.out_dim[i] = dims[i + 1];
        L.off_w[i] = o;
        o += (size_t)dims[i + 1] * dims[i];
        L.off_b[i] = o;
        o += dims[i + 1];
    }
    return L;
}

int nparams_for(int d_in) { return (int)(W * d_in + W + 2 * (W * W + W) + 2 * W + 2); }

void free_mlp(bse_mlp* m) {
    if (!m) return;
    cudaFree(m->d_p); cudaFree(m->d_g); cudaFree(m->d_m); cudaFree(m->d_v); cudaFree(m->d_w);
    for (int i = 0; i < 4; ++i) { cudaFree(m->d_z[i]); cudaFree(m->d_dz[i]); }
    for (int i = 0; i < 3; ++i) cudaFree(m->d_h[i]);
    cudaFree(m->d_part);
    delete m;
}

size_t fwd_smem(int K, int N) { return sizeof(__nv_bfloat16) * (((size_t)K * N + 7) / 8) * 8 + sizeof(float) * 32 * K; }

// Forward over a batch; the output pre-activation lands in d_z[3] ([B][2]).
int mlp_forward(bse_ctx* ctx, bse_mlp* m, int B, const float* X) {
    const Layout L = layout(m->d_in);
    const float* in = X;
    for (int i = 0; i < 4; ++i) {
        const int K = L.in_dim[i], N = L.out_dim[i];
        const size_t sm = fwd_smem(K, N);
        const int blocks = (B + 31) / 32;
        if (i < 3) {
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_lin_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_lin_fwd<true><<<blocks, TPB, sm, ctx->stream>>>(in, K, m->d_w + L.off_w[i], m->d_p + L.off_b[i], N, B,
                                                              m->d_z[i], m->d_h[i]);
            in = m->d_h[i];
        } else {
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_lin_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_lin_fwd<false><<<blocks, TPB, sm, ctx->stream>>>(in, K, m->d_w + L.off_w[i], m->d_p + L.off_b[i], N, B,
                                                               m->d_z[3], nullptr);
        }
    }
    return BSE_OK;
}

// Loss and gradients into m->d_g; the loss (mean over the batch of the squared
// error summed over Re, Im) into *loss.
int mlp_grads(bse_ctx* ctx, bse_mlp* m, int B, const float* X, const float* Y, double* loss) {
    const Layout L = layout(m->d_in);
    mlp_forward(ctx, m, B, X);
    const int nblk = std::min(256, (2 * B + TPB - 1) / TPB);
    k_mse<<<nblk, TPB, 0, ctx->stream>>>(m->d_z[3], Y, 2 * B, 1.f / B, m->d_dz[3], m->d_part);
    for (int i = 3; i >= 0; --i) {
        const int K = L.in_dim[i], N = L.out_dim[i];
        const float* in = (i == 0) ? X : m->d_h[i - 1];
        k_lin_bwd_weight<<<(N * (K + 1) + TPB - 1) / TPB, TPB, 0, ctx->stream>>>(m->d_dz[i], N, in, K, B,
                                                                               m->d_g + L.off_w[i], m->d_g + L.off_b[i]);
        if (i > 0)
            k_lin_bwd_data<<<(int)(((long long)B * K + TPB - 1) / TPB), TPB, 0, ctx->stream>>>(
                m->d_dz[i], N, m->d_w + L.off_w[i], K, B, m->d_z[i - 1], m->d_dz[i - 1]);
    }
    std::vector<double> part(nblk);
    BSE_CUDA_TRY(ctx, cudaMemcpyAsync(part.data(), m->d_part, sizeof(double) * nblk, cudaMemcpyDeviceToHost, ctx->stream));
    BSE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (double v : part) s += v;
    if (loss) *loss = s / B;
    return BSE_OK;
}

}  // namespace

// ================================================ pair data from the method
namespace {

// Band gauge at integer grid point g (L points per axis) from the generators.
__device__ void gauge_at(const double2* gen, int nb, const int g[3], int L, double2* U) {
    double2 A[BSE_MAX_BANDS * BSE_MAX_BANDS];
    for (int i = 0; i < nb * nb; ++i) A[i] = make_double2(0.0, 0.0);
    for (int a = 0; a < 3; ++a) {
        double s, c;
        sincospi(2.0 * g[a] / L, &s, &c);
        const double2* g0 = gen + (a * 2) * nb * nb;
        const double2* g1 = gen + (a * 2 + 1) * nb * nb;
        for (int i = 0; i < nb * nb; ++i) A[i] = cadd(A[i], cadd(cscale(g0[i], s), cscale(g1[i], 1.0 - c)));
    }
    dmat_expm_i(A, nb, U);
}

// One CTA per sampled dense pair (k, k'): the t x t blocks of the explicit
// model kernel (FP64, dense weight e_k / N_k) and of K^{M1} = (1/N_div) F K_c F^H
// (FP32 from the handle's tables), written as network features and targets.
template <typename T>
__global__ void __launch_bounds__(576) k_pairs(
    const int* __restrict__ kd1, const int* __restrict__ kd2, int nblocks, const double2* __restrict__ gen_v,
    const double2* __restrict__ gen_c, const double2* __restrict__ mu, const typename Cx<T>::V* __restrict__ Kc,
    const typename Cx<T>::V* __restrict__ Dv, const typename Cx<T>::V* __restrict__ Dc, const T* __restrict__ dE,
    int n, int nd, int nv, int nc, int nb1, double e_k, double inv_eps, double kappa, int shells, int exchange_on,
    int d_in, float* __restrict__ X, float* __restrict__ Y) {
    using V = typename Cx<T>::V;
    const int blk = blockIdx.x;
    if (blk >= nblocks) return;
    const int t = nv * nc, Ndiv = nd * nd * nd, L = n * nd, nk = n * n * n * Ndiv, Nc = t * n * n * n;
    constexpr int PT = 24;                     // t <= 24 (checked by the host)
    __shared__ double2 Uv[2][BSE_MAX_BANDS * BSE_MAX_BANDS], Uc[2][BSE_MAX_BANDS * BSE_MAX_BANDS];
    __shared__ double2 M[2][26][PT];
    __shared__ float2 Fa[PT * PT], Fb[PT * PT], Tm[PT * PT];
    __shared__ double hq;
    const int kk[2] = {kd1[blk], kd2[blk]};
    int g[2][3];
    for (int s = 0; s < 2; ++s) {
        const int cell = kk[s] / Ndiv, js = kk[s] % Ndiv;
        const Int3 ci = unflat3(cell, n), j = unflat3(js, nd);
        g[s][0] = ci.a * nd + j.a; g[s][1] = ci.b * nd + j.b; g[s][2] = ci.c * nd + j.c;
    }
    if (threadIdx.x < 2) gauge_at(gen_v, nv, g[threadIdx.x], L, Uv[threadIdx.x]);
    else if (threadIdx.x < 4) gauge_at(gen_c, nc, g[threadIdx.x - 2], L, Uc[threadIdx.x - 2]);
    else if (threadIdx.x == 4) {
        // direct-term shape h(k - k') on the dense grid (minimum image, ties averaged)
        int cand[3][2], ncand[3];
        for (int a = 0; a < 3; ++a) {
            const int r = imod(g[0][a] - g[1][a], L);
            if (2 * r < L) { cand[a][0] = r; ncand[a] = 1; }
            else if (2 * r > L) { cand[a][0] = r - L; ncand[a] = 1; }
            else { cand[a][0] = r; cand[a][1] = r - L; ncand[a] = 2; }
        }
        double acc = 0.0;
        int cnt = 0;
        for (int x = 0; x < ncand[0]; ++x)
            for (int y = 0; y < ncand[1]; ++y)
                for (int z = 0; z < ncand[2]; ++z) {
                    const double q[3] = {(double)cand[0][x] / L, (double)cand[1][y] / L, (double)cand[2][z] / L};
                    double v = 0.0;
                    for (int ga = -1; ga <= 1; ++ga)
                        for (int gb = -1; gb <= 1; ++gb)
                            for (int gc = -1; gc <= 1; ++gc) {
                                const int g2 = ga * ga + gb * gb + gc * gc;
                                if (shells == 1 && g2 != 0) continue;
                                const double qa = q[0] + ga, qb = q[1] + gb, qc = q[2] + gc;
                                v += exp(-(double)g2) * 4.0 * kPi / (qa * qa + qb * qb + qc * qc + kappa * kappa);
                            }
                    acc += v;
                    ++cnt;
                }
        hq = acc / cnt;
    }
    __syncthreads();
    // exchange form factors M_vc(k, G) = [U_v^H mu(k, G) U_c]_vc at both points
    for (int idx = threadIdx.x; idx < 2 * 26 * t; idx += blockDim.x) {
        const int s = idx / (26 * t), G = (idx / t) % 26, tr = idx % t, v = tr / nc, c = tr % nc;
        double hm[7];
        hm[0] = 1.0;
        for (int a = 0; a < 3; ++a) {
            double sn, cs;
            sincospi(2.0 * g[s][a] / L, &sn, &cs);
            hm[1 + 2 * a] = cs;
            hm[2 + 2 * a] = sn;
        }
        double2 acc = make_double2(0.0, 0.0);
        for (int mm = 0; mm < nv; ++mm)
            for (int mp = 0; mp < nc; ++mp) {
                double2 mv = make_double2(0.0, 0.0);
                for (int h = 0; h < 7; ++h) mv = cadd(mv, cscale(mu[((size_t)(h * 26 + G) * nv + mm) * nc + mp], hm[h]));
                acc = cadd(acc, cmul(cmulc(Uv[s][mm * nv + v], mv), Uc[s][mp * nc + c]));
            }
        M[s][G][tr] = acc;
    }
    // K^{M1} block, accumulated in Tm via the factored form
    float2 kacc = make_float2(0.f, 0.f);
    const int e1 = threadIdx.x / t, e2 = threadIdx.x % t;        // (vc, v'c') of this thread (blockDim >= t*t)
    const bool mine = threadIdx.x < t * t;
    const int cell0 = kk[0] / Ndiv, js0 = kk[0] % Ndiv, cell1 = kk[1] / Ndiv, js1 = kk[1] % Ndiv;
    const Int3 c0 = unflat3(cell0, n), c1 = unflat3(cell1, n);
    for (int l = 0; l < 8; ++l) {
        const double fa = interp_weight(js0, l, nd, nb1);
        if (fa == 0.0) continue;
        const int ca = flat3(c0.a + ((l >> 2) & 1), c0.b + ((l >> 1) & 1), c0.c + (l & 1), n);
        __syncthreads();
        // Fa[(vc), (n1 n2)] = f d_v^{n1} conj(d_c^{n2})
        for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
            const int row = idx / t, col = idx % t;
            const int v = row / nc, c = row % nc, n1 = col / nc, n2 = col % nc;
            const double2 dv = to_d2(Dv[((size_t)kk[0] * 8 + l) * nv * nv + n1 * nv + v]);
            const double2 dc = to_d2(Dc[((size_t)kk[0] * 8 + l) * nc * nc + n2 * nc + c]);
            const double2 f = cscale(cmul(dv, conjg(dc)), fa);
            Fa[idx] = make_float2((float)f.x, (float)f.y);
        }
        for (int lp = 0; lp < 8; ++lp) {
            const double fb = interp_weight(js1, lp, nd, nb1);
            if (fb == 0.0) continue;
            const int cb = flat3(c1.a + ((lp >> 2) & 1), c1.b + ((lp >> 1) & 1), c1.c + (lp & 1), n);
            __syncthreads();
            for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
                const int row = idx / t, col = idx % t;
                const int v = row / nc, c = row % nc, n3 = col / nc, n4 = col % nc;
                const double2 dv = to_d2(Dv[((size_t)kk[1] * 8 + lp) * nv * nv + n3 * nv + v]);
                const double2 dc = to_d2(Dc[((size_t)kk[1] * 8 + lp) * nc * nc + n4 * nc + c]);
                const double2 f = cscale(cmul(dv, conjg(dc)), fb);
                Fb[idx] = make_float2((float)f.x, (float)f.y);                    // F(k', k~'): conj taken below
            }
            __syncthreads();
            // Tm = Fa K_c(ca, cb)
            for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
                const int row = idx / t, col = idx % t;
                float2 s = make_float2(0.f, 0.f);
                for (int q = 0; q < t; ++q) {
                    const float2 a = Fa[row * t + q];
                    const double2 kv = to_d2(Kc[(size_t)(ca * t + q) * Nc + cb * t + col]);
                    const float2 k = make_float2((float)kv.x, (float)kv.y);
                    s = cadd(s, cmul(a, k));
                }
                Tm[idx] = s;
            }
            __syncthreads();
            if (mine) {       // K^{M1}[e1][e2] += sum_q Tm[e1][q] conj(Fb[e2][q])
                for (int q = 0; q < t; ++q) kacc = cadd(kacc, cmul(Tm[e1 * t + q], conjg(Fb[e2 * t + q])));
            }
        }
    }
    __syncthreads();
    if (!mine) return;
    // explicit element
    const int v = e1 / nc, c = e1 % nc, v2 = e2 / nc, c2 = e2 % nc;
    double2 ex = make_double2(0.0, 0.0);
    if (exchange_on) {
        int G = 0;
        for (int ga = -1; ga <= 1; ++ga)
            for (int gb = -1; gb <= 1; ++gb)
                for (int gc = -1; gc <= 1; ++gc) {
                    const int g2 = ga * ga + gb * gb + gc * gc;
                    if (g2 == 0) continue;
                    ex = cadd(ex, cscale(cmulc(M[0][G][e1], M[1][G][e2]), 4.0 * kPi / g2));
                    ++G;
                }
    }
    double2 ov = make_double2(0.0, 0.0), oc = make_double2(0.0, 0.0);
    for (int mm = 0; mm < nv; ++mm) ov = cadd(ov, cmulc(Uv[1][mm * nv + v2], Uv[0][mm * nv + v]));
    for (int mm = 0; mm < nc; ++mm) oc = cadd(oc, cmulc(Uc[0][mm * nc + c], Uc[1][mm * nc + c2]));
    const double2 kx = cscale(csub(cscale(ex, 2.0), cscale(cmul(ov, oc), hq * inv_eps)), e_k / nk);
    const double2 km1 = cscale(make_double2(kacc.x, kacc.y), 1.0 / Ndiv);
    const size_t row = (size_t)blk * t * t + threadIdx.x;
    Y[2 * row] = (float)((kx.x - km1.x) * nk);
    Y[2 * row + 1] = (float)((kx.y - km1.y) * nk);
    // features
    float* x = X + row * d_in;
    for (int i = 0; i < d_in; ++i) x[i] = 0.f;
    double qq = 0.0;
    for (int a = 0; a < 3; ++a) {
        int d = imod(g[0][a] - g[1][a], L);
        if (2 * d >= L) d -= L;
        const double q = (double)d / L;
        x[a] = (float)q;
        qq += q * q;
    }
    x[3] = (float)sqrt(qq);
    x[4 + e1] = 1.f;
    x[4 + t + e2] = 1.f;
    x[4 + 2 * t] = (float)dE[(size_t)kk[0] * t + e1];
    x[5 + 2 * t] = (float)dE[(size_t)kk[1] * t + e2];
}

}  // namespace

// ========================================== learned correction (stencil conv)
namespace {

// features of every (near offset, vc, v'c') with dE at its zone average
__global__ void k_stencil_features(const int* __restrict__ offs, int noff, int L, int t, const float* __restrict__ dEavg,
                                   int d_in, float* __restrict__ X) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)noff * t * t) return;
    const int o = (int)(i / (t * t)), e1 = (int)((i / t) % t), e2 = (int)(i % t);
    float* x = X + i * d_in;
    for (int k = 0; k < d_in; ++k) x[k] = 0.f;
    float qq = 0.f;
    for (int a = 0; a < 3; ++a) {
        const float q = (float)offs[3 * o + a] / L;
        x[a] = q;
        qq += q * q;
    }
    x[3] = sqrtf(qq);
    x[4 + e1] = 1.f;
    x[4 + t + e2] = 1.f;
    x[4 + 2 * t] = dEavg[e1];
    x[5 + 2 * t] = dEavg[e2];
}

// zone average of dE per transition (fixed order)
template <typename T>
__global__ void k_dE_avg(const T* __restrict__ dE, int nk, int t, float* __restrict__ out) {
    __shared__ double sh[256];
    const int tr = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < nk; k += 256) s += (double)dE[(size_t)k * t + tr];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[tr] = (float)(sh[0] / nk);
}

// T(delta) = (out(delta) + conj(out(-delta))^T) / (2 N_k), scattered onto the
// periodic grid kernel ker[e1][e2][x][y][z].
__global__ void k_stencil_scatter(const float* __restrict__ out, const int* __restrict__ offs, const int* __restrict__ neg,
                                  int noff, int L, int t, float inv_nk, float2* __restrict__ ker) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)noff * t * t) return;
    const int o = (int)(i / (t * t)), e1 = (int)((i / t) % t), e2 = (int)(i % t);
    const long long j = ((long long)neg[o] * t + e2) * t + e1;
    const float re = 0.5f * (out[2 * i] + out[2 * j]) * inv_nk;
    const float im = 0.5f * (out[2 * i + 1] - out[2 * j + 1]) * inv_nk;
    const int x = imod(offs[3 * o], L), y = imod(offs[3 * o + 1], L), z = imod(offs[3 * o + 2], L);
    ker[(((size_t)e1 * t + e2) * L + x) * L * L + (size_t)y * L + z] = make_float2(re, im);
}

// One axis of a separable DFT on [chan][L][L][L]: out_j = sum_n in_n w^{j n},
// w = exp(sign 2 pi i / L) taken from the table tw [L].
__global__ void k_dft_axis(const float2* __restrict__ in, float2* __restrict__ out, int L, long long nchan, int axis,
                           const float2* __restrict__ tw) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long L3 = (long long)L * L * L;
    if (i >= nchan * L3) return;
    const long long ch = i / L3;
    const int r = (int)(i % L3);
    const int x = r / (L * L), y = (r / L) % L, z = r % L;
    const int j = axis == 0 ? x : (axis == 1 ? y : z);
    const long long stride = axis == 0 ? (long long)L * L : (axis == 1 ? L : 1);
    const long long base = ch * L3 + r - (long long)j * stride;
    float2 acc = make_float2(0.f, 0.f);
    int ph = 0;
    for (int nn = 0; nn < L; ++nn) {
        acc = cadd(acc, cmul(in[base + nn * stride], tw[ph]));
        ph += j;
        if (ph >= L) ph -= L;
    }
    out[i] = acc;
}

// psi [chain][kd t + tr] -> grid [chain][tr][x][y][z]
template <typename T>
__global__ void k_to_grid(const typename Cx<T>::V* __restrict__ psi, int nchains, int n, int nd, int t,
                          float2* __restrict__ grid) {
    const int nk = n * n * n * nd * nd * nd, Ndiv = nd * nd * nd, L = n * nd;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nchains * nk * t) return;
    const int ch = (int)(i / ((long long)nk * t)), rem = (int)(i % ((long long)nk * t));
    const int kd = rem / t, tr = rem % t;
    const Int3 ci = unflat3(kd / Ndiv, n), j = unflat3(kd % Ndiv, nd);
    const int x = ci.a * nd + j.a, y = ci.b * nd + j.b, z = ci.c * nd + j.c;
    const double2 v = to_d2(psi[i]);
    grid[(((size_t)ch * t + tr) * L + x) * L * L + (size_t)y * L + z] = make_float2((float)v.x, (float)v.y);
}

// per frequency: out[ch][e1][xi] = sum_e2 That[e1][e2][xi] in[ch][e2][xi]; one
// thread per (e1, xi) serves every chain, so That is read once.
__global__ void __launch_bounds__(256) k_freq_mul(const float2* __restrict__ That, const float2* __restrict__ in,
                                                  int nchains, int t, int L3, float2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)t * L3) return;
    const int e1 = (int)(i / L3), xi = (int)(i % L3);
    float2 acc[BSE_MAX_CHAINS];
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) acc[ch] = make_float2(0.f, 0.f);
    for (int e2 = 0; e2 < t; ++e2) {
        const float2 T = That[((size_t)e1 * t + e2) * L3 + xi];
#pragma unroll
        for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch)
            if (ch < nchains) acc[ch] = cadd(acc[ch], cmul(T, in[((size_t)ch * t + e2) * L3 + xi]));
    }
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch)
        if (ch < nchains) out[((size_t)ch * t + e1) * L3 + xi] = acc[ch];
}

// One axis of the separable DFT, in place, on [chan][L][L][L] (L <= 64): a CTA
// stages 32 lines along `axis` in shared memory (loads and stores coalesced),
// and warp w computes outputs w, w + 8, ... of line `lane`:
// out_k = sum_n in_n w^{k n} with w^j = tw[j], in two stages (below).
__global__ void __launch_bounds__(256) k_dft_tile(float2* __restrict__ a, int L, long long nlines, int axis,
                                                  const float2* __restrict__ tw_g) {
    extern __shared__ float2 dsm[];
    const int P = (L & 1) ? L + 2 : L + 1;              // odd row pitch: conflict-free 8-byte rows
    float2* tw = dsm;
    float2* din = tw + 64;
    float2* dout = din + 32 * P;
    const long long L2 = (long long)L * L, L3 = L2 * L;
    const long long g0 = (long long)blockIdx.x * 32;
    for (int j = threadIdx.x; j < L; j += blockDim.x) tw[j] = tw_g[j];
    // line g = (ch L + u) L + v; element n of it at base + n * stride
    auto base = [&](long long g) -> long long {
        const long long ch = g / L2;
        const int u = (int)((g / L) % L), v = (int)(g % L);
        if (axis == 0) return ch * L3 + (long long)u * L + v;
        if (axis == 1) return ch * L3 + (long long)u * L2 + v;
        return ch * L3 + (long long)u * L2 + (long long)v * L;
    };
    const long long stride = axis == 0 ? L2 : (axis == 1 ? L : 1);
    const int n_el = 32 * L;
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
        const int l = axis == 2 ? i / L : i % 32, n = axis == 2 ? i % L : i / 32;
        const long long g = g0 + l;
        if (g < nlines) din[l * P + n] = a[base(g) + n * stride];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Two-stage Cooley-Tukey with L = A B (A the largest divisor <= sqrt L):
    // n = B n1 + n2, k = k1 + A k2,
    //   Y[n2][k1] = w^{n2 k1} sum_{n1} x[B n1 + n2] w^{B n1 k1}      (stage 1, into dout)
    //   X[k1 + A k2] = sum_{n2} Y[n2][k1] w^{A n2 k2}                 (stage 2, into din)
    // with every power of w read from the table (index mod L).
    int A = 1;
    for (int d = 2; d * d <= L; ++d)
        if (L % d == 0) A = d;
    const int B = L / A;
    for (int q = warp; q < L; q += 8) {
        const int n2 = q / A, k1 = q - n2 * A;
        float2 acc = make_float2(0.f, 0.f);
        int ph = 0;
        const int dph = (B * k1) % L;
        for (int n1 = 0; n1 < A; ++n1) {
            acc = cadd(acc, cmul(din[lane * P + B * n1 + n2], tw[ph]));
            ph += dph;
            if (ph >= L) ph -= L;
        }
        dout[lane * P + q] = cmul(acc, tw[(n2 * k1) % L]);
    }
    __syncthreads();
    for (int k = warp; k < L; k += 8) {
        const int k2 = k / A, k1 = k - k2 * A;
        float2 acc = make_float2(0.f, 0.f);
        int ph = 0;
        const int dph = (A * k2) % L;
        for (int n2 = 0; n2 < B; ++n2) {
            acc = cadd(acc, cmul(dout[lane * P + n2 * A + k1], tw[ph]));
            ph += dph;
            if (ph >= L) ph -= L;
        }
        din[lane * P + k] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
        const int l = axis == 2 ? i / L : i % 32, n = axis == 2 ? i % L : i / 32;
        const long long g = g0 + l;
        if (g < nlines) a[base(g) + n * stride] = din[l * P + n];
    }
}

// w[ch][kd t + tr] += grid[ch][tr][g(kd)] / L^3, and block partials of <psi, w>
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_add_learned(const float2* __restrict__ grid, const typename Cx<T>::V* __restrict__ psi,
                                                                 typename Cx<T>::V* __restrict__ w, int nchains, int n, int nd, int t,
                                                                 float scale, double2* __restrict__ part) {
    using V = typename Cx<T>::V;
    __shared__ double2 red[BSE_MAX_CHAINS][BSE_VEC_THREADS];
    const int nk = n * n * n * nd * nd * nd, Ndiv = nd * nd * nd, L = n * nd;
    const long long N = (long long)nk * t;
    double2 dot[BSE_MAX_CHAINS];
    float2 dotf[BSE_MAX_CHAINS];
    for (int c = 0; c < BSE_MAX_CHAINS; ++c) {
        dot[c] = make_double2(0.0, 0.0);
        dotf[c] = make_float2(0.f, 0.f);
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int kd = (int)(i / t), tr = (int)(i % t);
        const Int3 ci = unflat3(kd / Ndiv, n), j = unflat3(kd % Ndiv, nd);
        const int x = ci.a * nd + j.a, y = ci.b * nd + j.b, z = ci.c * nd + j.c;
        for (int ch = 0; ch < nchains; ++ch) {
            const float2 gv = grid[(((size_t)ch * t + tr) * L + x) * L * L + (size_t)y * L + z];
            if constexpr (std::is_same<T, float>::value) {
                // FP32 vectors: the update and this thread's products in FP32 (FP64 is slow per
                // element on GB300); the sums over threads below stay FP64
                const float2 wv = w[(size_t)ch * N + i];
                const float2 nw = make_float2(fmaf(gv.x, scale, wv.x), fmaf(gv.y, scale, wv.y));
                w[(size_t)ch * N + i] = nw;
                const float2 p = psi[(size_t)ch * N + i];
                for (int c = 0; c < BSE_MAX_CHAINS; ++c)
                    if (c == ch) {
                        dotf[c].x = fmaf(p.x, nw.x, fmaf(p.y, nw.y, dotf[c].x));
                        dotf[c].y = fmaf(p.x, nw.y, fmaf(-p.y, nw.x, dotf[c].y));
                    }
            } else {
                const double2 wv = to_d2(w[(size_t)ch * N + i]);
                const V nw = from_d2<V>(make_double2(wv.x + (double)gv.x * scale, wv.y + (double)gv.y * scale));
                w[(size_t)ch * N + i] = nw;
                const double2 p = to_d2(psi[(size_t)ch * N + i]), q = to_d2(nw);
                for (int c = 0; c < BSE_MAX_CHAINS; ++c)
                    if (c == ch) { dot[c].x += p.x * q.x + p.y * q.y; dot[c].y += p.x * q.y - p.y * q.x; }
            }
        }
    }
    if constexpr (std::is_same<T, float>::value)
        for (int c = 0; c < BSE_MAX_CHAINS; ++c) dot[c] = make_double2((double)dotf[c].x, (double)dotf[c].y);
    for (int c = 0; c < BSE_MAX_CHAINS; ++c) red[c][threadIdx.x] = dot[c];
    __syncthreads();
    for (int st = BSE_VEC_THREADS / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int c = 0; c < BSE_MAX_CHAINS; ++c) red[c][threadIdx.x] = cadd(red[c][threadIdx.x], red[c][threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x < nchains) part[(size_t)threadIdx.x * BSE_MAX_VEC_BLOCKS + blockIdx.x] = red[threadIdx.x][0];
}

int dft3(bse_ctx* ctx, float2* a, float2* tmp, int L, long long nchan, const float2* tw) {
    const long long tot = nchan * L * L * L;
    if (L <= 64) {
        // in place, one tile of 32 lines per CTA and axis
        const long long nlines = nchan * L * L;
        const int P = (L & 1) ? L + 2 : L + 1;
        const size_t smem = sizeof(float2) * (64 + 2 * 32 * (size_t)P);
        static bool attr = false;
        if (!attr) {
            BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_dft_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
            attr = true;
        }
        const unsigned blocks = (unsigned)((nlines + 31) / 32);
        for (int axis = 0; axis < 3; ++axis) k_dft_tile<<<blocks, 256, smem, ctx->stream>>>(a, L, nlines, axis, tw);
        return BSE_OK;
    }
    const int blocks = (int)((tot + 255) / 256);
    k_dft_axis<<<blocks, 256, 0, ctx->stream>>>(a, tmp, L, nchan, 0, tw);
    k_dft_axis<<<blocks, 256, 0, ctx->stream>>>(tmp, a, L, nchan, 1, tw);
    k_dft_axis<<<blocks, 256, 0, ctx->stream>>>(a, tmp, L, nchan, 2, tw);
    BSE_CUDA_TRY(ctx, cudaMemcpyAsync(a, tmp, sizeof(float2) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
    return BSE_OK;
}

}  // namespace

// Learned term for nchains vectors: w += T * psi (periodic convolution via
// separable DFTs), with the <psi, w> partials recomputed.
int bse_apply_learned(bse_ctx* ctx, const bse_interp* s, int nchains, const void* psi, void* w, double2* dot) {
    const int L = s->n * s->nd, t = s->t;
    const long long L3 = (long long)L * L * L;
    const long long nchan = (long long)nchains * t;
    float2* g = s->d_lgrid;
    float2* tmp = s->d_lgrid + (size_t)BSE_MAX_CHAINS * t * L3;
    const long long tot = (long long)nchains * s->nk * t;
    if (s->vec_prec == BSE_PREC_F64)
        k_to_grid<double><<<(int)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)psi, nchains, s->n, s->nd, t, g);
    else
        k_to_grid<float><<<(int)((tot + 255) / 256), 256, 0, ctx->stream>>>((const float2*)psi, nchains, s->n, s->nd, t, g);
    int rc = dft3(ctx, g, tmp, L, nchan, s->d_tw_fwd);
    if (rc != BSE_OK) return rc;
    k_freq_mul<<<(int)(((long long)t * L3 + 255) / 256), 256, 0, ctx->stream>>>(s->d_lker, g, nchains, t, (int)L3, tmp);
    rc = dft3(ctx, tmp, g, L, nchan, s->d_tw_inv);
    if (rc != BSE_OK) return rc;
    const int nb = (int)std::min<long long>(std::max<long long>((s->N + BSE_VEC_THREADS - 1) / BSE_VEC_THREADS, 1), BSE_MAX_VEC_BLOCKS);
    const float scale = 1.f / (float)L3;
    if (s->vec_prec == BSE_PREC_F64)
        k_add_learned<double><<<nb, BSE_VEC_THREADS, 0, ctx->stream>>>(tmp, (const double2*)psi, (double2*)w, nchains, s->n,
                                                                      s->nd, t, scale, dot);
    else
        k_add_learned<float><<<nb, BSE_VEC_THREADS, 0, ctx->stream>>>(tmp, (const float2*)psi, (float2*)w, nchains, s->n,
                                                                     s->nd, t, scale, dot);
    return BSE_OK;
}

// ================================================================ C ABI
extern "C" {

int bse_mlp_param_count(int d_in) { return d_in >= 1 ? nparams_for(d_in) : BSE_ERR_ARG; }

int bse_mlp_create(bse_ctx* ctx, int d_in, int max_batch, const float* init_params, bse_mlp** out) {
    if (!ctx || !out || !init_params) return BSE_ERR_ARG;
    *out = nullptr;
    if (d_in < 1 || d_in > 4096 || max_batch < 1 || max_batch > (1 << 22)) {
        ctx->err = "d_in must be in 1..4096 and max_batch in 1..2^22";
        return BSE_ERR_ARG;
    }
    const int np = nparams_for(d_in);
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(init_params[i])) { ctx->err = "non-finite initial parameter"; return BSE_ERR_ARG; }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    bse_mlp* m = new bse_mlp();
    m->d_in = d_in;
    m->nparams = np;
    m->max_batch = max_batch;
    const Layout L = layout(d_in);
    int rc = BSE_OK;
    auto A = [&](void** p, size_t bytes, const char* what) { if (rc == BSE_OK) rc = bse_alloc(ctx, p, bytes, what); };
    A((void**)&m->d_p, sizeof(float) * np, "MLP parameters");
    A((void**)&m->d_g, sizeof(float) * np, "MLP gradients");
    A((void**)&m->d_m, sizeof(float) * np, "Adam m");
    A((void**)&m->d_v, sizeof(float) * np, "Adam v");
    A((void**)&m->d_w, sizeof(__nv_bfloat16) * np, "BF16 weights");
    for (int i = 0; i < 4; ++i) {
        A((void**)&m->d_z[i], sizeof(float) * (size_t)max_batch * L.out_dim[i], "MLP pre-activations");
        A((void**)&m->d_dz[i], sizeof(float) * (size_t)max_batch * L.out_dim[i], "MLP gradients of z");
    }
    for (int i = 0; i < 3; ++i) A((void**)&m->d_h[i], sizeof(float) * (size_t)max_batch * W, "MLP activations");
    A((void**)&m->d_part, sizeof(double) * 256, "loss partials");
    if (rc != BSE_OK) { free_mlp(m); return rc; }
    cudaMemcpy(m->d_p, init_params, sizeof(float) * np, cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, sizeof(float) * np);
    cudaMemset(m->d_v, 0, sizeof(float) * np);
    k_to_bf16<<<(np + 255) / 256, 256, 0, ctx->stream>>>(m->d_p, np, m->d_w);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { free_mlp(m); ctx->err = "MLP set-up failed"; return BSE_ERR_CUDA; }
    *out = m;
    return BSE_OK;
}

void bse_mlp_free(bse_mlp* m) { free_mlp(m); }

int bse_mlp_get_params(bse_ctx* ctx, const bse_mlp* m, float* host) {
    if (!ctx || !m || !host) return BSE_ERR_ARG;
    BSE_CUDA_TRY(ctx, cudaMemcpy(host, m->d_p, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost));
    return BSE_OK;
}

int bse_mlp_forward(bse_ctx* ctx, bse_mlp* m, int batch, const float* X, float* out) {
    if (!ctx || !m || !X || !out) return BSE_ERR_ARG;
    if (batch < 1 || batch > m->max_batch) { ctx->err = "batch outside 1..max_batch"; return BSE_ERR_ARG; }
    mlp_forward(ctx, m, batch, X);
    BSE_CUDA_TRY(ctx, cudaMemcpyAsync(out, m->d_z[3], sizeof(float) * 2 * batch, cudaMemcpyDeviceToDevice, ctx->stream));
    BSE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return BSE_OK;
}

int bse_mlp_gradients(bse_ctx* ctx, bse_mlp* m, int batch, const float* X, const float* Y, float* grad_host, double* loss) {
    if (!ctx || !m || !X || !Y || !grad_host) return BSE_ERR_ARG;
    if (batch < 1 || batch > m->max_batch) { ctx->err = "batch outside 1..max_batch"; return BSE_ERR_ARG; }
    int rc = mlp_grads(ctx, m, batch, X, Y, loss);
    if (rc != BSE_OK) return rc;
    BSE_CUDA_TRY(ctx, cudaMemcpy(grad_host, m->d_g, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost));
    return BSE_OK;
}

int bse_mlp_train_step(bse_ctx* ctx, bse_mlp* m, int batch, const float* X, const float* Y, float lr, double* loss) {
    if (!ctx || !m || !X || !Y) return BSE_ERR_ARG;
    if (batch < 1 || batch > m->max_batch || !(lr > 0.f)) { ctx->err = "bad batch or learning rate"; return BSE_ERR_ARG; }
    int rc = mlp_grads(ctx, m, batch, X, Y, loss);
    if (rc != BSE_OK) return rc;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<(m->nparams + 255) / 256, 256, 0, ctx->stream>>>(m->d_p, m->d_g, m->d_m, m->d_v, m->nparams, lr, b1, b2, 1e-8f,
                                                              c1, c2, m->d_w);
    BSE_CUDA_TRY(ctx, cudaGetLastError());
    return BSE_OK;
}

int bse_pairs_generate(bse_ctx* ctx, const bse_interp* s, int nblocks, const int* host_kd, const int* host_kd2, float* X,
                       float* Y) {
    if (!ctx || !s || !host_kd || !host_kd2 || !X || !Y || nblocks < 1) return BSE_ERR_ARG;
    const bse_coarse* c = s->co;
    if (c->kc_prec == BSE_PREC_BF16) { ctx->err = "pair data needs a complex128 or complex64 K_c"; return BSE_ERR_UNSUPPORTED; }
    if (s->t > 24) { ctx->err = "pair data supports t <= 24"; return BSE_ERR_UNSUPPORTED; }
    const int pthreads = std::max(64, (s->t * s->t + 31) / 32 * 32);
    for (int i = 0; i < nblocks; ++i)
        if (host_kd[i] < 0 || host_kd[i] >= s->nk || host_kd2[i] < 0 || host_kd2[i] >= s->nk) {
            ctx->err = "dense index out of range";
            return BSE_ERR_ARG;
        }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    int *d1 = nullptr, *d2 = nullptr;
    int rc;
    if ((rc = bse_alloc(ctx, (void**)&d1, sizeof(int) * nblocks, "pair indices")) != BSE_OK) return rc;
    if ((rc = bse_alloc(ctx, (void**)&d2, sizeof(int) * nblocks, "pair indices")) != BSE_OK) { cudaFree(d1); return rc; }
    cudaMemcpy(d1, host_kd, sizeof(int) * nblocks, cudaMemcpyHostToDevice);
    cudaMemcpy(d2, host_kd2, sizeof(int) * nblocks, cudaMemcpyHostToDevice);
    const int d_in = 6 + 2 * s->t;
    if (s->vec_prec == BSE_PREC_F64)
        k_pairs<double><<<nblocks, pthreads, 0, ctx->stream>>>(d1, d2, nblocks, c->d_gen_v, c->d_gen_c, c->d_mu, (const double2*)c->d_kc,
                                                         (const double2*)s->d_Dv, (const double2*)s->d_Dc, (const double*)s->d_dE,
                                                         s->n, s->nd, s->nv, s->nc, s->nb1, c->e_k, 1.0 / c->eps_inf, c->kappa,
                                                         c->direct_shells, c->exchange_on, d_in, X, Y);
    else
        k_pairs<float><<<nblocks, pthreads, 0, ctx->stream>>>(d1, d2, nblocks, c->d_gen_v, c->d_gen_c, c->d_mu, (const float2*)c->d_kc,
                                                        (const float2*)s->d_Dv, (const float2*)s->d_Dc, (const float*)s->d_dE,
                                                        s->n, s->nd, s->nv, s->nc, s->nb1, c->e_k, 1.0 / c->eps_inf, c->kappa,
                                                        c->direct_shells, c->exchange_on, d_in, X, Y);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(d1);
    cudaFree(d2);
    if (e != cudaSuccess) { ctx->err = std::string("pair generation: ") + cudaGetErrorString(e); return BSE_ERR_CUDA; }
    return BSE_OK;
}

int bse_interp_set_learned(bse_ctx* ctx, bse_interp* s, bse_mlp* m, int radius) {
    if (!ctx || !s) return BSE_ERR_ARG;
    bse_invalidate_graph(s);                 // the captured step loop changes with the correction
    if (!m) {          // switch the learned correction off
        s->learned = 0;
        return BSE_OK;
    }
    const int t = s->t, L = s->n * s->nd;
    if (m->d_in != 6 + 2 * t) { ctx->err = "network input size does not match 6 + 2 t"; return BSE_ERR_ARG; }
    if (radius < 1 || 2 * radius > L) { ctx->err = "radius must satisfy 1 <= radius <= L/2"; return BSE_ERR_ARG; }
    if (s->scheme != BSE_SCHEME_M1) { ctx->err = "the learned correction replaces M3: set it on an M1 handle"; return BSE_ERR_ARG; }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return BSE_ERR_CUDA;
    std::vector<int> offs;
    for (int a = -radius; a <= radius; ++a)
        for (int b = -radius; b <= radius; ++b)
            for (int cc = -radius; cc <= radius; ++cc)
                if (a * a + b * b + cc * cc < radius * radius) { offs.push_back(a); offs.push_back(b); offs.push_back(cc); }
    const int noff = (int)offs.size() / 3;
    std::vector<int> neg(noff);
    for (int i = 0; i < noff; ++i)
        for (int j = 0; j < noff; ++j)
            if (offs[3 * j] == -offs[3 * i] && offs[3 * j + 1] == -offs[3 * i + 1] && offs[3 * j + 2] == -offs[3 * i + 2]) {
                neg[i] = j;
                break;
            }
    const long long L3 = (long long)L * L * L;
    const long long rows = (long long)noff * t * t;
    int rc = BSE_OK;
    int *d_offs = nullptr, *d_neg = nullptr;
    float *d_X = nullptr, *d_out = nullptr, *d_avg = nullptr;
    auto A = [&](void** p, size_t bytes, const char* what) { if (rc == BSE_OK) rc = bse_alloc(ctx, p, bytes, what); };
    A((void**)&d_offs, sizeof(int) * offs.size(), "stencil offsets");
    A((void**)&d_neg, sizeof(int) * noff, "stencil offsets");
    float2* d_ktmp = nullptr;
    A((void**)&d_X, sizeof(float) * (size_t)rows * m->d_in, "stencil features");
    A((void**)&d_out, sizeof(float) * 2 * (size_t)rows, "stencil outputs");
    A((void**)&d_avg, sizeof(float) * t, "dE averages");
    A((void**)&d_ktmp, sizeof(float2) * (size_t)t * t * L3, "kernel transform scratch");
    if (!s->d_lker) A((void**)&s->d_lker, sizeof(float2) * (size_t)t * t * L3, "learned kernel");
    if (!s->d_lgrid) A((void**)&s->d_lgrid, sizeof(float2) * 2 * (size_t)BSE_MAX_CHAINS * t * L3, "learned grids");
    if (!s->d_tw_fwd) A((void**)&s->d_tw_fwd, sizeof(float2) * 2 * L, "DFT twiddles");
    auto cleanup = [&]() {
        cudaFree(d_offs); cudaFree(d_neg); cudaFree(d_X); cudaFree(d_out); cudaFree(d_avg); cudaFree(d_ktmp);
    };
    if (rc != BSE_OK) { cleanup(); return rc; }
    s->d_tw_inv = s->d_tw_fwd + L;
    std::vector<float2> tw(2 * L);
    for (int j = 0; j < L; ++j) {
        const double ang = 2.0 * kPi * j / L;
        tw[j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));          // forward: exp(-2 pi i j / L)
        tw[L + j] = make_float2((float)std::cos(ang), (float)std::sin(ang));       // inverse: exp(+2 pi i j / L)
    }
    cudaMemcpy(s->d_tw_fwd, tw.data(), sizeof(float2) * 2 * L, cudaMemcpyHostToDevice);
    cudaMemcpy(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_neg, neg.data(), sizeof(int) * noff, cudaMemcpyHostToDevice);
    if (s->vec_prec == BSE_PREC_F64) k_dE_avg<double><<<t, 256, 0, ctx->stream>>>((const double*)s->d_dE, s->nk, t, d_avg);
    else k_dE_avg<float><<<t, 256, 0, ctx->stream>>>((const float*)s->d_dE, s->nk, t, d_avg);
    // network inference over every (near offset, vc, v'c'), in chunks of max_batch rows
    k_stencil_features<<<(int)((rows + 255) / 256), 256, 0, ctx->stream>>>(d_offs, noff, L, t, d_avg, m->d_in, d_X);
    for (long long r0 = 0; r0 < rows; r0 += m->max_batch) {
        const int nb = (int)std::min<long long>(m->max_batch, rows - r0);
        mlp_forward(ctx, m, nb, d_X + r0 * m->d_in);
        cudaMemcpyAsync(d_out + 2 * r0, m->d_z[3], sizeof(float) * 2 * nb, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    // Hermitian stencil on the periodic grid, then its DFT (one channel per band pair)
    cudaMemsetAsync(s->d_lker, 0, sizeof(float2) * (size_t)t * t * L3, ctx->stream);
    k_stencil_scatter<<<(int)((rows + 255) / 256), 256, 0, ctx->stream>>>(d_out, d_offs, d_neg, noff, L, t, 1.f / s->nk,
                                                                        s->d_lker);
    rc = dft3(ctx, s->d_lker, d_ktmp, L, (long long)t * t, s->d_tw_fwd);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    cleanup();
    if (rc != BSE_OK) return rc;
    if (e != cudaSuccess) { ctx->err = std::string("learned stencil: ") + cudaGetErrorString(e); return BSE_ERR_CUDA; }
    s->learned = 1;
    s->learned_radius = radius;
    return BSE_OK;
}

}  // extern "C"
