// Hot path: one interpolated H application per Lanczos step and the Lanczos
// vector updates (Sec. 2 Eqs. ai-ci; Sec. 4 Eqs. matmul1-matmul3, M3).
//
//   restrict   Q(k~) = sum_{uvw} sum_{k' in S(k~ - uvw)} f conj(Dv) psi Dc^T     (Eq. matmul1,
//              gathered per target coarse point by Eq. ordersums: no atomics)
//   K_c apply  R = K_c Q                                                         (Eq. matmul2)
//   near field u(k, k~) = sum_{k~'} A(k~,k~') [y1(k,k~') - h_head(q_c) z(k,k~')]  (M3)
//   prolong    w = dE psi + (1/N_div) sum_l f Dv^T (R(k~_l) + u(k,l)) conj(Dc)    (Eqs. matmul3, bse1)
//   Lanczos    a = Re<psi,w>, w -= a psi + b psi_prev, [CGS2], b' = ||w||, psi' = w / b'
//
// Every reduction is two-stage with a fixed order, so results are bitwise
// reproducible run to run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>

#include "bse_internal.cuh"

namespace {

constexpr int kRestrictWarps = 8;

// ----------------------------------------------------------------- restrict
// One CTA per target coarse point; warp w takes the (corner l, sub-point js)
// pairs w, w + 8, ... with non-zero weight; lane e owns coarse transition e
// (and e + 32).  OUT_BF16: write the split-BF16 operand of the tensor-core
// apply (rows: Re hi, Im hi, Re lo, Im lo per chain) instead of Q.
template <typename T, bool OUT_BF16>
__global__ void __launch_bounds__(256) k_restrict(
    const typename Cx<T>::V* __restrict__ psi, const typename Cx<T>::V* __restrict__ Dv,
    const typename Cx<T>::V* __restrict__ Dc, int n, int nd, int nv, int nc, int nb1, int nchains,
    int N, int Nc, typename Cx<T>::V* __restrict__ Q, __nv_bfloat16* __restrict__ Bop, int ldk,
    typename Cx<T>::V* __restrict__ X, const int* __restrict__ stop) {
    using V = typename Cx<T>::V;
    // per-warp staging of one (source point, corner) pair: psi rows of all
    // chains, Dv and Dc; reused at the end for the cross-warp reduction
    constexpr int WS = BSE_MAX_CHAINS * BSE_MAX_T + 2 * BSE_MAX_T;
    __shared__ V sm[kRestrictWarps * WS];
    const int t = nv * nc;
    const int Ndiv = nd * nd * nd;
    const int ic = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Int3 i = unflat3(ic, n);
    V* wps = sm + warp * WS;
    V* wdv = wps + BSE_MAX_CHAINS * BSE_MAX_T;
    V* wdc = wdv + BSE_MAX_T;
    V acc[BSE_MAX_CHAINS][2];
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) { acc[ch][0] = czero<V>(); acc[ch][1] = czero<V>(); }
    int n3q[2], n4q[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) { const int e = lane + 32 * q; n3q[q] = e / nc; n4q[q] = e % nc; }
    for (int p = warp; p < 8 * Ndiv; p += kRestrictWarps) {
        const int l = p / Ndiv, js = p % Ndiv;
        const T f = interp_weight_as<T>(js, l, nd, nb1);
        if (f == (T)0) continue;                                   // warp-uniform
        const int src = flat3(i.a - ((l >> 2) & 1), i.b - ((l >> 1) & 1), i.c - (l & 1), n);
        const size_t kd = (size_t)src * Ndiv + js;
        const V* dv = Dv + (kd * 8 + l) * nv * nv;
        const V* dc = Dc + (kd * 8 + l) * nc * nc;
        for (int ch = 0; ch < nchains; ++ch)
            for (int e = lane; e < t; e += 32) wps[ch * BSE_MAX_T + e] = psi[(size_t)ch * N + kd * t + e];
        for (int e = lane; e < nv * nv; e += 32) wdv[e] = dv[e];
        for (int e = lane; e < nc * nc; e += 32) wdc[e] = dc[e];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = lane + 32 * q;
            if (e >= t) break;
            const int n3 = n3q[q], n4 = n4q[q];
#pragma unroll
            for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
                if (ch >= nchains) break;
                const V* ps = wps + ch * BSE_MAX_T;
                V x = czero<V>();
                for (int vp = 0; vp < nv; ++vp) {
                    V inner = czero<V>();
                    for (int cp = 0; cp < nc; ++cp) inner = cadd(inner, cmul(ps[vp * nc + cp], wdc[n4 * nc + cp]));
                    x = cadd(x, cmulc(wdv[n3 * nv + vp], inner));
                }
                x = cscale(x, f);
                if (X) X[(((size_t)ch * (N / t) + kd) * 8 + l) * t + e] = x;
                acc[ch][q] = cadd(acc[ch][q], x);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    V (*red)[BSE_MAX_CHAINS][BSE_MAX_T] = reinterpret_cast<V (*)[BSE_MAX_CHAINS][BSE_MAX_T]>(sm);
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
        if (ch >= nchains) break;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = lane + 32 * q;
            if (e < t) red[warp][ch][e] = acc[ch][q];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nchains * t; idx += blockDim.x) {
        const int ch = idx / t, e = idx % t;
        V s = red[0][ch][e];
        for (int w = 1; w < kRestrictWarps; ++w) s = cadd(s, red[w][ch][e]);
        const int row = ic * t + e;
        if (!OUT_BF16) {
            Q[(size_t)ch * Nc + row] = s;
        } else {
            const float re = (float)s.x, im = (float)s.y;
            const __nv_bfloat16 rh = __float2bfloat16_rn(re), ih = __float2bfloat16_rn(im);
            const __nv_bfloat16 rl = __float2bfloat16_rn(re - __bfloat162float(rh));
            const __nv_bfloat16 il = __float2bfloat16_rn(im - __bfloat162float(ih));
            Bop[(size_t)(ch)*ldk + row] = rh;
            Bop[(size_t)(nchains + ch) * ldk + row] = ih;
            Bop[(size_t)(2 * nchains + ch) * ldk + row] = rl;
            Bop[(size_t)(3 * nchains + ch) * ldk + row] = il;
        }
    }
    (void)stop;
}

// ------------------------------------------------ staged restrict and prolong
// Both kernels take one coarse point (restrict) or one coarse cell (prolong)
// per CTA and walk its eight corners l.  For each corner the active
// (sub-point, corner) pairs (f != 0) come from per-CTA lists built with a warp
// ballot; their d rows, and the psi rows (restrict) or the R and u rows
// (prolong), are staged in shared memory by cp.async, double-buffered across
// corners, each row padded to an odd number of complex entries so that a warp
// reading one row per lane touches every bank at most twice.  Thread
// (chain c, item s) = (tid / 64, tid % 64) computes its pair from shared
// memory; the d tables are read from HBM once for all chains.
// Limits: N_div <= 64, <= 4 chains (= 256 threads / 64).

constexpr int odd_pad(int x) { return x | 1; }

__device__ __forceinline__ void cpa8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Active sub-points of every corner: cnt[l], list[l][i] = js (ascending),
// pos[l][js] = i or -1.  Warps 0-7 build corner l = warp.
__device__ __forceinline__ void corner_lists(int nd, int nb1, int* cnt, int* list, signed char* pos) {
    const int Ndiv = nd * nd * nd, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 8) {
        const int l = warp;
        int base = 0;
        for (int j0 = 0; j0 < Ndiv; j0 += 32) {
            const int js = j0 + lane;
            const bool act = js < Ndiv && interp_active(js, l, nd, nb1);
            const unsigned m = __ballot_sync(0xffffffffu, act);
            const int idx = base + __popc(m & ((1u << lane) - 1u));
            if (js < Ndiv) pos[l * 64 + js] = act ? (signed char)idx : (signed char)-1;
            if (act) list[l * 64 + idx] = js;
            base += __popc(m);
        }
        if (lane == 0) cnt[l] = base;
    }
}

template <int NV, int NC>
__host__ __device__ constexpr int restrict_st_buf(int nchains) {
    return 64 * (odd_pad(NV * NV) + odd_pad(NC * NC)) + nchains * 64 * odd_pad(NV * NC);
}
template <int NV, int NC>
size_t restrict_st_smem(int nchains) {
    const size_t a = 2 * (size_t)restrict_st_buf<NV, NC>(nchains), b = 256 * (size_t)odd_pad(NV * NC);
    return sizeof(float2) * std::max(a, b);
}

// Restrict (Eq. matmul1 gathered by Eq. ordersums), one CTA per target coarse
// point k~: x(k, l) = f conj(Dv) psi Dc^T for every active pair of the source
// cells k~ - l, written to X, and Q(k~) = sum of the x, summed over the 64 item
// threads of each chain in a fixed order.  XH: X holds the pieces for the
// tensor-core near field, FP16 (re, im) scaled by xscale[chain], t padded to a
// multiple of 4 with zeros.
template <int NV, int NC, bool OUT_BF16, bool XH>
__global__ void __launch_bounds__(256) k_restrict_st(
    const float2* __restrict__ psi, const float2* __restrict__ Dv, const float2* __restrict__ Dc, int n, int nd,
    int nb1, int nchains, int N, int Nc, float2* __restrict__ Q, __nv_bfloat16* __restrict__ Bop, int ldk,
    void* __restrict__ X, const float* __restrict__ xscale) {
    constexpr int t = NV * NC, RV = NV * NV, RC = NC * NC;
    constexpr int RVp = odd_pad(RV), RCp = odd_pad(RC), TP = odd_pad(t);
    extern __shared__ float2 st_sm[];
    __shared__ int cnt[8];
    __shared__ int list[8 * 64];
    __shared__ signed char pos[8 * 64];
    const int Ndiv = nd * nd * nd, nk = N / t;
    const int buf = restrict_st_buf<NV, NC>(nchains);
    const int ic = blockIdx.x, tid = threadIdx.x, c = tid >> 6, s = tid & 63;
    const Int3 i = unflat3(ic, n);
    corner_lists(nd, nb1, cnt, list, pos);
    __syncthreads();
    auto src_cell = [&](int l) { return flat3(i.a - ((l >> 2) & 1), i.b - ((l >> 1) & 1), i.c - (l & 1), n); };
    auto stage = [&](int l, float2* b) {
        const int m = cnt[l];
        const size_t cell0 = (size_t)src_cell(l) * Ndiv;
        float2* dv = b;
        float2* dc = dv + 64 * RVp;
        float2* ps = dc + 64 * RCp;
        for (int q = tid; q < m * RV; q += 256) {
            const int it = q / RV, k = q - it * RV;
            cpa8(dv + it * RVp + k, Dv + ((cell0 + list[l * 64 + it]) * 8 + l) * RV + k);
        }
        for (int q = tid; q < m * RC; q += 256) {
            const int it = q / RC, k = q - it * RC;
            cpa8(dc + it * RCp + k, Dc + ((cell0 + list[l * 64 + it]) * 8 + l) * RC + k);
        }
        for (int ch = 0; ch < nchains; ++ch)
            for (int q = tid; q < m * t; q += 256) {
                const int it = q / t, e = q - it * t;
                cpa8(ps + (ch * 64 + it) * TP + e, psi + (size_t)ch * N + (cell0 + list[l * 64 + it]) * t + e);
            }
    };
    float2 acc[t];
#pragma unroll
    for (int e = 0; e < t; ++e) acc[e] = make_float2(0.f, 0.f);
    stage(0, st_sm);
    cpa_commit();
    for (int l = 0; l < 8; ++l) {
        if (l + 1 < 8) {
            stage(l + 1, st_sm + ((l + 1) & 1) * buf);
            cpa_commit();
            cpa_wait1();
        } else {
            cpa_wait0();
        }
        __syncthreads();
        const float2* b = st_sm + (l & 1) * buf;
        if (c < nchains && s < cnt[l]) {
            const int js = list[l * 64 + s];
            const float f = interp_weight_f(js, l, nd, nb1);
            const float2* dv = b + s * RVp;
            const float2* dc = b + 64 * RVp + s * RCp;
            const float2* ps = b + 64 * (RVp + RCp) + (c * 64 + s) * TP;
            float2 x[NV][NC];
#pragma unroll
            for (int a = 0; a < NV; ++a)
#pragma unroll
                for (int bb = 0; bb < NC; ++bb) x[a][bb] = make_float2(0.f, 0.f);
#pragma unroll
            for (int vp = 0; vp < NV; ++vp) {
                float2 pr[NC];
#pragma unroll
                for (int cp = 0; cp < NC; ++cp) pr[cp] = ps[vp * NC + cp];
                float2 t1[NC];                                  // t1[n4] = sum_c' psi[vp][c'] Dc[n4][c']
#pragma unroll
                for (int n4 = 0; n4 < NC; ++n4) {
                    float2 sacc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int cp = 0; cp < NC; ++cp) {
                        const float2 d = dc[n4 * NC + cp];
                        sacc.x = fmaf(pr[cp].x, d.x, fmaf(-pr[cp].y, d.y, sacc.x));
                        sacc.y = fmaf(pr[cp].x, d.y, fmaf(pr[cp].y, d.x, sacc.y));
                    }
                    t1[n4] = sacc;
                }
#pragma unroll
                for (int n3 = 0; n3 < NV; ++n3) {
                    const float2 d = dv[n3 * NV + vp];             // x += conj(Dv[n3][vp]) t1
#pragma unroll
                    for (int n4 = 0; n4 < NC; ++n4) {
                        x[n3][n4].x = fmaf(d.x, t1[n4].x, fmaf(d.y, t1[n4].y, x[n3][n4].x));
                        x[n3][n4].y = fmaf(d.x, t1[n4].y, fmaf(-d.y, t1[n4].x, x[n3][n4].y));
                    }
                }
            }
            const size_t kd = (size_t)src_cell(l) * Ndiv + js;
            float2 xv[t];
#pragma unroll
            for (int a = 0; a < NV; ++a)
#pragma unroll
                for (int bb = 0; bb < NC; ++bb) {
                    const float2 v = make_float2(x[a][bb].x * f, x[a][bb].y * f);
                    xv[a * NC + bb] = v;
                    acc[a * NC + bb].x += v.x;
                    acc[a * NC + bb].y += v.y;
                }
            if constexpr (XH) {
                constexpr int TPAD = (t + 3) & ~3;
                const float sx = xscale[c];
                uint4* xo = reinterpret_cast<uint4*>(reinterpret_cast<__half2*>(X) + (((size_t)c * nk + kd) * 8 + l) * TPAD);
#pragma unroll
                for (int q4 = 0; q4 < TPAD / 4; ++q4) {
                    uint32_t w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = 4 * q4 + u;
                        const __half2 h = e < t ? __floats2half2_rn(xv[e].x * sx, xv[e].y * sx) : __floats2half2_rn(0.f, 0.f);
                        w[u] = *reinterpret_cast<const uint32_t*>(&h);
                    }
                    xo[q4] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else if (X) {
                float2* xo = reinterpret_cast<float2*>(X) + (((size_t)c * nk + kd) * 8 + l) * t;
#pragma unroll
                for (int e = 0; e < t; ++e) xo[e] = xv[e];
            }
        }
        __syncthreads();
    }
    // Q(k~): fixed-order sum over the 64 item threads of each chain
    float2* red = st_sm;
#pragma unroll
    for (int e = 0; e < t; ++e) red[tid * TP + e] = acc[e];
    __syncthreads();
    for (int idx = tid; idx < nchains * t; idx += 256) {
        const int ch = idx / t, e = idx - ch * t;
        float2 sum = make_float2(0.f, 0.f);
        for (int r = 0; r < 64; ++r) {
            const float2 v = red[(ch * 64 + r) * TP + e];
            sum.x += v.x;
            sum.y += v.y;
        }
        const int row = ic * t + e;
        if (!OUT_BF16) {
            Q[(size_t)ch * Nc + row] = sum;
        } else {
            const __nv_bfloat16 rh = __float2bfloat16_rn(sum.x), ih = __float2bfloat16_rn(sum.y);
            Bop[(size_t)ch * ldk + row] = rh;
            Bop[(size_t)(nchains + ch) * ldk + row] = ih;
            Bop[(size_t)(2 * nchains + ch) * ldk + row] = __float2bfloat16_rn(sum.x - __bfloat162float(rh));
            Bop[(size_t)(3 * nchains + ch) * ldk + row] = __float2bfloat16_rn(sum.y - __bfloat162float(ih));
        }
    }
}

template <int NV, int NC>
__host__ __device__ constexpr int prolong_st_buf(int nchains, bool near) {
    return 64 * (odd_pad(NV * NV) + odd_pad(NC * NC)) + nchains * odd_pad(NV * NC) +
           (near ? nchains * 64 * odd_pad(NV * NC) : 0);
}
// Epilogue rows (psi [chain][sub-point][TP] complex, dE [sub-point][TP] real) in
// complex units, and where they go: buffer 0 when they fit (it is free while
// corner 7 runs from buffer 1), else after both buffers.
template <int NV, int NC>
__host__ __device__ constexpr int prolong_st_eps(int nchains) {
    return nchains * 64 * odd_pad(NV * NC) + 32 * odd_pad(NV * NC);
}
template <int NV, int NC>
__host__ __device__ constexpr int prolong_st_eps_off(int nchains, bool near) {
    return prolong_st_eps<NV, NC>(nchains) <= prolong_st_buf<NV, NC>(nchains, near) ? 0 : 2 * prolong_st_buf<NV, NC>(nchains, near);
}
template <int NV, int NC>
size_t prolong_st_smem(int nchains, bool near) {
    const size_t a = 2 * (size_t)prolong_st_buf<NV, NC>(nchains, near);
    const size_t b = (size_t)prolong_st_eps_off<NV, NC>(nchains, near) + prolong_st_eps<NV, NC>(nchains);
    return sizeof(float2) * std::max(a, b);
}
constexpr int kProlongMaxCtas = BSE_MAX_VEC_BLOCKS;

// Prolong + diagonal (Eqs. matmul3, bse1), one CTA per coarse cell (grid-strided):
// w(k) = dE psi(k) + (1/N_div) sum_l f Dv^T (R(k~_l) + u(k, l)) conj(Dc) for the
// cell's sub-points k; w leaves through shared memory in coalesced rows; the
// CTA's FP64 partials of <psi, w> per chain go to part[chain][blockIdx.x].
template <int NV, int NC, bool NEAR>
__global__ void __launch_bounds__(256) k_prolong_st(
    const float2* __restrict__ R, const float2* __restrict__ Unf, const float2* __restrict__ Dv,
    const float2* __restrict__ Dc, const float* __restrict__ dE, const float2* __restrict__ psi, int n, int nd,
    int nb1, int nchains, int N, int Nc, float2* __restrict__ W, double2* __restrict__ part) {
    constexpr int t = NV * NC, RV = NV * NV, RC = NC * NC;
    constexpr int RVp = odd_pad(RV), RCp = odd_pad(RC), TP = odd_pad(t);
    extern __shared__ float2 st_sm[];
    __shared__ int cnt[8];
    __shared__ int list[8 * 64];
    __shared__ signed char pos[8 * 64];
    __shared__ double2 dred[256];
    const int Ndiv = nd * nd * nd, nk = N / t, nkc = nk / Ndiv;
    const int buf = prolong_st_buf<NV, NC>(nchains, NEAR);
    const int tid = threadIdx.x, c = tid >> 6, js = tid & 63;
    const float inv_ndiv = 1.f / (float)Ndiv;
    corner_lists(nd, nb1, cnt, list, pos);
    __syncthreads();
    double2 dot = make_double2(0.0, 0.0);
    for (int cell = blockIdx.x; cell < nkc; cell += gridDim.x) {
        const Int3 ci = unflat3(cell, n);
        const size_t cell0 = (size_t)cell * Ndiv;
        auto stage = [&](int l, float2* b) {
            const int m = cnt[l];
            float2* dv = b;
            float2* dc = dv + 64 * RVp;
            float2* rr = dc + 64 * RCp;
            float2* uu = rr + nchains * TP;
            for (int q = tid; q < m * RV; q += 256) {
                const int it = q / RV, k = q - it * RV;
                cpa8(dv + it * RVp + k, Dv + ((cell0 + list[l * 64 + it]) * 8 + l) * RV + k);
            }
            for (int q = tid; q < m * RC; q += 256) {
                const int it = q / RC, k = q - it * RC;
                cpa8(dc + it * RCp + k, Dc + ((cell0 + list[l * 64 + it]) * 8 + l) * RC + k);
            }
            const int cc = flat3(ci.a + ((l >> 2) & 1), ci.b + ((l >> 1) & 1), ci.c + (l & 1), n);
            for (int q = tid; q < nchains * t; q += 256) {
                const int ch = q / t, e = q - ch * t;
                cpa8(rr + ch * TP + e, R + (size_t)ch * Nc + (size_t)cc * t + e);
            }
            if (NEAR)
                for (int ch = 0; ch < nchains; ++ch)
                    for (int q = tid; q < m * t; q += 256) {
                        const int it = q / t, e = q - it * t;
                        cpa8(uu + (ch * 64 + it) * TP + e,
                             Unf + (((size_t)ch * nk + cell0 + list[l * 64 + it]) * 8 + l) * t + e);
                    }
        };
        float2* eps_ps = st_sm + prolong_st_eps_off<NV, NC>(nchains, NEAR);
        float* eps_de = reinterpret_cast<float*>(eps_ps + nchains * 64 * TP);
        auto stage_epilogue = [&]() {
            for (int ch = 0; ch < nchains; ++ch)
                for (int q = tid; q < Ndiv * t; q += 256) {
                    const int j = q / t, e = q - j * t;
                    cpa8(eps_ps + (ch * 64 + j) * TP + e, psi + (size_t)ch * N + cell0 * t + q);
                }
            for (int q = tid; q < Ndiv * t; q += 256) {
                const int j = q / t, e = q - j * t;
                cpa4(eps_de + j * TP + e, dE + cell0 * t + q);
            }
        };
        float2 sacc[NV][NC];
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int bb = 0; bb < NC; ++bb) sacc[a][bb] = make_float2(0.f, 0.f);
        stage(0, st_sm);
        cpa_commit();
        for (int l = 0; l < 8; ++l) {
            if (l + 1 < 8) stage(l + 1, st_sm + ((l + 1) & 1) * buf);
            else stage_epilogue();
            cpa_commit();
            cpa_wait1();
            __syncthreads();
            const float2* b = st_sm + (l & 1) * buf;
            const int p = js < Ndiv ? (int)pos[l * 64 + js] : -1;
            if (c < nchains && p >= 0) {
                const float f = interp_weight_f(js, l, nd, nb1);
                const float2* dv = b + p * RVp;
                const float2* dc = b + 64 * RVp + p * RCp;
                const float2* rr = b + 64 * (RVp + RCp) + c * TP;
                const float2* uu = b + 64 * (RVp + RCp) + nchains * TP + (c * 64 + p) * TP;
#pragma unroll
                for (int n1 = 0; n1 < NV; ++n1) {
                    float2 m[NC];
#pragma unroll
                    for (int n2 = 0; n2 < NC; ++n2) {
                        m[n2] = rr[n1 * NC + n2];
                        if (NEAR) { const float2 u = uu[n1 * NC + n2]; m[n2].x += u.x; m[n2].y += u.y; }
                    }
                    float2 tr[NC];                              // tr[c] = sum_n2 m[n2] conj(Dc[n2][c])
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) {
                        float2 a = make_float2(0.f, 0.f);
#pragma unroll
                        for (int n2 = 0; n2 < NC; ++n2) {
                            const float2 d = dc[n2 * NC + cc];
                            a.x = fmaf(m[n2].x, d.x, fmaf(m[n2].y, d.y, a.x));
                            a.y = fmaf(m[n2].y, d.x, fmaf(-m[n2].x, d.y, a.y));
                        }
                        tr[cc] = make_float2(a.x * f, a.y * f);
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const float2 d = dv[n1 * NV + v];
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            sacc[v][cc].x = fmaf(d.x, tr[cc].x, fmaf(-d.y, tr[cc].y, sacc[v][cc].x));
                            sacc[v][cc].y = fmaf(d.x, tr[cc].y, fmaf(d.y, tr[cc].x, sacc[v][cc].y));
                        }
                    }
                }
            }
            __syncthreads();
        }
        cpa_wait0();
        __syncthreads();
        // w = dE psi + s / N_div; <psi, w> in FP64; w written over the psi row
        if (c < nchains && js < Ndiv) {
            float2* row = eps_ps + (c * 64 + js) * TP;
            const float* de = eps_de + js * TP;
            float dre = 0.f, dim = 0.f;                         // the row's t products in FP32, rows summed in FP64
#pragma unroll
            for (int a = 0; a < NV; ++a)
#pragma unroll
                for (int bb = 0; bb < NC; ++bb) {
                    const int e = a * NC + bb;
                    const float2 pv = row[e];
                    const float d = de[e];
                    const float2 w = make_float2(fmaf(pv.x, d, sacc[a][bb].x * inv_ndiv), fmaf(pv.y, d, sacc[a][bb].y * inv_ndiv));
                    row[e] = w;
                    dre = fmaf(pv.x, w.x, fmaf(pv.y, w.y, dre));
                    dim = fmaf(pv.x, w.y, fmaf(-pv.y, w.x, dim));
                }
            dot.x += (double)dre;
            dot.y += (double)dim;
        }
        __syncthreads();
        for (int ch = 0; ch < nchains; ++ch)
            for (int q = tid; q < Ndiv * t; q += 256) {
                const int j = q / t, e = q - j * t;
                W[(size_t)ch * N + cell0 * t + q] = eps_ps[(ch * 64 + j) * TP + e];
            }
        __syncthreads();
    }
    // per-chain partial: fixed-order tree over the chain's 64 threads
    dred[tid] = dot;
    __syncthreads();
    for (int st = 32; st > 0; st >>= 1) {
        if ((tid & 63) < st) dred[tid] = cadd(dred[tid], dred[tid + st]);
        __syncthreads();
    }
    if (tid < nchains * 64 && (tid & 63) == 0) part[(size_t)(tid >> 6) * BSE_MAX_VEC_BLOCKS + blockIdx.x] = dred[tid];
}

// ------------------------------------------------- K_c apply on CUDA cores
// R[ch][i] = sum_j K[i][j] Q[ch][j]; one warp per row, fixed-order shuffle
// reduction.  Used for complex128 and complex64 storage.
template <typename T>
__global__ void __launch_bounds__(256) k_kc_apply_simt(const typename Cx<T>::V* __restrict__ K,
                                                      const typename Cx<T>::V* __restrict__ Q, int Nc,
                                                      int nchains, typename Cx<T>::V* __restrict__ R) {
    using V = typename Cx<T>::V;
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= Nc) return;
    V acc[BSE_MAX_CHAINS];
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) acc[ch] = czero<V>();
    const V* kr = K + (size_t)row * Nc;
    for (int j = lane; j < Nc; j += 32) {
        const V k = kr[j];
#pragma unroll
        for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch)
            if (ch < nchains) acc[ch] = cadd(acc[ch], cmul(k, Q[(size_t)ch * Nc + j]));
    }
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
        if (ch >= nchains) break;
        V v = acc[ch];
        for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) R[(size_t)ch * Nc + row] = v;
    }
}

// ---------------------------------------------------------------- near field
// Method 3 correction in coarse-basis form, one CTA per target dense point k:
//   phase 1: y1(k, s) = sum h_head(q_dense) x(k', k~_s), z(k, s) = sum x(k', k~_s) over the
//            near k' whose corner k~_s lies in slot s (lists built at set-up);
//   phase 2: u(k, l) = sum_s Hv(k~_l, k~_s) [y1 - h_head(q_coarse) z] Hc(k~_l, k~_s)^T.
// The prolong kernel applies F(k, k~_l) and 1/N_div.
template <typename T>
__global__ void __launch_bounds__(256) k_near_field(
    const typename Cx<T>::V* __restrict__ X, const NearEntry* __restrict__ list,
    const int* __restrict__ list_start, const T* __restrict__ hd, const typename Cx<T>::V* __restrict__ Hv,
    const typename Cx<T>::V* __restrict__ Hc, const T* __restrict__ hc, int n, int nd, int nv, int nc,
    int nb1, int smin, int ns1, int rmin, int nr1, int nchains, typename Cx<T>::V* __restrict__ U) {
    using V = typename Cx<T>::V;
    extern __shared__ unsigned char smem_raw[];
    const int t = nv * nc;
    const int nslot = ns1 * ns1 * ns1;
    V* y1 = reinterpret_cast<V*>(smem_raw);
    V* z = y1 + nslot * t;
    const int Ndiv = nd * nd * nd;
    const int nk = n * n * n * Ndiv;
    const int kd = blockIdx.x;
    const int cell = kd / Ndiv, js = kd % Ndiv;
    const Int3 ci = unflat3(cell, n);
    const int* st = list_start + (size_t)js * (nslot + 1);
    for (int ch = 0; ch < nchains; ++ch) {
        const V* Xc = X + (size_t)ch * nk * 8 * t;
        for (int idx = threadIdx.x; idx < nslot * t; idx += blockDim.x) {
            const int s = idx / t, e = idx % t;
            V ya = czero<V>(), za = czero<V>();
            for (int q = st[s]; q < st[s + 1]; ++q) {
                const NearEntry en = list[q];
                const int co1 = (en.co & 15) - 8, co2 = ((en.co >> 4) & 15) - 8, co3 = ((en.co >> 8) & 15) - 8;
                const int src = flat3(ci.a + co1, ci.b + co2, ci.c + co3, n);
                const V xv = Xc[(((size_t)src * Ndiv + en.js_src) * 8 + en.l_src) * t + e];
                ya = cadd(ya, cscale(xv, hd[en.near_idx]));
                za = cadd(za, xv);
            }
            y1[idx] = ya;
            z[idx] = za;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < 8 * t; idx += blockDim.x) {
            const int l = idx / t, e = idx % t;
            if (!interp_active(js, l, nd, nb1)) continue;
            const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
            const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
            const int n1 = e / nc, n2 = e % nc;
            V acc = czero<V>();
            for (int s = 0; s < nslot; ++s) {
                const Int3 so = unflat3(s, ns1);
                const int ra = so.a + smin - l1 - rmin, rb = so.b + smin - l2 - rmin, rc = so.c + smin - l3 - rmin;
                const int r = (ra * nr1 + rb) * nr1 + rc;
                const V* hv = Hv + ((size_t)kt * nr1 * nr1 * nr1 + r) * nv * nv + n1 * nv;
                const V* hcm = Hc + ((size_t)kt * nr1 * nr1 * nr1 + r) * nc * nc + n2 * nc;
                const T hcr = hc[r];
                const V* ys = y1 + s * t;
                const V* zs = z + s * t;
                for (int n3 = 0; n3 < nv; ++n3) {
                    V inner = czero<V>();
                    for (int n4 = 0; n4 < nc; ++n4) {
                        const V g = csub(ys[n3 * nc + n4], cscale(zs[n3 * nc + n4], hcr));
                        inner = cadd(inner, cmul(g, hcm[n4]));
                    }
                    acc = cadd(acc, cmul(hv[n3], inner));
                }
            }
            U[(((size_t)ch * nk + kd) * 8 + l) * t + e] = acc;
        }
        __syncthreads();
    }
}

// Method 3 correction, one CTA per (coarse cell C, chain): all N_div targets
// of C share the corners k~_l = C + l, the slots k~_s = C + o_s and hence the
// head blocks.  For each slot s:
//   (a) stage the slot's source rows x(k', k~_s) in shared memory: the pair
//       (js', l') of the active list names source cell C + o_s - l';
//   (b) y1(k, s) = sum h_head(q_dense) x, z(k, s) = sum x over the near sources
//       of every target k (per-(js, s) lists built at set-up);
//   (c) u(k, l) += Hv [y1 - h_head(q_coarse) z] Hc^T in factored form: each
//       thread owns one row n1 of one active (target, corner) pair, forms
//       T_row = G_row Hc^T, and gathers the other rows of T from its lane
//       group (NVP lanes, NVP >= nv a power of two) by shuffles.
template <typename T, int NVP>
__global__ void __launch_bounds__(512) k_near_cell(
    const typename Cx<T>::V* __restrict__ X, const int* __restrict__ clist, const int* __restrict__ cstart,
    const int* __restrict__ pairs, int npairs, const T* __restrict__ hd, int n_near,
    const typename Cx<T>::V* __restrict__ Hv, const typename Cx<T>::V* __restrict__ Hc, const T* __restrict__ hc,
    int n, int nd, int nv, int nc, int smin, int ns1, int rmin, int nr1, typename Cx<T>::V* __restrict__ U) {
    using V = typename Cx<T>::V;
    constexpr int MAXNC = BSE_MAX_BANDS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = nv * nc, tp = t + 1, Ndiv = nd * nd * nd, nslot = ns1 * ns1 * ns1, nrel = nr1 * nr1 * nr1;
    const int nk = n * n * n * Ndiv;
    const int cell = blockIdx.x, ch = blockIdx.y;
    // rows are padded to t + 1 elements so neighbouring rows start in different banks
    V* Xb = reinterpret_cast<V*>(smem_raw);          // [npairs][tp]  staged source rows
    V* Ua = Xb + (size_t)npairs * tp;                 // [npairs][tp]  accumulated u
    V* Y1 = Ua + (size_t)npairs * tp;                 // [Ndiv][tp]
    V* Zs = Y1 + (size_t)Ndiv * tp;                   // [Ndiv][tp]
    V* Hvs = Zs + (size_t)Ndiv * tp;                  // [8][nv*nv]
    V* Hcs = Hvs + 8 * nv * nv;                       // [8][nc*nc]
    T* hcs = reinterpret_cast<T*>(Hcs + 8 * nc * nc); // [8]
    T* hds = hcs + 8;                                 // [n_near]
    int* pcache = reinterpret_cast<int*>(hds + n_near);   // [npairs]   js | corner << 16
    int* scell = pcache + npairs;                     // [nslot][8] source cell of (slot, corner)
    const Int3 ci = unflat3(cell, n);
    const V* Xc = X + (size_t)ch * nk * 8 * t;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = tid; i < n_near; i += bd) hds[i] = hd[i];
    for (int i = tid; i < npairs; i += bd) pcache[i] = pairs[i];
    for (int i = tid; i < npairs * tp; i += bd) Ua[i] = czero<V>();
    for (int i = tid; i < nslot * 8; i += bd) {
        const int s = i >> 3, l = i & 7;
        const Int3 so = unflat3(s, ns1);
        scell[i] = flat3(ci.a + so.a + smin - ((l >> 2) & 1), ci.b + so.b + smin - ((l >> 1) & 1),
                         ci.c + so.c + smin - (l & 1), n);
    }
    const int lane = tid & 31, gbase = lane & ~(NVP - 1);
    const int rows_per_pass = bd / t;                 // staging: thread -> (row, element) without division
    const int e_st = tid % t, r_st = tid / t;
    __syncthreads();
    for (int s = 0; s < nslot; ++s) {
        const Int3 so = unflat3(s, ns1);
        const int oa = so.a + smin, ob = so.b + smin, oc = so.c + smin;
        // (a) source rows and the head blocks of the 8 corners
        if (r_st < rows_per_pass) {
            for (int p = r_st; p < npairs; p += rows_per_pass) {
                const int pk = pcache[p], js = pk & 0xFFFF, l = pk >> 16;
                const int sc = scell[s * 8 + l];
                Xb[p * tp + e_st] = Xc[(((size_t)sc * Ndiv + js) * 8 + l) * t + e_st];
            }
        }
        for (int idx = tid; idx < 8 * (nv * nv + nc * nc + 1); idx += bd) {
            const int l = idx & 7, q = idx >> 3;
            const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
            const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
            const int r = ((oa - l1 - rmin) * nr1 + (ob - l2 - rmin)) * nr1 + (oc - l3 - rmin);
            if (q < nv * nv) Hvs[l * nv * nv + q] = Hv[((size_t)kt * nrel + r) * nv * nv + q];
            else if (q < nv * nv + nc * nc) Hcs[l * nc * nc + (q - nv * nv)] = Hc[((size_t)kt * nrel + r) * nc * nc + (q - nv * nv)];
            else hcs[l] = hc[r];
        }
        __syncthreads();
        // (b) y1, z for every target of the cell
        const int* cs = cstart + s;
        if (r_st < rows_per_pass) {
            for (int j = r_st; j < Ndiv; j += rows_per_pass) {
                V y = czero<V>(), z = czero<V>();
                const int q1 = cs[(size_t)j * (nslot + 1) + 1];
                for (int q = cs[(size_t)j * (nslot + 1)]; q < q1; ++q) {
                    const int en = clist[q];
                    const V xv = Xb[(en & 0xFFFF) * tp + e_st];
                    y = cadd(y, cscale(xv, hds[en >> 16]));
                    z = cadd(z, xv);
                }
                Y1[j * tp + e_st] = y;
                Zs[j * tp + e_st] = z;
            }
        }
        __syncthreads();
        // (c) factored head application
        for (int base = 0; base < npairs * NVP; base += bd) {
            const int item = base + tid;
            const int p = item / NVP, n1 = item % NVP;
            const bool valid = (p < npairs) && (n1 < nv);
            int j = 0, l = 0;
            if (valid) { const int pk = pcache[p]; j = pk & 0xFFFF; l = pk >> 16; }
            V trow[MAXNC];
#pragma unroll
            for (int n2 = 0; n2 < MAXNC; ++n2) trow[n2] = czero<V>();
            if (valid) {
                const T hcl = hcs[l];
                const V* y = Y1 + j * tp + n1 * nc;
                const V* z = Zs + j * tp + n1 * nc;
                const V* hcm = Hcs + l * nc * nc;
                for (int n4 = 0; n4 < nc; ++n4) {
                    const V g = csub(y[n4], cscale(z[n4], hcl));
#pragma unroll
                    for (int n2 = 0; n2 < MAXNC; ++n2)
                        if (n2 < nc) trow[n2] = cadd(trow[n2], cmul(g, hcm[n2 * nc + n4]));
                }
            }
            V acc[MAXNC];
#pragma unroll
            for (int n2 = 0; n2 < MAXNC; ++n2) acc[n2] = czero<V>();
            for (int n3 = 0; n3 < nv; ++n3) {
                const V hv = valid ? Hvs[l * nv * nv + n1 * nv + n3] : czero<V>();
#pragma unroll
                for (int n2 = 0; n2 < MAXNC; ++n2) {
                    if (n2 < nc) {
                        V tv;
                        tv.x = __shfl_sync(0xffffffffu, trow[n2].x, gbase + n3);
                        tv.y = __shfl_sync(0xffffffffu, trow[n2].y, gbase + n3);
                        acc[n2] = cadd(acc[n2], cmul(hv, tv));
                    }
                }
            }
            if (valid) {
                V* ua = Ua + (size_t)p * tp + n1 * nc;
#pragma unroll
                for (int n2 = 0; n2 < MAXNC; ++n2)
                    if (n2 < nc) ua[n2] = cadd(ua[n2], acc[n2]);
            }
        }
        __syncthreads();
    }
    if (r_st < rows_per_pass) {
        for (int p = r_st; p < npairs; p += rows_per_pass) {
            const int pk = pcache[p], j = pk & 0xFFFF, l = pk >> 16;
            U[(((size_t)ch * nk + (size_t)cell * Ndiv + j) * 8 + l) * t + e_st] = Ua[p * tp + e_st];
        }
    }
}

// Register-blocked variant of k_near_cell for FP32 and compile-time band
// counts: one thread owns one active (target, corner) pair p and keeps its
// u block (NV x NC) in registers; per slot it forms the rows of
// T = [y1 - h_head(q_coarse) z] Hc^T one at a time and adds Hv T.  Phases (a)
// and (b) are those of k_near_cell.  Needs npairs <= blockDim.
template <int NV, int NC, int PF>
__global__ void __launch_bounds__(512) k_near_cell_rb(
    const float2* __restrict__ X, const int* __restrict__ clist, const int* __restrict__ cstart,
    const int* __restrict__ pairs, int npairs, const float* __restrict__ hd, int n_near,
    const float2* __restrict__ Hv, const float2* __restrict__ Hc, const float* __restrict__ hc,
    int n, int nd, int smin, int ns1, int rmin, int nr1, float2* __restrict__ U) {
    constexpr int t = NV * NC, tp = t + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Ndiv = nd * nd * nd, nslot = ns1 * ns1 * ns1, nrel = nr1 * nr1 * nr1;
    const int nk = n * n * n * Ndiv;
    const int cell = blockIdx.x, ch = blockIdx.y;
    float2* Xb = reinterpret_cast<float2*>(smem_raw);     // [npairs][tp]
    float2* Y1 = Xb + (size_t)npairs * tp;                 // [Ndiv][tp]
    float2* Zs = Y1 + (size_t)Ndiv * tp;                   // [Ndiv][tp]
    float2* Hvs = Zs + (size_t)Ndiv * tp;                  // [8][NV*NV]
    float2* Hcs = Hvs + 8 * NV * NV;                       // [8][NC*NC]
    float* hcs = reinterpret_cast<float*>(Hcs + 8 * NC * NC);
    float* hds = hcs + 8;
    int* pcache = reinterpret_cast<int*>(hds + n_near);
    int* scell = pcache + npairs;
    const Int3 ci = unflat3(cell, n);
    const float2* Xc = X + (size_t)ch * nk * 8 * t;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = tid; i < n_near; i += bd) hds[i] = hd[i];
    for (int i = tid; i < npairs; i += bd) pcache[i] = pairs[i];
    for (int i = tid; i < nslot * 8; i += bd) {
        const int s = i >> 3, l = i & 7;
        const Int3 so = unflat3(s, ns1);
        scell[i] = flat3(ci.a + so.a + smin - ((l >> 2) & 1), ci.b + so.b + smin - ((l >> 1) & 1),
                         ci.c + so.c + smin - (l & 1), n);
    }
    const int rows_per_pass = bd / t;
    const int e_st = tid % t, r_st = tid / t;
    const bool own = tid < npairs;
    int jo = 0, lo = 0;
    float2 u[NV][NC];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = 0; b < NC; ++b) u[a][b] = make_float2(0.f, 0.f);
    __syncthreads();
    if (own) { const int pk = pcache[tid]; jo = pk & 0xFFFF; lo = pk >> 16; }
    // PF > 0: the next slot's source rows are loaded into registers while the
    // current slot computes (PF >= rows per thread, checked by the launcher).
    float2 pf[PF > 0 ? PF : 1];
    auto fetch = [&](int s_) {
        if (r_st < rows_per_pass) {
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int p = r_st + k * rows_per_pass;
                if (p < npairs) {
                    const int pk = pcache[p], js = pk & 0xFFFF, l = pk >> 16;
                    pf[k] = Xc[(((size_t)scell[s_ * 8 + l] * Ndiv + js) * 8 + l) * t + e_st];
                }
            }
        }
    };
    if (PF > 0) fetch(0);
    for (int s = 0; s < nslot; ++s) {
        const Int3 so = unflat3(s, ns1);
        const int oa = so.a + smin, ob = so.b + smin, oc = so.c + smin;
        if (r_st < rows_per_pass) {
            if (PF > 0) {
#pragma unroll
                for (int k = 0; k < PF; ++k) {
                    const int p = r_st + k * rows_per_pass;
                    if (p < npairs) Xb[p * tp + e_st] = pf[k];
                }
            } else {
                for (int p = r_st; p < npairs; p += rows_per_pass) {
                    const int pk = pcache[p], js = pk & 0xFFFF, l = pk >> 16;
                    Xb[p * tp + e_st] = Xc[(((size_t)scell[s * 8 + l] * Ndiv + js) * 8 + l) * t + e_st];
                }
            }
        }
        for (int idx = tid; idx < 8 * (NV * NV + NC * NC + 1); idx += bd) {
            const int l = idx & 7, q = idx >> 3;
            const int l1 = (l >> 2) & 1, l2 = (l >> 1) & 1, l3 = l & 1;
            const int kt = flat3(ci.a + l1, ci.b + l2, ci.c + l3, n);
            const int r = ((oa - l1 - rmin) * nr1 + (ob - l2 - rmin)) * nr1 + (oc - l3 - rmin);
            if (q < NV * NV) Hvs[l * NV * NV + q] = Hv[((size_t)kt * nrel + r) * NV * NV + q];
            else if (q < NV * NV + NC * NC) Hcs[l * NC * NC + (q - NV * NV)] = Hc[((size_t)kt * nrel + r) * NC * NC + (q - NV * NV)];
            else hcs[l] = hc[r];
        }
        __syncthreads();
        if (PF > 0 && s + 1 < nslot) fetch(s + 1);
        const int* cs = cstart + s;
        if (r_st < rows_per_pass) {
            for (int j = r_st; j < Ndiv; j += rows_per_pass) {
                float2 y = make_float2(0.f, 0.f), z = make_float2(0.f, 0.f);
                const int q1 = cs[(size_t)j * (nslot + 1) + 1];
                for (int q = cs[(size_t)j * (nslot + 1)]; q < q1; ++q) {
                    const int en = clist[q];
                    const float2 xv = Xb[(en & 0xFFFF) * tp + e_st];
                    const float h = hds[en >> 16];
                    y.x = fmaf(h, xv.x, y.x);
                    y.y = fmaf(h, xv.y, y.y);
                    z.x += xv.x;
                    z.y += xv.y;
                }
                Y1[j * tp + e_st] = y;
                Zs[j * tp + e_st] = z;
            }
        }
        __syncthreads();
        if (own) {
            const float hcl = hcs[lo];
            const float2* hcm = Hcs + lo * NC * NC;
            const float2* hvm = Hvs + lo * NV * NV;
            const float2* yr = Y1 + jo * tp;
            const float2* zr = Zs + jo * tp;
#pragma unroll
            for (int n3 = 0; n3 < NV; ++n3) {
                float2 g[NC];
#pragma unroll
                for (int n4 = 0; n4 < NC; ++n4) {
                    const float2 yv = yr[n3 * NC + n4], zv = zr[n3 * NC + n4];
                    g[n4] = make_float2(fmaf(-hcl, zv.x, yv.x), fmaf(-hcl, zv.y, yv.y));
                }
                float2 tr[NC];
#pragma unroll
                for (int n2 = 0; n2 < NC; ++n2) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int n4 = 0; n4 < NC; ++n4) {
                        const float2 h = hcm[n2 * NC + n4];
                        acc.x = fmaf(g[n4].x, h.x, fmaf(-g[n4].y, h.y, acc.x));
                        acc.y = fmaf(g[n4].x, h.y, fmaf(g[n4].y, h.x, acc.y));
                    }
                    tr[n2] = acc;
                }
#pragma unroll
                for (int n1 = 0; n1 < NV; ++n1) {
                    const float2 h = hvm[n1 * NV + n3];
#pragma unroll
                    for (int n2 = 0; n2 < NC; ++n2) {
                        u[n1][n2].x = fmaf(h.x, tr[n2].x, fmaf(-h.y, tr[n2].y, u[n1][n2].x));
                        u[n1][n2].y = fmaf(h.x, tr[n2].y, fmaf(h.y, tr[n2].x, u[n1][n2].y));
                    }
                }
            }
        }
        __syncthreads();
    }
    if (own) {
        float2* dst = U + (((size_t)ch * nk + (size_t)cell * Ndiv + jo) * 8 + lo) * t;
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int b = 0; b < NC; ++b) dst[a * NC + b] = u[a][b];
    }
}

// ------------------------------------------------------- prolong + diagonal
// w = dE psi + (1/N_div) sum_l f Dv^T (R(k~_l) + u(k, l)) conj(Dc); one thread
// per dense element (kd, v, c) serving all chains; block partials of <psi, w>.
template <typename T, bool NEAR>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_prolong(
    const typename Cx<T>::V* __restrict__ R, const typename Cx<T>::V* __restrict__ Unf,
    const typename Cx<T>::V* __restrict__ Dv, const typename Cx<T>::V* __restrict__ Dc,
    const T* __restrict__ dE, const typename Cx<T>::V* __restrict__ psi, int n, int nd, int nv, int nc,
    int nb1, int nchains, int N, int Nc, typename Cx<T>::V* __restrict__ W, double2* __restrict__ part) {
    using V = typename Cx<T>::V;
    // per-warp staging: M = R(k~_l) + u(k, l) for all chains, Dv, Dc of one
    // (dense point, corner) pair; reused at the end for the block reduction
    constexpr int WS = BSE_MAX_CHAINS * BSE_MAX_T + 2 * BSE_MAX_T;
    constexpr int NW = BSE_VEC_THREADS / 32;
    __shared__ __align__(16) unsigned char smraw[NW * WS * sizeof(double2)];
    const int t = nv * nc;
    const int Ndiv = nd * nd * nd;
    const int nk = N / t;
    const T inv_ndiv = (T)1 / (T)Ndiv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V* wm = reinterpret_cast<V*>(smraw) + warp * WS;
    V* wdv = wm + BSE_MAX_CHAINS * BSE_MAX_T;
    V* wdc = wdv + BSE_MAX_T;
    int vq[2], cq[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) { const int e = lane + 32 * q; vq[q] = e / nc; cq[q] = e % nc; }
    double2 dot[BSE_MAX_CHAINS];
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) dot[ch] = make_double2(0.0, 0.0);
    for (int kd = blockIdx.x * NW + warp; kd < nk; kd += gridDim.x * NW) {
        const int cell = kd / Ndiv, js = kd % Ndiv;
        const Int3 ci = unflat3(cell, n);
        V acc[BSE_MAX_CHAINS][2];
#pragma unroll
        for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) { acc[ch][0] = czero<V>(); acc[ch][1] = czero<V>(); }
        for (int l = 0; l < 8; ++l) {
            const T f = interp_weight_as<T>(js, l, nd, nb1);
            if (f == (T)0) continue;                               // warp-uniform
            const int cc = flat3(ci.a + ((l >> 2) & 1), ci.b + ((l >> 1) & 1), ci.c + (l & 1), n);
            const V* dv = Dv + ((size_t)kd * 8 + l) * nv * nv;
            const V* dc = Dc + ((size_t)kd * 8 + l) * nc * nc;
            for (int ch = 0; ch < nchains; ++ch)
                for (int e = lane; e < t; e += 32) {
                    V r = R[(size_t)ch * Nc + (size_t)cc * t + e];
                    if (NEAR) r = cadd(r, Unf[(((size_t)ch * nk + kd) * 8 + l) * t + e]);
                    wm[ch * BSE_MAX_T + e] = r;
                }
            for (int e = lane; e < nv * nv; e += 32) wdv[e] = dv[e];
            for (int e = lane; e < nc * nc; e += 32) wdc[e] = dc[e];
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = lane + 32 * q;
                if (e >= t) break;
                const int v = vq[q], c = cq[q];
#pragma unroll
                for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
                    if (ch >= nchains) break;
                    const V* m = wm + ch * BSE_MAX_T;
                    V s = czero<V>();
                    for (int n1 = 0; n1 < nv; ++n1) {
                        V inner = czero<V>();
                        for (int n2 = 0; n2 < nc; ++n2) inner = cadd(inner, cmul(m[n1 * nc + n2], conjg(wdc[n2 * nc + c])));
                        s = cadd(s, cmul(wdv[n1 * nv + v], inner));
                    }
                    acc[ch][q] = cadd(acc[ch][q], cscale(s, f));
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = lane + 32 * q;
            if (e >= t) break;
            const size_t gid = (size_t)kd * t + e;
            const T de = dE[gid];
#pragma unroll
            for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
                if (ch >= nchains) break;
                const V p = psi[(size_t)ch * N + gid];
                const V w = cadd(cscale(p, de), cscale(acc[ch][q], inv_ndiv));
                W[(size_t)ch * N + gid] = w;
                const double2 pd = to_d2(p), wd = to_d2(w);
                dot[ch].x += pd.x * wd.x + pd.y * wd.y;
                dot[ch].y += pd.x * wd.y - pd.y * wd.x;
            }
        }
    }
    __syncthreads();
    double2 (*red)[BSE_VEC_THREADS] = reinterpret_cast<double2 (*)[BSE_VEC_THREADS]>(smraw);
    for (int ch = 0; ch < nchains; ++ch) red[ch][threadIdx.x] = dot[ch];
    __syncthreads();
    for (int s = BSE_VEC_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int ch = 0; ch < nchains; ++ch) red[ch][threadIdx.x] = cadd(red[ch][threadIdx.x], red[ch][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x < nchains) part[(size_t)threadIdx.x * BSE_MAX_VEC_BLOCKS + blockIdx.x] = red[threadIdx.x][0];
}

// ------------------------------------------------------------- Lanczos steps
__device__ inline double2 block_sum2(double2 v, double2* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double2 r = sh[0];
    __syncthreads();
    return r;
}

// a_i = Re sum(partials), one block per chain; the imaginary part is kept as a
// Hermiticity diagnostic.
__global__ void k_reduce_a(const double2* __restrict__ part, int nblk, int step, int m,
                           double* __restrict__ a, double* __restrict__ aim, const int* __restrict__ stop) {
    __shared__ double2 sh[256];
    const int ch = blockIdx.x;
    if (stop[ch]) return;
    double2 s = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s = cadd(s, part[(size_t)ch * BSE_MAX_VEC_BLOCKS + i]);
    s = block_sum2(s, sh);
    if (threadIdx.x == 0) {
        a[ch * m + step] = s.x;
        aim[ch * m + step] = s.y;
    }
}

// w <- w - a_i psi_i - b_i psi_{i-1}; block partials of ||w||^2.
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_lanczos_axpy(
    typename Cx<T>::V* __restrict__ W, const typename Cx<T>::V* __restrict__ psi,
    const typename Cx<T>::V* __restrict__ psi_prev, const double* __restrict__ a, const double* __restrict__ b,
    int step, int m, int N, int nchains, double* __restrict__ part, const int* __restrict__ stop) {
    using V = typename Cx<T>::V;
    __shared__ double2 sh[BSE_VEC_THREADS];
    for (int ch = 0; ch < nchains; ++ch) {
        if (stop[ch]) continue;
        const double ai = a[ch * m + step];
        const double bi = b[ch * (m + 1) + step];
        double nrm = 0.0;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
            const size_t o = (size_t)ch * N + g;
            const double2 w = to_d2(W[o]), p = to_d2(psi[o]), q = to_d2(psi_prev[o]);
            const double2 r = make_double2(w.x - ai * p.x - bi * q.x, w.y - ai * p.y - bi * q.y);
            const V rv = from_d2<V>(r);
            W[o] = rv;
            const double2 rd = to_d2(rv);
            nrm += rd.x * rd.x + rd.y * rd.y;
        }
        const double2 s = block_sum2(make_double2(nrm, 0.0), sh);
        if (threadIdx.x == 0) part[(size_t)ch * BSE_MAX_VEC_BLOCKS + blockIdx.x] = s.x;
    }
}

// Classical Gram-Schmidt pass, part 1: partials of h_j = <V_j, w>, j = 0..nb-1.
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_cgs_dots(const typename Cx<T>::V* __restrict__ basis,
                                                             const typename Cx<T>::V* __restrict__ W, int nb,
                                                             int mb, int N, int ch, int nblk,
                                                             double2* __restrict__ part) {
    __shared__ double2 sh[BSE_VEC_THREADS];
    const int j = blockIdx.y;
    const auto* vj = basis + ((size_t)ch * mb + j) * N;
    const auto* w = W + (size_t)ch * N;
    double2 s = make_double2(0.0, 0.0);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
        const double2 a = to_d2(vj[g]), b = to_d2(w[g]);
        s.x += a.x * b.x + a.y * b.y;
        s.y += a.x * b.y - a.y * b.x;
    }
    s = block_sum2(s, sh);
    if (threadIdx.x == 0) part[(size_t)j * nblk + blockIdx.x] = s;
    (void)nb;
}

__global__ void k_cgs_reduce(const double2* __restrict__ part, int nblk, double2* __restrict__ h) {
    __shared__ double2 sh[256];
    const int j = blockIdx.x;
    double2 s = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s = cadd(s, part[(size_t)j * nblk + i]);
    s = block_sum2(s, sh);
    if (threadIdx.x == 0) h[j] = s;
}

// Part 2: w <- w - sum_j h_j V_j; block partials of ||w||^2.
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_cgs_update(const typename Cx<T>::V* __restrict__ basis,
                                                               typename Cx<T>::V* __restrict__ W,
                                                               const double2* __restrict__ h, int nb, int mb,
                                                               int N, int ch, double* __restrict__ part) {
    using V = typename Cx<T>::V;
    __shared__ double2 sh[BSE_VEC_THREADS];
    double nrm = 0.0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
        double2 w = to_d2(W[(size_t)ch * N + g]);
        for (int j = 0; j < nb; ++j) {
            const double2 v = to_d2(basis[((size_t)ch * mb + j) * N + g]);
            const double2 hj = h[j];
            w.x -= hj.x * v.x - hj.y * v.y;
            w.y -= hj.x * v.y + hj.y * v.x;
        }
        const V wv = from_d2<V>(w);
        W[(size_t)ch * N + g] = wv;
        const double2 wd = to_d2(wv);
        nrm += wd.x * wd.x + wd.y * wd.y;
    }
    const double2 s = block_sum2(make_double2(nrm, 0.0), sh);
    if (threadIdx.x == 0) part[(size_t)ch * BSE_MAX_VEC_BLOCKS + blockIdx.x] = s.x;
}

// FP32 vectors, two complex entries per float4 (N even).  The vector update is
// FP32 arithmetic (the vectors are FP32); ||w||^2 is summed per thread in FP32
// over its few entries and across threads and blocks in FP64, in a fixed order.
// GB300 runs FP64 at 1/64 of the FP32 rate, so per-entry FP64 work would bound
// these kernels.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// w <- w - a_i psi_i - b_i psi_{i-1}; block partials of ||w||^2 (every chain in one pass).
__global__ void __launch_bounds__(256) k_lanczos_axpy4(float4* __restrict__ W, const float4* __restrict__ psi,
                                                       const float4* __restrict__ psi_prev, const double* __restrict__ a,
                                                       const double* __restrict__ b, int step, int m, int N4,
                                                       int nchains, double* __restrict__ part,
                                                       const int* __restrict__ stop) {
    __shared__ double red[BSE_MAX_CHAINS][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ch = 0; ch < nchains; ++ch) {
        const bool run = !stop[ch];
        const float ai = (float)a[ch * m + step], bi = (float)b[ch * (m + 1) + step];
        float nrm = 0.f;
        if (run)
            for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N4; g += gridDim.x * blockDim.x) {
                const size_t o = (size_t)ch * N4 + g;
                const float4 w = W[o], p = psi[o], q = psi_prev[o];
                float4 r;
                r.x = fmaf(-bi, q.x, fmaf(-ai, p.x, w.x));
                r.y = fmaf(-bi, q.y, fmaf(-ai, p.y, w.y));
                r.z = fmaf(-bi, q.z, fmaf(-ai, p.z, w.z));
                r.w = fmaf(-bi, q.w, fmaf(-ai, p.w, w.w));
                W[o] = r;
                nrm = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, nrm))));
            }
        const double ws = warp_sum_d((double)nrm);
        if (lane == 0) red[ch][warp] = ws;
    }
    __syncthreads();
    if (threadIdx.x < nchains && !stop[threadIdx.x]) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[(size_t)threadIdx.x * BSE_MAX_VEC_BLOCKS + blockIdx.x] = s;
    }
}

// One launch for a_i, the update and b_{i+1} (FP32 vectors, no
// reorthogonalisation; 512 threads per block, one block per SM, grid-stride).  GB300 issues FP64
// at a small fraction of its FP32 rate, so the FP64 work here is per block or
// per warp, never per element:
//  * a_i: warp 0 of every block sums the <psi, w> block partials of the H
//    application in FP64, in the same fixed order in every block (block 0
//    stores a_i and its imaginary part);
//  * the update and ||w||^2 in FP32 per thread and per warp (shuffles), the 8
//    warp sums of a block in FP64 into its partial;
//  * the last block to finish (a counter that it resets) sums the block
//    partials in FP64 in a fixed order into b_{i+1} and applies the breakdown
//    test b_{i+1} < 1e-12 max_j |a_j|.
template <int NCH>
__global__ void __launch_bounds__(512) k_lanczos_axpy4_ab(float4* __restrict__ W, const float4* __restrict__ psi,
                                                          const float4* __restrict__ psi_prev,
                                                          const double2* __restrict__ dot, int ndot, double* __restrict__ a,
                                                          double* __restrict__ aim, double* __restrict__ b, int step, int m,
                                                          int N4, double* __restrict__ part,
                                                          int* __restrict__ stop, int* __restrict__ ctr) {
    __shared__ float wsum[NCH][16];
    __shared__ double a_sh[NCH];
    __shared__ float ab_sh[NCH][2];
    __shared__ int run_sh[NCH];
    __shared__ int last_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const int run = stop[ch] == 0;                 // uniform over the grid until the last block
            // the imaginary part (a Hermiticity diagnostic) in block 0 only
            double2 s = make_double2(0.0, 0.0);
            if (run) {
                if (blockIdx.x == 0)
                    for (int i = lane; i < ndot; i += 32) s = cadd(s, dot[(size_t)ch * BSE_MAX_VEC_BLOCKS + i]);
                else
                    for (int i = lane; i < ndot; i += 32) s.x += dot[(size_t)ch * BSE_MAX_VEC_BLOCKS + i].x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_down_sync(0xffffffffu, s.x, o);
                if (blockIdx.x == 0) s.y += __shfl_down_sync(0xffffffffu, s.y, o);
            }
            if (lane == 0) {
                run_sh[ch] = run;
                a_sh[ch] = s.x;
                ab_sh[ch][0] = (float)s.x;
                ab_sh[ch][1] = (float)b[ch * (m + 1) + step];
                if (blockIdx.x == 0 && run) {
                    a[ch * m + step] = s.x;
                    aim[ch * m + step] = s.y;
                }
            }
        }
    }
    __syncthreads();
    float nrm[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        nrm[ch] = 0.f;
        if (!run_sh[ch]) continue;
        const float ai = ab_sh[ch][0], bi = ab_sh[ch][1];
        const int G = gridDim.x * blockDim.x;
        // two entries per pass: both loads in flight before either update
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N4; g += 2 * G) {
            const bool two = g + G < N4;
            const size_t o = (size_t)ch * N4 + g, o2 = o + G;
            const float4 w = W[o], p = psi[o], q = psi_prev[o];
            float4 w2 = make_float4(0.f, 0.f, 0.f, 0.f), p2 = w2, q2 = w2;
            if (two) { w2 = W[o2]; p2 = psi[o2]; q2 = psi_prev[o2]; }
            float4 r;
            r.x = fmaf(-bi, q.x, fmaf(-ai, p.x, w.x));
            r.y = fmaf(-bi, q.y, fmaf(-ai, p.y, w.y));
            r.z = fmaf(-bi, q.z, fmaf(-ai, p.z, w.z));
            r.w = fmaf(-bi, q.w, fmaf(-ai, p.w, w.w));
            W[o] = r;
            nrm[ch] = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, nrm[ch]))));
            if (two) {
                r.x = fmaf(-bi, q2.x, fmaf(-ai, p2.x, w2.x));
                r.y = fmaf(-bi, q2.y, fmaf(-ai, p2.y, w2.y));
                r.z = fmaf(-bi, q2.z, fmaf(-ai, p2.z, w2.z));
                r.w = fmaf(-bi, q2.w, fmaf(-ai, p2.w, w2.w));
                W[o2] = r;
                nrm[ch] = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, fmaf(r.w, r.w, nrm[ch]))));
            }
        }
    }
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        float x = nrm[ch];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) wsum[ch][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NCH && run_sh[threadIdx.x]) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)wsum[threadIdx.x][w];
        part[(size_t)threadIdx.x * BSE_MAX_VEC_BLOCKS + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_sh = atomicAdd(ctr, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last_sh || warp != 0) return;
    __threadfence();
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        if (!run_sh[ch]) continue;
        double s = 0.0, am = lane == 0 ? fabs(a_sh[ch]) : 0.0;
        for (int i = lane; i < (int)gridDim.x; i += 32) s += __ldcg(part + (size_t)ch * BSE_MAX_VEC_BLOCKS + i);
        for (int j = lane; j < step; j += 32) am = fmax(am, fabs(a[ch * m + j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            am = fmax(am, __shfl_down_sync(0xffffffffu, am, o));
        }
        if (lane == 0) {
            const double bn = sqrt(s);
            b[ch * (m + 1) + step + 1] = bn;
            if (!(bn >= 1e-12 * am)) stop[ch] = step + 1;
        }
    }
    if (lane == 0) *ctr = 0;
}

// psi_{i+1} = w / b_{i+1} (written over psi_{i-1}), also into the basis when kept.
__global__ void __launch_bounds__(256) k_lanczos_scale4(const float4* __restrict__ W, float4* __restrict__ out,
                                                        const double* __restrict__ b, int step, int m, int N4,
                                                        int nchains, float4* __restrict__ basis, int mb,
                                                        const int* __restrict__ stop) {
    // 1 / b_{i+1} once per block (FP64 is slow per element on GB300)
    __shared__ float inv_sh[BSE_MAX_CHAINS];
    if (threadIdx.x < nchains) inv_sh[threadIdx.x] = (float)(1.0 / b[threadIdx.x * (m + 1) + step + 1]);
    __syncthreads();
    for (int ch = 0; ch < nchains; ++ch) {
        if (stop[ch]) continue;
        const float inv = inv_sh[ch];
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N4; g += gridDim.x * blockDim.x) {
            const float4 w = W[(size_t)ch * N4 + g];
            const float4 v = make_float4(w.x * inv, w.y * inv, w.z * inv, w.w * inv);
            out[(size_t)ch * N4 + g] = v;
            if (basis) basis[((size_t)ch * mb + step + 1) * N4 + g] = v;
        }
    }
}

// b_{i+1} = sqrt(sum partials); breakdown when b_{i+1} < 1e-12 max_j |a_j|.
__global__ void k_reduce_b(const double* __restrict__ part, int nblk, int step, int m, const double* __restrict__ a,
                           double* __restrict__ b, int* __restrict__ stop) {
    __shared__ double2 sh[256];
    const int ch = blockIdx.x;
    if (stop[ch]) return;
    double s = 0.0, am = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[(size_t)ch * BSE_MAX_VEC_BLOCKS + i];
    for (int j = threadIdx.x; j <= step; j += blockDim.x) am = fmax(am, fabs(a[ch * m + j]));
    const double2 r = block_sum2(make_double2(s, 0.0), sh);
    // block maximum of |a_j| (the second component of sh is free)
    sh[threadIdx.x].y = am;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x].y = fmax(sh[threadIdx.x].y, sh[threadIdx.x + o].y);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double bn = sqrt(r.x);
        b[ch * (m + 1) + step + 1] = bn;
        if (!(bn >= 1e-12 * sh[0].y)) stop[ch] = step + 1;
    }
}

// psi_{i+1} = w / b_{i+1} (written over psi_{i-1}), also into the basis when kept.
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_lanczos_scale(
    const typename Cx<T>::V* __restrict__ W, typename Cx<T>::V* __restrict__ out, const double* __restrict__ b,
    int step, int m, int N, int nchains, typename Cx<T>::V* __restrict__ basis, int mb, const int* __restrict__ stop) {
    using V = typename Cx<T>::V;
    for (int ch = 0; ch < nchains; ++ch) {
        if (stop[ch]) continue;
        const double inv = 1.0 / b[ch * (m + 1) + step + 1];
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
            const double2 w = to_d2(W[(size_t)ch * N + g]);
            const V v = from_d2<V>(make_double2(w.x * inv, w.y * inv));
            out[(size_t)ch * N + g] = v;
            if (basis) basis[((size_t)ch * mb + step + 1) * N + g] = v;
        }
    }
}

// Start vectors: P(e) = sum_alpha e_alpha P^alpha; partial ||P||^2.
template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_dipole_start(const double2* __restrict__ P, const double* __restrict__ dirs,
                                                                  int N, int nchains, typename Cx<T>::V* __restrict__ out,
                                                                  double* __restrict__ part) {
    using V = typename Cx<T>::V;
    __shared__ double2 sh[BSE_VEC_THREADS];
    for (int ch = 0; ch < nchains; ++ch) {
        const double e0 = dirs[3 * ch], e1 = dirs[3 * ch + 1], e2 = dirs[3 * ch + 2];
        double nrm = 0.0;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
            const double2 p0 = P[g], p1 = P[(size_t)N + g], p2 = P[(size_t)2 * N + g];
            const double2 p = make_double2(e0 * p0.x + e1 * p1.x + e2 * p2.x, e0 * p0.y + e1 * p1.y + e2 * p2.y);
            out[(size_t)ch * N + g] = from_d2<V>(p);
            nrm += p.x * p.x + p.y * p.y;
        }
        const double2 s = block_sum2(make_double2(nrm, 0.0), sh);
        if (threadIdx.x == 0) part[(size_t)ch * BSE_MAX_VEC_BLOCKS + blockIdx.x] = s.x;
    }
}

// ||P||^2 per chain and psi_1 = P / ||P|| (in place); b_1 = 0.
template <typename T>
__global__ void k_start_norm(const double* __restrict__ part, int nblk, int m, double* __restrict__ pn2,
                             double* __restrict__ b) {
    __shared__ double2 sh[256];
    const int ch = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[(size_t)ch * BSE_MAX_VEC_BLOCKS + i];
    const double2 r = block_sum2(make_double2(s, 0.0), sh);
    if (threadIdx.x == 0) {
        pn2[ch] = r.x;
        if (b) b[ch * (m + 1)] = 0.0;
    }
}

template <typename T>
__global__ void __launch_bounds__(BSE_VEC_THREADS) k_start_scale(typename Cx<T>::V* __restrict__ v, const double* __restrict__ pn2,
                                                                 int N, int nchains, typename Cx<T>::V* __restrict__ zero_me,
                                                                 typename Cx<T>::V* __restrict__ basis, int mb) {
    using V = typename Cx<T>::V;
    for (int ch = 0; ch < nchains; ++ch) {
        const double inv = 1.0 / sqrt(pn2[ch]);
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
            const double2 p = to_d2(v[(size_t)ch * N + g]);
            const V s = from_d2<V>(make_double2(p.x * inv, p.y * inv));
            v[(size_t)ch * N + g] = s;
            zero_me[(size_t)ch * N + g] = czero<V>();
            if (basis) basis[((size_t)ch * mb) * N + g] = s;
        }
    }
}

// Continued fraction, one thread per (chain, omega), FP64 (Eq. fraccont).
__global__ void k_cont_frac(const double* __restrict__ a, const double* __restrict__ b, const int* __restrict__ steps,
                            const double* __restrict__ pn2, int m, int nchains, double pref, double eta, int nw,
                            const double* __restrict__ omega, double2* __restrict__ eps) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nchains * nw) return;
    const int ch = idx / nw, iw = idx % nw;
    const int ms = steps[ch];
    const double zr = omega[iw], zi = eta;
    // g = 1 / (z - a_m), then g = 1 / (z - a_i - b_{i+1}^2 g)
    double gr = 0.0, gi = 0.0;
    for (int i = ms - 1; i >= 0; --i) {
        const double b2 = (i == ms - 1) ? 0.0 : b[ch * (m + 1) + i + 1] * b[ch * (m + 1) + i + 1];
        const double dr = zr - a[ch * m + i] - b2 * gr;
        const double di = zi - b2 * gi;
        const double den = dr * dr + di * di;
        gr = dr / den;
        gi = -di / den;
    }
    eps[idx] = make_double2(1.0 - pref * pn2[ch] * gr, -pref * pn2[ch] * gi);
}

// Method 2 application w = H psi with the stored dense H (complex128 [N][N]),
// one warp per row (grid-stride over rows), every chain per row; block
// partials of <psi, w> for the Lanczos a_i.
constexpr int kM2Warps = 8;
__global__ void __launch_bounds__(32 * kM2Warps) k_m2_apply(const double2* __restrict__ H, const double2* __restrict__ psi,
                                                            int N, int nchains, double2* __restrict__ w,
                                                            double2* __restrict__ part) {
    __shared__ double2 red[BSE_MAX_CHAINS][kM2Warps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2 dot[BSE_MAX_CHAINS];
#pragma unroll
    for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) dot[ch] = make_double2(0.0, 0.0);
    for (int r = blockIdx.x * kM2Warps + warp; r < N; r += gridDim.x * kM2Warps) {
        double2 acc[BSE_MAX_CHAINS];
#pragma unroll
        for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) acc[ch] = make_double2(0.0, 0.0);
        const double2* hr = H + (size_t)r * N;
        for (int j = lane; j < N; j += 32) {
            const double2 h = hr[j];
#pragma unroll
            for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch)
                if (ch < nchains) acc[ch] = cadd(acc[ch], cmul(h, psi[(size_t)ch * N + j]));
        }
#pragma unroll
        for (int ch = 0; ch < BSE_MAX_CHAINS; ++ch) {
            if (ch >= nchains) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[ch].x += __shfl_xor_sync(0xffffffffu, acc[ch].x, o);
                acc[ch].y += __shfl_xor_sync(0xffffffffu, acc[ch].y, o);
            }
            if (lane == 0) {
                w[(size_t)ch * N + r] = acc[ch];
                dot[ch] = cadd(dot[ch], cmulc(psi[(size_t)ch * N + r], acc[ch]));
            }
        }
    }
    if (lane == 0)
        for (int ch = 0; ch < nchains; ++ch) red[ch][warp] = dot[ch];
    __syncthreads();
    if (threadIdx.x < nchains) {
        double2 sum = make_double2(0.0, 0.0);
        for (int k = 0; k < kM2Warps; ++k) sum = cadd(sum, red[threadIdx.x][k]);
        part[(size_t)threadIdx.x * BSE_MAX_VEC_BLOCKS + blockIdx.x] = sum;
    }
}

inline int m2_blocks(int N) { return std::min((N + kM2Warps - 1) / kM2Warps, BSE_MAX_VEC_BLOCKS); }

inline int vec_blocks(long long N) {
    long long b = (N + BSE_VEC_THREADS - 1) / BSE_VEC_THREADS;
    return (int)std::min<long long>(std::max<long long>(b, 1), BSE_MAX_VEC_BLOCKS);
}

// Raise a kernel's dynamic shared-memory limit when a launch needs more than the
// current one (by default 48 KB less the kernel's static shared memory); only
// ever raised: handles of different sizes share the attribute.
template <typename K>
void ensure_smem(K kernel, size_t bytes) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && (size_t)fa.maxDynamicSharedSizeBytes < bytes)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The staged FP32 restrict / prolong kernels serve 3x3, 4x4 and 4x6 bands with N_div <= 64.
inline bool staged_bands(const bse_interp* s) {
    return s->vec_prec == BSE_PREC_F32 && s->Ndiv <= 64 &&
           ((s->nv == 3 && s->nc == 3) || (s->nv == 4 && s->nc == 4) || (s->nv == 4 && s->nc == 6));
}

// Number of <psi, w> block partials one H application leaves in the dot buffer.
inline int dot_blocks(const bse_interp* s) {
    if (s->scheme == BSE_SCHEME_M2) return m2_blocks(s->N);
    if (!s->learned && staged_bands(s)) return std::min(s->co->nkc, kProlongMaxCtas);
    return vec_blocks(s->N);
}

// FP32 pieces (X32, [chain][nk][8][t]) -> FP16 pieces for the tensor-core near
// field ([chain][nk][8][tpad], scaled by xscale[chain], zero padding).
__global__ void __launch_bounds__(256) k_pieces_to_half(const float2* __restrict__ X32, int nk, int t, int tpad,
                                                        int nchains, const float* __restrict__ xscale,
                                                        __half2* __restrict__ Xh) {
    const long long n = (long long)nchains * nk * 8 * tpad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long piece = i / tpad;
        const int e = (int)(i - piece * tpad), ch = (int)(piece / ((long long)nk * 8));
        const float sx = xscale[ch];
        const float2 v = e < t ? X32[piece * t + e] : make_float2(0.f, 0.f);
        Xh[i] = __floats2half2_rn(v.x * sx, v.y * sx);
    }
}

// FP16 piece scale per chain from the input's 2-norm (bse_near_tc_xscale on
// the device): the largest power of two with scale dbound ||psi|| <= 2^15.
__global__ void __launch_bounds__(256) k_chain_xscale(const float2* __restrict__ psi, int N, double dbound,
                                                      float* __restrict__ xscale) {
    __shared__ double2 sh[256];
    const int ch = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float2 v = psi[(size_t)ch * N + i];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    const double2 r = block_sum2(make_double2(s, 0.0), sh);
    if (threadIdx.x == 0) {
        const double b = fmax(dbound * fmax(sqrt(r.x), 1e-300), 1e-300);
        int e = 0;
        frexp(32768.0 / b, &e);
        xscale[ch] = (float)ldexp(1.0, e - 1);
    }
}

// Restrict: staged FP32 kernel for 3x3, 4x4 and 4x6 bands (N_div <= 64), generic otherwise.
// xh: the pieces go to X as FP16 for the tensor-core near field (scaled by
// xscale); the generic kernel then writes FP32 pieces to x32 first.
template <typename T>
void launch_restrict(bse_ctx* ctx, const bse_interp* s, int nchains, const void* psi, void* Q, __nv_bfloat16* bop,
                     void* X, bool xh, const float* xscale, void* x32) {
    using V = typename Cx<T>::V;
    const bse_coarse* c = s->co;
    cudaStream_t st = ctx->stream;
    const bool bf = c->kc_prec == BSE_PREC_BF16;
    if constexpr (std::is_same<T, float>::value) {
        const float2* p = (const float2*)psi;
        const float2* dv = (const float2*)s->d_Dv;
        const float2* dc = (const float2*)s->d_Dc;
#define BSE_ST_RESTRICT_V(NV_, NC_, BF_, XH_)                                                                       \
    {                                                                                                               \
        const size_t smem = restrict_st_smem<NV_, NC_>(nchains);                                                    \
        ensure_smem(k_restrict_st<NV_, NC_, BF_, XH_>, smem);                                                       \
        k_restrict_st<NV_, NC_, BF_, XH_><<<c->nkc, 256, smem, st>>>(p, dv, dc, s->n, s->nd, s->nb1, nchains, s->N, \
                                                                    c->Nc, BF_ ? nullptr : (float2*)Q, BF_ ? bop : nullptr, \
                                                                    BF_ ? c->ldk : 0, X, xscale);                   \
    }
#define BSE_ST_RESTRICT(NV_, NC_)                                                                                   \
    if (s->nv == NV_ && s->nc == NC_ && s->Ndiv <= 64) {                                                            \
        if (bf && xh) BSE_ST_RESTRICT_V(NV_, NC_, true, true)                                                       \
        else if (bf) BSE_ST_RESTRICT_V(NV_, NC_, true, false)                                                       \
        else if (xh) BSE_ST_RESTRICT_V(NV_, NC_, false, true)                                                       \
        else BSE_ST_RESTRICT_V(NV_, NC_, false, false)                                                              \
        return;                                                                                                     \
    }
        BSE_ST_RESTRICT(3, 3)
        BSE_ST_RESTRICT(4, 4)
        BSE_ST_RESTRICT(4, 6)
#undef BSE_ST_RESTRICT
#undef BSE_ST_RESTRICT_V
    }
    void* xout = xh ? x32 : X;
    if (bf)
        k_restrict<T, true><<<c->nkc, 256, 0, st>>>((const V*)psi, (const V*)s->d_Dv, (const V*)s->d_Dc, s->n, s->nd,
                                                   s->nv, s->nc, s->nb1, nchains, s->N, c->Nc, nullptr, bop, c->ldk,
                                                   (V*)xout, nullptr);
    else
        k_restrict<T, false><<<c->nkc, 256, 0, st>>>((const V*)psi, (const V*)s->d_Dv, (const V*)s->d_Dc, s->n, s->nd,
                                                    s->nv, s->nc, s->nb1, nchains, s->N, c->Nc, (V*)Q, nullptr, 0,
                                                    (V*)xout, nullptr);
    if (xh) {
        const long long n = (long long)nchains * s->nk * 8 * s->nf_tc_tpad;
        const int g = (int)std::min<long long>((n + 255) / 256, 4096);
        k_pieces_to_half<<<g, 256, 0, st>>>((const float2*)x32, s->nk, s->t, s->nf_tc_tpad, nchains, xscale, (__half2*)X);
    }
}

// Prolong + diagonal: staged FP32 kernel for 3x3, 4x4 and 4x6 bands (N_div <= 64), generic otherwise.
template <typename T>
void launch_prolong(bse_ctx* ctx, const bse_interp* s, int nchains, const void* R, const void* U, const void* psi,
                    void* W, double2* dot) {
    using V = typename Cx<T>::V;
    const bse_coarse* c = s->co;
    cudaStream_t st = ctx->stream;
    const int nb = vec_blocks(s->N);
    const bool m3 = U != nullptr;
    if constexpr (std::is_same<T, float>::value) {
#define BSE_ST_PROLONG(NV_, NC_)                                                                                     \
    if (s->nv == NV_ && s->nc == NC_ && s->Ndiv <= 64) {                                                             \
        const size_t smem = prolong_st_smem<NV_, NC_>(nchains, m3);                                                  \
        const int g = std::min(c->nkc, kProlongMaxCtas);                                                             \
        if (m3) {                                                                                                    \
            ensure_smem(k_prolong_st<NV_, NC_, true>, smem);                                                         \
            k_prolong_st<NV_, NC_, true><<<g, 256, smem, st>>>(                                                      \
                (const float2*)R, (const float2*)U, (const float2*)s->d_Dv, (const float2*)s->d_Dc,                  \
                (const float*)s->d_dE, (const float2*)psi, s->n, s->nd, s->nb1, nchains, s->N, c->Nc, (float2*)W,    \
                dot);                                                                                                \
        } else {                                                                                                     \
            ensure_smem(k_prolong_st<NV_, NC_, false>, smem);                                                        \
            k_prolong_st<NV_, NC_, false><<<g, 256, smem, st>>>(                                                     \
                (const float2*)R, nullptr, (const float2*)s->d_Dv, (const float2*)s->d_Dc, (const float*)s->d_dE,    \
                (const float2*)psi, s->n, s->nd, s->nb1, nchains, s->N, c->Nc, (float2*)W, dot);                     \
        }                                                                                                            \
        return;                                                                                                      \
    }
        BSE_ST_PROLONG(3, 3)
        BSE_ST_PROLONG(4, 4)
        BSE_ST_PROLONG(4, 6)
#undef BSE_ST_PROLONG
    }
    if (m3)
        k_prolong<T, true><<<nb, BSE_VEC_THREADS, 0, st>>>((const V*)R, (const V*)U, (const V*)s->d_Dv,
                                                          (const V*)s->d_Dc, (const T*)s->d_dE, (const V*)psi, s->n,
                                                          s->nd, s->nv, s->nc, s->nb1, nchains, s->N, c->Nc, (V*)W, dot);
    else
        k_prolong<T, false><<<nb, BSE_VEC_THREADS, 0, st>>>((const V*)R, nullptr, (const V*)s->d_Dv,
                                                           (const V*)s->d_Dc, (const T*)s->d_dE, (const V*)psi, s->n,
                                                           s->nd, s->nv, s->nc, s->nb1, nchains, s->N, c->Nc, (V*)W, dot);
}

struct Timer {
    bse_ctx* ctx;
    bool on;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int cls;
    Timer(bse_ctx* c, bool enabled, int k) : ctx(c), on(enabled), cls(k) {
        if (on) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, ctx->stream);
        }
    }
    ~Timer() {
        if (on) {
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ctx->kt_ms[cls] += ms;
            ctx->kt_n[cls] += 1;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    }
};

// One application of H to nchains vectors psi -> w (device, vector precision),
// block partials of <psi, w> into s->d_part_dot.
// The tensor-core near field serves this application (FP16 pieces from restrict).
inline bool near_tc_active(const bse_interp* s) {
    return s->scheme == BSE_SCHEME_M3 && s->nf_tc && !s->nf_force_cuda_cores;
}

// unit: every psi has 2-norm 1 (the Lanczos vectors), so the FP16 piece scale
// set up for unit vectors applies; otherwise it is computed from the norms.
template <typename T>
int apply_h_typed(bse_ctx* ctx, bse_interp* s, int nchains, const void* psi_v, void* w_v, bool prof, bool unit) {
    using V = typename Cx<T>::V;
    const bse_coarse* c = s->co;
    cudaStream_t st = ctx->stream;
    const V* psi = (const V*)psi_v;
    V* W = (V*)w_v;
    if (s->scheme == BSE_SCHEME_M2) {
        if constexpr (std::is_same<T, double>::value) {
            Timer tm(ctx, prof, KC_KCAPPLY);
            k_m2_apply<<<m2_blocks(s->N), 32 * kM2Warps, 0, st>>>((const double2*)s->d_H2, psi, s->N, nchains, W,
                                                                 s->d_part_dot);
        }
        return BSE_OK;
    }
    const bool m3 = s->scheme == BSE_SCHEME_M3;
    const bool xh = near_tc_active(s);
    void* X = m3 ? s->d_X : nullptr;
    const float* xscale = unit ? s->d_xscale : s->d_xscale_gen;
    if (xh && !unit)
        k_chain_xscale<<<nchains, 256, 0, st>>>((const float2*)psi, s->N, s->dbound, s->d_xscale_gen);
    {
        Timer tm(ctx, prof, KC_RESTRICT);
        launch_restrict<T>(ctx, s, nchains, psi, s->d_Q, s->d_Bop, X, xh, xscale, s->d_U);
    }
    // The K_c apply and the near field read only what restrict wrote.  With the
    // tensor-core near field (one CTA per coarse cell, so its last wave leaves
    // SMs idle) the apply runs on the lane's auxiliary stream at the lowest
    // scheduling priority and the near field at the highest: the apply's CTAs
    // take SMs only once every near-field CTA has one, and share the chunks of
    // K_c among themselves.  Profiled runs keep the kernels one after another.
    const int ln = ctx->lane;
    if (xh && c->kc_prec == BSE_PREC_BF16 && !prof && ctx->aux[ln]) {
        BSE_CUDA_TRY(ctx, cudaEventRecord(ctx->aux_fork[ln], st));
        BSE_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->aux[ln], ctx->aux_fork[ln], 0));
        int rc = bse_near_tc_launch(ctx, s, nchains, X, xscale, s->d_U, true, ctx->prio_greatest);
        if (rc != BSE_OK) return rc;
        if ((rc = bse_tc_apply(ctx, s, nchains, ctx->aux[ln], true, ctx->prio_least)) != BSE_OK) return rc;
        BSE_CUDA_TRY(ctx, cudaEventRecord(ctx->aux_join[ln], ctx->aux[ln]));
        BSE_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->aux_join[ln], 0));
    } else {
        {
            Timer tm(ctx, prof, KC_KCAPPLY);
            if (c->kc_prec == BSE_PREC_BF16) {
                int rc = bse_tc_apply(ctx, s, nchains, st, false, 0);
                if (rc != BSE_OK) return rc;
            } else {
                k_kc_apply_simt<T><<<(c->Nc + 7) / 8, 256, 0, st>>>((const V*)c->d_kc, (const V*)s->d_Q, c->Nc, nchains, (V*)s->d_R);
            }
        }
        if (m3) {
            Timer tm(ctx, prof, KC_NEAR);
            int rc = bse_launch_near_field(ctx, s, nchains, X, xscale, s->d_U);
            if (rc != BSE_OK) return rc;
        }
    }
    {
        Timer tm(ctx, prof, KC_PROLONG);
        launch_prolong<T>(ctx, s, nchains, s->d_R, m3 ? s->d_U : nullptr, psi, W, s->d_part_dot);
    }
    if (s->learned) {
        Timer tm(ctx, prof, KC_NEAR);
        int rc = bse_apply_learned(ctx, s, nchains, psi, W, s->d_part_dot);
        if (rc != BSE_OK) return rc;
    }
    return BSE_OK;
}

// Convergence check of the Sec. 5.1 stopping rule (BSE_STOP_CONVERGED): eps on
// the rule's frequencies from the first `ms` steps (Eq. fraccont, bottom-up,
// FP64, as k_cont_frac), against the previous check's eps, which it replaces.
// Block maxima of |d Re eps|, |Re eps|, |d Im eps|, |Im eps| go to `part`.
constexpr int kConvThreads = 64;
__global__ void __launch_bounds__(kConvThreads) k_conv_eval(const double* __restrict__ a, const double* __restrict__ b,
                                                            int ms, int m, const double* __restrict__ pn2, double pref,
                                                            double eta, const double* __restrict__ omega, int nw,
                                                            double2* __restrict__ eps_prev, double* __restrict__ part,
                                                            const int* __restrict__ stop) {
    __shared__ double red[4][kConvThreads];
    const int ch = blockIdx.y;
    if (stop[ch]) return;                                        // uniform over the block
    const int iw = blockIdx.x * kConvThreads + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (iw < nw) {
        const double zr = omega[iw], zi = eta;
        double gr = 0.0, gi = 0.0;
        for (int i = ms - 1; i >= 0; --i) {
            const double bb = (i == ms - 1) ? 0.0 : b[ch * (m + 1) + i + 1];
            const double b2 = bb * bb;
            const double dr = zr - a[ch * m + i] - b2 * gr, di = zi - b2 * gi;
            const double den = dr * dr + di * di;
            gr = dr / den;
            gi = -di / den;
        }
        const double2 e = make_double2(1.0 - pref * pn2[ch] * gr, -pref * pn2[ch] * gi);
        const double2 o = eps_prev[(size_t)ch * nw + iw];
        eps_prev[(size_t)ch * nw + iw] = e;
        v[0] = fabs(e.x - o.x);
        v[1] = fabs(e.x);
        v[2] = fabs(e.y - o.y);
        v[3] = fabs(e.y);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int s = kConvThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = fmax(red[q][threadIdx.x], red[q][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x < 4) part[((size_t)ch * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// Stop decision: a chain whose spectrum moved by at most tol (relative to its
// largest |Re eps| and |Im eps|) since the previous check stops after `ms`
// steps; the stop word records -ms (a breakdown records +steps).
__global__ void k_conv_decide(const double* __restrict__ part, int nblk, int ms, int first, double tol,
                              int* __restrict__ stop) {
    const int ch = blockIdx.x;
    if (threadIdx.x != 0 || stop[ch]) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < nblk; ++i)
        for (int q = 0; q < 4; ++q) v[q] = fmax(v[q], part[((size_t)ch * nblk + i) * 4 + q]);
    if (!first && v[0] <= tol * v[1] && v[2] <= tol * v[3]) stop[ch] = -ms;
}

// The stopping rule as one system's run sees it (prefactor s_eps / N_k).
struct StopRule {
    double tol, pref, eta;
    int every, nw;
    const double* omega;
};

inline StopRule stop_rule_for(const bse_ctx* ctx, const bse_interp* s) {
    return StopRule{ctx->stop_tol, ctx->stop_seps / (double)s->nk, ctx->stop_eta, ctx->stop_every, ctx->stop_nw,
                    ctx->d_stop_omega};
}

void drop_graph(bse_interp* s) {
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    ++s->state_serial;
}

// Buffers of a Haydock run, kept in the handle: coefficients for m steps, the
// start directions and norms, the CGS2 basis, the convergence-check state for
// nw frequencies.  Replacing any of them invalidates a cached graph.
template <typename T>
int ensure_state(bse_ctx* ctx, bse_interp* s, int m, bool reorth, int nw) {
    using V = typename Cx<T>::V;
    int rc;
    if (!s->d_dirs) {
        if ((rc = bse_alloc(ctx, (void**)&s->d_dirs, sizeof(double) * 3 * BSE_MAX_CHAINS, "directions")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_pn2, sizeof(double) * BSE_MAX_CHAINS, "norms")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_lz_ctr, sizeof(int), "Lanczos counter")) != BSE_OK) return rc;
        BSE_CUDA_TRY(ctx, cudaMemset(s->d_lz_ctr, 0, sizeof(int)));
    }
    if (s->m_alloc < m) {
        drop_graph(s);
        cudaFree(s->d_a); cudaFree(s->d_aim); cudaFree(s->d_b);
        s->d_a = s->d_aim = s->d_b = nullptr;
        s->m_alloc = 0;
        if ((rc = bse_alloc(ctx, (void**)&s->d_a, sizeof(double) * BSE_MAX_CHAINS * m, "a")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_aim, sizeof(double) * BSE_MAX_CHAINS * m, "a imag")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_b, sizeof(double) * BSE_MAX_CHAINS * (m + 1), "b")) != BSE_OK) return rc;
        s->m_alloc = m;
    }
    if (reorth && s->basis_m < m + 1) {
        drop_graph(s);
        cudaFree(s->d_basis); cudaFree(s->d_cgs_part); cudaFree(s->d_cgs_h);
        s->d_basis = nullptr; s->d_cgs_part = s->d_cgs_h = nullptr;
        s->basis_m = 0;
        if ((rc = bse_alloc(ctx, &s->d_basis, sizeof(V) * BSE_MAX_CHAINS * (size_t)(m + 1) * s->N, "Lanczos basis")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_cgs_part, sizeof(double2) * (size_t)(m + 1) * BSE_MAX_VEC_BLOCKS, "CGS partials")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_cgs_h, sizeof(double2) * (size_t)(m + 1), "CGS coefficients")) != BSE_OK) return rc;
        s->basis_m = m + 1;
    }
    if (nw > s->eps_nw) {
        drop_graph(s);
        cudaFree(s->d_eps_prev); cudaFree(s->d_conv_part);
        s->d_eps_prev = nullptr; s->d_conv_part = nullptr;
        s->eps_nw = 0;
        const int nblk = (nw + kConvThreads - 1) / kConvThreads;
        if ((rc = bse_alloc(ctx, (void**)&s->d_eps_prev, sizeof(double2) * BSE_MAX_CHAINS * (size_t)nw, "previous spectrum")) != BSE_OK) return rc;
        if ((rc = bse_alloc(ctx, (void**)&s->d_conv_part, sizeof(double) * BSE_MAX_CHAINS * 4 * (size_t)nblk, "check maxima")) != BSE_OK) return rc;
        s->eps_nw = nw;
    }
    return BSE_OK;
}

// Enqueue the whole Haydock loop for one system on ctx->stream (start vectors
// from s->d_dirs).  With a stopping rule the convergence check runs every
// rule->every steps; with `poll` the host reads the stop words after each
// check and stops enqueueing once every chain has stopped.
template <typename T>
int enqueue_chains(bse_ctx* ctx, bse_interp* s, int nch, int m, bool reorth, bool prof, const StopRule* rule,
                   bool poll) {
    using V = typename Cx<T>::V;
    cudaStream_t st = ctx->stream;
    const int N = s->N;
    const int nb = vec_blocks(N);
    V* A = (V*)s->d_vec[0];
    V* B = (V*)s->d_vec[1];
    V* W = (V*)s->d_vec[2];
    V* basis = reorth ? (V*)s->d_basis : nullptr;
    const int mb = s->basis_m;
    // FP32 vectors with an even length: float4 update kernels, one float4 per thread and chain
    const bool vec4 = std::is_same<T, float>::value && (N % 2) == 0;
    const int nb4 = (int)std::min<long long>(std::max<long long>((N / 2 + 255) / 256, 1), BSE_MAX_VEC_BLOCKS);
    cudaMemsetAsync(s->d_stop, 0, sizeof(int) * BSE_MAX_CHAINS, st);
    // psi_1 = P / ||P|| in B, psi_0 = 0 in A
    k_dipole_start<T><<<nb, BSE_VEC_THREADS, 0, st>>>(s->d_P, s->d_dirs, N, nch, B, s->d_part_nrm);
    k_start_norm<T><<<nch, 256, 0, st>>>(s->d_part_nrm, nb, m, s->d_pn2, s->d_b);
    k_start_scale<T><<<nb, BSE_VEC_THREADS, 0, st>>>(B, s->d_pn2, N, nch, A, basis, mb);
    for (int i = 0; i < m; ++i) {
        int rc = apply_h_typed<T>(ctx, s, nch, B, W, prof, true);
        if (rc != BSE_OK) return rc;
        Timer tm(ctx, prof, KC_LANCZOS);
        if (vec4 && !reorth) {
            // a_i, the update and b_{i+1} in one launch, then the scale
#define BSE_AXPY_AB(NCH_)                                                                                       \
    k_lanczos_axpy4_ab<NCH_><<<nbab, 512, 0, st>>>((float4*)W, (const float4*)B, (const float4*)A, s->d_part_dot,    \
                                                  dot_blocks(s), s->d_a, s->d_aim, s->d_b, i, m, N / 2, s->d_part_nrm, \
                                                  s->d_stop, s->d_lz_ctr)
            // one block of 512 threads per SM: every block sums the <psi, w> partials in FP64
            const int nbab = std::min((N / 2 + 511) / 512, std::max(ctx->sm_count, 1));
            if (nch == 1) BSE_AXPY_AB(1);
            else if (nch == 2) BSE_AXPY_AB(2);
            else if (nch == 3) BSE_AXPY_AB(3);
            else BSE_AXPY_AB(4);
#undef BSE_AXPY_AB
        } else {
        k_reduce_a<<<nch, 256, 0, st>>>(s->d_part_dot, dot_blocks(s), i, m, s->d_a, s->d_aim, s->d_stop);
        if (vec4)
            k_lanczos_axpy4<<<nb4, 256, 0, st>>>((float4*)W, (const float4*)B, (const float4*)A, s->d_a, s->d_b, i, m,
                                                 N / 2, nch, s->d_part_nrm, s->d_stop);
        else
            k_lanczos_axpy<T><<<nb, BSE_VEC_THREADS, 0, st>>>(W, B, A, s->d_a, s->d_b, i, m, N, nch, s->d_part_nrm, s->d_stop);
        if (reorth) {
            for (int ch = 0; ch < nch; ++ch)
                for (int pass = 0; pass < 2; ++pass) {
                    dim3 g(nb, i + 1);
                    k_cgs_dots<T><<<g, BSE_VEC_THREADS, 0, st>>>(basis, W, i + 1, mb, N, ch, nb, s->d_cgs_part);
                    k_cgs_reduce<<<i + 1, 256, 0, st>>>(s->d_cgs_part, nb, s->d_cgs_h);
                    k_cgs_update<T><<<nb, BSE_VEC_THREADS, 0, st>>>(basis, W, s->d_cgs_h, i + 1, mb, N, ch, s->d_part_nrm);
                }
        }
        k_reduce_b<<<nch, 256, 0, st>>>(s->d_part_nrm, nb, i, m, s->d_a, s->d_b, s->d_stop);
        }
        if (rule && (i + 1) % rule->every == 0) {
            const int nblk = (rule->nw + kConvThreads - 1) / kConvThreads;
            k_conv_eval<<<dim3(nblk, nch), kConvThreads, 0, st>>>(s->d_a, s->d_b, i + 1, m, s->d_pn2, rule->pref, rule->eta,
                                                                  rule->omega, rule->nw, s->d_eps_prev, s->d_conv_part,
                                                                  s->d_stop);
            k_conv_decide<<<nch, 32, 0, st>>>(s->d_conv_part, nblk, i + 1, (i + 1) == rule->every ? 1 : 0, rule->tol,
                                              s->d_stop);
        }
        if (vec4)
            k_lanczos_scale4<<<nb4, 256, 0, st>>>((const float4*)W, (float4*)A, s->d_b, i, m, N / 2, nch, (float4*)basis,
                                                  mb, s->d_stop);
        else
            k_lanczos_scale<T><<<nb, BSE_VEC_THREADS, 0, st>>>(W, A, s->d_b, i, m, N, nch, basis, mb, s->d_stop);
        std::swap(A, B);
        if (poll && rule && (i + 1) % rule->every == 0) {
            int stop[BSE_MAX_CHAINS] = {0, 0, 0, 0};
            BSE_CUDA_TRY(ctx, cudaMemcpyAsync(stop, s->d_stop, sizeof(int) * BSE_MAX_CHAINS, cudaMemcpyDeviceToHost, st));
            BSE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
            bool all = true;
            for (int ch = 0; ch < nch; ++ch) all = all && stop[ch] != 0;
            if (all) break;
        }
    }
    return BSE_OK;
}

// Copy a run's results to the host; steps_done from the stop words (+k: a
// breakdown after k steps, -k: converged after k steps, 0: all m steps).
int finish_run(bse_ctx* ctx, bse_interp* s, int nch, int m, double* a, double* b, double* pnorm2, int* steps_done,
               int* warn) {
    cudaStream_t st = ctx->stream;
    int stop[BSE_MAX_CHAINS] = {0, 0, 0, 0};
    cudaMemcpyAsync(pnorm2, s->d_pn2, sizeof(double) * nch, cudaMemcpyDeviceToHost, st);
    for (int ch = 0; ch < nch; ++ch) {
        cudaMemcpyAsync(a + (size_t)ch * m, s->d_a + (size_t)ch * m, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(b + (size_t)ch * (m + 1), s->d_b + (size_t)ch * (m + 1), sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, st);
    }
    cudaMemcpyAsync(stop, s->d_stop, sizeof(int) * BSE_MAX_CHAINS, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("Haydock run: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    for (int ch = 0; ch < nch; ++ch) {
        steps_done[ch] = stop[ch] > 0 ? stop[ch] : (stop[ch] < 0 ? -stop[ch] : m);
        if (stop[ch] > 0) *warn = BSE_WARN_BREAKDOWN;
        // coefficients past the last step are left undefined on the device: zero them
        for (int i = steps_done[ch]; i < m; ++i) a[(size_t)ch * m + i] = 0.0;
        for (int i = steps_done[ch] + 1; i <= m; ++i) b[(size_t)ch * (m + 1) + i] = 0.0;
    }
    return BSE_OK;
}

int read_status(bse_ctx* ctx) {
    int status = 0;
    BSE_CUDA_TRY(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        ctx->err = bse_timeout_message(status);
        cudaMemset(ctx->d_status, 0, sizeof(int));
        return BSE_ERR_TIMEOUT;
    }
    return BSE_OK;
}

template <typename T>
int run_chains_typed(bse_ctx* ctx, bse_interp* s, int nch, const double* pol_dirs, int m, int flags, double* a,
                     double* b, double* pnorm2, int* steps_done) {
    const bool reorth = flags & BSE_REORTH_CGS2;
    const bool prof = flags & BSE_PROFILE;
    const bool conv = flags & BSE_STOP_CONVERGED;
    const bool graph = (flags & BSE_USE_GRAPH) && !prof && !conv;
    int rc = ensure_state<T>(ctx, s, m, reorth, conv ? ctx->stop_nw : 0);
    if (rc != BSE_OK) return rc;
    cudaStream_t st = ctx->stream;
    BSE_CUDA_TRY(ctx, cudaMemcpyAsync(s->d_dirs, pol_dirs, sizeof(double) * 3 * nch, cudaMemcpyHostToDevice, st));
    if (prof) for (int k = 0; k < KC_COUNT; ++k) { ctx->kt_ms[k] = 0; ctx->kt_n[k] = 0; }
    if (graph) {
        const long long key[6] = {ctx->serial, nch, m, flags & (BSE_REORTH_CGS2 | BSE_USE_GRAPH), s->state_serial,
                                  ctx->wait_cycles};
        if (!s->graph || !std::equal(key, key + 6, s->graph_key)) {
            if (s->graph) cudaGraphExecDestroy(s->graph);
            s->graph = nullptr;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = enqueue_chains<T>(ctx, s, nch, m, reorth, false, nullptr, false);
                e = cudaStreamEndCapture(st, &g);
            }
            if (e == cudaSuccess && rc == BSE_OK) e = cudaGraphInstantiate(&s->graph, g, cudaGraphInstantiateFlagUseNodePriority);
            if (g) cudaGraphDestroy(g);
            if (rc != BSE_OK) return rc;
            if (e != cudaSuccess) {
                s->graph = nullptr;
                ctx->err = std::string("graph capture: ") + cudaGetErrorString(e);
                return BSE_ERR_CUDA;
            }
            std::copy(key, key + 6, s->graph_key);
        }
        BSE_CUDA_TRY(ctx, cudaGraphLaunch(s->graph, st));
    } else {
        StopRule rule{};
        if (conv) rule = stop_rule_for(ctx, s);
        rc = enqueue_chains<T>(ctx, s, nch, m, reorth, prof, conv ? &rule : nullptr, conv);
        if (rc != BSE_OK) return rc;
    }
    int warn = BSE_OK;
    if ((rc = finish_run(ctx, s, nch, m, a, b, pnorm2, steps_done, &warn)) != BSE_OK) return rc;
    if ((rc = read_status(ctx)) != BSE_OK) return rc;
    return warn;
}

template <typename T>
int dipoles_typed(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, void* p_out, double* pnorm2) {
    cudaStream_t st = ctx->stream;
    int rc = ensure_state<T>(ctx, s, 1, false, 0);
    if (rc != BSE_OK) return rc;
    cudaMemcpyAsync(s->d_dirs, pol_dirs, sizeof(double) * 3 * npol, cudaMemcpyHostToDevice, st);
    const int nb = vec_blocks(s->N);
    k_dipole_start<T><<<nb, BSE_VEC_THREADS, 0, st>>>(s->d_P, s->d_dirs, s->N, npol, (typename Cx<T>::V*)p_out, s->d_part_nrm);
    k_start_norm<T><<<npol, 256, 0, st>>>(s->d_part_nrm, nb, 0, s->d_pn2, nullptr);
    cudaMemcpyAsync(pnorm2, s->d_pn2, sizeof(double) * npol, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("dipoles: ") + cudaGetErrorString(e); return BSE_ERR_CUDA; }
    return BSE_OK;
}

}  // namespace

void bse_release_run_state(bse_interp* s) {
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    cudaFree(s->d_dirs); cudaFree(s->d_pn2); cudaFree(s->d_eps_prev); cudaFree(s->d_conv_part); cudaFree(s->d_lz_ctr);
    s->d_dirs = nullptr; s->d_pn2 = nullptr; s->d_eps_prev = nullptr; s->d_conv_part = nullptr; s->d_lz_ctr = nullptr;
}

void bse_release_ctx_state(bse_ctx* ctx) {
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    ctx->batch_graph = nullptr;
    for (int k = 0; k < 8; ++k) {
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
        if (ctx->side_join[k]) cudaEventDestroy(ctx->side_join[k]);
        ctx->side[k] = nullptr;
        ctx->side_join[k] = nullptr;
    }
    if (ctx->side_fork) cudaEventDestroy(ctx->side_fork);
    ctx->side_fork = nullptr;
    for (int k = 0; k < 9; ++k) {
        if (ctx->aux[k]) cudaStreamDestroy(ctx->aux[k]);
        if (ctx->aux_fork[k]) cudaEventDestroy(ctx->aux_fork[k]);
        if (ctx->aux_join[k]) cudaEventDestroy(ctx->aux_join[k]);
        ctx->aux[k] = nullptr;
        ctx->aux_fork[k] = nullptr;
        ctx->aux_join[k] = nullptr;
    }
    cudaFree(ctx->cf_buf);
    ctx->cf_buf = nullptr;
    ctx->cf_bytes = 0;
    cudaFree(ctx->d_stop_omega);
    ctx->d_stop_omega = nullptr;
}

void bse_invalidate_graph(bse_interp* s) { drop_graph(s); }

// Auxiliary streams (lowest priority, non-blocking) and fork / join events of
// the concurrent K_c apply, one set per lane; created with the context.
int bse_prepare_aux(bse_ctx* ctx) {
    BSE_CUDA_TRY(ctx, cudaDeviceGetStreamPriorityRange(&ctx->prio_least, &ctx->prio_greatest));
    for (int k = 0; k < 9; ++k) {
        BSE_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ctx->aux[k], cudaStreamNonBlocking, ctx->prio_least));
        BSE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->aux_fork[k], cudaEventDisableTiming));
        BSE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->aux_join[k], cudaEventDisableTiming));
    }
    return BSE_OK;
}

int bse_apply_once(bse_ctx* ctx, bse_interp* s, int nvec, const void* x, void* y, bool profile) {
    int rc = (s->vec_prec == BSE_PREC_F64) ? apply_h_typed<double>(ctx, s, nvec, x, y, profile, false)
                                           : apply_h_typed<float>(ctx, s, nvec, x, y, profile, false);
    if (rc != BSE_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("apply H: ") + cudaGetErrorString(e); return BSE_ERR_CUDA; }
    return read_status(ctx);
}

int bse_run_chains(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, int nsteps, int flags, double* a,
                   double* b, double* pnorm2, int* steps_done) {
    if (s->vec_prec == BSE_PREC_F64)
        return run_chains_typed<double>(ctx, s, npol, pol_dirs, nsteps, flags, a, b, pnorm2, steps_done);
    return run_chains_typed<float>(ctx, s, npol, pol_dirs, nsteps, flags, a, b, pnorm2, steps_done);
}

// Many independent systems in one CUDA graph: every system's whole Haydock
// loop is captured on one of up to 8 side streams forked from the context
// stream (longest systems first, each onto the least-loaded stream) and
// joined back, so the batch is a single graph launch whose branches run
// concurrently on the GPU.  The instantiated graph stays in the context and is
// replayed while the same systems (by serial), chain counts, steps and flags
// come back; with BSE_STOP_CONVERGED the stopped chains skip their work.
int bse_run_batch(bse_ctx* ctx, bse_interp* const* sys, int nsys, const int* npol, const double* pol_dirs, int m,
                  int flags, double* a, double* b, double* pnorm2, int* steps_done) {
    const bool reorth = flags & BSE_REORTH_CGS2;
    const bool conv = flags & BSE_STOP_CONVERGED;
    cudaStream_t main_st = ctx->stream;
    std::vector<int> first(nsys);
    int rc = BSE_OK, off = 0;
    std::vector<long long> key = {ctx->serial, m, flags, conv ? (long long)ctx->stop_every : 0, ctx->wait_cycles};
    for (int i = 0; i < nsys; ++i) {
        bse_interp* s = sys[i];
        rc = (s->vec_prec == BSE_PREC_F64) ? ensure_state<double>(ctx, s, m, reorth, conv ? ctx->stop_nw : 0)
                                           : ensure_state<float>(ctx, s, m, reorth, conv ? ctx->stop_nw : 0);
        if (rc != BSE_OK) return rc;
        BSE_CUDA_TRY(ctx, cudaMemcpyAsync(s->d_dirs, pol_dirs + 3 * off, sizeof(double) * 3 * npol[i],
                                          cudaMemcpyHostToDevice, main_st));
        first[i] = off;
        off += npol[i];
        key.push_back(s->serial);
        key.push_back(s->state_serial);
        key.push_back(npol[i]);
    }
    if (conv) {
        // the rule's numbers are baked into the captured kernels
        long long bits[3];
        std::memcpy(&bits[0], &ctx->stop_tol, 8);
        std::memcpy(&bits[1], &ctx->stop_seps, 8);
        std::memcpy(&bits[2], &ctx->stop_eta, 8);
        key.insert(key.end(), bits, bits + 3);
        key.push_back(ctx->stop_nw);
        key.push_back((long long)(uintptr_t)ctx->d_stop_omega);
    }
    const int K = std::min(nsys, 8);
    if (!ctx->side_fork) {
        BSE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->side_fork, cudaEventDisableTiming));
        for (int k = 0; k < 8; ++k) {
            BSE_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking));
            BSE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->side_join[k], cudaEventDisableTiming));
        }
    }
    cudaError_t e = cudaSuccess;
    if (!ctx->batch_graph || key != ctx->batch_key) {
        if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
        ctx->batch_graph = nullptr;
        std::vector<int> order(nsys);
        std::vector<double> cost(nsys);
        for (int i = 0; i < nsys; ++i) {
            const bse_interp* s = sys[i];
            order[i] = i;
            cost[i] = (double)s->co->Nc * s->co->Nc * npol[i] + (double)s->N * npol[i] * 64.0 +
                      (s->scheme == BSE_SCHEME_M3 ? (double)s->nk * s->npairs * s->t * npol[i] * 8.0 : 0.0);
        }
        std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(main_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaEventRecord(ctx->side_fork, main_st);
            for (int k = 0; k < K; ++k) cudaStreamWaitEvent(ctx->side[k], ctx->side_fork, 0);
            std::vector<double> load(K, 0.0);
            for (int i : order) {
                const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[k] += cost[i];
                ctx->stream = ctx->side[k];
                ctx->lane = 1 + k;
                StopRule rule{};
                if (conv) rule = stop_rule_for(ctx, sys[i]);
                rc = (sys[i]->vec_prec == BSE_PREC_F64)
                         ? enqueue_chains<double>(ctx, sys[i], npol[i], m, reorth, false, conv ? &rule : nullptr, false)
                         : enqueue_chains<float>(ctx, sys[i], npol[i], m, reorth, false, conv ? &rule : nullptr, false);
                ctx->stream = main_st;
                ctx->lane = 0;
                if (rc != BSE_OK) break;
            }
            for (int k = 0; k < K; ++k) {
                cudaEventRecord(ctx->side_join[k], ctx->side[k]);
                cudaStreamWaitEvent(main_st, ctx->side_join[k], 0);
            }
            e = cudaStreamEndCapture(main_st, &g);
        }
        ctx->stream = main_st;
        ctx->lane = 0;
        if (e == cudaSuccess && rc == BSE_OK) e = cudaGraphInstantiate(&ctx->batch_graph, g, cudaGraphInstantiateFlagUseNodePriority);
        if (g) cudaGraphDestroy(g);
        if (rc != BSE_OK) return rc;
        if (e != cudaSuccess) {
            ctx->batch_graph = nullptr;
            ctx->err = std::string("batched Haydock graph: ") + cudaGetErrorString(e);
            return BSE_ERR_CUDA;
        }
        ctx->batch_key = key;
    }
    BSE_CUDA_TRY(ctx, cudaGraphLaunch(ctx->batch_graph, main_st));
    int warn = BSE_OK;
    for (int i = 0; i < nsys; ++i) {
        const int o = first[i];
        rc = finish_run(ctx, sys[i], npol[i], m, a + (size_t)o * m, b + (size_t)o * (m + 1), pnorm2 + o,
                        steps_done + o, &warn);
        if (rc != BSE_OK) return rc;
    }
    if ((rc = read_status(ctx)) != BSE_OK) return rc;
    return warn;
}

int bse_make_dipoles(bse_ctx* ctx, bse_interp* s, int npol, const double* pol_dirs, void* p_out, double* pnorm2) {
    if (s->vec_prec == BSE_PREC_F64) return dipoles_typed<double>(ctx, s, npol, pol_dirs, p_out, pnorm2);
    return dipoles_typed<float>(ctx, s, npol, pol_dirs, p_out, pnorm2);
}

// Continued fraction on the device; its buffers are one grow-only block of the
// context (no allocation once it is large enough).
int bse_cf_device(bse_ctx* ctx, int nchains, int nsteps, const int* steps_done, const double* a, const double* b,
                  const double* pnorm2, double prefactor, double eta, int nw, const double* omega, double* eps) {
    cudaStream_t st = ctx->stream;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t oa = 0, ob = oa + al(sizeof(double) * nchains * nsteps), op = ob + al(sizeof(double) * nchains * (nsteps + 1));
    const size_t ow = op + al(sizeof(double) * nchains), os = ow + al(sizeof(double) * nw);
    const size_t oe = os + al(sizeof(int) * nchains), total = oe + al(sizeof(double2) * nchains * nw);
    if (total > ctx->cf_bytes) {
        cudaFree(ctx->cf_buf);
        ctx->cf_buf = nullptr;
        ctx->cf_bytes = 0;
        int rc = bse_alloc(ctx, &ctx->cf_buf, total, "continued-fraction buffers");
        if (rc != BSE_OK) return rc;
        ctx->cf_bytes = total;
    }
    unsigned char* base = static_cast<unsigned char*>(ctx->cf_buf);
    double* d_a = (double*)(base + oa);
    double* d_b = (double*)(base + ob);
    double* d_pn = (double*)(base + op);
    double* d_w = (double*)(base + ow);
    int* d_s = (int*)(base + os);
    double2* d_eps = (double2*)(base + oe);
    cudaMemcpyAsync(d_a, a, sizeof(double) * nchains * nsteps, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_b, b, sizeof(double) * nchains * (nsteps + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_pn, pnorm2, sizeof(double) * nchains, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_w, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_s, steps_done, sizeof(int) * nchains, cudaMemcpyHostToDevice, st);
    k_cont_frac<<<(nchains * nw + 127) / 128, 128, 0, st>>>(d_a, d_b, d_s, d_pn, nsteps, nchains, prefactor, eta, nw, d_w, d_eps);
    cudaMemcpyAsync(eps, d_eps, sizeof(double2) * nchains * nw, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("continued fraction: ") + cudaGetErrorString(e); return BSE_ERR_CUDA; }
    return BSE_OK;
}

namespace {

// The H application of apply_h_typed with every per-call buffer taken from
// `sc` instead of the handle; enqueues only (no allocation, no sync).
template <typename T>
int apply_scratch_typed(bse_ctx* ctx, const bse_interp* s, int nchains, const void* psi_v, void* w_v,
                        const ApplyScratch& sc) {
    using V = typename Cx<T>::V;
    const bse_coarse* c = s->co;
    cudaStream_t st = ctx->stream;
    const V* psi = (const V*)psi_v;
    V* W = (V*)w_v;
    if (s->scheme == BSE_SCHEME_M2) {
        if constexpr (std::is_same<T, double>::value)
            k_m2_apply<<<m2_blocks(s->N), 32 * kM2Warps, 0, st>>>((const double2*)s->d_H2, psi, s->N, nchains, W, sc.dot);
        return BSE_OK;
    }
    const bool m3 = s->scheme == BSE_SCHEME_M3;
    const bool xh = near_tc_active(s);
    void* X = m3 ? sc.X : nullptr;
    if (xh) k_chain_xscale<<<nchains, 256, 0, st>>>((const float2*)psi, s->N, s->dbound, s->d_xscale_gen);
    if (c->kc_prec == BSE_PREC_BF16) {
        BSE_CUDA_TRY(ctx, cudaMemsetAsync(sc.bop, 0, sizeof(__nv_bfloat16) * 16 * (size_t)c->ldk, st));
        launch_restrict<T>(ctx, s, nchains, psi, nullptr, sc.bop, X, xh, s->d_xscale_gen, sc.U);
        int rc = bse_tc_apply_scratch(ctx, s, nchains, sc.bop, sc.part, sc.R);
        if (rc != BSE_OK) return rc;
    } else {
        launch_restrict<T>(ctx, s, nchains, psi, sc.Q, nullptr, X, xh, s->d_xscale_gen, sc.U);
        k_kc_apply_simt<T><<<(c->Nc + 7) / 8, 256, 0, st>>>((const V*)c->d_kc, (const V*)sc.Q, c->Nc, nchains, (V*)sc.R);
    }
    if (m3) {
        int rc = bse_launch_near_field(ctx, s, nchains, X, s->d_xscale_gen, sc.U);
        if (rc != BSE_OK) return rc;
    }
    launch_prolong<T>(ctx, s, nchains, sc.R, m3 ? sc.U : nullptr, psi, W, sc.dot);
    return BSE_OK;
}

}  // namespace

int bse_apply_scratch(bse_ctx* ctx, const bse_interp* s, int nvec, const void* x, void* y, const ApplyScratch& sc) {
    return (s->vec_prec == BSE_PREC_F64) ? apply_scratch_typed<double>(ctx, s, nvec, x, y, sc)
                                         : apply_scratch_typed<float>(ctx, s, nvec, x, y, sc);
}

namespace {

template <typename T, int NVP>
int launch_near_cell(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, void* U) {
    using V = typename Cx<T>::V;
    const int smem = (int)s->cell_smem;
    if (smem > 48 * 1024)
        BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_cell<T, NVP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid(s->co->nkc, nchains);
    k_near_cell<T, NVP><<<grid, 512, smem, ctx->stream>>>(
        (const V*)X, s->d_clist, s->d_cstart, s->d_pairs, s->npairs, (const T*)s->d_hd, s->n_near, (const V*)s->d_Hv,
        (const V*)s->d_Hc, (const T*)s->d_hc, s->n, s->nd, s->nv, s->nc, s->smin, s->ns1, s->rmin, s->nr1, (V*)U);
    return BSE_OK;
}

template <int NV, int NC, int PF>
int launch_near_rb(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, void* U) {
    constexpr int t = NV * NC, tp = t + 1;
    const size_t bytes = sizeof(float2) * ((size_t)s->npairs * tp + 2 * (size_t)s->Ndiv * tp + 8 * (NV * NV + NC * NC)) +
                         sizeof(float) * (8 + (size_t)s->n_near) + sizeof(int) * ((size_t)s->npairs + 8 * (size_t)s->nslot);
    const int smem = (int)bytes;
    if (smem > 48 * 1024)
        BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_cell_rb<NV, NC, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // one thread per active (target, corner) pair; with at most 256 pairs and no
    // register prefetch, 256-thread CTAs let two CTAs share an SM (128 registers)
    dim3 grid(s->co->nkc, nchains);
    const int bd = (PF == 0 && s->npairs <= 256) ? 256 : 512;
    k_near_cell_rb<NV, NC, PF><<<grid, bd, smem, ctx->stream>>>(
        (const float2*)X, s->d_clist, s->d_cstart, s->d_pairs, s->npairs, (const float*)s->d_hd, s->n_near,
        (const float2*)s->d_Hv, (const float2*)s->d_Hc, (const float*)s->d_hc, s->n, s->nd, s->smin, s->ns1, s->rmin,
        s->nr1, (float2*)U);
    return BSE_OK;
}

template <typename T>
int launch_near_typed(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, const float* xscale, void* U) {
    using V = typename Cx<T>::V;
    if constexpr (std::is_same<T, float>::value) {
        if (near_tc_active(s)) return bse_near_tc_launch(ctx, s, nchains, X, xscale, U);
        if (s->cell_smem && s->npairs <= 512) {
            // rows of the slot staging each of the 512 threads owns
            const int rows = (s->npairs + 512 / s->t - 1) / (512 / s->t);
            if (s->nv == 3 && s->nc == 3)
                return rows <= 8 ? launch_near_rb<3, 3, 8>(ctx, s, nchains, X, U) : launch_near_rb<3, 3, 0>(ctx, s, nchains, X, U);
            if (s->nv == 4 && s->nc == 4)
                return rows <= 12 ? launch_near_rb<4, 4, 12>(ctx, s, nchains, X, U) : launch_near_rb<4, 4, 0>(ctx, s, nchains, X, U);
            if (s->nv == 4 && s->nc == 6) return launch_near_rb<4, 6, 0>(ctx, s, nchains, X, U);
        }
    }
    if (s->cell_smem) {
        if (s->nv <= 1) return launch_near_cell<T, 1>(ctx, s, nchains, X, U);
        if (s->nv <= 2) return launch_near_cell<T, 2>(ctx, s, nchains, X, U);
        if (s->nv <= 4) return launch_near_cell<T, 4>(ctx, s, nchains, X, U);
        return launch_near_cell<T, 8>(ctx, s, nchains, X, U);
    }
    const size_t smem = sizeof(V) * 2 * s->nslot * s->t;
    if (smem > 48 * 1024)
        BSE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_near_field<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_near_field<T><<<s->nk, 256, smem, ctx->stream>>>((const V*)X, s->d_list, s->d_list_start, (const T*)s->d_hd,
                                                      (const V*)s->d_Hv, (const V*)s->d_Hc, (const T*)s->d_hc, s->n,
                                                      s->nd, s->nv, s->nc, s->nb1, s->smin, s->ns1, s->rmin, s->nr1,
                                                      nchains, (V*)U);
    return BSE_OK;
}

}  // namespace

// M3 near field for nchains chains: X pieces in, u pieces out (both [chain][nk][8][t]).
int bse_launch_near_field(bse_ctx* ctx, const bse_interp* s, int nchains, const void* X, const float* xscale, void* U) {
    return (s->vec_prec == BSE_PREC_F64) ? launch_near_typed<double>(ctx, s, nchains, X, xscale, U)
                                         : launch_near_typed<float>(ctx, s, nchains, X, xscale, U);
}
