// Set-up kernels: band gauge, coarse kernel K_c, dense tables, M3 tables.
//
// Everything the Haydock loop reads is built here on the device, from the
// model parameters alone (Sec. 2 model inputs, Sec. 3 double-grid tables).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "bse_dmat.cuh"
#include "bse_internal.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ small matrices
// n x n complex matrices (n <= 8) held by one thread, row-major.
struct Mat {
    double2 v[BSE_MAX_BANDS * BSE_MAX_BANDS];
};


// E = expm(i A) for Hermitian A (dmat_expm_i: scaling and squaring of the Taylor series).
__device__ void expm_i(const Mat& A, int n, Mat& E) { dmat_expm_i(A.v, n, E.v); }

// Fractional coordinate of point p of an (n * nd)^3 grid in coarse-major order.
__device__ inline void point_frac(int p, int n, int nd, double k[3], int g[3]) {
    const int Ndiv = nd * nd * nd;
    const int ic = p / Ndiv, js = p % Ndiv;
    const Int3 i = unflat3(ic, n), j = unflat3(js, nd);
    g[0] = i.a * nd + j.a; g[1] = i.b * nd + j.b; g[2] = i.c * nd + j.c;
    const double L = (double)(n * nd);
    for (int a = 0; a < 3; ++a) k[a] = g[a] / L;
}

// Band gauge U(k) = expm(i sum_a [sin(2 pi k_a) G_a0 + (1 - cos 2 pi k_a) G_a1]).
__global__ void k_gauge(const double2* __restrict__ gen, int nb, int n, int nd, int npts,
                        double2* __restrict__ U) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    double k[3];
    int g[3];
    point_frac(p, n, nd, k, g);
    Mat A, E;
    for (int i = 0; i < nb * nb; ++i) A.v[i] = make_double2(0.0, 0.0);
    for (int a = 0; a < 3; ++a) {
        double s, c;
        sincospi(2.0 * k[a], &s, &c);
        const double2* g0 = gen + (a * 2 + 0) * nb * nb;
        const double2* g1 = gen + (a * 2 + 1) * nb * nb;
        for (int i = 0; i < nb * nb; ++i)
            A.v[i] = cadd(A.v[i], cadd(cscale(g0[i], s), cscale(g1[i], 1.0 - c)));
    }
    expm_i(A, nb, E);
    for (int i = 0; i < nb * nb; ++i) U[(size_t)p * nb * nb + i] = E.v[i];
}

__device__ inline void harmonics(const double k[3], double c[7]) {
    c[0] = 1.0;
    for (int a = 0; a < 3; ++a) {
        double s, co;
        sincospi(2.0 * k[a], &s, &co);
        c[1 + 2 * a] = co;
        c[2 + 2 * a] = s;
    }
}

// Minimum-image shape tables over all index differences of an L^3 grid:
// mode 0: h(q) = sum_G exp(-|G|^2) 4 pi / (|q + G|^2 + kappa^2) over `shells` G;
// mode 1: head 1 / (|q|^2 + kappa^2).  Ties (difference L/2) average the images.
__global__ void k_shape_table(int L, double kappa, int shells, int h_const, double h0, int mode,
                              double* __restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L * L * L) return;
    if (mode == 0 && h_const) { out[idx] = h0; return; }
    const Int3 d = unflat3(idx, L);
    int cand[3][2], nc[3];
    const int dd[3] = {d.a, d.b, d.c};
    for (int a = 0; a < 3; ++a) {
        const int r = dd[a];
        if (2 * r < L) { cand[a][0] = r; nc[a] = 1; }
        else if (2 * r > L) { cand[a][0] = r - L; nc[a] = 1; }
        else { cand[a][0] = r; cand[a][1] = r - L; nc[a] = 2; }
    }
    double acc = 0.0;
    int cnt = 0;
    for (int x = 0; x < nc[0]; ++x)
        for (int y = 0; y < nc[1]; ++y)
            for (int z = 0; z < nc[2]; ++z) {
                const double q[3] = {(double)cand[0][x] / L, (double)cand[1][y] / L, (double)cand[2][z] / L};
                double v = 0.0;
                if (mode == 1) {
                    v = 1.0 / (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + kappa * kappa);
                } else {
                    for (int ga = -1; ga <= 1; ++ga)
                        for (int gb = -1; gb <= 1; ++gb)
                            for (int gc = -1; gc <= 1; ++gc) {
                                const int g2 = ga * ga + gb * gb + gc * gc;
                                if (shells == 1 && g2 != 0) continue;
                                const double qa = q[0] + ga, qb = q[1] + gb, qc = q[2] + gc;
                                v += exp(-(double)g2) * 4.0 * kPi / (qa * qa + qb * qb + qc * qc + kappa * kappa);
                            }
                }
                acc += v;
                ++cnt;
            }
    out[idx] = acc / cnt;
}

// Exchange form factors on the coarse mesh: M_vc(k~, G) = [U_v^H mu(k~, G) U_c]_vc.
__global__ void k_form_factors(const double2* __restrict__ Uv, const double2* __restrict__ Uc,
                               const double2* __restrict__ mu, int n, int nv, int nc,
                               double2* __restrict__ M) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nkc = n * n * n;
    if (idx >= nkc * 26) return;
    const int ic = idx / 26, G = idx % 26;
    double k[3];
    int g[3];
    point_frac(ic, n, 1, k, g);
    double c[7];
    harmonics(k, c);
    const double2* uv = Uv + (size_t)ic * nv * nv;
    const double2* uc = Uc + (size_t)ic * nc * nc;
    for (int v = 0; v < nv; ++v)
        for (int cc = 0; cc < nc; ++cc) {
            double2 s = make_double2(0.0, 0.0);
            for (int m = 0; m < nv; ++m)
                for (int mp = 0; mp < nc; ++mp) {
                    double2 muv = make_double2(0.0, 0.0);
                    for (int h = 0; h < 7; ++h)
                        muv = cadd(muv, cscale(mu[((size_t)(h * 26 + G) * nv + m) * nc + mp], c[h]));
                    s = cadd(s, cmul(cmulc(uv[m * nv + v], muv), uc[mp * nc + cc]));
                }
            M[((size_t)ic * 26 + G) * nv * nc + v * nc + cc] = s;
        }
}

// K_c element (Eq. bse2 in the model, coarse weight e_k / n^3):
//   K = pref [ 2 sum_G v(G) conj(M_i(G)) M_j(G) - O^v O^c h(k~_i - k~_j) / eps_inf ].
// 16 x 16 tiles; the form factors of the tile's rows and columns are staged in
// shared memory.  Output in the storage precision of the handle.
template <int PREC>
__global__ void k_build_kc(const double2* __restrict__ M, const double2* __restrict__ Uv,
                           const double2* __restrict__ Uc, const double* __restrict__ htab, int n,
                           int nv, int nc, double pref, double inv_eps, int exchange_on, int Nc,
                           int ldk, void* __restrict__ out, __nv_bfloat16* __restrict__ kr,
                           __nv_bfloat16* __restrict__ ki) {
    __shared__ double2 Mi[16][26];
    __shared__ double2 Mj[16][26];
    const int t = nv * nc;
    const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
    const int tid = threadIdx.y * 16 + threadIdx.x;
    for (int e = tid; e < 16 * 26; e += 256) {
        const int r = e / 26, G = e % 26;
        const int i = i0 + r, j = j0 + r;
        Mi[r][G] = (i < Nc) ? M[((size_t)(i / t) * 26 + G) * t + (i % t)] : make_double2(0.0, 0.0);
        Mj[r][G] = (j < Nc) ? M[((size_t)(j / t) * 26 + G) * t + (j % t)] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
    if (i >= Nc || j >= Nc) return;
    double2 ex = make_double2(0.0, 0.0);
    if (exchange_on) {
        int G = 0;
        for (int ga = -1; ga <= 1; ++ga)
            for (int gb = -1; gb <= 1; ++gb)
                for (int gc = -1; gc <= 1; ++gc) {
                    const int g2 = ga * ga + gb * gb + gc * gc;
                    if (g2 == 0) continue;
                    const double vG = 4.0 * kPi / g2;
                    ex = cadd(ex, cscale(cmulc(Mi[threadIdx.y][G], Mj[threadIdx.x][G]), vG));
                    ++G;
                }
    }
    const int ic = i / t, tr = i % t, v = tr / nc, c = tr % nc;
    const int jc = j / t, tq = j % t, v2 = tq / nc, c2 = tq % nc;
    const double2* uva = Uv + (size_t)ic * nv * nv;
    const double2* uvb = Uv + (size_t)jc * nv * nv;
    const double2* uca = Uc + (size_t)ic * nc * nc;
    const double2* ucb = Uc + (size_t)jc * nc * nc;
    double2 ov = make_double2(0.0, 0.0), oc = make_double2(0.0, 0.0);
    for (int m = 0; m < nv; ++m) ov = cadd(ov, cmulc(uvb[m * nv + v2], uva[m * nv + v]));   // Uv[a]_mv conj(Uv[b]_mv2)
    for (int m = 0; m < nc; ++m) oc = cadd(oc, cmulc(uca[m * nc + c], ucb[m * nc + c2]));   // conj(Uc[a]_mc) Uc[b]_mc2
    const Int3 ia = unflat3(ic, n), ib = unflat3(jc, n);
    const double h = htab[flat3(ia.a - ib.a, ia.b - ib.b, ia.c - ib.c, n)];
    const double2 d = cscale(cmul(ov, oc), h * inv_eps);
    const double2 kv = cscale(csub(cscale(ex, 2.0), d), pref);
    if (PREC == BSE_PREC_F64) {
        reinterpret_cast<double2*>(out)[(size_t)i * Nc + j] = kv;
    } else if (PREC == BSE_PREC_F32) {
        reinterpret_cast<float2*>(out)[(size_t)i * Nc + j] = make_float2((float)kv.x, (float)kv.y);
    } else {
        kr[(size_t)i * ldk + j] = __double2bfloat16(kv.x);
        ki[(size_t)i * ldk + j] = __double2bfloat16(kv.y);
    }
}

// ---------------------------------------------------------------- Method 2
// Dense interpolation matrix (Eq. interpwfn) F [N][Nc], complex128:
// F[(kd, v, c), (k~_l, n1, n2)] += f(kd, l) d_v^{n1} conj(d_c^{n2}); one thread per row.
__global__ void k_m2_F(const double2* __restrict__ Dv, const double2* __restrict__ Dc, int n, int nd, int nv, int nc,
                       int nb1, int N, int Nc, double2* __restrict__ F) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const int t = nv * nc, kd = row / t, tr = row % t, v = tr / nc, c = tr % nc;
    const int Ndiv = nd * nd * nd, ic = kd / Ndiv, js = kd % Ndiv;
    const Int3 i = unflat3(ic, n);
    double2* fr = F + (size_t)row * Nc;
    for (int l = 0; l < 8; ++l) {
        const double f = interp_weight(js, l, nd, nb1);
        if (f == 0.0) continue;
        const int cic = flat3(i.a + ((l >> 2) & 1), i.b + ((l >> 1) & 1), i.c + (l & 1), n);
        const double2* dv = Dv + ((size_t)kd * 8 + l) * nv * nv;
        const double2* dc = Dc + ((size_t)kd * 8 + l) * nc * nc;
        for (int n1 = 0; n1 < nv; ++n1)
            for (int n2 = 0; n2 < nc; ++n2) {
                const double2 val = cscale(cmul(dv[n1 * nv + v], conjg(dc[n2 * nc + c])), f);
                double2* dst = fr + (size_t)cic * t + n1 * nc + n2;
                *dst = cadd(*dst, val);
            }
    }
}

// Head of Eq. diverg for every coarse pair and the remainder:
//   A[(i, n1 n2), (j, n3 n4)] = alpha O^v_{n1 n3}(i, j) O^c_{n2 n4}(i, j),
//   Kmod = K_c - A h_head(q_coarse(i - j)).
__global__ void k_m2_heads(const double2* __restrict__ Uv, const double2* __restrict__ Uc,
                           const double* __restrict__ hh, const double2* __restrict__ Kc, int n, int nv, int nc,
                           double alpha, int Nc, double2* __restrict__ A, double2* __restrict__ Kmod) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Nc * Nc) return;
    const int t = nv * nc, i = (int)(e / Nc), j = (int)(e % Nc);
    const int ic = i / t, jc = j / t, n1 = (i % t) / nc, n2 = (i % t) % nc, n3 = (j % t) / nc, n4 = (j % t) % nc;
    double2 ov = make_double2(0.0, 0.0), oc = make_double2(0.0, 0.0);
    for (int m = 0; m < nv; ++m)
        ov = cadd(ov, cmul(Uv[((size_t)ic * nv + m) * nv + n1], conjg(Uv[((size_t)jc * nv + m) * nv + n3])));
    for (int m = 0; m < nc; ++m)
        oc = cadd(oc, cmul(conjg(Uc[((size_t)ic * nc + m) * nc + n2]), Uc[((size_t)jc * nc + m) * nc + n4]));
    const double2 a = cscale(cmul(ov, oc), alpha);
    const Int3 ia = unflat3(ic, n), ib = unflat3(jc, n);
    const double hc = hh[flat3(ia.a - ib.a, ia.b - ib.b, ia.c - ib.c, n)];
    A[e] = a;
    Kmod[e] = csub(Kc[e], cscale(a, hc));
}

// C [M][Nn] = X [M][K] Y [K][Nn] (conj_y = 0) or X Y^H with Y [Nn][K] (conj_y = 1),
// complex128, 16 x 16 tiles staged in shared memory.
__global__ void k_m2_gemm(const double2* __restrict__ X, const double2* __restrict__ Y, int M, int Nn, int K,
                          int conj_y, double2* __restrict__ C) {
    __shared__ double2 xs[16][17], ys[16][17];
    const int r = blockIdx.y * 16 + threadIdx.y, col = blockIdx.x * 16 + threadIdx.x;
    double2 acc = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int kx = k0 + threadIdx.x, ky = k0 + threadIdx.y;
        xs[threadIdx.y][threadIdx.x] = (r < M && kx < K) ? X[(size_t)r * K + kx] : make_double2(0.0, 0.0);
        const int yc = blockIdx.x * 16 + threadIdx.x;
        double2 yv = make_double2(0.0, 0.0);
        if (yc < Nn && ky < K) yv = conj_y ? conjg(Y[(size_t)yc * K + ky]) : Y[(size_t)ky * Nn + yc];
        ys[threadIdx.y][threadIdx.x] = yv;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc = cadd(acc, cmul(xs[threadIdx.y][kk], ys[kk][threadIdx.x]));
        __syncthreads();
    }
    if (r < M && col < Nn) C[(size_t)r * Nn + col] = acc;
}

// H = diag(dE) + (HA h_head(q_dense) + H) / N_div in place (H holds F Kmod F^H).
__global__ void k_m2_combine(const double2* __restrict__ HA, const double* __restrict__ hd, const double* __restrict__ dE,
                             int n, int nd, int t, int N, double2* __restrict__ H) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)N * N) return;
    const int i = (int)(e / N), j = (int)(e % N);
    const int L = n * nd, Ndiv = nd * nd * nd;
    const int ki = i / t, kj = j / t;
    const Int3 ci = unflat3(ki / Ndiv, n), si = unflat3(ki % Ndiv, nd), cj = unflat3(kj / Ndiv, n), sj = unflat3(kj % Ndiv, nd);
    const double h = hd[flat3((ci.a - cj.a) * nd + si.a - sj.a, (ci.b - cj.b) * nd + si.b - sj.b,
                              (ci.c - cj.c) * nd + si.c - sj.c, L)];
    double2 v = cscale(cadd(cscale(HA[e], h), H[e]), 1.0 / Ndiv);
    if (i == j) v.x += dE[i];
    H[e] = v;
}

// K_c given by the caller (complex128 [Nc][Nc]) converted to the storage precision.
template <int PREC>
__global__ void k_kc_from_user(const double2* __restrict__ user, int Nc, int ldk, void* __restrict__ out,
                               __nv_bfloat16* __restrict__ kr, __nv_bfloat16* __restrict__ ki) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)Nc * Nc) return;
    const double2 v = user[e];
    const long long i = e / Nc, j = e % Nc;
    if (PREC == BSE_PREC_F64) {
        reinterpret_cast<double2*>(out)[e] = v;
    } else if (PREC == BSE_PREC_F32) {
        reinterpret_cast<float2*>(out)[e] = make_float2((float)v.x, (float)v.y);
    } else {
        kr[i * ldk + j] = __double2bfloat16(v.x);
        ki[i * ldk + j] = __double2bfloat16(v.y);
    }
}

// Dense table given by the caller (FP64 / complex128 host data copied to `tmp`)
// into the vector precision.
template <typename T>
__global__ void k_real_to(const double* __restrict__ src, long long n, T* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}
template <typename V>
__global__ void k_cplx_to(const double2* __restrict__ src, long long n, V* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = from_d2<V>(src[i]);
}

// Dense tables, one thread per dense point kd:
//   Delta E_vc(k) (exact on the dense mesh), dipoles P^alpha_vc(k) = [U_v^T pi^alpha conj(U_c)],
//   and for all 8 corners d = U(k~)^H U(k) for both manifolds (Eq. completeness).
template <typename T>
__global__ void k_dense_tables(const double2* __restrict__ Uvd, const double2* __restrict__ Ucd,
                               const double2* __restrict__ Uvc, const double2* __restrict__ Ucc,
                               const double* __restrict__ offsets, const double2* __restrict__ dip,
                               int n, int nd, int nv, int nc, double e_gap, double band_width,
                               T* __restrict__ dE, typename Cx<T>::V* __restrict__ Dv,
                               typename Cx<T>::V* __restrict__ Dc, double2* __restrict__ P) {
    using V = typename Cx<T>::V;
    const int nk = n * n * n * nd * nd * nd;
    const int kd = blockIdx.x * blockDim.x + threadIdx.x;
    if (kd >= nk) return;
    const int t = nv * nc, N = nk * t;
    const int Ndiv = nd * nd * nd;
    double k[3];
    int g[3];
    point_frac(kd, n, nd, k, g);
    double band = e_gap;
    for (int a = 0; a < 3; ++a) band += band_width * (1.0 - cospi(2.0 * k[a]));
    for (int tr = 0; tr < t; ++tr) dE[(size_t)kd * t + tr] = (T)(band + offsets[tr]);
    const double2* uv = Uvd + (size_t)kd * nv * nv;
    const double2* uc = Ucd + (size_t)kd * nc * nc;
    double c[7];
    harmonics(k, c);
    for (int al = 0; al < 3; ++al)
        for (int v = 0; v < nv; ++v)
            for (int cc = 0; cc < nc; ++cc) {
                double2 s = make_double2(0.0, 0.0);
                for (int m = 0; m < nv; ++m)
                    for (int mp = 0; mp < nc; ++mp) {
                        double2 pim = make_double2(0.0, 0.0);
                        for (int h = 0; h < 7; ++h)
                            pim = cadd(pim, cscale(dip[((size_t)(h * 3 + al) * nv + m) * nc + mp], c[h]));
                        s = cadd(s, cmul(cmul(uv[m * nv + v], pim), conjg(uc[mp * nc + cc])));
                    }
                P[(size_t)al * N + (size_t)kd * t + v * nc + cc] = s;
            }
    const int ic = kd / Ndiv;
    const Int3 i = unflat3(ic, n);
    for (int l = 0; l < 8; ++l) {
        const int cic = flat3(i.a + ((l >> 2) & 1), i.b + ((l >> 1) & 1), i.c + (l & 1), n);
        const double2* cv = Uvc + (size_t)cic * nv * nv;
        const double2* ccm = Ucc + (size_t)cic * nc * nc;
        for (int np = 0; np < nv; ++np)
            for (int v = 0; v < nv; ++v) {
                double2 s = make_double2(0.0, 0.0);
                for (int m = 0; m < nv; ++m) s = cadd(s, cmulc(cv[m * nv + np], uv[m * nv + v]));
                Dv[((size_t)kd * 8 + l) * nv * nv + np * nv + v] = from_d2<V>(s);
            }
        for (int np = 0; np < nc; ++np)
            for (int cc = 0; cc < nc; ++cc) {
                double2 s = make_double2(0.0, 0.0);
                for (int m = 0; m < nc; ++m) s = cadd(s, cmulc(ccm[m * nc + np], uc[m * nc + cc]));
                Dc[((size_t)kd * 8 + l) * nc * nc + np * nc + cc] = from_d2<V>(s);
            }
    }
}

// Head factors of Eq. diverg for coarse pairs (k~, k~ + r), r in the relative box:
//   Hv = alpha O^v(k~, k~'), Hc = O^c(k~, k~'); hc[r] = h_head(q_coarse(r)).
template <typename T>
__global__ void k_heads(const double2* __restrict__ Uv, const double2* __restrict__ Uc,
                        const double* __restrict__ hhead_coarse, int n, int nv, int nc, int rmin,
                        int nr1, double alpha, typename Cx<T>::V* __restrict__ Hv,
                        typename Cx<T>::V* __restrict__ Hc, T* __restrict__ hc) {
    using V = typename Cx<T>::V;
    const int nrel = nr1 * nr1 * nr1;
    const int nkc = n * n * n;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nkc * nrel) return;
    const int ic = idx / nrel, r = idx % nrel;
    const Int3 rr = unflat3(r, nr1);
    const int ra = rr.a + rmin, rb = rr.b + rmin, rc = rr.c + rmin;
    const Int3 i = unflat3(ic, n);
    const int jc = flat3(i.a + ra, i.b + rb, i.c + rc, n);
    const double2* uva = Uv + (size_t)ic * nv * nv;
    const double2* uvb = Uv + (size_t)jc * nv * nv;
    const double2* uca = Uc + (size_t)ic * nc * nc;
    const double2* ucb = Uc + (size_t)jc * nc * nc;
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
            double2 s = make_double2(0.0, 0.0);
            for (int m = 0; m < nv; ++m) s = cadd(s, cmulc(uvb[m * nv + b], uva[m * nv + a]));
            Hv[(size_t)idx * nv * nv + a * nv + b] = from_d2<V>(cscale(s, alpha));
        }
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
            double2 s = make_double2(0.0, 0.0);
            for (int m = 0; m < nc; ++m) s = cadd(s, cmulc(uca[m * nc + a], ucb[m * nc + b]));
            Hc[(size_t)idx * nc * nc + a * nc + b] = from_d2<V>(s);
        }
    if (ic == 0) hc[r] = (T)hhead_coarse[flat3(ra, rb, rc, n)];
}

// h_head at the dense near offsets: 1 / (|delta / L|^2 + kappa^2) (near pairs never tie).
template <typename T>
__global__ void k_near_head(const int* __restrict__ offs, int n_near, int L, double kappa,
                            T* __restrict__ hd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_near) return;
    const double qa = (double)offs[3 * i] / L, qb = (double)offs[3 * i + 1] / L,
                 qc = (double)offs[3 * i + 2] / L;
    hd[i] = (T)(1.0 / (qa * qa + qb * qb + qc * qc + kappa * kappa));
}

inline int blocks_for(long long n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace

int bse_alloc(bse_ctx* ctx, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("device allocation of ") + what + " (" + std::to_string(bytes) +
                   " bytes) failed: " + cudaGetErrorString(e);
        *p = nullptr;
        return BSE_ERR_OOM;
    }
    return BSE_OK;
}

#define TRY(x)                     \
    do {                           \
        int rc_ = (x);             \
        if (rc_ != BSE_OK) return rc_; \
    } while (0)

int bse_setup_coarse_device(bse_ctx* ctx, bse_coarse* c, const void* user_kc) {
    const int n = c->n, nv = c->nv, nc = c->nc, nkc = c->nkc, Nc = c->Nc;
    cudaStream_t st = ctx->stream;
    TRY(bse_alloc(ctx, (void**)&c->d_Uv, sizeof(double2) * nkc * nv * nv, "coarse Uv"));
    TRY(bse_alloc(ctx, (void**)&c->d_Uc, sizeof(double2) * nkc * nc * nc, "coarse Uc"));
    k_gauge<<<blocks_for(nkc, 64), 64, 0, st>>>(c->d_gen_v, nv, n, 1, nkc, c->d_Uv);
    k_gauge<<<blocks_for(nkc, 64), 64, 0, st>>>(c->d_gen_c, nc, n, 1, nkc, c->d_Uc);
    double2* d_M = nullptr;
    double* d_h = nullptr;
    if (!user_kc) {
        TRY(bse_alloc(ctx, (void**)&d_M, sizeof(double2) * nkc * 26 * nv * nc, "form factors"));
        TRY(bse_alloc(ctx, (void**)&d_h, sizeof(double) * nkc, "shape table"));
        k_form_factors<<<blocks_for((long long)nkc * 26, 64), 64, 0, st>>>(c->d_Uv, c->d_Uc, c->d_mu, n, nv, nc, d_M);
        k_shape_table<<<blocks_for(nkc, 128), 128, 0, st>>>(n, c->kappa, c->direct_shells, c->h_const, c->h0, 0, d_h);
    }
    size_t bytes;
    if (c->kc_prec == BSE_PREC_F64) bytes = sizeof(double2) * (size_t)Nc * Nc;
    else if (c->kc_prec == BSE_PREC_F32) bytes = sizeof(float2) * (size_t)Nc * Nc;
    else bytes = 2 * sizeof(__nv_bfloat16) * (size_t)Nc * c->ldk;
    int rc = bse_alloc(ctx, &c->d_kc, bytes, "K_c");
    if (rc != BSE_OK) { cudaFree(d_M); cudaFree(d_h); return rc; }
    if (c->kc_prec == BSE_PREC_BF16) {
        c->d_kr = reinterpret_cast<__nv_bfloat16*>(c->d_kc);
        c->d_ki = c->d_kr + (size_t)Nc * c->ldk;
        cudaMemsetAsync(c->d_kc, 0, bytes, st);                 // zero the padding columns
    }
    const double pref = c->e_k / nkc;
    dim3 bs(16, 16), gs(blocks_for(Nc, 16), blocks_for(Nc, 16));
    if (user_kc) {
        const long long ne = (long long)Nc * Nc;
        const double2* u = static_cast<const double2*>(user_kc);
        if (c->kc_prec == BSE_PREC_F64)
            k_kc_from_user<BSE_PREC_F64><<<blocks_for(ne, 256), 256, 0, st>>>(u, Nc, c->ldk, c->d_kc, nullptr, nullptr);
        else if (c->kc_prec == BSE_PREC_F32)
            k_kc_from_user<BSE_PREC_F32><<<blocks_for(ne, 256), 256, 0, st>>>(u, Nc, c->ldk, c->d_kc, nullptr, nullptr);
        else
            k_kc_from_user<BSE_PREC_BF16><<<blocks_for(ne, 256), 256, 0, st>>>(u, Nc, c->ldk, nullptr, c->d_kr, c->d_ki);
    } else if (c->kc_prec == BSE_PREC_F64)
        k_build_kc<BSE_PREC_F64><<<gs, bs, 0, st>>>(d_M, c->d_Uv, c->d_Uc, d_h, n, nv, nc, pref, 1.0 / c->eps_inf,
                                                   c->exchange_on, Nc, c->ldk, c->d_kc, nullptr, nullptr);
    else if (c->kc_prec == BSE_PREC_F32)
        k_build_kc<BSE_PREC_F32><<<gs, bs, 0, st>>>(d_M, c->d_Uv, c->d_Uc, d_h, n, nv, nc, pref, 1.0 / c->eps_inf,
                                                   c->exchange_on, Nc, c->ldk, c->d_kc, nullptr, nullptr);
    else
        k_build_kc<BSE_PREC_BF16><<<gs, bs, 0, st>>>(d_M, c->d_Uv, c->d_Uc, d_h, n, nv, nc, pref, 1.0 / c->eps_inf,
                                                    c->exchange_on, Nc, c->ldk, nullptr, c->d_kr, c->d_ki);
    cudaError_t e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(d_M);
    cudaFree(d_h);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        ctx->err = std::string("coarse set-up kernels: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return BSE_ERR_CUDA;
    }
    return BSE_OK;
}

namespace {

// Replace the model's dense tables by the caller's (bse_dense_inputs), after
// k_dense_tables has written the model's.
// Largest Frobenius norm of the caller's overlap blocks over the pieces of
// non-zero weight (host arrays [nk][8][nb][nb] complex128).
double max_block_norm(const double* d, const bse_interp* s, int nb) {
    double best = 0.0;
    for (int kd = 0; kd < s->nk; ++kd)
        for (int l = 0; l < 8; ++l) {
            if (!interp_active(kd % s->Ndiv, l, s->nd, s->nb1)) continue;
            const double* p = d + ((size_t)kd * 8 + l) * nb * nb * 2;
            double f = 0.0;
            for (int q = 0; q < 2 * nb * nb; ++q) f += p[q] * p[q];
            best = std::max(best, std::sqrt(f));
        }
    return best;
}

template <typename T>
int apply_dense_inputs(bse_ctx* ctx, bse_interp* s, const bse_dense_inputs* in) {
    using V = typename Cx<T>::V;
    const double bv = in->Dv ? max_block_norm(in->Dv, s, s->nv) : std::sqrt((double)s->nv);
    const double bc = in->Dc ? max_block_norm(in->Dc, s, s->nc) : std::sqrt((double)s->nc);
    s->dbound = bv * bc;
    cudaStream_t st = ctx->stream;
    const long long N = s->N, nDv = (long long)s->nk * 8 * s->nv * s->nv, nDc = (long long)s->nk * 8 * s->nc * s->nc;
    const long long most = std::max(std::max(N, nDv), nDc);
    double2* tmp = nullptr;
    TRY(bse_alloc(ctx, (void**)&tmp, sizeof(double2) * (size_t)most, "dense input staging"));
    cudaError_t e = cudaSuccess;
    if (in->dE && e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp, in->dE, sizeof(double) * N, cudaMemcpyHostToDevice, st);
        k_real_to<T><<<blocks_for(N, 256), 256, 0, st>>>((const double*)tmp, N, (T*)s->d_dE);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (in->P && e == cudaSuccess) e = cudaMemcpyAsync(s->d_P, in->P, sizeof(double2) * 3 * N, cudaMemcpyHostToDevice, st);
    if (in->Dv && e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp, in->Dv, sizeof(double2) * nDv, cudaMemcpyHostToDevice, st);
        k_cplx_to<V><<<blocks_for(nDv, 256), 256, 0, st>>>(tmp, nDv, (V*)s->d_Dv);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (in->Dc && e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp, in->Dc, sizeof(double2) * nDc, cudaMemcpyHostToDevice, st);
        k_cplx_to<V><<<blocks_for(nDc, 256), 256, 0, st>>>(tmp, nDc, (V*)s->d_Dc);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        ctx->err = std::string("dense inputs: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    return BSE_OK;
}

// Method 2 set-up (FP64): the dense interpolated Hamiltonian, built with
// temporaries F, A, Kmod, F M and F A F^H that are freed again.
int build_m2(bse_ctx* ctx, bse_interp* s) {
    const bse_coarse* c = s->co;
    cudaStream_t st = ctx->stream;
    const int N = s->N, Nc = c->Nc, L = s->n * s->nd;
    double2 *F = nullptr, *A = nullptr, *Km = nullptr, *T = nullptr, *HA = nullptr;
    double *hh = nullptr, *hd = nullptr;
    int rc = BSE_OK;
    auto cleanup = [&]() { cudaFree(F); cudaFree(A); cudaFree(Km); cudaFree(T); cudaFree(HA); cudaFree(hh); cudaFree(hd); };
    if ((rc = bse_alloc(ctx, &s->d_H2, sizeof(double2) * (size_t)N * N, "Method 2 Hamiltonian")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&F, sizeof(double2) * (size_t)N * Nc, "M2 F")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&A, sizeof(double2) * (size_t)Nc * Nc, "M2 head")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&Km, sizeof(double2) * (size_t)Nc * Nc, "M2 remainder")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&T, sizeof(double2) * (size_t)N * Nc, "M2 temporary")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&HA, sizeof(double2) * (size_t)N * N, "M2 head part")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&hh, sizeof(double) * c->nkc, "coarse head table")) != BSE_OK ||
        (rc = bse_alloc(ctx, (void**)&hd, sizeof(double) * (size_t)L * L * L, "dense head table")) != BSE_OK) {
        cleanup();
        return rc;
    }
    cudaMemsetAsync(F, 0, sizeof(double2) * (size_t)N * Nc, st);
    k_m2_F<<<blocks_for(N, 128), 128, 0, st>>>((const double2*)s->d_Dv, (const double2*)s->d_Dc, s->n, s->nd, s->nv,
                                               s->nc, s->nb1, N, Nc, F);
    k_shape_table<<<blocks_for(c->nkc, 128), 128, 0, st>>>(s->n, c->kappa, 27, 0, 0.0, 1, hh);
    k_shape_table<<<blocks_for((long long)L * L * L, 128), 128, 0, st>>>(L, c->kappa, 27, 0, 0.0, 1, hd);
    k_m2_heads<<<blocks_for((long long)Nc * Nc, 256), 256, 0, st>>>(c->d_Uv, c->d_Uc, hh, (const double2*)c->d_kc, s->n,
                                                                   s->nv, s->nc, c->alpha, Nc, A, Km);
    const dim3 b16(16, 16);
    // H <- F Kmod F^H, HA <- F A F^H
    k_m2_gemm<<<dim3(blocks_for(Nc, 16), blocks_for(N, 16)), b16, 0, st>>>(F, Km, N, Nc, Nc, 0, T);
    k_m2_gemm<<<dim3(blocks_for(N, 16), blocks_for(N, 16)), b16, 0, st>>>(T, F, N, N, Nc, 1, (double2*)s->d_H2);
    k_m2_gemm<<<dim3(blocks_for(Nc, 16), blocks_for(N, 16)), b16, 0, st>>>(F, A, N, Nc, Nc, 0, T);
    k_m2_gemm<<<dim3(blocks_for(N, 16), blocks_for(N, 16)), b16, 0, st>>>(T, F, N, N, Nc, 1, HA);
    k_m2_combine<<<blocks_for((long long)N * N, 256), 256, 0, st>>>(HA, hd, (const double*)s->d_dE, s->n, s->nd, s->t,
                                                                    N, (double2*)s->d_H2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        ctx->err = std::string("Method 2 set-up: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    return BSE_OK;
}

template <typename T>
int setup_interp_typed(bse_ctx* ctx, bse_interp* s, const bse_dense_inputs* dense) {
    using V = typename Cx<T>::V;
    const bse_coarse* c = s->co;
    const int n = s->n, nd = s->nd, nk = s->nk, nv = s->nv, nc = s->nc, t = s->t, N = s->N;
    cudaStream_t st = ctx->stream;
    // dense tables
    double2 *d_Uvd = nullptr, *d_Ucd = nullptr;
    TRY(bse_alloc(ctx, (void**)&d_Uvd, sizeof(double2) * (size_t)nk * nv * nv, "dense Uv"));
    TRY(bse_alloc(ctx, (void**)&d_Ucd, sizeof(double2) * (size_t)nk * nc * nc, "dense Uc"));
    TRY(bse_alloc(ctx, &s->d_dE, sizeof(T) * (size_t)N, "dE"));
    TRY(bse_alloc(ctx, &s->d_Dv, sizeof(V) * (size_t)nk * 8 * nv * nv, "Dv"));
    TRY(bse_alloc(ctx, &s->d_Dc, sizeof(V) * (size_t)nk * 8 * nc * nc, "Dc"));
    TRY(bse_alloc(ctx, (void**)&s->d_P, sizeof(double2) * 3 * (size_t)N, "dipoles"));
    k_gauge<<<blocks_for(nk, 64), 64, 0, st>>>(c->d_gen_v, nv, n, nd, nk, d_Uvd);
    k_gauge<<<blocks_for(nk, 64), 64, 0, st>>>(c->d_gen_c, nc, n, nd, nk, d_Ucd);
    k_dense_tables<T><<<blocks_for(nk, 64), 64, 0, st>>>(d_Uvd, d_Ucd, c->d_Uv, c->d_Uc, c->d_offsets, c->d_dip, n,
                                                        nd, nv, nc, c->e_gap, c->band_width, (T*)s->d_dE,
                                                        (V*)s->d_Dv, (V*)s->d_Dc, s->d_P);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_Uvd);
    cudaFree(d_Ucd);
    if (e != cudaSuccess) {
        ctx->err = std::string("dense set-up kernels: ") + cudaGetErrorString(e);
        return BSE_ERR_CUDA;
    }
    s->dbound = std::sqrt((double)nv) * std::sqrt((double)nc);
    if (dense) TRY(apply_dense_inputs<T>(ctx, s, dense));
    // scratch
    const size_t nvec = BSE_MAX_CHAINS;
    TRY(bse_alloc(ctx, &s->d_Q, sizeof(V) * nvec * c->Nc, "Q"));
    TRY(bse_alloc(ctx, &s->d_R, sizeof(V) * nvec * c->Nc, "R"));
    for (int q = 0; q < 3; ++q) TRY(bse_alloc(ctx, &s->d_vec[q], sizeof(V) * nvec * N, "Lanczos vectors"));
    TRY(bse_alloc(ctx, (void**)&s->d_part_dot, sizeof(double2) * nvec * BSE_MAX_VEC_BLOCKS, "dot partials"));
    TRY(bse_alloc(ctx, (void**)&s->d_part_nrm, sizeof(double) * nvec * BSE_MAX_VEC_BLOCKS, "norm partials"));
    TRY(bse_alloc(ctx, (void**)&s->d_stop, sizeof(int) * nvec, "stop flags"));
    if (s->scheme == BSE_SCHEME_M2) {
        if constexpr (std::is_same<T, double>::value) TRY(build_m2(ctx, s));
    }
    if (s->scheme == BSE_SCHEME_M3) {
        TRY(bse_alloc(ctx, &s->d_X, sizeof(V) * nvec * nk * 8 * t, "restricted pieces X"));
        TRY(bse_alloc(ctx, &s->d_U, sizeof(V) * nvec * nk * 8 * t, "near-field pieces"));
        // near offsets and contribution lists (integer bookkeeping on the host)
        const int R2 = (int)std::floor(s->width * s->width * nd * nd + 1e-9);
        const int rad = (int)std::floor(std::sqrt((double)R2) + 1e-12);
        std::vector<int> offs;
        for (int a = -rad; a <= rad; ++a)
            for (int b = -rad; b <= rad; ++b)
                for (int cc = -rad; cc <= rad; ++cc)
                    if (a * a + b * b + cc * cc <= R2) { offs.push_back(a); offs.push_back(b); offs.push_back(cc); }
        s->n_near = (int)offs.size() / 3;
        s->smin = floordiv(-rad, nd);
        const int smax = floordiv(nd - 1 + rad, nd) + 1;
        s->ns1 = smax - s->smin + 1;
        s->nslot = s->ns1 * s->ns1 * s->ns1;
        s->rmin = s->smin - 1;
        s->nr1 = smax - s->rmin + 1;
        s->nrel = s->nr1 * s->nr1 * s->nr1;
        if (s->ns1 > 15 || s->smin < -8 || smax > 7) {
            ctx->err = "M3 width too large for the near-field tables";
            return BSE_ERR_UNSUPPORTED;
        }
        const int Ndiv = s->Ndiv;
        std::vector<std::vector<NearEntry>> per_slot((size_t)Ndiv * s->nslot);
        for (int js = 0; js < Ndiv; ++js) {
            const Int3 j = unflat3(js, nd);
            for (int q = 0; q < s->n_near; ++q) {
                const int g[3] = {j.a + offs[3 * q], j.b + offs[3 * q + 1], j.c + offs[3 * q + 2]};
                int co[3], jp[3];
                for (int a = 0; a < 3; ++a) { co[a] = floordiv(g[a], nd); jp[a] = g[a] - co[a] * nd; }
                const int jsp = (jp[0] * nd + jp[1]) * nd + jp[2];
                for (int l = 0; l < 8; ++l) {
                    if (interp_weight(jsp, l, nd, s->nb1) == 0.0) continue;
                    const int o[3] = {co[0] + ((l >> 2) & 1), co[1] + ((l >> 1) & 1), co[2] + (l & 1)};
                    const int slot = ((o[0] - s->smin) * s->ns1 + (o[1] - s->smin)) * s->ns1 + (o[2] - s->smin);
                    NearEntry ent;
                    ent.co = (co[0] + 8) | ((co[1] + 8) << 4) | ((co[2] + 8) << 8);
                    ent.js_src = jsp;
                    ent.l_src = l;
                    ent.near_idx = q;
                    per_slot[(size_t)js * s->nslot + slot].push_back(ent);
                }
            }
        }
        std::vector<NearEntry> flat;
        std::vector<int> start((size_t)Ndiv * (s->nslot + 1));
        for (int js = 0; js < Ndiv; ++js) {
            for (int sl = 0; sl < s->nslot; ++sl) {
                start[(size_t)js * (s->nslot + 1) + sl] = (int)flat.size();
                const auto& v = per_slot[(size_t)js * s->nslot + sl];
                flat.insert(flat.end(), v.begin(), v.end());
            }
            start[(size_t)js * (s->nslot + 1) + s->nslot] = (int)flat.size();
        }
        TRY(bse_alloc(ctx, (void**)&s->d_list, sizeof(NearEntry) * flat.size(), "near list"));
        TRY(bse_alloc(ctx, (void**)&s->d_list_start, sizeof(int) * start.size(), "near list starts"));
        BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_list, flat.data(), sizeof(NearEntry) * flat.size(), cudaMemcpyHostToDevice));
        BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_list_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
        // Cell-batched form: the same contributions, with the source named by its
        // (js', corner) pair index, so one coarse cell's targets share a slot's
        // source rows staged in shared memory.
        {
            // corner-major order: neighbouring threads share a corner's head blocks
            std::vector<int> pairs, pidx((size_t)Ndiv * 8, -1);
            for (int l = 0; l < 8; ++l)
                for (int js = 0; js < Ndiv; ++js)
                    if (interp_weight(js, l, nd, s->nb1) != 0.0) {
                        pidx[(size_t)js * 8 + l] = (int)pairs.size();
                        pairs.push_back(js | (l << 16));
                    }
            s->npairs = (int)pairs.size();
            std::vector<int> clist, cstart((size_t)Ndiv * (s->nslot + 1));
            for (int js = 0; js < Ndiv; ++js) {
                for (int sl = 0; sl < s->nslot; ++sl) {
                    cstart[(size_t)js * (s->nslot + 1) + sl] = (int)clist.size();
                    for (const NearEntry& en : per_slot[(size_t)js * s->nslot + sl])
                        clist.push_back(pidx[(size_t)en.js_src * 8 + en.l_src] | (en.near_idx << 16));
                }
                cstart[(size_t)js * (s->nslot + 1) + s->nslot] = (int)clist.size();
            }
            const size_t vs = sizeof(V), ts = sizeof(T);
            const size_t tp = t + 1;                   // padded row stride (bank spread)
            const size_t smem = vs * (2 * (size_t)s->npairs * tp + 2 * (size_t)Ndiv * tp + 8 * (nv * nv + nc * nc)) +
                                ts * (8 + (size_t)s->n_near) + sizeof(int) * ((size_t)s->npairs + 8 * (size_t)s->nslot);
            int maxsm = 0;
            cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
            const bool fits = s->n_near < 65536 && s->npairs < 65536 && smem + 1024 <= (size_t)maxsm;
            s->cell_smem = fits ? smem : 0;
            if (fits) {
                TRY(bse_alloc(ctx, (void**)&s->d_pairs, sizeof(int) * pairs.size(), "near pairs"));
                TRY(bse_alloc(ctx, (void**)&s->d_clist, sizeof(int) * clist.size(), "cell near list"));
                TRY(bse_alloc(ctx, (void**)&s->d_cstart, sizeof(int) * cstart.size(), "cell near list starts"));
                BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice));
                BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_clist, clist.data(), sizeof(int) * clist.size(), cudaMemcpyHostToDevice));
                BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_cstart, cstart.data(), sizeof(int) * cstart.size(), cudaMemcpyHostToDevice));
            }
        }
        int* d_offs = nullptr;
        double* d_hh = nullptr;
        TRY(bse_alloc(ctx, (void**)&d_offs, sizeof(int) * offs.size(), "near offsets"));
        TRY(bse_alloc(ctx, (void**)&d_hh, sizeof(double) * c->nkc, "coarse head table"));
        BSE_CUDA_TRY(ctx, cudaMemcpy(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice));
        TRY(bse_alloc(ctx, &s->d_hd, sizeof(T) * s->n_near, "near head values"));
        TRY(bse_alloc(ctx, &s->d_Hv, sizeof(V) * (size_t)c->nkc * s->nrel * nv * nv, "Hv"));
        TRY(bse_alloc(ctx, &s->d_Hc, sizeof(V) * (size_t)c->nkc * s->nrel * nc * nc, "Hc"));
        TRY(bse_alloc(ctx, &s->d_hc, sizeof(T) * s->nrel, "hc"));
        k_near_head<T><<<blocks_for(s->n_near, 128), 128, 0, st>>>(d_offs, s->n_near, n * nd, c->kappa, (T*)s->d_hd);
        k_shape_table<<<blocks_for(c->nkc, 128), 128, 0, st>>>(n, c->kappa, 27, 0, 0.0, 1, d_hh);
        k_heads<T><<<blocks_for((long long)c->nkc * s->nrel, 64), 64, 0, st>>>(
            c->d_Uv, c->d_Uc, d_hh, n, nv, nc, s->rmin, s->nr1, c->alpha, (V*)s->d_Hv, (V*)s->d_Hc, (T*)s->d_hc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d_offs);
        cudaFree(d_hh);
        if (e != cudaSuccess) {
            ctx->err = std::string("M3 set-up kernels: ") + cudaGetErrorString(e);
            return BSE_ERR_CUDA;
        }
        TRY(bse_near_tc_prepare(ctx, s, per_slot));
        if (s->nf_tc) {
            // FP16 piece scales for unit-norm vectors (every Lanczos vector), and
            // room for the scales bse_apply_h computes from its inputs' norms
            const float xs = bse_near_tc_xscale(s, 1.0 + 1e-3);
            const float h4[4] = {xs, xs, xs, xs};
            TRY(bse_alloc(ctx, (void**)&s->d_xscale, sizeof(float) * 4, "piece scales"));
            TRY(bse_alloc(ctx, (void**)&s->d_xscale_gen, sizeof(float) * 4, "piece scales"));
            BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_xscale, h4, sizeof(h4), cudaMemcpyHostToDevice));
            BSE_CUDA_TRY(ctx, cudaMemcpy(s->d_xscale_gen, h4, sizeof(h4), cudaMemcpyHostToDevice));
        }
    }
    if (c->kc_prec == BSE_PREC_BF16) TRY(bse_tc_prepare(ctx, s));
    return BSE_OK;
}

}  // namespace

int bse_setup_interp_device(bse_ctx* ctx, bse_interp* s, const bse_dense_inputs* dense) {
    if (s->vec_prec == BSE_PREC_F64) return setup_interp_typed<double>(ctx, s, dense);
    return setup_interp_typed<float>(ctx, s, dense);
}
