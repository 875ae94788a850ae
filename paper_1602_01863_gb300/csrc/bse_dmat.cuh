// Small dense complex matrices held by one thread (n <= BSE_MAX_BANDS,
// row-major double2 arrays), shared by the set-up kernels (band gauge) and the
// pair-data kernel of the learned residual.
#pragma once

#include "bse_internal.cuh"

// C = A B
__device__ inline void dmat_mul(const double2* A, const double2* B, double2* C, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = 0; k < n; ++k) s = cadd(s, cmul(A[i * n + k], B[k * n + j]));
            C[i * n + j] = s;
        }
}

// E = expm(i A) for Hermitian A by scaling and squaring of the Taylor series:
// X = i A / 2^s with ||A||_F / 2^s <= 1/2, E = sum_{k<=24} X^k / k!, then s squarings.
__device__ inline void dmat_expm_i(const double2* A, int n, double2* E) {
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += A[i].x * A[i].x + A[i].y * A[i].y;
    fro = sqrt(fro);
    int s = 0;
    while (fro > 0.5) { fro *= 0.5; ++s; }
    const double sc = ldexp(1.0, -s);
    double2 X[BSE_MAX_BANDS * BSE_MAX_BANDS], term[BSE_MAX_BANDS * BSE_MAX_BANDS], tmp[BSE_MAX_BANDS * BSE_MAX_BANDS];
    for (int i = 0; i < n * n; ++i) {
        X[i] = make_double2(-A[i].y * sc, A[i].x * sc);   // i A / 2^s
        E[i] = make_double2((i / n == i % n) ? 1.0 : 0.0, 0.0);
        term[i] = E[i];
    }
    for (int k = 1; k <= 24; ++k) {
        dmat_mul(term, X, tmp, n);
        const double inv = 1.0 / k;
        for (int i = 0; i < n * n; ++i) {
            term[i] = cscale(tmp[i], inv);
            E[i] = cadd(E[i], term[i]);
        }
    }
    for (int q = 0; q < s; ++q) {
        dmat_mul(E, E, tmp, n);
        for (int i = 0; i < n * n; ++i) E[i] = tmp[i];
    }
}
