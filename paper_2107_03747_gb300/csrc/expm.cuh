// expm.cuh -- exact exponential of a traceless anti-Hermitian 3x3 matrix.
//
// For X = iQ (Q Hermitian, traceless) the Cayley-Hamilton theorem gives
// Q^3 = c1 Q + c0 1 with c1 = tr(Q^2)/2 and c0 = det Q, so every power of Q is
// Q^n = alpha_n 1 + beta_n Q + gamma_n Q^2 with the scalar recursion
//   alpha_{n+1} = c0 gamma_n,  beta_{n+1} = alpha_n + c1 gamma_n,  gamma_{n+1} = beta_n,
// and exp(iQ) = f0 1 + f1 Q + f2 Q^2 with f = sum_n i^n (alpha_n, beta_n, gamma_n)/n!
// (the Cayley-Hamilton form of the exponential used by Morningstar & Peardon,
// Phys. Rev. D 69 (2004) 054501, here with the coefficient functions summed as
// their convergent power series instead of the trigonometric closed form).  The
// series is summed in blocks of four terms until the next block is below the
// working precision; arguments with ||Q||_F > 1 are scaled by 2^-s first and the
// result squared s times.  The result is exact to rounding in either precision.
#pragma once

#include "su3.cuh"

namespace tgf {

template <class T>
struct series_tol;
template <>
struct series_tol<double> {
    static constexpr double v = 1e-18;
};
template <>
struct series_tol<float> {
    static constexpr float v = 1e-9f;
};

// Entries of M = f0 + f1 Q + f2 Q^2 (complex f, Hermitian Q and Q^2).  Diagonal: real q = Q_ii,
// u = (Q^2)_ii.  Off-diagonal pair: m_ij = f1 q + f2 u and m_ji = f1 q* + f2 u* for q = Q_ij,
// u = (Q^2)_ij.
template <class T>
__device__ __forceinline__ void set_diag_entry(cx<T>& m, const cx<T>& f0, const cx<T>& f1, const cx<T>& f2, T q, T u) {
    m = {f0.re + f1.re * q + f2.re * u, f0.im + f1.im * q + f2.im * u};
}
template <class T>
__device__ __forceinline__ void set_offdiag_pair(cx<T>& mij, cx<T>& mji, const cx<T>& f1, const cx<T>& f2,
                                                 const cx<T>& q, const cx<T>& u) {
    mij = {f1.re * q.re - f1.im * q.im + f2.re * u.re - f2.im * u.im,
           f1.re * q.im + f1.im * q.re + f2.re * u.im + f2.im * u.re};
    mji = {f1.re * q.re + f1.im * q.im + f2.re * u.re + f2.im * u.im,
           -f1.re * q.im + f1.im * q.re - f2.re * u.im + f2.im * u.re};
}
// FP32 on packed pairs (su3.cuh): with P = f1 q.re + f2 u.re = (A, D) and R = f1 q.im + f2 u.im =
// (C, B) (f as packed (re, im)), m_ij = (A - B, D + C) = P + (-1, +1) swap(R) and
// m_ji = (A + B, D - C) = P + (+1, -1) swap(R): 6 packed instructions per pair instead of 16.
template <>
__device__ __forceinline__ void set_diag_entry<float>(cx<float>& m, const cx<float>& f0, const cx<float>& f1,
                                                      const cx<float>& f2, float q, float u) {
    unpack2(ffma2(as2(f2), pack2(u, u), ffma2(as2(f1), pack2(q, q), as2(f0))), m);
}
template <>
__device__ __forceinline__ void set_offdiag_pair<float>(cx<float>& mij, cx<float>& mji, const cx<float>& f1,
                                                        const cx<float>& f2, const cx<float>& q, const cx<float>& u) {
    const f32x2 P = ffma2(as2(f2), re2(u), fmul2(as2(f1), re2(q)));
    cx<float> R;
    unpack2(ffma2(as2(f2), im2(u), fmul2(as2(f1), im2(q))), R);
    unpack2(ffma2(sw2(R), pack2(-1.f, 1.f), P), mij);
    unpack2(ffma2(sw2(R), pack2(1.f, -1.f), P), mji);
}

// exp(X) for X given by its 8 parameters (see alg8); with MINUS_ONE, exp(X) - 1 with the unit
// matrix taken out of the series (f0 - 1 summed from its second term), so that small X keep
// their full relative precision.
template <class T, bool MINUS_ONE = false>
__device__ __forceinline__ void expm_su3(mat3<T>& m, const alg8<T>& x) {
    // Q = -i X
    const T q00 = x.v[0], q11 = x.v[1], q22 = -(x.v[0] + x.v[1]);
    cx<T> q01 = {x.v[3], -x.v[2]};
    cx<T> q02 = {x.v[5], -x.v[4]};
    cx<T> q12 = {x.v[7], -x.v[6]};
    T n01 = q01.re * q01.re + q01.im * q01.im;
    T n02 = q02.re * q02.re + q02.im * q02.im;
    T n12 = q12.re * q12.re + q12.im * q12.im;
    T c1 = T(0.5) * (q00 * q00 + q11 * q11 + q22 * q22) + n01 + n02 + n12;
    // det Q = q00 q11 q22 + 2 Re(q01 q12 conj(q02)) - q00 |q12|^2 - q11 |q02|^2 - q22 |q01|^2
    T pr = q01.re * q12.re - q01.im * q12.im;
    T pi = q01.re * q12.im + q01.im * q12.re;
    T c0 = q00 * q11 * q22 + T(2) * (pr * q02.re + pi * q02.im) - q00 * n12 - q11 * n02 - q22 * n01;

    int s = 0;
    T sc = T(1);
    T r2 = T(2) * c1;  // ||Q||_F^2
    if (r2 > T(1)) {
        // smallest s with ||Q 2^-s||_F <= 1
        while (r2 > T(1) && s < 60) {
            r2 *= T(0.25);
            sc *= T(0.5);
            ++s;
        }
        c1 *= sc * sc;
        c0 *= sc * sc * sc;
    }

    // f_j = sum_n i^n (alpha_n, beta_n, gamma_n) / n!, summed four terms at a time
    // (i^n cycles i, -1, -i, +1 within a block; at most 20 terms, ||Q||_F <= 1 here)
    T a = T(1), b = T(0), g = T(0);
    // f0 starts at 1 (the n = 0 term) unless the unit matrix is taken out; with scaling and
    // squaring the full matrix is needed first and 1 is subtracted at the end
    T f0r = (MINUS_ONE && s == 0) ? T(0) : T(1), f0i = T(0), f1r = T(0), f1i = T(0), f2r = T(0), f2i = T(0);
    const T tol = series_tol<T>::v;
#pragma unroll
    for (int blk = 0; blk < 5; ++blk) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T inv = T(1) / T(4 * blk + k + 1);
            const T an = c0 * g * inv;
            const T bn = fma(c1, g, a) * inv;
            const T gn = b * inv;
            a = an; b = bn; g = gn;
            if (k == 0) { f0i += a; f1i += b; f2i += g; }
            if (k == 1) { f0r -= a; f1r -= b; f2r -= g; }
            if (k == 2) { f0i -= a; f1i -= b; f2i -= g; }
            if (k == 3) { f0r += a; f1r += b; f2r += g; }
        }
        if (fabs(a) + fabs(b) + fabs(g) < tol) break;
    }
    // Q scaled by sc for the polynomial
    const T s00 = q00 * sc, s11 = q11 * sc, s22 = q22 * sc;
    q01.re *= sc; q01.im *= sc;
    q02.re *= sc; q02.im *= sc;
    q12.re *= sc; q12.im *= sc;
    n01 *= sc * sc; n02 *= sc * sc; n12 *= sc * sc;
    // Q^2 (Hermitian): diagonal and upper triangle
    const T d0 = s00 * s00 + n01 + n02;
    const T d1 = n01 + s11 * s11 + n12;
    const T d2 = n02 + n12 + s22 * s22;
    // (Q^2)_01 = (q00 + q11) q01 + q02 conj(q12)
    cx<T> u01 = {(s00 + s11) * q01.re + q02.re * q12.re + q02.im * q12.im,
                 (s00 + s11) * q01.im + q02.im * q12.re - q02.re * q12.im};
    // (Q^2)_02 = (q00 + q22) q02 + q01 q12
    cx<T> u02 = {(s00 + s22) * q02.re + q01.re * q12.re - q01.im * q12.im,
                 (s00 + s22) * q02.im + q01.re * q12.im + q01.im * q12.re};
    // (Q^2)_12 = conj(q01) q02 + (q11 + q22) q12
    cx<T> u12 = {q01.re * q02.re + q01.im * q02.im + (s11 + s22) * q12.re,
                 q01.re * q02.im - q01.im * q02.re + (s11 + s22) * q12.im};
    // M = f0 + f1 Q + f2 Q^2
    const cx<T> f0 = {f0r, f0i}, f1 = {f1r, f1i}, f2 = {f2r, f2i};
    set_diag_entry(m.e[0][0], f0, f1, f2, s00, d0);
    set_diag_entry(m.e[1][1], f0, f1, f2, s11, d1);
    set_diag_entry(m.e[2][2], f0, f1, f2, s22, d2);
    set_offdiag_pair(m.e[0][1], m.e[1][0], f1, f2, q01, u01);
    set_offdiag_pair(m.e[0][2], m.e[2][0], f1, f2, q02, u02);
    set_offdiag_pair(m.e[1][2], m.e[2][1], f1, f2, q12, u12);
#pragma unroll 1
    for (int k = 0; k < s; ++k) {
        mat3<T> t = m;
        mul_nn(m, t, t);
    }
    if (MINUS_ONE && s > 0) {
        m.e[0][0].re -= T(1);
        m.e[1][1].re -= T(1);
        m.e[2][2].re -= T(1);
    }
}

}  // namespace tgf
