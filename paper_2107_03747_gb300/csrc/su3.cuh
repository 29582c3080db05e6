// su3.cuh -- 3x3 complex matrix arithmetic in registers, templated on the real type.
//
// Products are written out entry by entry so that the compiler keeps every operand
// in registers and contracts the multiply-adds into FMAs; no shared memory, no
// loops that survive unrolling.
#pragma once

#include <cuda_runtime.h>

namespace tgf {

template <class T>
struct cx {
    T re, im;
};

template <class T>
struct mat3 {
    cx<T> e[3][3];
};

template <class T>
__device__ __forceinline__ void set_zero(mat3<T>& a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.e[i][j] = {T(0), T(0)};
}

template <class T>
__device__ __forceinline__ void add_to(mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a.e[i][j].re += b.e[i][j].re;
            a.e[i][j].im += b.e[i][j].im;
        }
}

// Products rounded on their own, never contracted into a neighbouring add.  The scalar sums below
// that mix products and adds are written as explicit chains of fma and mul_rn, so every kernel
// that inlines them rounds the same way (the compiler may otherwise contract a b - c d either way,
// and differently in different kernels).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// a *= (zr + i zi)
template <class T>
__device__ __forceinline__ void scale_cx(mat3<T>& a, T zr, T zi) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T r = a.e[i][j].re, m = a.e[i][j].im;
            a.e[i][j].re = fma(r, zr, -mul_rn(m, zi));
            a.e[i][j].im = fma(r, zi, mul_rn(m, zr));
        }
}

// c = a b
template <class T>
__device__ __forceinline__ void mul_nn(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = a.e[i][0].re * b.e[0][j].re - a.e[i][0].im * b.e[0][j].im;
            T im = a.e[i][0].re * b.e[0][j].im + a.e[i][0].im * b.e[0][j].re;
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                re = fma(a.e[i][k].re, b.e[k][j].re, re);
                re = fma(-a.e[i][k].im, b.e[k][j].im, re);
                im = fma(a.e[i][k].re, b.e[k][j].im, im);
                im = fma(a.e[i][k].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

// c = a b^+
template <class T>
__device__ __forceinline__ void mul_nd(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // sum_k a_ik conj(b_jk)
            T re = a.e[i][0].re * b.e[j][0].re + a.e[i][0].im * b.e[j][0].im;
            T im = a.e[i][0].im * b.e[j][0].re - a.e[i][0].re * b.e[j][0].im;
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                re = fma(a.e[i][k].re, b.e[j][k].re, re);
                re = fma(a.e[i][k].im, b.e[j][k].im, re);
                im = fma(a.e[i][k].im, b.e[j][k].re, im);
                im = fma(-a.e[i][k].re, b.e[j][k].im, im);
            }
            c.e[i][j] = {re, im};
        }
}

// c = a^+ b
template <class T>
__device__ __forceinline__ void mul_dn(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // sum_k conj(a_ki) b_kj
            T re = a.e[0][i].re * b.e[0][j].re + a.e[0][i].im * b.e[0][j].im;
            T im = a.e[0][i].re * b.e[0][j].im - a.e[0][i].im * b.e[0][j].re;
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                re = fma(a.e[k][i].re, b.e[k][j].re, re);
                re = fma(a.e[k][i].im, b.e[k][j].im, re);
                im = fma(a.e[k][i].re, b.e[k][j].im, im);
                im = fma(-a.e[k][i].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

// c = a b + w with the product formed first and w added once: when a b is small next to w (the
// flow's update W + (exp(X) - 1) W) every rounding of the product is relative to the small term,
// and the sum rounds only once on top of w
template <class T>
__device__ __forceinline__ void mul_nn_plus(mat3<T>& c, const mat3<T>& a, const mat3<T>& b, const mat3<T>& w) {
    mul_nn(c, a, b);
    add_to(c, w);
}

// c += a b^+
template <class T>
__device__ __forceinline__ void mul_nd_acc(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = c.e[i][j].re, im = c.e[i][j].im;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(a.e[i][k].re, b.e[j][k].re, re);
                re = fma(a.e[i][k].im, b.e[j][k].im, re);
                im = fma(a.e[i][k].im, b.e[j][k].re, im);
                im = fma(-a.e[i][k].re, b.e[j][k].im, im);
            }
            c.e[i][j] = {re, im};
        }
}

// c += a^+ b
template <class T>
__device__ __forceinline__ void mul_dn_acc(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = c.e[i][j].re, im = c.e[i][j].im;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(a.e[k][i].re, b.e[k][j].re, re);
                re = fma(a.e[k][i].im, b.e[k][j].im, re);
                im = fma(a.e[k][i].re, b.e[k][j].im, im);
                im = fma(-a.e[k][i].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

// Rows 0 and 1 of c = a b^+ and of c = a b (row 2 of c untouched): with a, b in SU(3) the product
// is in SU(3) and its row 2 follows as conj(row0 x row1) (rebuild_row2), so a factor stored as
// two rows needs no rebuilt third row of its own.
template <class T>
__device__ __forceinline__ void mul_nd_top(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = T(0), im = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(a.e[i][k].re, b.e[j][k].re, re);
                re = fma(a.e[i][k].im, b.e[j][k].im, re);
                im = fma(a.e[i][k].im, b.e[j][k].re, im);
                im = fma(-a.e[i][k].re, b.e[j][k].im, im);
            }
            c.e[i][j] = {re, im};
        }
}
template <class T>
__device__ __forceinline__ void mul_nn_top(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T re = T(0), im = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(a.e[i][k].re, b.e[k][j].re, re);
                re = fma(-a.e[i][k].im, b.e[k][j].im, re);
                im = fma(a.e[i][k].re, b.e[k][j].im, im);
                im = fma(a.e[i][k].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

// rows 0 and 1 of c = a b + w (the product formed first, as mul_nn_plus)
template <class T>
__device__ __forceinline__ void mul_nn_plus_top(mat3<T>& c, const mat3<T>& a, const mat3<T>& b, const mat3<T>& w) {
    mul_nn_top(c, a, b);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c.e[i][j].re += w.e[i][j].re;
            c.e[i][j].im += w.e[i][j].im;
        }
}

// c += a^+ b^+
template <class T>
__device__ __forceinline__ void mul_dd_acc(mat3<T>& c, const mat3<T>& a, const mat3<T>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // sum_k conj(a_ki) conj(b_jk)
            T re = c.e[i][j].re, im = c.e[i][j].im;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(a.e[k][i].re, b.e[j][k].re, re);
                re = fma(-a.e[k][i].im, b.e[j][k].im, re);
                im = fma(-a.e[k][i].re, b.e[j][k].im, im);
                im = fma(-a.e[k][i].im, b.e[j][k].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

// ---------------------------------------------------------------------------------------------
// FP32 products on packed pairs.  A complex entry (re, im) sits in one 64-bit register pair and
// the products run on fma.rn.f32x2, two lanes per instruction.  Broadcasting one half of a pair
// ((x, x)) and swapping its halves are free operand forms of the packed instructions; negating a
// half is not.  So each entry of a product is built from two sign-free accumulators
//   p = sum_k x_k * v_k,   q = sum_k y_k * swap(v_k)
// (x, y the broadcast real and imaginary parts of one factor, v the packed entries of the other)
// and one final packed FMA applies the signs: that is 7 packed instructions per entry instead of
// 12 scalar ones.  The FMA pipe time is about the same; the instruction issue, which bounds the
// FP32 stage kernel, drops by about 40 % per product.  Each lane rounds like a scalar FMA; only
// the order of the additions differs from the scalar forms above.
// ---------------------------------------------------------------------------------------------

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, cx<float>& z) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(z.re), "=f"(z.im) : "l"(v));
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 fmul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 as2(const cx<float>& z) { return pack2(z.re, z.im); }   // (re, im)
__device__ __forceinline__ f32x2 sw2(const cx<float>& z) { return pack2(z.im, z.re); }   // (im, re)
__device__ __forceinline__ f32x2 re2(const cx<float>& z) { return pack2(z.re, z.re); }   // (re, re)
__device__ __forceinline__ f32x2 im2(const cx<float>& z) { return pack2(z.im, z.im); }   // (im, im)

// Sign patterns of the final combine.  With p = sum x v and q = sum y swap(v):
//   a b      : re = sum(ar br - ai bi), im = sum(ar bi + ai br)  ->  c = p + (-1, +1) q
//   a b^+    : re = sum(ar br + ai bi), im = sum(ai br - ar bi)  ->  c = q + (+1, -1) p
//   a^+ b    : re = sum(ar br + ai bi), im = sum(ar bi - ai br)  ->  c = p + (+1, -1) q
// where (ar, ai) is the entry of the left factor and (br, bi) that of the right one.

// c = a b
template <>
__device__ __forceinline__ void mul_nn<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(-1.f, 1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[0][j]));
            f32x2 q = fmul2(im2(a.e[i][0]), sw2(b.e[0][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[k][j]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[k][j]), q);
            }
            unpack2(ffma2(q, s, p), c.e[i][j]);
        }
}

// c = a b^+
template <>
__device__ __forceinline__ void mul_nd<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[j][0]));
            f32x2 q = fmul2(im2(a.e[i][0]), sw2(b.e[j][0]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[j][k]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[j][k]), q);
            }
            unpack2(ffma2(p, s, q), c.e[i][j]);
        }
}

// c = a^+ b
template <>
__device__ __forceinline__ void mul_dn<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[0][i]), as2(b.e[0][j]));
            f32x2 q = fmul2(im2(a.e[0][i]), sw2(b.e[0][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[k][i]), as2(b.e[k][j]), p);
                q = ffma2(im2(a.e[k][i]), sw2(b.e[k][j]), q);
            }
            unpack2(ffma2(q, s, p), c.e[i][j]);
        }
}

// c = a b + w: the packed product, then one packed add of w per entry
__device__ __forceinline__ f32x2 fadd2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
template <>
__device__ __forceinline__ void mul_nn_plus<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b,
                                                   const mat3<float>& w) {
    const f32x2 s = pack2(-1.f, 1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[0][j]));
            f32x2 q = fmul2(im2(a.e[i][0]), sw2(b.e[0][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[k][j]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[k][j]), q);
            }
            unpack2(fadd2(ffma2(q, s, p), as2(w.e[i][j])), c.e[i][j]);
        }
}

// c += a b^+ (the old c enters the accumulator that the combine adds unscaled)
template <>
__device__ __forceinline__ void mul_nd_acc<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[j][0]));
            f32x2 q = ffma2(im2(a.e[i][0]), sw2(b.e[j][0]), as2(c.e[i][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[j][k]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[j][k]), q);
            }
            unpack2(ffma2(p, s, q), c.e[i][j]);
        }
}

// c += a^+ b
template <>
__device__ __forceinline__ void mul_dn_acc<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = ffma2(re2(a.e[0][i]), as2(b.e[0][j]), as2(c.e[i][j]));
            f32x2 q = fmul2(im2(a.e[0][i]), sw2(b.e[0][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[k][i]), as2(b.e[k][j]), p);
                q = ffma2(im2(a.e[k][i]), sw2(b.e[k][j]), q);
            }
            unpack2(ffma2(q, s, p), c.e[i][j]);
        }
}

// c += a^+ b^+ = conj(a^T b^T): with p = sum re(a_ki) (b_jk) and q = sum im(a_ki) swap(b_jk) the
// entry is (p.x - q.x, -p.y - q.y), two sign-applying FMAs onto c
template <>
__device__ __forceinline__ void mul_dd_acc<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 sp = pack2(1.f, -1.f), sq = pack2(-1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[0][i]), as2(b.e[j][0]));
            f32x2 q = fmul2(im2(a.e[0][i]), sw2(b.e[j][0]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[k][i]), as2(b.e[j][k]), p);
                q = ffma2(im2(a.e[k][i]), sw2(b.e[j][k]), q);
            }
            unpack2(ffma2(q, sq, ffma2(p, sp, as2(c.e[i][j]))), c.e[i][j]);
        }
}

// rows 0 and 1 of c = a b^+ and c = a b on packed pairs
template <>
__device__ __forceinline__ void mul_nd_top<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(1.f, -1.f);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[j][0]));
            f32x2 q = fmul2(im2(a.e[i][0]), sw2(b.e[j][0]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[j][k]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[j][k]), q);
            }
            unpack2(ffma2(p, s, q), c.e[i][j]);
        }
}
template <>
__device__ __forceinline__ void mul_nn_top<float>(mat3<float>& c, const mat3<float>& a, const mat3<float>& b) {
    const f32x2 s = pack2(-1.f, 1.f);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            f32x2 p = fmul2(re2(a.e[i][0]), as2(b.e[0][j]));
            f32x2 q = fmul2(im2(a.e[i][0]), sw2(b.e[0][j]));
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                p = ffma2(re2(a.e[i][k]), as2(b.e[k][j]), p);
                q = ffma2(im2(a.e[i][k]), sw2(b.e[k][j]), q);
            }
            unpack2(ffma2(q, s, p), c.e[i][j]);
        }
}

// Row 2 of an SU(3) matrix from rows 0 and 1: r2 = conj(r0 x r1).
template <class T>
__device__ __forceinline__ void rebuild_row2(mat3<T>& u) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int a = (j + 1) % 3, b = (j + 2) % 3;
        // (p q - r v)^* with p = r0_a, q = r1_b, r = r0_b, v = r1_a
        const cx<T> p = u.e[0][a], q = u.e[1][b], r = u.e[0][b], v = u.e[1][a];
        const T rv_re = fma(r.re, v.re, -mul_rn(r.im, v.im));
        const T rv_im = fma(r.re, v.im, mul_rn(r.im, v.re));
        const T re = fma(p.re, q.re, fma(-p.im, q.im, -rv_re));
        const T im = fma(p.re, q.im, fma(p.im, q.re, -rv_im));
        u.e[2][j] = {re, -im};
    }
}

// The 8 real parameters of a traceless anti-Hermitian matrix
//   X = [[ i a0,      b01,      b02 ],
//        [ -b01^*,    i a1,     b12 ],
//        [ -b02^*,   -b12^*,    i a2 ]],   a2 = -a0 - a1,
// stored as {a0, a1, b01.re, b01.im, b02.re, b02.im, b12.re, b12.im}.
template <class T>
struct alg8 {
    T v[8];
};

// -P_ta(M) with P_ta(M) = (M - M^+)/2 - tr(M - M^+)/6 * 1: the flow force from Omega = U Sigma.
template <class T>
__device__ __forceinline__ void minus_proj_ta(alg8<T>& z, const mat3<T>& m) {
    const T third = T(1) / T(3);
    T tr = (m.e[0][0].im + m.e[1][1].im + m.e[2][2].im) * third;
    z.v[0] = -(m.e[0][0].im - tr);
    z.v[1] = -(m.e[1][1].im - tr);
    // b_jk = -(m_jk - conj(m_kj))/2
    z.v[2] = -T(0.5) * (m.e[0][1].re - m.e[1][0].re);
    z.v[3] = -T(0.5) * (m.e[0][1].im + m.e[1][0].im);
    z.v[4] = -T(0.5) * (m.e[0][2].re - m.e[2][0].re);
    z.v[5] = -T(0.5) * (m.e[0][2].im + m.e[2][0].im);
    z.v[6] = -T(0.5) * (m.e[1][2].re - m.e[2][1].re);
    z.v[7] = -T(0.5) * (m.e[1][2].im + m.e[2][1].im);
}

}  // namespace tgf
