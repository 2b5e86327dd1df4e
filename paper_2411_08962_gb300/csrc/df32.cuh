// Double-FP32 ("df32") arithmetic: a value is an unevaluated sum hi + lo of two
// floats, about 44 significant bits.  Built from the error-free
// transformations TwoSum (Knuth) and the FMA form of TwoProd (Ogita, Rump,
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005).
// The sums and products use the __fadd_rn / __fmul_rn intrinsics, which the
// compiler never contracts into FMAs or reassociates, so the transformations
// stay error-free whatever the -fmad setting.
#pragma once

#include <cuda_runtime.h>

namespace wick {

struct df {
    float h, l;
};
struct cdf {
    df x, y;  // real, imaginary
};

// a * b = p + e exactly
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

// a + b = s + e exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// acc += (p.h + p.l): the high parts are added error-free, the low parts and
// the rounding error of the high sum are collected in acc.l (renormalised by
// the reader).
__device__ __forceinline__ void acc_add(df &acc, df p) {
    const df s = two_sum(acc.h, p.h);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, p.l));
}

// acc += a * b with a an exact float, b a df32 value
__device__ __forceinline__ void acc_fma(df &acc, float a, df b) {
    df p = two_prod(a, b.h);
    p.l = fmaf(a, b.l, p.l);
    acc_add(acc, p);
}

// complex acc += a * b, a an exact float complex, b df32 complex
__device__ __forceinline__ void cacc_fma(cdf &acc, float2 a, const cdf &b) {
    acc_fma(acc.x, a.x, b.x);
    acc_fma(acc.x, -a.y, b.y);
    acc_fma(acc.y, a.x, b.y);
    acc_fma(acc.y, a.y, b.x);
}

// complex acc += w * a * b, a and b exact float complex, w a small integer
__device__ __forceinline__ void cacc_fma3(cdf &acc, float w, float2 a, float2 b) {
    // products of exact floats are exact as (p, e); the integer weight scales
    // both parts (exact for |w| a power of two, else one rounding of ~2^-48)
    df p;
    p = two_prod(a.x, b.x); p.h = __fmul_rn(p.h, w); p.l = __fmul_rn(p.l, w); acc_add(acc.x, p);
    p = two_prod(-a.y, b.y); p.h = __fmul_rn(p.h, w); p.l = __fmul_rn(p.l, w); acc_add(acc.x, p);
    p = two_prod(a.x, b.y); p.h = __fmul_rn(p.h, w); p.l = __fmul_rn(p.l, w); acc_add(acc.y, p);
    p = two_prod(a.y, b.x); p.h = __fmul_rn(p.h, w); p.l = __fmul_rn(p.l, w); acc_add(acc.y, p);
}

__device__ __forceinline__ double to_double(df a) { return (double)a.h + (double)a.l; }

// split a double into hi + lo floats (exact to ~2^-48 relative)
__device__ __forceinline__ df split_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// (a.h + a.l) * (b.h + b.l), rounded to df32
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
    const float s = __fadd_rn(p.h, p.l);
    return {s, __fsub_rn(p.l, __fsub_rn(s, p.h))};
}

__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.h, b.h);
    const float e = __fadd_rn(__fadd_rn(s.l, a.l), b.l);
    const float r = __fadd_rn(s.h, e);
    return {r, __fsub_rn(e, __fsub_rn(r, s.h))};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

// ---------------------------------------------------------------------------
// Packed form on the sm_100-family f32x2 instructions: one 64-bit register
// holds two float lanes, and add/sub/mul/fma.rn.f32x2 work on both at once.
// A packed double-FP32 value is a pair (h, l) of such registers.
// ---------------------------------------------------------------------------
typedef unsigned long long f2x;

__device__ __forceinline__ f2x pk(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2x v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct pdf {
    f2x h, l;
};

// acc += A * (Bh + Bl) lane-wise, given nA = -A.  np = RN(-A*Bh) = -RN(A*Bh), so
// fma(A, Bh, np) is the exact product error (TwoProd); the high sum is the
// TwoSum of acc.h and RN(A*Bh) written with np; low parts are collected in acc.l.
__device__ __forceinline__ void pacc(pdf &acc, f2x A, f2x nA, f2x Bh, f2x Bl) {
    const f2x np = mul2(nA, Bh);
    f2x e = fma2(A, Bh, np);
    e = fma2(A, Bl, e);
    const f2x s = sub2(acc.h, np);
    const f2x bb = sub2(s, acc.h);
    const f2x t = sub2(acc.h, sub2(s, bb));
    const f2x u = add2(np, bb);
    acc.h = s;
    acc.l = add2(acc.l, add2(sub2(t, u), e));
}

// the same with an exact (float) second factor: no low part to multiply
__device__ __forceinline__ void pacc_exact(pdf &acc, f2x A, f2x nA, f2x B) {
    const f2x np = mul2(nA, B);
    const f2x e = fma2(A, B, np);
    const f2x s = sub2(acc.h, np);
    const f2x bb = sub2(s, acc.h);
    const f2x t = sub2(acc.h, sub2(s, bb));
    const f2x u = add2(np, bb);
    acc.h = s;
    acc.l = add2(acc.l, add2(sub2(t, u), e));
}

__device__ __forceinline__ f2x swap2(f2x v) {
    float a, b;
    upk(v, a, b);
    return pk(b, a);
}

// a + b for packed double-FP32 values, renormalised
__device__ __forceinline__ pdf padd(pdf a, pdf b) {
    const f2x s = add2(a.h, b.h);
    const f2x bb = sub2(s, a.h);
    const f2x err = add2(sub2(a.h, sub2(s, bb)), sub2(b.h, bb));
    const f2x lo = add2(add2(a.l, b.l), err);
    const f2x r = add2(s, lo);
    return {r, sub2(lo, sub2(r, s))};
}

__device__ __forceinline__ cdf cdf_mul(const cdf &a, const cdf &b) {
    return {df_add(df_mul(a.x, b.x), df_neg(df_mul(a.y, b.y))), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}

}  // namespace wick
