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

__device__ __forceinline__ cdf cdf_mul(const cdf &a, const cdf &b) {
    return {df_add(df_mul(a.x, b.x), df_neg(df_mul(a.y, b.y))), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}

}  // namespace wick
