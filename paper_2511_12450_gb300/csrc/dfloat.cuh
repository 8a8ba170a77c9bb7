// dfloat.cuh -- double-float arithmetic: a real number as an unevaluated sum hi + lo of two
// FP32 values (|lo| <= ulp(hi) / 2), about 48 significant bits, carried by FP32 instructions.
//
// Built from two error-free transformations: Knuth's two-sum (the exact rounding error of
// an addition, six additions) and the two-product by fused multiply-add (the exact error of
// a product, one FMA).  A multiply-accumulate acc += a b computes a.hi b.hi and its exact
// error, adds the cross terms a.hi b.lo + a.lo b.hi (a.lo b.lo, below 2^-48 relative, is
// dropped), and adds the product into acc by two-sum followed by renormalisation: 13 FP32
// operations.  On a part whose FP64 rate is 1/58 of its FP32 rate, a complex
// multiply-accumulate (four of these, 52 operations) costs less than one DFMA's issue time
// of the four a complex FP64 FMA needs.
#pragma once
#include <cuda_runtime.h>

namespace lfmm {

// complex double-float: (re.hi, re.lo, im.hi, im.lo), 16 bytes like a complex double
typedef float4 dfc;

__device__ __forceinline__ void df_acc(float& ah, float& al, float bh, float bl, float ch, float cl) {
    // (ah, al) += (bh, bl) (ch, cl); the product is rounded on its own (__fmul_rn is never
    // contracted into the following addition), as the two-sum below requires
    const float p = __fmul_rn(bh, ch);
    float pe = fmaf(bh, ch, -p);
    pe = fmaf(bh, cl, pe);
    pe = fmaf(bl, ch, pe);
    const float s = ah + p;
    const float v = s - ah;
    float e = (ah - (s - v)) + (p - v);
    e += al + pe;
    ah = s + e;
    al = e - (ah - s);
}
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
    const float s = ah + bh;
    const float v = s - ah;
    float e = (ah - (s - v)) + (bh - v);
    e += al + bl;
    ah = s + e;
    al = e - (ah - s);
}
// acc += a b (complex)
__device__ __forceinline__ void dfc_fma(dfc& acc, const dfc& a, const dfc& b) {
    df_acc(acc.x, acc.y, a.x, a.y, b.x, b.y);
    df_acc(acc.x, acc.y, -a.z, -a.w, b.z, b.w);
    df_acc(acc.z, acc.w, a.x, a.y, b.z, b.w);
    df_acc(acc.z, acc.w, a.z, a.w, b.x, b.y);
}
__device__ __forceinline__ void dfc_add(dfc& acc, const dfc& b) {
    df_add(acc.x, acc.y, b.x, b.y);
    df_add(acc.z, acc.w, b.z, b.w);
}
// (-1)^k v by sign-bit flips (no arithmetic)
__device__ __forceinline__ dfc dfc_sign(const dfc& v, int k) {
    const unsigned m = ((unsigned)k & 1u) << 31;
    return make_float4(__uint_as_float(__float_as_uint(v.x) ^ m), __uint_as_float(__float_as_uint(v.y) ^ m),
                       __uint_as_float(__float_as_uint(v.z) ^ m), __uint_as_float(__float_as_uint(v.w) ^ m));
}
__device__ __forceinline__ dfc dfc_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// split a double into hi + lo (hi the nearest float, lo the nearest float to the rest)
__device__ __forceinline__ void df_split(double d, float& hi, float& lo) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}
__device__ __forceinline__ dfc to_dfc(double re, double im) {
    dfc r;
    df_split(re, r.x, r.y);
    df_split(im, r.z, r.w);
    return r;
}
__device__ __forceinline__ double df_value(float hi, float lo) { return (double)hi + (double)lo; }

}  // namespace lfmm
