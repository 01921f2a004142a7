// dfloat.cuh -- double-float ("double-word") arithmetic: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about
// 48 significant bits.  B300 runs FP32 at many times its FP64 rate, so the
// transforms of the complex128-accuracy path can run in this arithmetic.
//
// Building blocks (error-free transformations and the double-word
// algorithms with proven bounds of Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017):
//   two_sum        a + b = s + e exactly (6 operations, any a, b)
//   fast_two_sum   the same when |a| >= |b| (3 operations)
//   two_prod       a b = p + e exactly with one FMA
//   add            DWPlusDW, relative error <= 3 u^2        (u = 2^-24)
//   mul            DWTimesDW with FMA, relative error <= 5 u^2
//   mul by FP32    DWTimesFP with FMA, relative error <= 2 u^2
// No FP32 rounding may be reassociated or fused here: the FMAs are explicit
// and the sums contain no products the compiler could contract.
#pragma once

#include <cuda_runtime.h>

namespace ctap {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
    __host__ __device__ constexpr df(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ constexpr df(int i) : hi(static_cast<float>(i)), lo(0.0f) {}
    __host__ __device__ explicit operator double() const
    {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

struct alignas(16) df2 {
    df x, y;
};

namespace dfw {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// The same on PAIRS of independent values (the real and the imaginary part
// of one complex value) with the FP32-pair instructions of the sm_100
// family: element by element the same IEEE round-to-nearest operations in
// the same order, so the results are bitwise those of the scalar forms.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = padd(a, b);
    const float2 bb = psub(s, a);
    e = padd(psub(a, psub(s, bb)), psub(b, bb));
}
// two_sum(a, -b) without forming -b: (-b) - bb = -(b + bb) exactly, and
// x + (-y) rounds as x - y
__device__ __forceinline__ void two_diff2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = psub(a, b);
    const float2 bb = psub(s, a);
    e = psub(psub(a, psub(s, bb)), padd(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = padd(a, b);
    e = psub(b, psub(s, a));
}
// DWPlusDW on pairs (SUB: the second operand negated), hi and lo parts
template <bool SUB>
__device__ __forceinline__ void dw_add2(float2 xh, float2 xl, float2 yh, float2 yl, float2 &zh, float2 &zl)
{
    float2 sh, sl, th, tl, vh, vl;
    if constexpr (SUB) {
        two_diff2(xh, yh, sh, sl);
        two_diff2(xl, yl, th, tl);
    } else {
        two_sum2(xh, yh, sh, sl);
        two_sum2(xl, yl, th, tl);
    }
    const float2 c = padd(sl, th);
    fast_two_sum2(sh, c, vh, vl);
    const float2 w = padd(tl, vl);
    fast_two_sum2(vh, w, zh, zl);
}

__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
// DWTimesDW on pairs
__device__ __forceinline__ void dw_mul2(float2 xh, float2 xl, float2 yh, float2 yl, float2 &zh, float2 &zl)
{
    const float2 ch = pmul(xh, yh);
    const float2 cl1 = pfma(xh, yh, pneg(ch));
    const float2 tl0 = pmul(xl, yl);
    const float2 tl1 = pfma(xh, yl, tl0);
    const float2 cl2 = pfma(xl, yh, tl1);
    const float2 cl3 = padd(cl1, cl2);
    fast_two_sum2(ch, cl3, zh, zl);
}

}  // namespace dfw

// a pair of double-float values (two lanes of FP32 pairs): hi parts, lo parts
struct dfp {
    float2 h, l;
};
// a b + c on pairs (the product, then the sum: as fmadd on each element)
__device__ __forceinline__ dfp fmadd2(const dfp &a, const dfp &b, const dfp &c)
{
    dfp t, z;
    dfw::dw_mul2(a.h, a.l, b.h, b.l, t.h, t.l);
    dfw::dw_add2<false>(t.h, t.l, c.h, c.l, z.h, z.l);
    return z;
}

__device__ __forceinline__ df operator+(df x, df y)
{
    float sh, sl, th, tl, vh, vl, zh, zl;
    dfw::two_sum(x.hi, y.hi, sh, sl);
    dfw::two_sum(x.lo, y.lo, th, tl);
    const float c = __fadd_rn(sl, th);
    dfw::fast_two_sum(sh, c, vh, vl);
    const float w = __fadd_rn(tl, vl);
    dfw::fast_two_sum(vh, w, zh, zl);
    return df(zh, zl);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y)
{
    float ch, cl1;
    dfw::two_prod(x.hi, y.hi, ch, cl1);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    const float cl3 = __fadd_rn(cl1, cl2);
    float zh, zl;
    dfw::fast_two_sum(ch, cl3, zh, zl);
    return df(zh, zl);
}
// product with an FP32 number (DWTimesFP)
__device__ __forceinline__ df mul_f(df x, float y)
{
    float ch, cl1;
    dfw::two_prod(x.hi, y, ch, cl1);
    const float cl3 = __fmaf_rn(x.lo, y, cl1);
    float zh, zl;
    dfw::fast_two_sum(ch, cl3, zh, zl);
    return df(zh, zl);
}
__device__ __forceinline__ df &operator+=(df &x, df y) { return x = x + y; }
__device__ __forceinline__ df &operator-=(df &x, df y) { return x = x - y; }
__device__ __forceinline__ df &operator*=(df &x, df y) { return x = x * y; }
__device__ __forceinline__ bool operator<(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// a b + c (a product and a sum, each with its double-word bound)
__device__ __forceinline__ df fmadd(df a, df b, df c) { return a * b + c; }

// exact multiplication by s = +-1 (the half-turn sign of a lifted rotation)
__device__ __forceinline__ df sign_mul(df x, df s) { return df(x.hi * s.hi, x.lo * s.hi); }

// transcendental helpers through FP64 (used only off the hot path:
// imaginary-time factors and large kick angles)
__device__ __forceinline__ df dexp(df x) { return df(::exp(static_cast<double>(x))); }

}  // namespace ctap
