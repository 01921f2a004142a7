// device_fft.cuh -- shared-memory / register FFT building blocks for the
// split-step passes (the transforms of the Fourier split-operator step,
// Sec. IV).  sm_103a, FP32 (complex64) and FP64 (complex128).
//
// Every non-trivial twiddle is a rotation applied by three shears
// ("lifting": x += p y; y += u x; x += p y with p = -tan(phi/2), u = sin phi).
// A product of shears has determinant exactly 1 whatever the rounding of p
// and u, and the inverse rotation is the same three shears with -p, -u, so
// an inverse transform written as the exact mirror of the forward one undoes
// it up to rounding noise only.  This removes the systematic norm drift that
// FP32-rounded cos/sin twiddles give over thousands of steps.
//
// Transforms are mixed-radix Stockham stages: each thread gathers R points
// from shared memory, rotates them by the stage twiddles, runs an R-point DFT
// in registers (radix-2 decimation in frequency, outputs in bit-reversed
// register order) and scatters the results in natural order.  The inverse
// stage is the exact mirror (gather, inverse register DFT, inverse twiddles,
// scatter) and stages run in reverse order, so a forward/inverse pair returns
// N times the input.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "dfloat.cuh"

namespace ctap {

template <class T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<df> { using type = df2; };     // double-float complex (16 bytes)
template <class T> using Cx = typename CxT<T>::type;

// Rotation by phi with |phi| <= pi/2 times a sign s = +-1, in lifting form:
// multiplying by exp(i a) == s * rotate(phi).  f is a spare slot that
// imaginary-time tables use for a real factor.
template <class T> struct alignas(4 * sizeof(T)) Lift { T p, u, s, f; };

constexpr double kPi = 3.14159265358979323846264338327950288;

// --------------------------------------------------------------- helpers
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
__host__ __device__ constexpr int brev(int k, int n)
{
    int r = 0;
    for (int b = 1; b < n; b <<= 1) { r = (r << 1) | (k & 1); k >>= 1; }
    return r;
}

// Taylor series evaluated at compile time (|x| <= pi/2): used only for the
// fixed rotations inside the register DFTs.
__host__ __device__ constexpr double ce_sin(double x)
{
    double t = x, s = x;
    for (int n = 1; n < 24; ++n) { t = -t * x * x / double((2 * n) * (2 * n + 1)); s += t; }
    return s;
}
__host__ __device__ constexpr double ce_cos(double x)
{
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 24; ++n) { t = -t * x * x / double((2 * n - 1) * (2 * n)); s += t; }
    return s;
}

template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
// compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1
template <int N, class F> __device__ __forceinline__ void sfor(F &&f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return ::exp(x); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// v <- rotate(phi) v          (p = -tan(phi/2), u = sin(phi))
template <class T> __device__ __forceinline__ void rot_f(Cx<T> &v, T p, T u)
{
    v.x = fmadd(p, v.y, v.x);
    v.y = fmadd(u, v.x, v.y);
    v.x = fmadd(p, v.y, v.x);
}
// exact mirror: v <- rotate(-phi) v
template <class T> __device__ __forceinline__ void rot_b(Cx<T> &v, T p, T u)
{
    v.x = fmadd(-p, v.y, v.x);
    v.y = fmadd(-u, v.x, v.y);
    v.x = fmadd(-p, v.y, v.x);
}
template <class T> __device__ __forceinline__ void lift_f(Cx<T> &v, const Lift<T> &w)
{
    rot_f<T>(v, w.p, w.u);
    v.x *= w.s;
    v.y *= w.s;
}
template <class T> __device__ __forceinline__ void lift_b(Cx<T> &v, const Lift<T> &w)
{
    v.x *= w.s;
    v.y *= w.s;
    rot_b<T>(v, w.p, w.u);
}
// double-float: the half-turn sign s = +-1 is applied exactly
template <> __device__ __forceinline__ void lift_f<df>(df2 &v, const Lift<df> &w)
{
    rot_f<df>(v, w.p, w.u);
    v.x = sign_mul(v.x, w.s);
    v.y = sign_mul(v.y, w.s);
}
template <> __device__ __forceinline__ void lift_b<df>(df2 &v, const Lift<df> &w)
{
    v.x = sign_mul(v.x, w.s);
    v.y = sign_mul(v.y, w.s);
    rot_b<df>(v, w.p, w.u);
}

// Twiddle exp(-2 pi i J/R) of a radix-2 level of size R, J < R/2, reduced to
// identity (mode 0), a rotation with |phi| < pi/2 (1), times -i (2), or a
// rotation then times -i (3).
template <int R, int J> struct RegTw {
    static constexpr int mode = (J == 0) ? 0 : (4 * J < R ? 1 : (4 * J == R ? 2 : 3));
    static constexpr double phi =
        mode == 1 ? -2.0 * kPi * J / R : (mode == 3 ? -2.0 * kPi * (J - R / 4) / R : 0.0);
    static constexpr double p = -ce_sin(phi / 2) / ce_cos(phi / 2);
    static constexpr double u = ce_sin(phi);
};

// Complex sum and difference of the butterflies.  Double-float: both
// components at once in FP32-pair instructions (bitwise the scalar result,
// half the instructions).
template <class T> __device__ __forceinline__ Cx<T> cx_add(const Cx<T> &a, const Cx<T> &b)
{
    Cx<T> r;
    r.x = a.x + b.x;
    r.y = a.y + b.y;
    return r;
}
template <class T> __device__ __forceinline__ Cx<T> cx_sub(const Cx<T> &a, const Cx<T> &b)
{
    Cx<T> r;
    r.x = a.x - b.x;
    r.y = a.y - b.y;
    return r;
}
template <bool SUB> __device__ __forceinline__ df2 cx_addsub_df(const df2 &a, const df2 &b)
{
    float2 zh, zl;
    dfw::dw_add2<SUB>(make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo),
                      make_float2(b.x.hi, b.y.hi), make_float2(b.x.lo, b.y.lo), zh, zl);
    return df2{df(zh.x, zl.x), df(zh.y, zl.y)};
}
template <> __device__ __forceinline__ df2 cx_add<df>(const df2 &a, const df2 &b) { return cx_addsub_df<false>(a, b); }
template <> __device__ __forceinline__ df2 cx_sub<df>(const df2 &a, const df2 &b) { return cx_addsub_df<true>(a, b); }

// Two double-float complex values rotated at once (the x parts as one pair,
// the y parts as another): a by the lifting pair (pa, ua), b by (pb, ub);
// BACK: the exact mirror (rot_b).  Element by element the operations of
// rot_f / rot_b, so bitwise their results.
// (P, U: the coefficient pairs, already negated for the mirror)
__device__ __forceinline__ void rot2_dfp(df2 &a, df2 &b, const dfp &P, const dfp &U)
{
    dfp X{make_float2(a.x.hi, b.x.hi), make_float2(a.x.lo, b.x.lo)};
    dfp Y{make_float2(a.y.hi, b.y.hi), make_float2(a.y.lo, b.y.lo)};
    X = fmadd2(P, Y, X);
    Y = fmadd2(U, X, Y);
    X = fmadd2(P, Y, X);
    a.x = df(X.h.x, X.l.x);
    b.x = df(X.h.y, X.l.y);
    a.y = df(Y.h.x, Y.l.x);
    b.y = df(Y.h.y, Y.l.y);
}
template <bool BACK>
__device__ __forceinline__ void rot2_df(df2 &a, df2 &b, const df &pa, const df &ua, const df &pb, const df &ub)
{
    const float sg = BACK ? -1.0f : 1.0f;          // exact negation of the coefficients
    const dfp P{make_float2(sg * pa.hi, sg * pb.hi), make_float2(sg * pa.lo, sg * pb.lo)};
    const dfp U{make_float2(sg * ua.hi, sg * ub.hi), make_float2(sg * ua.lo, sg * ub.lo)};
    rot2_dfp(a, b, P, U);
}
// lift_f / lift_b of two double-float values at once (bitwise the single forms)
__device__ __forceinline__ void lift2_f(df2 &a, df2 &b, const Lift<df> &wa, const Lift<df> &wb)
{
    rot2_df<false>(a, b, wa.p, wa.u, wb.p, wb.u);
    a.x = sign_mul(a.x, wa.s);
    a.y = sign_mul(a.y, wa.s);
    b.x = sign_mul(b.x, wb.s);
    b.y = sign_mul(b.y, wb.s);
}
__device__ __forceinline__ void lift2_b(df2 &a, df2 &b, const Lift<df> &wa, const Lift<df> &wb)
{
    a.x = sign_mul(a.x, wa.s);
    a.y = sign_mul(a.y, wa.s);
    b.x = sign_mul(b.x, wb.s);
    b.y = sign_mul(b.y, wb.s);
    rot2_df<true>(a, b, wa.p, wa.u, wb.p, wb.u);
}
// lift_f / lift_b of two values, each with its own twiddle (double-float:
// both at once; otherwise one after the other)
template <class T>
__device__ __forceinline__ void lift_pair_f(Cx<T> &a, Cx<T> &b, const Lift<T> &wa, const Lift<T> &wb)
{
    if constexpr (std::is_same<T, df>::value) {
        lift2_f(a, b, wa, wb);
    } else {
        lift_f<T>(a, wa);
        lift_f<T>(b, wb);
    }
}
template <class T>
__device__ __forceinline__ void lift_pair_b(Cx<T> &a, Cx<T> &b, const Lift<T> &wa, const Lift<T> &wb)
{
    if constexpr (std::is_same<T, df>::value) {
        lift2_b(a, b, wa, wb);
    } else {
        lift_b<T>(a, wa);
        lift_b<T>(b, wb);
    }
}
// both components of a double-float complex value times s (x *= s, y *= s)
__device__ __forceinline__ void cx_scale_df(df2 &v, const df &s)
{
    float2 zh, zl;
    dfw::dw_mul2(make_float2(v.x.hi, v.y.hi), make_float2(v.x.lo, v.y.lo), make_float2(s.hi, s.hi),
                 make_float2(s.lo, s.lo), zh, zl);
    v.x = df(zh.x, zl.x);
    v.y = df(zh.y, zl.y);
}

// Forward R-point DFT (exp(-2 pi i jk/R)) of v[OFF + k*ST], in place; output
// frequency k lands in register OFF + brev(k, R)*ST.
template <int R, int OFF, int ST, class T> __device__ __forceinline__ void dft_fwd(Cx<T> *v)
{
    if constexpr (std::is_same<T, df>::value && R >= 4) {
        // double-float: the same butterflies with the rotations of levels j
        // and j + R/4 (one angle; the second then times -i) done as pairs
        constexpr int H = R / 2, Q4 = R / 4;
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const Cx<T> a = v[OFF + j * ST], b = v[OFF + (j + H) * ST];
            v[OFF + j * ST] = cx_add<T>(a, b);
            v[OFF + (j + H) * ST] = cx_sub<T>(a, b);
        });
        sfor<Q4>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            static_assert(RegTw<R, j + Q4>::mode == (j == 0 ? 2 : 3), "paired levels");
            Cx<T> &d1 = v[OFF + (j + H) * ST];
            Cx<T> &d2 = v[OFF + (j + Q4 + H) * ST];
            if constexpr (W::mode == 1) rot2_df<false>(d1, d2, T(W::p), T(W::u), T(W::p), T(W::u));
            T t = d2.x;                                 // times -i
            d2.x = d2.y;
            d2.y = -t;
        });
        dft_fwd<H, OFF, ST, T>(v);
        dft_fwd<H, OFF + H * ST, ST, T>(v);
    } else if constexpr (R > 1) {
        constexpr int H = R / 2;
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            const Cx<T> a = v[OFF + j * ST], b = v[OFF + (j + H) * ST];
            v[OFF + j * ST] = cx_add<T>(a, b);
            Cx<T> d = cx_sub<T>(a, b);
            if constexpr (W::mode == 1 || W::mode == 3) rot_f<T>(d, T(W::p), T(W::u));
            if constexpr (W::mode >= 2) { T t = d.x; d.x = d.y; d.y = -t; }   // times -i
            v[OFF + (j + H) * ST] = d;
        });
        dft_fwd<H, OFF, ST, T>(v);
        dft_fwd<H, OFF + H * ST, ST, T>(v);
    }
}

// Exact mirror of dft_fwd: input in bit-reversed register order, output
// natural, R times the inverse DFT.
template <int R, int OFF, int ST, class T> __device__ __forceinline__ void dft_inv(Cx<T> *v)
{
    if constexpr (std::is_same<T, df>::value && R >= 4) {
        constexpr int H = R / 2, Q4 = R / 4;
        dft_inv<H, OFF, ST, T>(v);
        dft_inv<H, OFF + H * ST, ST, T>(v);
        sfor<Q4>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            Cx<T> &d1 = v[OFF + (j + H) * ST];
            Cx<T> &d2 = v[OFF + (j + Q4 + H) * ST];
            T t = d2.x;                                 // times +i
            d2.x = -d2.y;
            d2.y = t;
            if constexpr (W::mode == 1) rot2_df<true>(d1, d2, T(W::p), T(W::u), T(W::p), T(W::u));
        });
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const Cx<T> a = v[OFF + j * ST], d = v[OFF + (j + H) * ST];
            v[OFF + j * ST] = cx_add<T>(a, d);
            v[OFF + (j + H) * ST] = cx_sub<T>(a, d);
        });
    } else if constexpr (R > 1) {
        constexpr int H = R / 2;
        dft_inv<H, OFF, ST, T>(v);
        dft_inv<H, OFF + H * ST, ST, T>(v);
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            Cx<T> a = v[OFF + j * ST], d = v[OFF + (j + H) * ST];
            if constexpr (W::mode >= 2) { T t = d.x; d.x = -d.y; d.y = t; }  // times +i
            if constexpr (W::mode == 1 || W::mode == 3) rot_b<T>(d, T(W::p), T(W::u));
            v[OFF + j * ST] = cx_add<T>(a, d);
            v[OFF + (j + H) * ST] = cx_sub<T>(a, d);
        });
    }
}

// Addressing of the batch of lines in a shared-memory tile:
// base(line) = (line >> lgA) * S1 + (line & (A-1)) * S2; element e of a line
// sits at base + e * es.
struct LineMap {
    int lgA, S1, S2, es;
    __device__ __forceinline__ int base(int line) const
    {
        return (line >> lgA) * S1 + (line & ((1 << lgA) - 1)) * S2;
    }
};

// One Stockham stage of radix R on 2^lgLines lines of length 2^lgL in shared
// memory; Ns = 2^lgNs; tw holds exp(-2 pi i e/(Ns R)), e < Ns R.
// NT threads, each holding up to MAXV points.
template <int R, int MAXV, int NT, class T>
__device__ __forceinline__ void stage_fwd(Cx<T> *sm, const LineMap lm, int lgLines, int lgL,
                                          int lgNs, const Lift<T> *__restrict__ tw)
{
    constexpr int Q = MAXV / R;
    constexpr int lgR = ilog2(R);
    static_assert(Q >= 1, "radix larger than the per-thread capacity");
    const int lgLr = lgL - lgR;
    const int ntasks = 1 << (lgLines + lgLr);
    const int lmask = (1 << lgLines) - 1;
    Cx<T> v[Q][R];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int q = threadIdx.x + i * NT;
        if (q < ntasks) {
            const int base = lm.base(q & lmask), j = q >> lgLines;
#pragma unroll
            for (int r = 0; r < R; ++r) v[i][r] = sm[base + (j + (r << lgLr)) * lm.es];
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int q = threadIdx.x + i * NT;
        if (q < ntasks) {
            const int base = lm.base(q & lmask), j = q >> lgLines;
            const int jm = j & ((1 << lgNs) - 1);
            if (lgNs > 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) lift_f<T>(v[i][r], tw[jm * r]);
            }
            dft_fwd<R, 0, 1, T>(v[i]);
            const int idxD = ((j >> lgNs) << (lgNs + lgR)) + jm;
            sfor<R>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                sm[base + (idxD + (k << lgNs)) * lm.es] = v[i][brev(k, R)];
            });
        }
    }
    __syncthreads();
}

// Exact mirror of stage_fwd.
template <int R, int MAXV, int NT, class T>
__device__ __forceinline__ void stage_inv(Cx<T> *sm, const LineMap lm, int lgLines, int lgL,
                                          int lgNs, const Lift<T> *__restrict__ tw)
{
    constexpr int Q = MAXV / R;
    constexpr int lgR = ilog2(R);
    static_assert(Q >= 1, "radix larger than the per-thread capacity");
    const int lgLr = lgL - lgR;
    const int ntasks = 1 << (lgLines + lgLr);
    const int lmask = (1 << lgLines) - 1;
    Cx<T> v[Q][R];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int q = threadIdx.x + i * NT;
        if (q < ntasks) {
            const int base = lm.base(q & lmask), j = q >> lgLines;
            const int jm = j & ((1 << lgNs) - 1);
            const int idxD = ((j >> lgNs) << (lgNs + lgR)) + jm;
            sfor<R>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                v[i][brev(k, R)] = sm[base + (idxD + (k << lgNs)) * lm.es];
            });
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int q = threadIdx.x + i * NT;
        if (q < ntasks) {
            const int base = lm.base(q & lmask), j = q >> lgLines;
            const int jm = j & ((1 << lgNs) - 1);
            dft_inv<R, 0, 1, T>(v[i]);
            if (lgNs > 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) lift_b<T>(v[i][r], tw[jm * r]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) sm[base + (j + (r << lgLr)) * lm.es] = v[i][r];
        }
    }
    __syncthreads();
}

// Radix plan of one axis: nst Stockham stages, stage s has radix R[s],
// Ns = 2^lgNs[s] and its twiddle table at tw + off[s].
struct AxisPlan {
    int lgL;
    int nst;
    int R[4];
    int lgNs[4];
    int off[4];
};

template <int MAXV, int NT, class T>
__device__ __forceinline__ void axis_fwd(Cx<T> *sm, const LineMap lm, int lgLines,
                                         const AxisPlan &ap, const Lift<T> *__restrict__ tw)
{
    for (int s = 0; s < ap.nst; ++s) {
        const Lift<T> *t = tw + ap.off[s];
        switch (ap.R[s]) {
        case 2: stage_fwd<2, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 4: stage_fwd<4, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 8: stage_fwd<8, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 16: stage_fwd<16, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        default:
            if constexpr (MAXV >= 32) stage_fwd<32, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t);
            break;
        }
    }
}

template <int MAXV, int NT, class T>
__device__ __forceinline__ void axis_inv(Cx<T> *sm, const LineMap lm, int lgLines,
                                         const AxisPlan &ap, const Lift<T> *__restrict__ tw)
{
    for (int s = ap.nst - 1; s >= 0; --s) {
        const Lift<T> *t = tw + ap.off[s];
        switch (ap.R[s]) {
        case 2: stage_inv<2, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 4: stage_inv<4, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 8: stage_inv<8, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        case 16: stage_inv<16, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t); break;
        default:
            if constexpr (MAXV >= 32) stage_inv<32, MAXV, NT, T>(sm, lm, lgLines, ap.lgL, ap.lgNs[s], t);
            break;
        }
    }
}

// ---------------------------------------------------------------- kicks
// exp(i a) = s * rotate(phi), |phi| <= pi/2, from the angle a at run time.
// Half-angle sine and cosine from their Taylor series on |h| <= pi/4.
__device__ __forceinline__ void lift_from_angle(float a, float &p, float &u, float &s)
{
    const float m = rintf(a * 0.318309886183790671f);          // half-turns
    float phi = fmadd(-m, 3.14159274101257324f, a);            // pi split hi/lo
    phi = fmadd(-m, -8.74227765734758577e-08f, phi);
    s = (static_cast<int>(m) & 1) ? -1.0f : 1.0f;
    const float h = 0.5f * phi, h2 = h * h;
    float sn = fmadd(h2, 2.75573192e-06f, -1.98412698e-04f);    // 1/9!, -1/7!
    sn = fmadd(h2, sn, 8.33333333e-03f);                       // 1/5!
    sn = fmadd(h2, sn, -1.66666667e-01f);                      // -1/3!
    sn = fmadd(h2 * h, sn, h);
    float cs = fmadd(h2, -2.75573192e-07f, 2.48015873e-05f);    // -1/10!, 1/8!
    cs = fmadd(h2, cs, -1.38888889e-03f);                      // -1/6!
    cs = fmadd(h2, cs, 4.16666667e-02f);                       // 1/4!
    cs = fmadd(h2, cs, -0.5f);
    cs = fmadd(h2, cs, 1.0f);
    p = -sn / cs;
    u = 2.0f * sn * cs;
}

__device__ __forceinline__ void lift_from_angle(double a, double &p, double &u, double &s)
{
    const double m = rint(a * 0.318309886183790671538);
    double phi = fmadd(-m, 3.141592653589793116, a);
    phi = fmadd(-m, 1.2246467991473532e-16, phi);
    s = (static_cast<long long>(m) & 1) ? -1.0 : 1.0;
    const double h = 0.5 * phi, h2 = h * h;
    // sin(h) = h sum (-h^2)^n/(2n+1)!, cos(h) = sum (-h^2)^n/(2n)!, n <= 10
    double sn = 1.0 / 51090942171709440000.0;                  // 1/21!
    double cs = 1.0 / 2432902008176640000.0;                   // 1/20!
    const double fs[10] = {-1.0 / 121645100408832000.0, 1.0 / 355687428096000.0,
                           -1.0 / 1307674368000.0, 1.0 / 6227020800.0, -1.0 / 39916800.0,
                           1.0 / 362880.0, -1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0, 1.0};
    const double fc[10] = {-1.0 / 6402373705728000.0, 1.0 / 20922789888000.0,
                           -1.0 / 87178291200.0, 1.0 / 479001600.0, -1.0 / 3628800.0,
                           1.0 / 40320.0, -1.0 / 720.0, 1.0 / 24.0, -1.0 / 2.0, 1.0};
#pragma unroll
    for (int i = 0; i < 10; ++i) {          // Horner in h^2, signs in the coefficients
        sn = fmadd(sn, h2, fs[i]);
        cs = fmadd(cs, h2, fc[i]);
    }
    sn *= h;
    p = -sn / cs;
    u = 2.0 * sn * cs;
}

// double-float kick coefficients for |th| <= 0.1: p = -tan(-th/2), u = sin(-th)
// from their odd Taylor series in double-float arithmetic (terms through
// th^11, below 2^-48 relative)
__device__ __forceinline__ void lift_small(df th, df &p, df &u)
{
    const df a = -th, a2 = a * a;
    df s = fmadd(a2, df(-2.5052108385441720e-08), df(2.7557319223985893e-06));
    s = fmadd(a2, s, df(-1.9841269841269841e-04));
    s = fmadd(a2, s, df(8.3333333333333333e-03));
    s = fmadd(a2, s, df(-1.6666666666666667e-01));
    u = fmadd(a2 * a, s, a);
    const df h = mul_f(a, 0.5f), h2 = h * h;
    df t = fmadd(h2, df(3.5921280365724810e-03), df(8.8632355299021966e-03));
    t = fmadd(h2, t, df(2.1869488536155203e-02));
    t = fmadd(h2, t, df(5.3968253968253968e-02));
    t = fmadd(h2, t, df(1.3333333333333333e-01));
    t = fmadd(h2, t, df(3.3333333333333333e-01));
    p = -fmadd(h2 * h, t, h);
}

// lift_small for two angles at once (the coefficients as pairs): element by
// element the operations of lift_small, so bitwise its results
__device__ __forceinline__ dfp dfp_const(double c)
{
    const df d(c);
    return dfp{make_float2(d.hi, d.hi), make_float2(d.lo, d.lo)};
}
__device__ __forceinline__ dfp dfp_mul(const dfp &x, const dfp &y)
{
    dfp z;
    dfw::dw_mul2(x.h, x.l, y.h, y.l, z.h, z.l);
    return z;
}
__device__ __forceinline__ void lift_small2(df th0, df th1, dfp &p, dfp &u)
{
    const dfp a{make_float2(-th0.hi, -th1.hi), make_float2(-th0.lo, -th1.lo)};
    const dfp a2 = dfp_mul(a, a);
    dfp s = fmadd2(a2, dfp_const(-2.5052108385441720e-08), dfp_const(2.7557319223985893e-06));
    s = fmadd2(a2, s, dfp_const(-1.9841269841269841e-04));
    s = fmadd2(a2, s, dfp_const(8.3333333333333333e-03));
    s = fmadd2(a2, s, dfp_const(-1.6666666666666667e-01));
    u = fmadd2(dfp_mul(a2, a), s, a);
    // h = a/2 as mul_f(a, 0.5f) (DWTimesFP)
    dfp h;
    {
        const float2 y = make_float2(0.5f, 0.5f);
        const float2 ch = dfw::pmul(a.h, y);
        const float2 cl1 = dfw::pfma(a.h, y, dfw::pneg(ch));
        const float2 cl3 = dfw::pfma(a.l, y, cl1);
        dfw::fast_two_sum2(ch, cl3, h.h, h.l);
    }
    const dfp h2 = dfp_mul(h, h);
    dfp t = fmadd2(h2, dfp_const(3.5921280365724810e-03), dfp_const(8.8632355299021966e-03));
    t = fmadd2(h2, t, dfp_const(2.1869488536155203e-02));
    t = fmadd2(h2, t, dfp_const(5.3968253968253968e-02));
    t = fmadd2(h2, t, dfp_const(1.3333333333333333e-01));
    t = fmadd2(h2, t, dfp_const(3.3333333333333333e-01));
    const dfp q = fmadd2(dfp_mul(h2, h), t, h);
    p = dfp{dfw::pneg(q.h), dfw::pneg(q.l)};
}

// double-float angle: reduced and evaluated in FP64 (kicks use the
// double-float series above for small angles instead)
__device__ __forceinline__ void lift_from_angle(df a, df &p, df &u, df &s)
{
    double pd, ud, sd;
    lift_from_angle(static_cast<double>(a), pd, ud, sd);
    p = df(pd);
    u = df(ud);
    s = df(sd);
}

}  // namespace ctap
