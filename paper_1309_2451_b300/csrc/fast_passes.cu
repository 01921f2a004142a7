// fast_passes.cu -- specialised XY and Z passes (complex64 and complex128).
//
// Same HBM layout and the same arithmetic definition as the generic passes
// in kernels.cu (natural kx order, natural k' order, rows j P + r), so plans
// can mix them.  What changes is how the work stays on chip.
//
// Every middle stage is done IN PLACE per task: a task writes its results
// back to exactly the shared-memory positions it read, so a stage needs no
// "load all / barrier / store all" and a task is one small register DFT in a
// runtime loop (compact code: the fully unrolled alternative stalled on
// instruction fetch).  For that, real-space x and y are kept inside shared
// memory in digit-swapped order (position RA (x mod RB) + x div RB for
// x = RA RB points); HBM always sees natural order.
//
// XY pass (NX = RA RB columns, LY = YA YB rows of one plane's row class):
//   P1  inverse x, last Stockham stage, read straight from HBM, rotated back;
//   P2  inverse x, first stage, in place;
//   P3a inverse y, last stage (in place);
//   P3b inverse y first stage -> potential factor -> forward y first stage,
//       in registers, in place;
//   P3c forward y, last stage (in place);
//   P4  forward x, first stage, in place;
//   P5  forward x, last stage, straight to HBM.
//
// Z pass (NZ = ZA ZB, tile NZ x C, C = P W, 256 or 512 threads):
//   Z1  read P rows per z (two columns per thread), finish the forward
//       y-transform (cross twiddle + P-point DFT), write the tile;
//   Z2  forward z, first stage, in place;
//   Z3  forward z last stage, kinetic factor, inverse last stage, in
//       registers, in place;
//   Z4  inverse z, first stage, in place;
//   Z5  inverse cross DFT, store.
//   Tile columns are XOR-swizzled per z (column ^ W (z mod 16/W)) so that
//   the z-major accesses of Z1/Z5 and the column accesses of Z2-Z4 are both
//   free of bank conflicts.
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace ctap {

namespace {

constexpr int kFastNT = 512;

// exp(-i th) as a lifted rotation for |th| <= 0.5 (no half-turn reduction):
// rotation angle a = -th; u = sin(a), p = -tan(a/2) from odd Taylor series
// (own; |a/2| <= 0.25).
__device__ __forceinline__ void lift_small(float th, float &p, float &u)
{
    const float a = -th, a2 = a * a;
    float s = fmadd(a2, 2.75573192e-06f, -1.98412698e-04f);      // 1/9!, -1/7!
    s = fmadd(a2, s, 8.33333333e-03f);                           // 1/5!
    s = fmadd(a2, s, -1.66666667e-01f);                          // -1/3!
    u = fmadd(a2 * a, s, a);
    const float h = 0.5f * a, h2 = h * h;                        // tan h series
    float t = fmadd(h2, 8.86323552e-03f, 2.18694885e-02f);        // 1382/155925, 62/2835
    t = fmadd(h2, t, 5.39682540e-02f);                           // 17/315
    t = fmadd(h2, t, 1.33333333e-01f);                           // 2/15
    t = fmadd(h2, t, 3.33333333e-01f);                           // 1/3
    p = -fmadd(h2 * h, t, h);
}

// exp(-i th) for the real-time kick: the short series for complex64 when
// |th| <= 0.5, the general half-turn reduction otherwise (always for FP64)
// |th| <= 0.16: the same odd series truncated after the fifth-order terms
// (omitted terms below th^7/5040 = 5e-10 and 17 (th/2)^7/315 = 1e-9)
__device__ __forceinline__ void lift_tiny(float th, float &p, float &u)
{
    const float a = -th, a2 = a * a;
    u = fmadd(a2 * a, fmadd(a2, 8.33333333e-03f, -1.66666667e-01f), a);     // a - a^3/6 + a^5/120
    const float h = 0.5f * a, h2 = h * h;
    p = -fmadd(h2 * h, fmadd(h2, 1.33333333e-01f, 3.33333333e-01f), h);    // -(h + h^3/3 + 2h^5/15)
}

// small: 2 for |th| <= 0.16, 1 for |th| <= 0.5, 0 for any angle
__device__ __forceinline__ void kick_rt(float2 &v, float th, int small)
{
    if (small == 2) {
        float p, u;
        lift_tiny(th, p, u);
        rot_f<float>(v, p, u);
    } else if (small) {
        float p, u;
        lift_small(th, p, u);
        rot_f<float>(v, p, u);
    } else {
        float p, u, s;
        lift_from_angle(-th, p, u, s);
        rot_f<float>(v, p, u);
        v.x *= s;
        v.y *= s;
    }
}
// FP64: |th| <= 0.1 uses odd Taylor series without division (own; next
// terms below 1e-18 relative), otherwise the general reduction.
__device__ __forceinline__ void lift_small(double th, double &p, double &u)
{
    const double a = -th, a2 = a * a;
    double s = fmadd(a2, -2.5052108385441720e-08, 2.7557319223985893e-06);   // -1/11!, 1/9!
    s = fmadd(a2, s, -1.9841269841269841e-04);                               // -1/7!
    s = fmadd(a2, s, 8.3333333333333333e-03);                                // 1/5!
    s = fmadd(a2, s, -1.6666666666666667e-01);                               // -1/3!
    u = fmadd(a2 * a, s, a);
    const double h = 0.5 * a, h2 = h * h;
    double t = fmadd(h2, 3.5921280365724810e-03, 8.8632355299021966e-03);    // 21844/6081075, 1382/155925
    t = fmadd(h2, t, 2.1869488536155203e-02);                                // 62/2835
    t = fmadd(h2, t, 5.3968253968253968e-02);                                // 17/315
    t = fmadd(h2, t, 1.3333333333333333e-01);                                // 2/15
    t = fmadd(h2, t, 3.3333333333333333e-01);                                // 1/3
    p = -fmadd(h2 * h, t, h);
}

__device__ __forceinline__ void kick_rt(double2 &v, double th, int small)
{
    if (small) {
        double p, u;
        lift_small(th, p, u);
        rot_f<double>(v, p, u);
        return;
    }
    double p, u, s;
    lift_from_angle(-th, p, u, s);
    rot_f<double>(v, p, u);
    v.x *= s;
    v.y *= s;
}

// double-float kick: the double-float series for |th| <= 0.1, the FP64
// reduction otherwise
__device__ __forceinline__ void kick_rt(df2 &v, df th, int small)
{
    df p, u, s;
    if (small && fabsf(th.hi) <= 0.1f) {
        lift_small(th, p, u);
        rot_f<df>(v, p, u);
        return;
    }
    lift_from_angle(-th, p, u, s);
    rot_f<df>(v, p, u);
    v.x = sign_mul(v.x, s);
    v.y = sign_mul(v.y, s);
}
// two kicks at once when both angles take the short series (bitwise
// kick_rt on each; otherwise kick_rt on each)
__device__ __forceinline__ void kick_rt2(df2 &v0, df2 &v1, df th0, df th1, int small)
{
    if (small && fabsf(th0.hi) <= 0.1f && fabsf(th1.hi) <= 0.1f) {
        dfp p, u;
        lift_small2(th0, th1, p, u);
        rot2_dfp(v0, v1, p, u);
        return;
    }
    kick_rt(v0, th0, small);
    kick_rt(v1, th1, small);
}
__device__ __forceinline__ void ld2(const df2 *p, df2 &a, df2 &b)
{
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st2(df2 *p, const df2 &a, const df2 &b)
{
    p[0] = a;
    p[1] = b;
}

__device__ __forceinline__ float norm2(const float2 &v) { return fmadd(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ double norm2(const double2 &v) { return fmadd(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ df norm2(const df2 &v) { return v.x * v.x + v.y * v.y; }

template <class T>
__device__ __forceinline__ void kick_one(Cx<T> &v, T th, int imag, int small)
{
    if (imag) {
        const T f = dexp(-th);
        v.x *= f;
        v.y *= f;
    } else {
        kick_rt(v, th, small);
    }
}

template <class T>
__device__ __forceinline__ void kick_sep(Cx<T> &v, const Lift<T> &a, const Lift<T> &b,
                                         const Lift<T> &c, int imag)
{
    if (imag) {
        const T f = a.f * b.f * c.f;
        v.x *= f;
        v.y *= f;
    } else {
        rot_f<T>(v, a.p, a.u);
        rot_f<T>(v, b.p, b.u);
        rot_f<T>(v, c.p, c.u);
        const T s = a.s * b.s * c.s;
        v.x *= s;
        v.y *= s;
    }
}

// R consecutive complex values as R/2 128-bit shared-memory accesses
// (p must be 16-byte aligned)
// two consecutive complex64 values move as one 16-byte access; complex128
// values are 16 bytes each already
__device__ __forceinline__ void ld2(const float2 *p, float2 &a, float2 &b)
{
    const float4 w = *reinterpret_cast<const float4 *>(p);
    a = make_float2(w.x, w.y);
    b = make_float2(w.z, w.w);
}
__device__ __forceinline__ void st2(float2 *p, const float2 &a, const float2 &b)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &a, double2 &b)
{
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st2(double2 *p, const double2 &a, const double2 &b)
{
    p[0] = a;
    p[1] = b;
}
// streaming (evict-first) global access of one complex128 value
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(double2 *p, const double2 &v) { __stcs(p, v); }
template <int R, class C2> __device__ __forceinline__ void load_pairs(const C2 *p, C2 (&v)[R])
{
#pragma unroll
    for (int i = 0; i < R; i += 2) ld2(p + i, v[i], v[i + 1]);
}
template <int R, class C2> __device__ __forceinline__ void store_pairs(C2 *p, const C2 (&v)[R])
{
#pragma unroll
    for (int i = 0; i < R; i += 2) st2(p + i, v[i], v[i + 1]);
}
// compiler-only fence: keeps table loads from being hoisted en masse (the
// hoisted loads of a 32-point stage otherwise exceed the register file)
__device__ __forceinline__ void hoist_fence() { asm volatile("" ::: "memory"); }

template <int NQ, int NT = kFastNT> __device__ void block_sum(double (&acc)[NQ], double *out)
{
    __shared__ double red[NT / 32][NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][q] = v;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double v = (lane < NT / 32) ? red[lane][q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) out[q] = v;
        }
    }
}

}  // namespace

// ======================================================================= XY
// HOT: the steady real-time step with the product potential (full kick, no
// reductions, small angles) compiled without per-point flag tests.
// threads per XY CTA (register budget): the hot complex64 variant fits in 64
// registers and runs 1024 threads (32 warps hide more shared-memory and
// HBM latency); the other complex64 variants 512, complex128 256
// threads per XY CTA: complex64 512 (1024 for the hot steady variant, which
// fits 64 registers), complex128 256 (255 registers), double-float 512 (its
// arithmetic is chains of dependent FP32 operations: warps matter more than
// registers, and one task per thread fits 128)
template <class T, bool HOT = false> __host__ __device__ constexpr int xy_threads()
{
    return sizeof(T) == 4 ? (HOT ? 1024 : 512) : (std::is_same<T, df>::value ? 512 : 256);
}

template <class T, int NX, int RA, int RB, int LY, int YA, int YB, bool IN_MIXED, bool OUT_MIXED,
          bool HOT>
__global__ void __launch_bounds__(xy_threads<T, HOT>()) xy_fast_kernel(const XYArgs<T> a)
{
    static_assert(RA * RB == NX && YA * YB == LY, "radix split");
    using C2 = Cx<T>;
    constexpr int NT = xy_threads<T, HOT>();
    constexpr int PITCH = NX + 2;          // even: rows stay 16-byte aligned
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *sm = reinterpret_cast<C2 *>(smraw);
    __shared__ T gtab[LY];              // g(y), y = r + P jy
    __shared__ T htab[NX];              // H(x, z) tau at swapped position
    __shared__ Lift<T> ytab[LY];        // separable y factor
    // complex64 observables: per-CTA tables so that the per-point work is FP32
    // only (g(y) of the tile's rows and H(x, z) rounded to FP32 as before;
    // guide membership of each column decided once, in FP64)
    __shared__ float obs_g[sizeof(T) == 4 ? LY : 1];
    __shared__ float obs_h[sizeof(T) == 4 ? NX : 1];
    __shared__ unsigned char obs_in[sizeof(T) == 4 ? NX : 1];

    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int z = blockIdx.x >> g.lgP, r = blockIdx.x & (g.P - 1);
    const int zl = z & (g.nz - 1);          // replica-local z (z counts planes over the batch)
    const long long pbase = (long long)z * g.plane;
    const C2 *src = a.src + pbase;
    C2 *dst = a.dst + pbase;
    // x and y twiddles staged in shared memory (after the tile)
    // wx[rr RA + j] = exp(-2 pi i j rr/NX) (j < RA, rr < RB): the twiddles of
    // the last x stage in the order the 16 lanes of a row read them (one
    // table row per rr: consecutive lanes, consecutive entries, no conflicts)
    Lift<T> *wx = reinterpret_cast<Lift<T> *>(sm + LY * PITCH);
    Lift<T> *wy = wx + NX;                                            // exp(-2 pi i e/LY)
    for (int e = t; e < NX + LY; e += NT)
        wx[e] = e < NX ? a.tw[g.fast_x_off + (e % RA) * (e / RA)] : a.tw[g.fast_y_off + e - NX];
    // hot instantiations: the steady pass (merged kick), the first pass of a
    // run (natural in, half kick) and the last (natural out, half kick)
    const int flags = HOT ? ((IN_MIXED && OUT_MIXED) ? XY_KICK_FULL : XY_KICK_HALF) : a.flags;
    const Kick<T> &k = a.k;
    const bool kick = (flags & (XY_KICK_HALF | XY_KICK_FULL | XY_KICK_SPLIT)) != 0;
    const bool full = (flags & XY_KICK_FULL) != 0;
    const T tau = full ? k.tau_full : k.tau_half;
    // additive z-only term of the product form: one phase for the whole plane
    const T thz = k.vz ? k.vz[zl] * tau : T(0);

    auto swx = [](int x) { return RA * (x % RB) + x / RB; };     // natural x -> position
    auto unswx = [](int p) { return p / RA + RB * (p % RA); };   // position -> natural x
    auto swy = [](int jy) { return YA * (jy % YB) + jy / YB; };

    if constexpr (sizeof(T) == 4 && !HOT) {
        if (flags & XY_RED_OBS) {
            if (t < LY && a.vform_obs == VF_PRODUCT) obs_g[t] = (float)a.rd.g64[r + t * g.P];
            if (t < NX) {
                const double xq = g.box[0] + (double)t * g.dx;
                unsigned m = 0;
                if (a.rd.xc) {
                    m |= fabs(xq - a.rd.xc[zl]) < a.rd.hw ? 1u : 0u;
                    m |= fabs(xq - a.rd.xc[g.nz + zl]) < a.rd.hw ? 2u : 0u;
                    m |= fabs(xq - a.rd.xc[2 * g.nz + zl]) < a.rd.hw ? 4u : 0u;
                }
                obs_in[t] = (unsigned char)m;
                obs_h[t] = (a.vform_obs == VF_PRODUCT) ? (float)a.rd.H64[(long long)z * g.nx + t] : 0.0f;
            }
        }
    }
    if (t < LY) {
        const int y = r + t * g.P;
        if (HOT || k.form == VF_PRODUCT) gtab[t] = k.g[y];
        // (the observables pass has no kick and no separable tables)
        else if (k.form == VF_SEPARABLE && kick) ytab[t] = (full ? k.sep_full : k.sep_half)[g.nx + y];
    }
    if (t < NX && (HOT || k.form == VF_PRODUCT))
        htab[t] = k.H[(long long)z * g.nx + unswx(t)] * tau;

    if constexpr (IN_MIXED) {
        // P1: inverse x, last stage (Ns = RA, radix RB) from HBM.  All loads of
        // the thread's tasks are issued before the first is used, and before
        // the barrier that publishes the staged tables (their latencies overlap).
        {
            constexpr int NTASK = LY * RA;
            constexpr int Q = (NTASK + NT - 1) / NT;
            C2 v[Q][RB];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int q = t + i * NT;
                if (NTASK % NT == 0 || q < NTASK) {
                    const int j = q % RA, row = q / RA;
                    const C2 *rowp = src + ((long long)(row * g.P + r) << g.lgnx);
                    sfor<RB>([&](auto kc) {
                        constexpr int kk = decltype(kc)::value;
                        v[i][brev(kk, RB)] = rowp[j + RA * kk];
                    });
                }
            }
            __syncthreads();   // staged tables are read from here on
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int q = t + i * NT;
                if (NTASK % NT == 0 || q < NTASK) {
                    const int j = q % RA, row = q / RA;
                    dft_inv<RB, 0, 1, T>(v[i]);
#pragma unroll
                    for (int rr = 1; rr + 1 < RB; rr += 2)
                        lift_pair_b<T>(v[i][rr], v[i][rr + 1], wx[rr * RA + j], wx[(rr + 1) * RA + j]);
                    lift_b<T>(v[i][RB - 1], wx[(RB - 1) * RA + j]);
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) sm[row * PITCH + j + RA * rr] = v[i][rr];
                }
            }
        }
        __syncthreads();
        // P2: inverse x, first stage (radix RA), in place on block j
        for (int q = t; q < LY * RB; q += NT) {
            const int row = q % LY, j = q / LY;
            C2 *bp = sm + row * PITCH + RA * j;
            C2 v[RA], w[RA];
            load_pairs<RA>(bp, w);
#pragma unroll
            for (int kk = 0; kk < RA; ++kk) v[brev(kk, RA)] = w[kk];
            dft_inv<RA, 0, 1, T>(v);
            store_pairs<RA>(bp, v);
        }
        __syncthreads();
        // P3a: inverse y, last stage (Ns = YA, radix YB), in place; two columns
        for (int q = t; q < (NX / 2) * YA; q += NT) {
            const int p = (q % (NX / 2)) * 2, i = q / (NX / 2);
            C2 v[YB], w[YB];
            sfor<YB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                ld2(sm + (i + YA * kk) * PITCH + p, v[brev(kk, YB)], w[brev(kk, YB)]);
            });
            dft_inv<YB, 0, 1, T>(v);
            dft_inv<YB, 0, 1, T>(w);
#pragma unroll
            for (int rr = 1; rr < YB; ++rr) {
                const Lift<T> tw = wy[i * rr];
                lift_pair_b<T>(v[rr], w[rr], tw, tw);
            }
#pragma unroll
            for (int rr = 0; rr < YB; ++rr) st2(sm + (i + YA * rr) * PITCH + p, v[rr], w[rr]);
        }
    } else {
        __syncthreads();   // staged tables are read from here on
        // natural rows into the swapped tile: a task moves the RB consecutive
        // points x = RB a + c of one row (16-byte loads); they land at swapped
        // positions RA c + a, consecutive across the lanes (conflict-free)
        for (int q = t; q < LY * RA; q += NT) {
            const int a = q % RA, jy = q / RA;
            const C2 *rowp = src + ((long long)(jy * g.P + r) << g.lgnx) + RB * a;
            C2 *smr = sm + swy(jy) * PITCH + a;
            C2 v[RB];
#pragma unroll
            for (int c = 0; c < RB; c += 2) ld2(rowp + c, v[c], v[c + 1]);
#pragma unroll
            for (int c = 0; c < RB; ++c) smr[RA * c] = v[c];
        }
    }
    __syncthreads();

    // P3b: y first stage: inverse -> potential factor -> forward, in registers;
    // two adjacent column positions per task
    {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        double gacc[2] = {0.0, 0.0};
        // adjoint gradient partial of one task: sum_y Im(conj(v) psi) g(y), times D_j(z,x)
        auto grad_task = [&](const C2 (&vv)[YA], int i, int x) {
            const C2 *ps = static_cast<const C2 *>(a.gd.psi) + pbase + x;
            double t1 = 0.0;
            if constexpr (std::is_same<T, float>::value) {
                float tf = 0.0f;                // the column's partial in FP32 (complex64 data)
#pragma unroll
                for (int rr = 0; rr < YA; ++rr) {
                    const int y = r + (i + YB * rr) * g.P;
                    const C2 q = ps[(long long)y << g.lgnx];
                    tf = fmadd(fmadd(vv[rr].x, q.y, -vv[rr].y * q.x), (float)a.gd.g64[y], tf);
                }
                t1 = tf;
            } else {
#pragma unroll
                for (int rr = 0; rr < YA; ++rr) {
                    const int y = r + (i + YB * rr) * g.P;
                    const C2 q = ps[(long long)y << g.lgnx];
                    t1 += ((double)vv[rr].x * (double)q.y - (double)vv[rr].y * (double)q.x) * a.gd.g64[y];
                }
            }
            gacc[0] += t1 * a.gd.D1[(long long)z * g.nx + x];
            gacc[1] += t1 * a.gd.D3[(long long)z * g.nx + x];
        };
        for (int q = t; q < (NX / 2) * YB; q += NT) {
            const int p0 = (q % (NX / 2)) * 2, i = q / (NX / 2);
            C2 v[2][YA];
            if constexpr (IN_MIXED) {
                sfor<YA>([&](auto kc) {
                    constexpr int kk = decltype(kc)::value;
                    ld2(sm + (YA * i + kk) * PITCH + p0, v[0][brev(kk, YA)], v[1][brev(kk, YA)]);
                });
                dft_inv<YA, 0, 1, T>(v[0]);
                dft_inv<YA, 0, 1, T>(v[1]);
            } else {
#pragma unroll
                for (int rr = 0; rr < YA; ++rr) ld2(sm + (YA * i + rr) * PITCH + p0, v[0][rr], v[1][rr]);
            }
            // v[c][rr] is the real-space point jy = i + YB rr, y = r + P jy, x = unswx(p0 + c)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int p = p0 + c, x = unswx(p);
                if (!HOT && (flags & XY_RED_OBS)) {
                    const double vz64 = a.rd.vz64 ? a.rd.vz64[zl] : 0.0;
                    const double vxz = (a.vform_obs == VF_SEPARABLE)
                                           ? a.rd.Vsep[x] + a.rd.Vsep[g.nx + g.ny + zl] : 0.0;
                    if constexpr (std::is_same<T, float>::value) {
                        // complex64: products and the column's YA-term partial sums in
                        // FP32 (the data carry 24 bits), FP64 from there on; FP64
                        // arithmetic per point would bind this pass to B300's FP64 rate
                        const float hz32 = obs_h[x], vz32 = (float)vz64;
                        const unsigned m = obs_in[x];
                        float sd = 0.0f, svd = 0.0f;
#pragma unroll
                        for (int rr = 0; rr < YA; ++rr) {
                            const int jy = i + YB * rr, y = r + jy * g.P;
                            const C2 u = v[c][rr];
                            const float d = fmadd(u.x, u.x, u.y * u.y);
                            float V = 0.0f;
                            if (a.vform_obs == VF_DENSE) V = k.Vd[pbase + ((long long)y << g.lgnx) + x];
                            else if (a.vform_obs == VF_PRODUCT) V = fmadd(obs_g[jy], hz32, vz32);
                            else if (a.vform_obs == VF_SEPARABLE) V = (float)(vxz + a.rd.Vsep[g.nx + y]);
                            sd += d;
                            svd = fmadd(V, d, svd);
                        }
                        acc[0] += sd;
                        acc[1] += svd;
                        if (m) {
                            const double sdd = (double)sd;
                            acc[2] += (m & 1u) ? sdd : 0.0;
                            acc[3] += (m & 2u) ? sdd : 0.0;
                            acc[4] += (m & 4u) ? sdd : 0.0;
                        }
                    } else {
                        const double xq = g.box[0] + (double)x * g.dx;
                        bool in0 = false, in1 = false, in2 = false;
                        if (a.rd.xc) {
                            in0 = fabs(xq - a.rd.xc[zl]) < a.rd.hw;
                            in1 = fabs(xq - a.rd.xc[g.nz + zl]) < a.rd.hw;
                            in2 = fabs(xq - a.rd.xc[2 * g.nz + zl]) < a.rd.hw;
                        }
                        const double hz =
                            (a.vform_obs == VF_PRODUCT) ? a.rd.H64[(long long)z * g.nx + x] : 0.0;
#pragma unroll
                        for (int rr = 0; rr < YA; ++rr) {
                            const int y = r + (i + YB * rr) * g.P;
                            const C2 u = v[c][rr];
                            const double d = (double)u.x * (double)u.x + (double)u.y * (double)u.y;
                            double V = 0.0;
                            if (a.vform_obs == VF_DENSE) V = (double)k.Vd[pbase + ((long long)y << g.lgnx) + x];
                            else if (a.vform_obs == VF_PRODUCT) V = a.rd.g64[y] * hz + vz64;
                            else if (a.vform_obs == VF_SEPARABLE) V = vxz + a.rd.Vsep[g.nx + y];
                            acc[0] += d;
                            acc[1] += V * d;
                            acc[2] += in0 ? d : 0.0;
                            acc[3] += in1 ? d : 0.0;
                            acc[4] += in2 ? d : 0.0;
                        }
                    }
                }
                if (!HOT && (flags & XY_GRAD_PRE)) grad_task(v[c], i, x);
                if (HOT) {
                    const T hx = htab[p];
                    const int tier = a.small_angle;     // 1 or 2 (uniform across the grid)
                    if constexpr (std::is_same<T, df>::value && YA % 2 == 0) {
                        // double-float: two rows per kick (pairs of FP32 pairs)
#pragma unroll
                        for (int rr = 0; rr < YA; rr += 2)
                            kick_rt2(v[c][rr], v[c][rr + 1], fmadd(gtab[i + YB * rr], hx, thz),
                                     fmadd(gtab[i + YB * (rr + 1)], hx, thz), tier);
                    } else {
#pragma unroll
                        for (int rr = 0; rr < YA; ++rr) kick_rt(v[c][rr], fmadd(gtab[i + YB * rr], hx, thz), tier);
                    }
                    // (the hot variant is only chosen when the short series applies)
                } else if (kick) {
                    // norm partial of the column in the element type (FP32 for complex64)
                    T nrm = T(0);
                    if (k.form == VF_SEPARABLE) {
                        const Lift<T> *tb = full ? k.sep_full : k.sep_half;
                        const Lift<T> lx = tb[x], lz = tb[g.nx + g.ny + zl];
                        const Lift<T> hx = k.sep_half[x], hz = k.sep_half[g.nx + g.ny + zl];
#pragma unroll
                        for (int rr = 0; rr < YA; ++rr) {
                            const int jy = i + YB * rr;
                            kick_sep<T>(v[c][rr], lx, ytab[jy], lz, k.imag);
                            if (flags & XY_RED_NORM) nrm += norm2(v[c][rr]);
                            if (flags & XY_STATE_OUT)
                                a.state_out[pbase + ((long long)(r + jy * g.P) << g.lgnx) + x] = v[c][rr];
                        }
                        if (flags & XY_GRAD) grad_task(v[c], i, x);
                        if (flags & XY_KICK_SPLIT) {
#pragma unroll
                            for (int rr = 0; rr < YA; ++rr)
                                kick_sep<T>(v[c][rr], hx, k.sep_half[g.nx + r + (i + YB * rr) * g.P], hz,
                                            k.imag);
                        }
                    } else {
                        const int small = a.small_angle;
                        const T hx = (k.form == VF_PRODUCT) ? htab[p] : T(0);
                        auto angle = [&](int rr) -> T {
                            const int jy = i + YB * rr;
                            return (k.form == VF_PRODUCT)
                                       ? fmadd(gtab[jy], hx, thz)
                                       : k.Vd[pbase + ((long long)(r + jy * g.P) << g.lgnx) + x] * tau;
                        };
                        // double-float real time: two rows per kick (pairs of FP32 pairs)
                        auto kick_rows = [&]() {
                            if constexpr (std::is_same<T, df>::value && YA % 2 == 0) {
                                if (!k.imag) {
#pragma unroll
                                    for (int rr = 0; rr < YA; rr += 2)
                                        kick_rt2(v[c][rr], v[c][rr + 1], angle(rr), angle(rr + 1), small);
                                    return;
                                }
                            }
#pragma unroll
                            for (int rr = 0; rr < YA; ++rr) kick_one<T>(v[c][rr], angle(rr), k.imag, small);
                        };
                        kick_rows();
#pragma unroll
                        for (int rr = 0; rr < YA; ++rr) {
                            const int jy = i + YB * rr;
                            if (flags & XY_RED_NORM) nrm += norm2(v[c][rr]);
                            if (flags & XY_STATE_OUT)
                                a.state_out[pbase + ((long long)(r + jy * g.P) << g.lgnx) + x] = v[c][rr];
                        }
                        if (flags & XY_GRAD) grad_task(v[c], i, x);
                        if (flags & XY_KICK_SPLIT) kick_rows();
                    }
                    if (flags & XY_RED_NORM) acc[0] += (double)nrm;
                }
            }
            if constexpr (OUT_MIXED) {
                dft_fwd<YA, 0, 1, T>(v[0]);
                dft_fwd<YA, 0, 1, T>(v[1]);
                sfor<YA>([&](auto kc) {
                    constexpr int kk = decltype(kc)::value;
                    st2(sm + (YA * i + kk) * PITCH + p0, v[0][brev(kk, YA)], v[1][brev(kk, YA)]);
                });
            } else {
#pragma unroll
                for (int rr = 0; rr < YA; ++rr) st2(sm + (YA * i + rr) * PITCH + p0, v[0][rr], v[1][rr]);
            }
        }
        if (!HOT) {
            if (flags & XY_RED_OBS) block_sum<5, NT>(acc, a.partials + (long long)blockIdx.x * 5);
            else if (flags & XY_RED_NORM) {
                double n1[1] = {acc[0]};
                block_sum<1, NT>(n1, a.partials + blockIdx.x);
            }
            if (flags & (XY_GRAD | XY_GRAD_PRE)) {
                __shared__ double gtot[2];
                block_sum<2, NT>(gacc, gtot);
                __syncthreads();
                if (t == 0) {
                    a.gd.acc[2 * blockIdx.x] += a.gd.coef * gtot[0];
                    a.gd.acc[2 * blockIdx.x + 1] += a.gd.coef * gtot[1];
                }
            }
        }
    }
    __syncthreads();

    if constexpr (OUT_MIXED) {
        // P3c: forward y, last stage (Ns = YA, radix YB), in place; two columns
        for (int q = t; q < (NX / 2) * YA; q += NT) {
            const int p = (q % (NX / 2)) * 2, i = q / (NX / 2);
            C2 v[YB], w[YB];
#pragma unroll
            for (int rr = 0; rr < YB; ++rr) ld2(sm + (i + YA * rr) * PITCH + p, v[rr], w[rr]);
#pragma unroll
            for (int rr = 1; rr < YB; ++rr) {
                const Lift<T> tw = wy[i * rr];
                lift_pair_f<T>(v[rr], w[rr], tw, tw);
            }
            dft_fwd<YB, 0, 1, T>(v);
            dft_fwd<YB, 0, 1, T>(w);
            sfor<YB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                st2(sm + (i + YA * kk) * PITCH + p, v[brev(kk, YB)], w[brev(kk, YB)]);
            });
        }
        __syncthreads();
        // P4: forward x, first stage (radix RA), in place on block j
        for (int q = t; q < LY * RB; q += NT) {
            const int row = q % LY, j = q / LY;
            C2 *bp = sm + row * PITCH + RA * j;
            C2 v[RA], w[RA];
            load_pairs<RA>(bp, v);
            dft_fwd<RA, 0, 1, T>(v);
#pragma unroll
            for (int kk = 0; kk < RA; ++kk) w[kk] = v[brev(kk, RA)];
            store_pairs<RA>(bp, w);
        }
        __syncthreads();
        // P5: forward x, last stage (Ns = RA, radix RB), straight to HBM
        for (int q = t; q < LY * RA; q += NT) {
            const int j = q % RA, row = q / RA;
            C2 v[RB];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) v[rr] = sm[row * PITCH + j + RA * rr];
#pragma unroll
            for (int rr = 1; rr + 1 < RB; rr += 2)
                lift_pair_f<T>(v[rr], v[rr + 1], wx[rr * RA + j], wx[(rr + 1) * RA + j]);
            lift_f<T>(v[RB - 1], wx[(RB - 1) * RA + j]);
            dft_fwd<RB, 0, 1, T>(v);
            C2 *rowp = dst + ((long long)(row * g.P + r) << g.lgnx);
            sfor<RB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                rowp[j + RA * kk] = v[brev(kk, RB)];
            });
        }
    } else {
        // natural rows out of the swapped tile (mirror of the natural load)
        for (int q = t; q < LY * RA; q += NT) {
            const int a = q % RA, jy = q / RA;
            C2 *rowp = dst + ((long long)(jy * g.P + r) << g.lgnx) + RB * a;
            const C2 *smr = sm + swy(jy) * PITCH + a;
            C2 v[RB];
#pragma unroll
            for (int c = 0; c < RB; ++c) v[c] = smr[RA * c];
#pragma unroll
            for (int c = 0; c < RB; c += 2) st2(rowp + c, v[c], v[c + 1]);
        }
    }
}

// ======================================================================== Z
// threads per Z CTA: 1024-point lines hold 32 points per stage task and need
// the 255-register budget of 256 threads; shorter lines fit 512 threads
// (complex128 always uses 256)
template <class T> __host__ __device__ constexpr int z_threads(int nz)
{
    return (sizeof(T) == 8 || nz >= 1024) ? 256 : 512;
}

template <class T, int NZ, int ZA, int ZB, int P, int W>
__global__ void __launch_bounds__(z_threads<T>(NZ), (sizeof(T) == 4 && P * W == 8) ? 2 : 1)
    z_fast_kernel(const ZArgs<T> a)
{
    static_assert(ZA * ZB == NZ, "NZ = ZA ZB");
    using C2 = Cx<T>;
    constexpr int NT = z_threads<T>(NZ);
    constexpr int C = P * W;
    constexpr int V2 = (sizeof(T) == 4 && W >= 2) ? 2 : 1;   // columns per load task
    static_assert(C >= 8, "tile needs at least 8 columns");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *sm = reinterpret_cast<C2 *>(smraw);
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int tl = blockIdx.x & ((1 << g.lgzt) - 1);          // tile within the replica
    const long long roff = (long long)(blockIdx.x >> g.lgzt) * g.rstride;
    const int kp = tl >> g.nblk_lg, b = tl & ((1 << g.nblk_lg) - 1);
    // C >= 16: rows of 16 complex span all 32 banks; rotate W-column blocks by
    //          z so the W-lane groups of Z1/Z5 land on distinct banks.
    // C == 8:  two rows share the 32 banks; rotate column pairs by z/2 (Z1/Z5)
    //          and shift every other block of 32 rows by half the banks (rows
    //          z and z + 32 meet in Z3): 8 padding slots after every 32 rows.
    // complex128: a row of 8 values spans all 32 banks; rotate W-column blocks
    //          by z so the lanes of Z1/Z5 (one column, 8 rows) spread out.
    auto at = [](int zz, int col) {
        if constexpr (sizeof(T) == 8) {
            constexpr int SWM = (W < 8) ? (8 / W - 1) : 0;
            return zz * C + (col ^ ((zz & SWM) * W));
        } else if constexpr (C >= 16) {
            constexpr int SWM = (W < 16) ? (16 / W - 1) : 0;
            return zz * C + (col ^ ((zz & SWM) * W));
        } else {
            return zz * C + (zz >> 5) * 8 + (col ^ (((zz >> 1) & 3) * 2));
        }
    };
    const Lift<T> *wc = a.tw + g.cross_off;    // exp(-2 pi i e/ny)
    const long long colbase = roff + ((long long)(kp * P) << g.lgnx) + (b * W);
    // z twiddles exp(-2 pi i e/NZ) and z kinetic factors, staged in shared
    // memory (L1 would lose them to the streaming tile loads)
    constexpr int TILE = NZ * C + ((sizeof(T) == 4 && C == 8) ? (NZ / 32) * 8 : 0);   // + row-block padding
    Lift<T> *wz = reinterpret_cast<Lift<T> *>(sm + TILE);
    Lift<T> *kz = wz + NZ;
    for (int e = t; e < NZ; e += NT) {
        wz[e] = a.tw[g.fast_z_off + e];
        if (!a.observe) kz[e] = a.kin[g.nx + g.ny + e];
        else if constexpr (std::is_same<T, float>::value)        // k_z^2/2 in FP32
            reinterpret_cast<float *>(kz)[e] = (float)a.k2h[g.nx + g.ny + e];
    }

    Lift<T> cw[P];
#pragma unroll
    for (int rr = 1; rr < P; ++rr) cw[rr] = wc[(rr * kp) & (g.ny - 1)];

    // Z1: load P rows per (z, column pair), forward cross DFT, write the tile.
    // Every load of the thread is issued before any is used (one DRAM latency
    // per tile instead of one per task).
    {
        constexpr int NTASK = NZ * (W / V2);
        constexpr int Q = (NTASK + NT - 1) / NT;
        C2 v[Q][V2][P];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            if (NTASK % NT == 0 || q < NTASK) {
                const int xo = (q % (W / V2)) * V2, zz = q / (W / V2);
                const C2 *p = a.src + (long long)zz * g.plane + colbase + xo;
#pragma unroll
                for (int rr = 0; rr < P; ++rr) {
                    if constexpr (V2 == 2) {
                        const float4 w4 = __ldcs(reinterpret_cast<const float4 *>(p + ((long long)rr << g.lgnx)));
                        v[i][0][rr] = make_float2(w4.x, w4.y);
                        v[i][1][rr] = make_float2(w4.z, w4.w);
                    } else {
                        v[i][0][rr] = ld_stream(p + ((long long)rr << g.lgnx));
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            if (NTASK % NT == 0 || q < NTASK) {
                const int xo = (q % (W / V2)) * V2, zz = q / (W / V2);
#pragma unroll
                for (int c = 0; c < V2; ++c) {
#pragma unroll
                    for (int rr = 1; rr < P; ++rr) lift_f<T>(v[i][c][rr], cw[rr]);
                    dft_fwd<P, 0, 1, T>(v[i][c]);
                }
                sfor<P>([&](auto kc) {
                    constexpr int k2 = decltype(kc)::value;
                    if constexpr (V2 == 2) {
                        const C2 e0 = v[i][0][brev(k2, P)], e1 = v[i][1][brev(k2, P)];
                        *reinterpret_cast<float4 *>(sm + at(zz, k2 * W + xo)) =
                            make_float4(e0.x, e0.y, e1.x, e1.y);
                    } else {
                        sm[at(zz, k2 * W + xo)] = v[i][0][brev(k2, P)];
                    }
                });
            }
        }
    }
    __syncthreads();

    // Z2: forward z, first stage (radix ZA) on rows j + ZB r, in place
    for (int q = t; q < C * ZB; q += NT) {
        const int col = q % C, j = q / C;
        C2 v[ZA];
#pragma unroll
        for (int rr = 0; rr < ZA; ++rr) v[rr] = sm[at(j + ZB * rr, col)];
        dft_fwd<ZA, 0, 1, T>(v);
        sfor<ZA>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            sm[at(j + ZB * kk, col)] = v[brev(kk, ZA)];
        });
    }
    __syncthreads();

    // Z3: last stage on the contiguous rows ZB jp + j, kinetic factor, inverse
    {
        const T sc = a.inv_n * (a.scale ? (T)(*a.scale) : T(1));
        double acc[1] = {0.0};
        for (int q = t; q < C * ZA; q += NT) {
            const int col = q % C, jp = q / C;
            const int kx = b * W + (col % W);
            const int ky = kp + ((col / W) << g.lgLy);
            C2 v[ZB];
#pragma unroll
            for (int j = 0; j < ZB; ++j) v[j] = sm[at(ZB * jp + j, col)];
            sfor<ZB - 1>([&](auto jc) {
                constexpr int j = decltype(jc)::value + 1;
                if constexpr (j % 4 == 0) hoist_fence();
                lift_f<T>(v[j], wz[jp * j]);
            });
            dft_fwd<ZB, 0, 1, T>(v);
            // register brev(k2) holds kz = jp + ZA k2
            if (a.observe) {
                const double kxy = a.k2h[kx] + a.k2h[g.nx + ky];
                if constexpr (std::is_same<T, float>::value) {
                    // complex64: the task's 32 terms in FP32, FP64 from there on
                    const float *k2z = reinterpret_cast<const float *>(kz);
                    const float kxyf = (float)kxy;
                    float sk = 0.0f;
                    sfor<ZB>([&](auto kc) {
                        constexpr int k2 = decltype(kc)::value;
                        sk = fmadd(kxyf + k2z[jp + ZA * k2], norm2(v[brev(k2, ZB)]), sk);
                    });
                    acc[0] += sk;
                } else {
                    sfor<ZB>([&](auto kc) {
                        constexpr int k2 = decltype(kc)::value;
                        const C2 u = v[brev(k2, ZB)];
                        acc[0] += (kxy + a.k2h[g.nx + g.ny + jp + ZA * k2]) *
                                  ((double)u.x * (double)u.x + (double)u.y * (double)u.y);
                    });
                }
                continue;
            }
            const Lift<T> ax = a.kin[kx], ay = a.kin[g.nx + ky];
            sfor<ZB>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                if constexpr (k2 % 4 == 0) hoist_fence();
                C2 &u = v[brev(k2, ZB)];
                const Lift<T> az = kz[jp + ZA * k2];
                if (a.imag) {
                    const T f = ax.f * ay.f * az.f * sc;
                    u.x *= f;
                    u.y *= f;
                } else {
                    rot_f<T>(u, ax.p, ax.u);
                    rot_f<T>(u, ay.p, ay.u);
                    rot_f<T>(u, az.p, az.u);
                    const T s = ax.s * ay.s * az.s * sc;
                    u.x *= s;
                    u.y *= s;
                }
            });
            dft_inv<ZB, 0, 1, T>(v);
            sfor<ZB - 1>([&](auto jc) {
                constexpr int j = decltype(jc)::value + 1;
                if constexpr (j % 4 == 0) hoist_fence();
                lift_b<T>(v[j], wz[jp * j]);
            });
#pragma unroll
            for (int j = 0; j < ZB; ++j) sm[at(ZB * jp + j, col)] = v[j];
        }
        if (a.observe) {
            block_sum<1, NT>(acc, a.partials + blockIdx.x);
            return;
        }
    }
    __syncthreads();

    // Z4: inverse z, first stage, in place
    for (int q = t; q < C * ZB; q += NT) {
        const int col = q % C, j = q / C;
        C2 v[ZA];
        sfor<ZA>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            v[brev(kk, ZA)] = sm[at(j + ZB * kk, col)];
        });
        dft_inv<ZA, 0, 1, T>(v);
#pragma unroll
        for (int rr = 0; rr < ZA; ++rr) sm[at(j + ZB * rr, col)] = v[rr];
    }
    __syncthreads();

    // Z5: inverse cross DFT and store
    for (int q = t; q < NZ * (W / V2); q += NT) {
        const int xo = (q % (W / V2)) * V2, zz = q / (W / V2);
        C2 v[V2][P];
        sfor<P>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            if constexpr (V2 == 2) {
                const float4 w4 = *reinterpret_cast<const float4 *>(sm + at(zz, k2 * W + xo));
                v[0][brev(k2, P)] = make_float2(w4.x, w4.y);
                v[1][brev(k2, P)] = make_float2(w4.z, w4.w);
            } else {
                v[0][brev(k2, P)] = sm[at(zz, k2 * W + xo)];
            }
        });
#pragma unroll
        for (int c = 0; c < V2; ++c) {
            dft_inv<P, 0, 1, T>(v[c]);
#pragma unroll
            for (int rr = 1; rr < P; ++rr) lift_b<T>(v[c][rr], cw[rr]);
        }
        C2 *p = a.dst + (long long)zz * g.plane + colbase + xo;
#pragma unroll
        for (int rr = 0; rr < P; ++rr) {
            if constexpr (V2 == 2)
                __stcs(reinterpret_cast<float4 *>(p + ((long long)rr << g.lgnx)),
                       make_float4(v[0][rr].x, v[0][rr].y, v[1][rr].x, v[1][rr].y));
            else
                st_stream(p + ((long long)rr << g.lgnx), v[0][rr]);
        }
    }
}

// ------------------------------------------------ asynchronous copies
namespace {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kRingCHZ = 128;            // z-rows per ring chunk
constexpr int kRingNT = 256;             // threads of a ring CTA

}  // namespace

// =================================================================== XY ring
// Persistent form of the steady complex64 XY pass (nx = 256, 64-row tiles,
// product potential, real time, in place): one 1024-thread CTA per SM walks
// over the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  A tile is two
// 32-row halves in a ring of three half buffers (3 x 32 x 258 x 8 B =
// 198 KB).  The next tile's first half arrives by 16-byte asynchronous copies
// (cp.async, no registers held), one 8-row round after each of the first
// four transform phases, so that the copy requests leave between arithmetic;
// its second half is issued as soon as the store phase has read the current
// tile back into registers.  The last inverse x stage then reads shared
// memory instead of HBM, and a tile's HBM load no longer stalls its SM.
// Same arithmetic, tables and HBM layout as the steady xy_fast_kernel.
template <int NX, int RA, int RB, int LY, int YA, int YB>
__global__ void __launch_bounds__(1024, 1) xy_ring_kernel(const XYArgs<float> a, int ntiles)
{
    static_assert(RA * RB == NX && YA * YB == LY && LY == 64 && YA == 8 && YB == 8, "64-row tiles");
    using T = float;
    using C2 = float2;
    constexpr int NT = 1024;
    constexpr int PITCH = NX + 2;
    constexpr int HR = LY / 2;                   // rows per half buffer
    constexpr int HB = HR * PITCH;               // complex values per half buffer
    constexpr int PPR = NX / 2;                  // 16-byte pieces per row
    constexpr int RPI = NT / PPR;                // rows per copy round
    constexpr int NCR = HR / RPI;                // copy rounds per half
    static_assert(LY * RA == NT && LY * RB == NT && (NX / 2) * YA == NT && (NX / 2) * YB == NT &&
                      NCR == 4 && HR % YA == 0,
                  "one task per thread in every phase, four copy rounds per half");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *bufs = reinterpret_cast<C2 *>(smraw);
    Lift<T> *wx = reinterpret_cast<Lift<T> *>(bufs + 3 * HB);   // as in xy_fast_kernel
    Lift<T> *wy = wx + NX;
    __shared__ T gtab[2][LY];                    // g(y) of the tile's rows, per tile
    __shared__ T htab[2][NX];                    // H(x, z) tau at swapped position, per tile
    __shared__ T thzs[2];                        // z-only phase, per tile

    const Geom &g = a.g;
    const Kick<T> &k = a.k;
    const int t = threadIdx.x;
    const int G = gridDim.x;
    const int nmine = (ntiles - (int)blockIdx.x + G - 1) / G;
    const T tau = k.tau_full;
    const int tier = a.small_angle;
    auto unswx = [](int p) { return p / RA + RB * (p % RA); };
    // half h of the i-th tile of this CTA: buffers rotate by two halves per tile
    auto half_buf = [&](int i, int h) { return bufs + ((2 * i + h) % 3) * HB; };
    const int cpiece = t % PPR, crow = t / PPR;
    // copy rounds [m0, m1) of half h of the i-th tile: thread t moves piece
    // t % PPR of rows crow + RPI m of the half
    auto issue = [&](int i, int h, int m0, int m1) {
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        const C2 *src = a.src + (long long)z * g.plane +
                        ((long long)((h * HR + crow + RPI * m0) * g.P + r) << g.lgnx) + 2 * cpiece;
        C2 *dst = half_buf(i, h) + (crow + RPI * m0) * PITCH + 2 * cpiece;
        const long long rstep = (long long)(RPI * g.P) << g.lgnx;
        for (int m = m0; m < m1; ++m) {
            cp_async16(dst, src);
            src += rstep;
            dst += RPI * PITCH;
        }
    };
    auto load_tabs = [&](int i) {
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        if (t < LY) gtab[i & 1][t] = k.g[r + t * g.P];
        if (t < NX) htab[i & 1][t] = k.H[(long long)z * g.nx + unswx(t)] * tau;
        if (t == 0) thzs[i & 1] = k.vz ? k.vz[z & (g.nz - 1)] * tau : T(0);
    };

    if (nmine > 0) {
        issue(0, 0, 0, NCR);
        issue(0, 1, 0, NCR);
        load_tabs(0);
    }
    cp_async_commit();
    for (int e = t; e < NX + LY; e += NT)
        wx[e] = e < NX ? a.tw[g.fast_x_off + (e % RA) * (e / RA)] : a.tw[g.fast_y_off + e - NX];

    for (int i = 0; i < nmine; ++i) {
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        const bool more = i + 1 < nmine;
        if (more) load_tabs(i + 1);
        cp_async_wait<0>();
        __syncthreads();                         // tile i (and its tables) visible
        C2 *const b0 = half_buf(i, 0);
        C2 *const b1 = half_buf(i, 1);
        const T *gt = gtab[i & 1];
        const T *ht = htab[i & 1];
        const T thz = thzs[i & 1];

        // P1: inverse x, last stage (radix RB) in place
        {
            const int j = t % RA, rw = t / RA;
            C2 *rp = (rw < HR ? b0 : b1) + (rw % HR) * PITCH;
            C2 v[RB];
            sfor<RB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v[brev(kk, RB)] = rp[j + RA * kk];
            });
            dft_inv<RB, 0, 1, T>(v);
#pragma unroll
            for (int rr = 1; rr < RB; ++rr) lift_b<T>(v[rr], wx[rr * RA + j]);
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) rp[j + RA * rr] = v[rr];
        }
        if (more) issue(i + 1, 0, 0, 1);
        __syncthreads();
        // P2: inverse x, first stage (radix RA), in place on block j
        {
            const int rw = t % LY, j = t / LY;
            C2 *bp = (rw < HR ? b0 : b1) + (rw % HR) * PITCH + RA * j;
            C2 v[RA], w[RA];
            load_pairs<RA>(bp, w);
#pragma unroll
            for (int kk = 0; kk < RA; ++kk) v[brev(kk, RA)] = w[kk];
            dft_inv<RA, 0, 1, T>(v);
            store_pairs<RA>(bp, v);
        }
        if (more) issue(i + 1, 0, 1, 2);
        __syncthreads();
        // P3a: inverse y, last stage (radix YB) on rows ii + YA kk, two
        // columns; row ii + YA kk lies in the first half for kk < HR / YA
        {
            const int p = (t % (NX / 2)) * 2, ii = t / (NX / 2);
            C2 *r0 = b0 + ii * PITCH + p, *r1 = b1 + ii * PITCH + p;
            C2 v[YB], w[YB];
            sfor<YB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                ld2((kk < HR / YA ? r0 : r1) + YA * (kk % (HR / YA)) * PITCH, v[brev(kk, YB)],
                    w[brev(kk, YB)]);
            });
            dft_inv<YB, 0, 1, T>(v);
            dft_inv<YB, 0, 1, T>(w);
#pragma unroll
            for (int rr = 1; rr < YB; ++rr) {
                const Lift<T> tw = wy[ii * rr];
                lift_b<T>(v[rr], tw);
                lift_b<T>(w[rr], tw);
            }
#pragma unroll
            for (int rr = 0; rr < YB; ++rr)
                st2((rr < HR / YA ? r0 : r1) + YA * (rr % (HR / YA)) * PITCH, v[rr], w[rr]);
        }
        if (more) issue(i + 1, 0, 2, 3);
        __syncthreads();
        // P3b: inverse y first stage -> potential factor -> forward y first
        // stage in registers; rows YA ii + kk lie in one half buffer
        {
            const int p0 = (t % (NX / 2)) * 2, ii = t / (NX / 2);
            C2 *rb = (ii < HR / YA ? b0 : b1) + ((YA * ii) % HR) * PITCH + p0;
            C2 v[2][YA];
            sfor<YA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                ld2(rb + kk * PITCH, v[0][brev(kk, YA)], v[1][brev(kk, YA)]);
            });
            dft_inv<YA, 0, 1, T>(v[0]);
            dft_inv<YA, 0, 1, T>(v[1]);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const T hx = ht[p0 + c];
#pragma unroll
                for (int rr = 0; rr < YA; ++rr) kick_rt(v[c][rr], fmadd(gt[ii + YB * rr], hx, thz), tier);
            }
            dft_fwd<YA, 0, 1, T>(v[0]);
            dft_fwd<YA, 0, 1, T>(v[1]);
            sfor<YA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                st2(rb + kk * PITCH, v[0][brev(kk, YA)], v[1][brev(kk, YA)]);
            });
        }
        if (more) issue(i + 1, 0, 3, 4);
        cp_async_commit();
        __syncthreads();
        // P3c: forward y, last stage (radix YB), in place
        {
            const int p = (t % (NX / 2)) * 2, ii = t / (NX / 2);
            C2 *r0 = b0 + ii * PITCH + p, *r1 = b1 + ii * PITCH + p;
            C2 v[YB], w[YB];
#pragma unroll
            for (int rr = 0; rr < YB; ++rr)
                ld2((rr < HR / YA ? r0 : r1) + YA * (rr % (HR / YA)) * PITCH, v[rr], w[rr]);
#pragma unroll
            for (int rr = 1; rr < YB; ++rr) {
                const Lift<T> tw = wy[ii * rr];
                lift_f<T>(v[rr], tw);
                lift_f<T>(w[rr], tw);
            }
            dft_fwd<YB, 0, 1, T>(v);
            dft_fwd<YB, 0, 1, T>(w);
            sfor<YB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                st2((kk < HR / YA ? r0 : r1) + YA * (kk % (HR / YA)) * PITCH, v[brev(kk, YB)],
                    w[brev(kk, YB)]);
            });
        }
        __syncthreads();
        // P4: forward x, first stage (radix RA), in place on block j
        {
            const int rw = t % LY, j = t / LY;
            C2 *bp = (rw < HR ? b0 : b1) + (rw % HR) * PITCH + RA * j;
            C2 v[RA], w[RA];
            load_pairs<RA>(bp, v);
            dft_fwd<RA, 0, 1, T>(v);
#pragma unroll
            for (int kk = 0; kk < RA; ++kk) w[kk] = v[brev(kk, RA)];
            store_pairs<RA>(bp, w);
        }
        __syncthreads();
        // P5: forward x, last stage, to HBM.  The task is read back first so
        // that the tile's first half buffer can take the next tile's second half
        {
            const int j = t % RA, rw = t / RA;
            const C2 *rp = (rw < HR ? b0 : b1) + (rw % HR) * PITCH;
            C2 v[RB];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) v[rr] = rp[j + RA * rr];
            __syncthreads();                     // tile i's buffers are free
            if (more) issue(i + 1, 1, 0, NCR);
            cp_async_commit();
#pragma unroll
            for (int rr = 1; rr < RB; ++rr) lift_f<T>(v[rr], wx[rr * RA + j]);
            dft_fwd<RB, 0, 1, T>(v);
            C2 *op = a.dst + (long long)z * g.plane + ((long long)(rw * g.P + r) << g.lgnx);
            sfor<RB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                op[j + RA * kk] = v[brev(kk, RB)];
            });
        }
    }
    cp_async_wait<0>();
}

// =================================================================== Z ring
// Persistent form of the complex64 Z pass for 1024-point lines and 16-column
// tiles (P = 4 row classes, W = 4 columns): one CTA per SM walks over tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  The tile lives in a ring of
// twelve 128-row chunks of shared memory (a tile is eight chunks).  While a
// tile is transformed, 16-byte asynchronous copies (cp.async, no registers
// held) bring in the first half of the next tile, one chunk after each of
// the four transform phases so that the copy requests trickle out between
// arithmetic instead of stalling every warp at once; the second half follows
// as soon as the store phase has read the current tile back.  The
// HBM load latency of a tile is thereby hidden behind the previous tile's
// shared-memory phases instead of stalling the SM.
//
// Phases per tile: Z1 cross twiddle + P-point DFT in place, Z2-Z4 as in
// z_fast_kernel, Z5 inverse cross DFT and streaming stores.  Same arithmetic
// and HBM layout as z_fast_kernel.

template <int NZ, int ZA, int ZB, int P, int W, int NT>
__global__ void __launch_bounds__(NT, 1) z_ring_kernel(const ZArgs<float> a, int ntiles)
{
    static_assert(ZA * ZB == NZ && ZA == 32 && ZB == 32, "1024-point lines as 32 x 32");
    static_assert(P * W == 16 && W == 4, "16-column tiles of 32-byte row segments");
    static_assert((NT == 256 || NT == 512) && kRingCHZ % (NT / 8) == 0 && NZ * (W / 2) % NT == 0,
                  "copy and read-back rounds divide evenly");
    using T = float;
    using C2 = float2;
    constexpr int C = P * W;
    constexpr int CHZ = kRingCHZ;
    constexpr int NCH = NZ / CHZ;                  // chunks per tile (8)
    constexpr int NRING = NCH + NCH / 2;           // ring slots (12)
    constexpr int CHE = CHZ * C;                   // complex values per chunk
    constexpr int SWM = 16 / W - 1;
    // shared-memory swizzle of a 16-column z-row: the 32-byte group of each
    // row class moves with z mod 4 and its 16-byte halves swap with bit 2 of
    // z, so that every access pattern below (16-byte copies and reads of
    // eight z-rows, 8-byte column sweeps) meets each bank once per wavefront
    auto swz = [](int z) { return ((z & SWM) * W) | (((z >> 2) & 1) * 2); };
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *ring = reinterpret_cast<C2 *>(smraw);
    Lift<T> *wz = reinterpret_cast<Lift<T> *>(ring + NRING * CHE);
    Lift<T> *kz = wz + NZ;
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int G = gridDim.x;
    const int nmine = (ntiles - (int)blockIdx.x + G - 1) / G;
    const int nblk_mask = (1 << g.nblk_lg) - 1;
    const Lift<T> *wc = a.tw + g.cross_off;

    // ring slot of chunk c of the i-th tile of this CTA
    auto slot_of = [](int i, int c) {
        int s = (i % 3) * 8 + c;           // 8 i mod 12 = 0, 8, 4 for i mod 3 = 0, 1, 2
        s -= (s >= NRING) ? NRING : 0;
        s -= (s >= NRING) ? NRING : 0;
        return s;
    };
    // asynchronous copy of chunks [c0, c1) of the i-th tile into the ring.
    // Thread t always moves the same 16-byte piece (half h of row class r)
    // of z-rows t/8 + 32 m, so its addresses advance by fixed strides.
    const int ch = t & 1, cr = (t >> 1) & (P - 1), czl = t >> 3;
    const int cdst = czl * C + ((cr * W + 2 * ch) ^ swz(czl));
    auto issue = [&](int i, int c0, int c1) {
        const int tile = blockIdx.x + i * G;
        const int tl = tile & ((1 << g.lgzt) - 1);
        const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
        const C2 *src = a.src + (long long)(tile >> g.lgzt) * g.rstride +
                        ((long long)(kp * P + cr) << g.lgnx) + b * W + 2 * ch +
                        (long long)(c0 * CHZ + czl) * g.plane;
        const long long zstep = (long long)(NT / 8) * g.plane;
        for (int c = c0; c < c1; ++c) {
            C2 *dst = ring + slot_of(i, c) * CHE + cdst;
#pragma unroll
            for (int m = 0; m < CHZ / (NT / 8); ++m) {
                cp_async16(dst + m * (NT / 8) * C, src);
                src += zstep;
            }
        }
    };
    // per-tile tables, double buffered: kinetic x factors of the W columns,
    // kinetic y factors of the P classes, cross twiddles
    __shared__ Lift<T> tabs[2][W + 2 * P];
    auto load_tabs = [&](int i) {
        if (t < W + 2 * P) {
            const int tile = blockIdx.x + i * G;
            const int tl = tile & ((1 << g.lgzt) - 1);
            const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
            Lift<T> v;
            if (t < W) v = a.kin[b * W + t];
            else if (t < W + P) v = a.kin[g.nx + kp + ((t - W) << g.lgLy)];
            else v = wc[((t - W - P) * kp) & (g.ny - 1)];
            tabs[i & 1][t] = v;
        }
    };

    if (nmine > 0) {
        issue(0, 0, NCH);
        load_tabs(0);
    }
    cp_async_commit();
    for (int e = t; e < NZ; e += NT) {
        wz[e] = a.tw[g.fast_z_off + e];
        kz[e] = a.kin[g.nx + g.ny + e];
    }
    const T sc = a.inv_n * (a.scale ? (T)(*a.scale) : T(1));

    for (int i = 0; i < nmine; ++i) {
        const int tile = blockIdx.x + i * G;
        const int tl = tile & ((1 << g.lgzt) - 1);
        const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
        const long long roff = (long long)(tile >> g.lgzt) * g.rstride;
        if (i + 1 < nmine) load_tabs(i + 1);
        cp_async_wait<0>();
        __syncthreads();                         // tile i (and its tables) visible
        const Lift<T> *tb = tabs[i & 1];

        int sb[NCH];                             // ring offset of each chunk of tile i
#pragma unroll
        for (int c = 0; c < NCH; ++c) sb[c] = slot_of(i, c) * CHE;
        auto at = [&](int zz, int col) {
            int s = slot_of(i, zz / CHZ);
            return s * CHE + (zz % CHZ) * C + (col ^ swz(zz));
        };
        const long long colbase = roff + ((long long)(kp * P) << g.lgnx) + (b * W);

        // Z1: cross twiddle + forward P-point DFT, in place (two columns per task)
        for (int q = t; q < NZ * (W / 2); q += NT) {
            const int xo = (q % (W / 2)) * 2, zz = q / (W / 2);
            C2 v[2][P];
#pragma unroll
            for (int rr = 0; rr < P; ++rr) {
                const float4 w4 = *reinterpret_cast<const float4 *>(ring + at(zz, rr * W + xo));
                v[0][rr] = make_float2(w4.x, w4.y);
                v[1][rr] = make_float2(w4.z, w4.w);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
#pragma unroll
                for (int rr = 1; rr < P; ++rr) lift_f<T>(v[c][rr], tb[W + P + rr]);
                dft_fwd<P, 0, 1, T>(v[c]);
            }
            sfor<P>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                const C2 e0 = v[0][brev(k2, P)], e1 = v[1][brev(k2, P)];
                *reinterpret_cast<float4 *>(ring + at(zz, k2 * W + xo)) = make_float4(e0.x, e0.y, e1.x, e1.y);
            });
        }
        if (i + 1 < nmine) issue(i + 1, 0, 1);   // next tile, first half, chunk 0
        __syncthreads();

        // Z2: forward z, first stage (radix ZA) on rows j + ZB rr, in place.
        // Row j + ZB rr lies in chunk rr / 4 (ZB = 32, 128-row chunks).
        for (int q = t; q < C * ZB; q += NT) {
            const int col = q % C, j = q / C;
            const int off = j * C + (col ^ swz(j));
            C2 v[ZA];
#pragma unroll
            for (int rr = 0; rr < ZA; ++rr) v[rr] = ring[sb[rr / 4] + (rr % 4) * ZB * C + off];
            dft_fwd<ZA, 0, 1, T>(v);
            sfor<ZA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                ring[sb[kk / 4] + (kk % 4) * ZB * C + off] = v[brev(kk, ZA)];
            });
        }
        if (i + 1 < nmine) issue(i + 1, 1, 2);   // next tile, first half, chunk 1
        __syncthreads();

        // Z3: last stage on the contiguous rows ZB jp + j, kinetic factor, inverse
        for (int q = t; q < C * ZA; q += NT) {
            const int col = q % C, jp = q / C;
            const int rowbase = slot_of(i, (ZB * jp) / CHZ) * CHE + ((ZB * jp) % CHZ) * C;
            C2 v[ZB];
#pragma unroll
            for (int j = 0; j < ZB; ++j) v[j] = ring[rowbase + j * C + (col ^ swz(j))];
            sfor<ZB - 1>([&](auto jc) {
                constexpr int j = decltype(jc)::value + 1;
                if constexpr (j % 4 == 0) hoist_fence();
                lift_f<T>(v[j], wz[jp * j]);
            });
            dft_fwd<ZB, 0, 1, T>(v);
            const Lift<T> ax = tb[col % W], ay = tb[W + col / W];
            sfor<ZB>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                if constexpr (k2 % 4 == 0) hoist_fence();
                C2 &u = v[brev(k2, ZB)];
                const Lift<T> az = kz[jp + ZA * k2];
                if (a.imag) {
                    const T f = ax.f * ay.f * az.f * sc;
                    u.x *= f;
                    u.y *= f;
                } else {
                    rot_f<T>(u, ax.p, ax.u);
                    rot_f<T>(u, ay.p, ay.u);
                    rot_f<T>(u, az.p, az.u);
                    const T s = ax.s * ay.s * az.s * sc;
                    u.x *= s;
                    u.y *= s;
                }
            });
            dft_inv<ZB, 0, 1, T>(v);
            sfor<ZB - 1>([&](auto jc) {
                constexpr int j = decltype(jc)::value + 1;
                if constexpr (j % 4 == 0) hoist_fence();
                lift_b<T>(v[j], wz[jp * j]);
            });
#pragma unroll
            for (int j = 0; j < ZB; ++j) ring[rowbase + j * C + (col ^ swz(j))] = v[j];
        }
        if (i + 1 < nmine) issue(i + 1, 2, 3);   // next tile, first half, chunk 2
        __syncthreads();

        // Z4: inverse z, first stage, in place
        for (int q = t; q < C * ZB; q += NT) {
            const int col = q % C, j = q / C;
            const int off = j * C + (col ^ swz(j));
            C2 v[ZA];
            sfor<ZA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v[brev(kk, ZA)] = ring[sb[kk / 4] + (kk % 4) * ZB * C + off];
            });
            dft_inv<ZA, 0, 1, T>(v);
#pragma unroll
            for (int rr = 0; rr < ZA; ++rr) ring[sb[rr / 4] + (rr % 4) * ZB * C + off] = v[rr];
        }
        if (i + 1 < nmine) issue(i + 1, 3, 4);   // next tile, first half, chunk 3
        cp_async_commit();
        __syncthreads();

        // Z5: the whole tile is read back to registers first (R5 rounds of
        // 4 x 16 bytes per thread; the cross twiddles too), so its ring
        // slots are free before the stores start: the next tile's second half
        // is copied in while this tile's inverse cross DFTs and stores run,
        // and no store waits for registers a later load would overwrite.
        // Two lanes write the two halves of each 32-byte row segment in the
        // same instruction (16 sectors per warp store: measured to drain
        // faster per SM than one lane per segment with 256-bit stores).
        constexpr int R5 = NZ * (W / 2) / NT;
        static_assert(R5 * NT == NCH * CHZ * (W / 2), "round m reads chunk m * NCH / R5 on");
        C2 v[R5][2][P];
        auto read_back = [&](int m) {
            const int q = m * NT + t;
            const int xo = (q % (W / 2)) * 2, zz = q / (W / 2);
            sfor<P>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                const float4 w4 = *reinterpret_cast<const float4 *>(ring + at(zz, k2 * W + xo));
                v[m][0][brev(k2, P)] = make_float2(w4.x, w4.y);
                v[m][1][brev(k2, P)] = make_float2(w4.z, w4.w);
            });
        };
        // the next tile's second half goes to this tile's first-half slots:
        // only those must be read back before it is issued
#pragma unroll
        for (int m = 0; m < R5 / 2; ++m) read_back(m);
        Lift<T> cw[P];
#pragma unroll
        for (int rr = 1; rr < P; ++rr) cw[rr] = tb[W + P + rr];
        __syncthreads();                         // tile i's first half and tables are free
        if (i + 1 < nmine) issue(i + 1, NCH / 2, NCH);
        cp_async_commit();
#pragma unroll
        for (int m = R5 / 2; m < R5; ++m) read_back(m);
#pragma unroll
        for (int m = 0; m < R5; ++m) {
            const int q = m * NT + t;
            const int xo = (q % (W / 2)) * 2, zz = q / (W / 2);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                dft_inv<P, 0, 1, T>(v[m][c]);
#pragma unroll
                for (int rr = 1; rr < P; ++rr) lift_b<T>(v[m][c][rr], cw[rr]);
            }
            C2 *p = a.dst + (long long)zz * g.plane + colbase + xo;
#pragma unroll
            for (int rr = 0; rr < P; ++rr)
                __stcs(reinterpret_cast<float4 *>(p + ((long long)rr << g.lgnx)),
                       make_float4(v[m][0][rr].x, v[m][0][rr].y, v[m][1][rr].x, v[m][1][rr].y));
        }
    }
    cp_async_wait<0>();
}

// ================================================================ dispatch
namespace {

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <class T, int NX, int RA, int RB, int LY, int YA, int YB>
bool try_xy(const XYArgs<T> &a, cudaStream_t st)
{
    if (a.g.nx != NX || a.g.Ly != LY) return false;
    const bool in = (a.flags & XY_IN_MIXED) != 0, out = (a.flags & XY_OUT_MIXED) != 0;
    const size_t smem = (size_t)LY * (NX + 2) * sizeof(Cx<T>) + (NX + LY) * sizeof(Lift<T>);
    static bool cfg = false;      // one flag for all five variants of this shape
    if (!cfg) {
        const int sz = (int)smem;
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, true, true>, attr, sz);
        cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, true, false>, attr, sz);
        cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, false, false>, attr, sz);
        cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, true, false>, attr, sz);
        cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, false, false>, attr, sz);
        if constexpr (sizeof(T) == 4) {
            cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, true, true>, attr, sz);
            cudaFuncSetAttribute(xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, false, true>, attr, sz);
        }
        cfg = true;
    }
    const int grid = xy_grid(a.g);
    constexpr int NT = xy_threads<T>();
    const bool hot = a.flags == (XY_IN_MIXED | XY_OUT_MIXED | XY_KICK_FULL) &&
                     a.k.form == VF_PRODUCT && !a.k.imag && a.small_angle;
    if constexpr (std::is_same<T, float>::value && NX == 256 && LY == 64 && RA == 16 && YA == 8) {
        if (hot && a.ring && a.src == a.dst) {
            constexpr int HB = (LY / 2) * (NX + 2);
            const size_t rsmem = 3 * HB * sizeof(Cx<T>) + (NX + LY) * sizeof(Lift<T>);
            static bool rcfg = false;
            if (!rcfg) {
                cudaFuncSetAttribute(xy_ring_kernel<NX, RA, RB, LY, YA, YB>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
                rcfg = true;
            }
            xy_ring_kernel<NX, RA, RB, LY, YA, YB><<<std::min(grid, sm_count()), 1024, rsmem, st>>>(a, grid);
            return true;
        }
    }
    if constexpr (sizeof(T) == 4) {
        const bool hot_kick = a.k.form == VF_PRODUCT && !a.k.imag && a.small_angle;
        if (hot_kick && a.flags == (XY_KICK_HALF | XY_OUT_MIXED)) {
            xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, true, true><<<grid, xy_threads<T, true>(), smem, st>>>(a);
            return true;
        }
        if (hot_kick && a.flags == (XY_IN_MIXED | XY_KICK_HALF)) {
            xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, false, true><<<grid, xy_threads<T, true>(), smem, st>>>(a);
            return true;
        }
    }
    if (hot)
        xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, true, true><<<grid, xy_threads<T, true>(), smem, st>>>(a);
    else if (in && out)
        xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, true, false><<<grid, NT, smem, st>>>(a);
    else if (in)
        xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, true, false, false><<<grid, NT, smem, st>>>(a);
    else if (out)
        xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, true, false><<<grid, NT, smem, st>>>(a);
    else
        xy_fast_kernel<T, NX, RA, RB, LY, YA, YB, false, false, false><<<grid, NT, smem, st>>>(a);
    return true;
}

template <class T, int NZ, int ZA, int ZB, int P, int W>
bool try_z(const ZArgs<T> &a, cudaStream_t st)
{
    if (a.g.nz != NZ || a.g.P != P || a.g.w != W) return false;
    constexpr int C = P * W;
    const size_t tile = (size_t)NZ * C + ((sizeof(T) == 4 && C == 8) ? (NZ / 32) * 8 : 0);
    const size_t smem = tile * sizeof(Cx<T>) + 2 * NZ * sizeof(Lift<T>);
    static bool cfg = false;
    if (!cfg) {
        cudaFuncSetAttribute(z_fast_kernel<T, NZ, ZA, ZB, P, W>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    if constexpr (std::is_same<T, float>::value && NZ == 1024 && P == 4 && W == 4) {
        if (a.ring && !a.observe && a.src == a.dst) {
            constexpr int NRING = 12;
            const size_t rsmem = (size_t)NRING * kRingCHZ * P * W * sizeof(Cx<T>) +
                                 2 * NZ * sizeof(Lift<T>);
            static bool rcfg = false;
            if (!rcfg) {
                cudaFuncSetAttribute(z_ring_kernel<NZ, ZA, ZB, P, W, kRingNT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
                rcfg = true;
            }
            const int ntiles = z_grid(a.g);
            const int grid = std::min(ntiles, sm_count());
            z_ring_kernel<NZ, ZA, ZB, P, W, kRingNT><<<grid, kRingNT, rsmem, st>>>(a, ntiles);
            return true;
        }
    }
    z_fast_kernel<T, NZ, ZA, ZB, P, W><<<z_grid(a.g), z_threads<T>(NZ), smem, st>>>(a);
    return true;
}

}  // namespace

// Rows per XY tile of the specialised passes: 64 for complex64, 32 for
// complex128 (a tile is then 128 KB either way).
int fast_rows(int esize) { return esize == 8 ? 64 : 32; }

bool fast_xy_supported(int esize, int nx, int Ly)
{
    return Ly == fast_rows(esize) && (nx == 256 || nx == 128 || nx == 64);
}

bool fast_z_supported(int esize, int nz, int P, int w)
{
    if (esize == 8)
        return (nz == 1024 && ((P == 4 && w == 4) || (P == 1 && w == 16) || (P == 2 && w == 8))) ||
               (nz == 512 && ((P == 4 && w == 8) || (P == 2 && w == 16))) ||
               (nz == 256 && ((P == 4 && w == 16) || (P == 2 && w == 32) || (P == 1 && w == 64)));
    return (nz == 1024 && ((P == 8 && w == 1) || (P == 2 && w == 4) || (P == 4 && w == 2))) ||
           (nz == 512 && ((P == 8 && w == 2) || (P == 4 && w == 4))) ||
           (nz == 256 && ((P == 8 && w == 4) || (P == 4 && w == 8)));
}

bool launch_xy_fast(const XYArgs<float> &a, cudaStream_t st)
{
    return try_xy<float, 256, 16, 16, 64, 8, 8>(a, st) || try_xy<float, 128, 16, 8, 64, 8, 8>(a, st) ||
           try_xy<float, 64, 8, 8, 64, 8, 8>(a, st);
}

bool launch_xy_fast(const XYArgs<double> &a, cudaStream_t st)
{
    return try_xy<double, 256, 16, 16, 32, 4, 8>(a, st) ||
           try_xy<double, 128, 16, 8, 32, 4, 8>(a, st) || try_xy<double, 64, 8, 8, 32, 4, 8>(a, st);
}

bool launch_z_fast(const ZArgs<float> &a, cudaStream_t st)
{
    return try_z<float, 1024, 32, 32, 4, 4>(a, st) || try_z<float, 1024, 32, 32, 1, 16>(a, st) ||
           try_z<float, 1024, 32, 32, 2, 8>(a, st) || try_z<float, 512, 32, 16, 4, 8>(a, st) ||
           try_z<float, 512, 32, 16, 2, 16>(a, st) || try_z<float, 256, 16, 16, 4, 16>(a, st) ||
           try_z<float, 256, 16, 16, 2, 32>(a, st) || try_z<float, 256, 16, 16, 1, 64>(a, st);
}

// Double-float: the specialised XY pass for 256-point rows (16-point
// register DFTs) and the three-stage Z pass of z3_df_pass.cuh for
// 1024-point z-lines (fully unrolled 32-point register DFTs in double-float
// arithmetic are too large to compile); other z lengths take the generic Z
// pass.
bool launch_xy_fast(const XYArgs<df> &a, cudaStream_t st)
{
    return try_xy<df, 256, 16, 16, 32, 4, 8>(a, st);
}
bool launch_z_fast(const ZArgs<df> &a, cudaStream_t st)
{
    return launch_z3_df_p8(a, st) || launch_z3_df_p4(a, st) || launch_z3_df_p2(a, st);
}

bool launch_z_fast(const ZArgs<double> &a, cudaStream_t st)
{
    return try_z<double, 1024, 32, 32, 8, 1>(a, st) || try_z<double, 1024, 32, 32, 2, 4>(a, st) ||
           try_z<double, 1024, 32, 32, 4, 2>(a, st) || try_z<double, 512, 32, 16, 8, 2>(a, st) ||
           try_z<double, 512, 32, 16, 4, 4>(a, st) || try_z<double, 256, 16, 16, 8, 4>(a, st) ||
           try_z<double, 256, 16, 16, 4, 8>(a, st);
}

}  // namespace ctap
