// z3_df_pass.cuh -- the specialised Z pass of the double-float path.
//
// 1024-point z-lines in three register stages (16 x 4 x 16) instead of the
// two 32-point stages of z_fast_kernel: fully unrolled 32-point register
// DFTs in double-float arithmetic are too large to compile; one 16-point
// task per thread fits the 128-register budget of 512 threads.
// Each (P, W) tile geometry is instantiated in its own translation unit
// (z3_df_p8.cu, z3_df_p4.cu, z3_df_p2.cu) so that the build compiles them in
// parallel.  Observables launches stop after the forward transform with the
// FP64 kinetic-energy sum (one partial per CTA).
#pragma once

#include "kernels.cuh"

namespace ctap {

namespace z3df {

// streaming (evict-first) global access of one double-float complex value
// (hi, lo of the real part, then of the imaginary part)
__device__ __forceinline__ df2 ld_stream(const df2 *p)
{
    const float4 w = __ldcs(reinterpret_cast<const float4 *>(p));
    return df2{df(w.x, w.y), df(w.z, w.w)};
}
__device__ __forceinline__ void st_stream(df2 *p, const df2 &v)
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo));
}
// compiler-only fence: keeps the twiddle-table loads of a stage from being
// hoisted en masse
__device__ __forceinline__ void hoist_fence() { asm volatile("" ::: "memory"); }

// fixed-order sum of one FP64 value over the CTA (warp shuffles, then the
// warp sums in order by warp 0); thread 0 writes it
template <int NT> __device__ __forceinline__ void cta_sum(double v, double *out)
{
    __shared__ double red[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double w = (lane < NT / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (lane == 0) *out = w;
    }
}

// Z pass with three register stages, NZ = ZA ZM ZB (1024 = 16 x 4 x 16), for
// complex128-sized elements.  It exists for the double-float path: the
// 32-point register DFTs of z_fast_kernel are too large to compile in
// double-float arithmetic.  Same tile, swizzle, cross DFT, HBM layout and
// kinetic factors as z_fast_kernel; the z transform is a three-level
// decimation in frequency, z = ZM ZB n1 + ZB n2 + n3 -> kz = k1 + ZA k2 +
// ZA ZM k3:
//   Z2  radix ZA over n1 (rows n2' + ZM ZB n1, n2' = ZB n2 + n3);
//   Z2b twiddle exp(-2 pi i n2' k1/NZ), radix ZM over n2;
//   Z3  twiddle exp(-2 pi i n3 k2/(ZM ZB)), radix ZB over the ZB contiguous
//       rows n3, the kinetic factor (real time: the (kx, ky) rotation of the
//       column from its table entry, then the kz one), and the exact mirror
//       back;
//   Z4b, Z4 the mirrors of Z2b and Z2.
template <class T, int NZ, int ZA, int ZM, int ZB, int P, int W, int NT>
__global__ void __launch_bounds__(NT, 1) z_fast3_kernel(const ZArgs<T> a)
{
    static_assert(ZA * ZM * ZB == NZ, "NZ = ZA ZM ZB");
    static_assert(sizeof(T) == 8, "complex128-sized elements");
    using C2 = Cx<T>;
    constexpr int C = P * W;
    constexpr int N2 = ZM * ZB;
    static_assert(C >= 8, "tile needs at least 8 columns");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *sm = reinterpret_cast<C2 *>(smraw);
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int tl = blockIdx.x & ((1 << g.lgzt) - 1);
    const long long roff = (long long)(blockIdx.x >> g.lgzt) * g.rstride;
    const int kp = tl >> g.nblk_lg, b = tl & ((1 << g.nblk_lg) - 1);
    // a row of 8 values spans all 32 banks; W-column blocks rotate with z
    auto at = [](int zz, int col) {
        constexpr int SWM = (W < 8) ? (8 / W - 1) : 0;
        return zz * C + (col ^ ((zz & SWM) * W));
    };
    const Lift<T> *wc = a.tw + g.cross_off;
    const long long colbase = roff + ((long long)(kp * P) << g.lgnx) + (b * W);
    Lift<T> *wz = reinterpret_cast<Lift<T> *>(sm + NZ * C);    // exp(-2 pi i e/NZ)
    Lift<T> *kz = wz + NZ;                                      // z kinetic factors
    for (int e = t; e < NZ; e += NT) {
        wz[e] = a.tw[g.fast_z_off + e];
        if (!a.observe) kz[e] = a.kin[g.nx + g.ny + e];
    }
    Lift<T> cw[P];
#pragma unroll
    for (int rr = 1; rr < P; ++rr) cw[rr] = wc[(rr * kp) & (g.ny - 1)];

    // Z1: load P rows per (z, column), forward cross DFT, write the tile;
    // every load of the thread is issued before any is used
    {
        constexpr int NTASK = NZ * W;
        constexpr int Q = NTASK / NT;
        static_assert(NTASK % NT == 0, "whole tasks per thread");
        C2 v[Q][P];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int xo = q % W, zz = q / W;
            const C2 *p = a.src + (long long)zz * g.plane + colbase + xo;
#pragma unroll
            for (int rr = 0; rr < P; ++rr) v[i][rr] = ld_stream(p + ((long long)rr << g.lgnx));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int xo = q % W, zz = q / W;
            // the lifted rotations in pairs (bitwise the single forms)
#pragma unroll
            for (int rr = 1; rr + 1 < P; rr += 2) lift2_f(v[i][rr], v[i][rr + 1], cw[rr], cw[rr + 1]);
            lift_f<T>(v[i][P - 1], cw[P - 1]);
            dft_fwd<P, 0, 1, T>(v[i]);
            sfor<P>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                sm[at(zz, k2 * W + xo)] = v[i][brev(k2, P)];
            });
        }
    }
    __syncthreads();

    // Z2: forward z, radix ZA over n1, in place (natural k1 order)
    for (int q = t; q < C * N2; q += NT) {
        const int col = q % C, j = q / C;
        C2 v[ZA];
#pragma unroll
        for (int rr = 0; rr < ZA; ++rr) v[rr] = sm[at(j + N2 * rr, col)];
        dft_fwd<ZA, 0, 1, T>(v);
        sfor<ZA>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            sm[at(j + N2 * kk, col)] = v[brev(kk, ZA)];
        });
    }
    __syncthreads();

    // Z2b: twiddle of the first level, radix ZM over n2
    for (int q = t; q < C * ZA * ZB; q += NT) {
        const int col = q % C, r2 = q / C;
        const int n3 = r2 % ZB, k1 = r2 / ZB;
        const int base = n3 + N2 * k1;
        C2 v[ZM];
#pragma unroll
        for (int n2 = 0; n2 < ZM; ++n2) v[n2] = sm[at(base + ZB * n2, col)];
#pragma unroll
        for (int n2 = 0; n2 < ZM; n2 += 2)
            lift2_f(v[n2], v[n2 + 1], wz[(ZB * n2 + n3) * k1], wz[(ZB * (n2 + 1) + n3) * k1]);
        dft_fwd<ZM, 0, 1, T>(v);
        sfor<ZM>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            sm[at(base + ZB * k2, col)] = v[brev(k2, ZM)];
        });
    }
    __syncthreads();

    // Z3: twiddle of the second level, radix ZB over the contiguous rows,
    // kinetic factor, inverse
    {
        const T sc = a.inv_n * (a.scale ? (T)(*a.scale) : T(1));
        double acc = 0.0;                              // observables: sum k^2/2 |psi_k|^2
        for (int q = t; q < C * ZA * ZM; q += NT) {
            const int col = q % C, r2 = q / C;
            const int k2 = r2 % ZM, k1 = r2 / ZM;
            const int base = ZB * k2 + N2 * k1;
            const int kx = b * W + (col % W);
            const int ky = kp + ((col / W) << g.lgLy);
            C2 v[ZB];
#pragma unroll
            for (int j = 0; j < ZB; ++j) v[j] = sm[at(base + j, col)];
            sfor<(ZB - 1) / 2>([&](auto jc) {
                constexpr int j = 2 * decltype(jc)::value + 1;
                if constexpr (j % 4 == 1) hoist_fence();
                lift2_f(v[j], v[j + 1], wz[ZA * j * k2], wz[ZA * (j + 1) * k2]);
            });
            lift_f<T>(v[ZB - 1], wz[ZA * (ZB - 1) * k2]);
            dft_fwd<ZB, 0, 1, T>(v);
            // register brev(k3) holds kz = k1 + ZA k2 + ZA ZM k3
            const int kzb = k1 + ZA * k2;
            if (a.observe) {                           // forward only: the kinetic sum in FP64
                const double kxy2 = a.k2h[kx] + a.k2h[g.nx + ky];
                sfor<ZB>([&](auto kc) {
                    constexpr int k3 = decltype(kc)::value;
                    const C2 u = v[brev(k3, ZB)];
                    const double ux = (double)u.x, uy = (double)u.y;
                    acc += (kxy2 + a.k2h[g.nx + g.ny + kzb + ZA * ZM * k3]) * (ux * ux + uy * uy);
                });
                continue;
            }
            const Lift<T> ax = a.kin[kx], ay = a.kin[g.nx + ky];
            // real time: the (kx, ky) rotation as one table entry (FP64 angle)
            const Lift<T> *kxy = static_cast<const Lift<T> *>(a.kin_xy);
            const Lift<T> axy = kxy ? kxy[(long long)ky * g.nx + kx] : ax;
            // two frequencies at a time: the three rotations as pairs, the
            // scale on both components at once
            sfor<ZB / 2>([&](auto kc) {
                constexpr int k3 = 2 * decltype(kc)::value;
                if constexpr (k3 % 4 == 0) hoist_fence();
                C2 &u0 = v[brev(k3, ZB)], &u1 = v[brev(k3 + 1, ZB)];
                const Lift<T> az0 = kz[kzb + ZA * ZM * k3], az1 = kz[kzb + ZA * ZM * (k3 + 1)];
                if (a.imag) {
                    cx_scale_df(u0, ax.f * ay.f * az0.f * sc);
                    cx_scale_df(u1, ax.f * ay.f * az1.f * sc);
                } else if (kxy) {
                    rot2_df<false>(u0, u1, axy.p, axy.u, axy.p, axy.u);
                    rot2_df<false>(u0, u1, az0.p, az0.u, az1.p, az1.u);
                    cx_scale_df(u0, axy.s * az0.s * sc);
                    cx_scale_df(u1, axy.s * az1.s * sc);
                } else {
                    rot2_df<false>(u0, u1, ax.p, ax.u, ax.p, ax.u);
                    rot2_df<false>(u0, u1, ay.p, ay.u, ay.p, ay.u);
                    rot2_df<false>(u0, u1, az0.p, az0.u, az1.p, az1.u);
                    cx_scale_df(u0, ax.s * ay.s * az0.s * sc);
                    cx_scale_df(u1, ax.s * ay.s * az1.s * sc);
                }
            });
            dft_inv<ZB, 0, 1, T>(v);
            sfor<(ZB - 1) / 2>([&](auto jc) {
                constexpr int j = 2 * decltype(jc)::value + 1;
                if constexpr (j % 4 == 1) hoist_fence();
                lift2_b(v[j], v[j + 1], wz[ZA * j * k2], wz[ZA * (j + 1) * k2]);
            });
            lift_b<T>(v[ZB - 1], wz[ZA * (ZB - 1) * k2]);
#pragma unroll
            for (int j = 0; j < ZB; ++j) sm[at(base + j, col)] = v[j];
        }
        if (a.observe) {                               // one partial per CTA, nothing stored
            cta_sum<NT>(acc, a.partials + blockIdx.x);
            return;
        }
    }
    __syncthreads();

    // Z4b: mirror of Z2b
    for (int q = t; q < C * ZA * ZB; q += NT) {
        const int col = q % C, r2 = q / C;
        const int n3 = r2 % ZB, k1 = r2 / ZB;
        const int base = n3 + N2 * k1;
        C2 v[ZM];
        sfor<ZM>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            v[brev(k2, ZM)] = sm[at(base + ZB * k2, col)];
        });
        dft_inv<ZM, 0, 1, T>(v);
#pragma unroll
        for (int n2 = 0; n2 < ZM; n2 += 2)
            lift2_b(v[n2], v[n2 + 1], wz[(ZB * n2 + n3) * k1], wz[(ZB * (n2 + 1) + n3) * k1]);
#pragma unroll
        for (int n2 = 0; n2 < ZM; ++n2) sm[at(base + ZB * n2, col)] = v[n2];
    }
    __syncthreads();

    // Z4: mirror of Z2
    for (int q = t; q < C * N2; q += NT) {
        const int col = q % C, j = q / C;
        C2 v[ZA];
        sfor<ZA>([&](auto kc) {
            constexpr int kk = decltype(kc)::value;
            v[brev(kk, ZA)] = sm[at(j + N2 * kk, col)];
        });
        dft_inv<ZA, 0, 1, T>(v);
#pragma unroll
        for (int rr = 0; rr < ZA; ++rr) sm[at(j + N2 * rr, col)] = v[rr];
    }
    __syncthreads();

    // Z5: inverse cross DFT and store
    for (int q = t; q < NZ * W; q += NT) {
        const int xo = q % W, zz = q / W;
        C2 v[P];
        sfor<P>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            v[brev(k2, P)] = sm[at(zz, k2 * W + xo)];
        });
        dft_inv<P, 0, 1, T>(v);
#pragma unroll
        for (int rr = 1; rr + 1 < P; rr += 2) lift2_b(v[rr], v[rr + 1], cw[rr], cw[rr + 1]);
        lift_b<T>(v[P - 1], cw[P - 1]);
        C2 *p = a.dst + (long long)zz * g.plane + colbase + xo;
#pragma unroll
        for (int rr = 0; rr < P; ++rr) st_stream(p + ((long long)rr << g.lgnx), v[rr]);
    }
}

// 512 threads: double-float arithmetic is a chain of dependent FP32
// operations, so the pass wants warps more than registers.  One 16-point
// task is live per thread and fits 128 registers without spills (ptxas -v);
// measured at 256x256x1024, 6.39 ms per launch against 10.2 ms at 256
// threads (255 registers) and 8.9 ms for the generic Z pass.
constexpr int kZ3NT = 512;

// launch on the plan's stream when the geometry is this instantiation's
template <int NZ, int ZA, int ZM, int ZB, int P, int W> bool try_z3(const ZArgs<df> &a, cudaStream_t st)
{
    if (a.g.nz != NZ || a.g.P != P || a.g.w != W) return false;
    const size_t smem = (size_t)NZ * P * W * sizeof(Cx<df>) + 2 * NZ * sizeof(Lift<df>);
    static bool cfg = false;
    if (!cfg) {
        cudaFuncSetAttribute(z_fast3_kernel<df, NZ, ZA, ZM, ZB, P, W, kZ3NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    z_fast3_kernel<df, NZ, ZA, ZM, ZB, P, W, kZ3NT><<<z_grid(a.g), kZ3NT, smem, st>>>(a);
    return true;
}

}  // namespace z3df

}  // namespace ctap
