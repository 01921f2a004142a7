// fast_passes.cu -- specialised complex64 XY and Z passes.
//
// Same HBM layout and the same arithmetic definition as the generic passes
// in kernels.cu (natural kx order, natural k' order, rows j P + r), so plans
// can mix them; what changes is how the work is kept on chip:
//
// XY pass (NX = RA * RB columns, LY rows, NX threads):
//   P1  inverse x, last Stockham stage, read straight from HBM (coalesced
//       rows), rotated back, written to shared memory;
//   P2  inverse x, first stage (shared -> shared);
//   P3  one thread per column: the whole LY-point y-line in registers:
//       inverse y DFT, potential factor, forward y DFT (no shared-memory
//       round trip between them);
//   P4  forward x, first stage;  P5 forward x, last stage, written straight
//       to HBM.
//   4 shared-memory round trips per point instead of 11.
//
// Z pass (NZ = ZA * ZB, tile NZ x (P W), 512 threads):
//   Z1  read P rows per z from HBM, finish the forward y-transform (cross
//       twiddle + P-point DFT) in registers, write the tile;
//   Z2  forward z, first stage;
//   Z3  forward z last stage, kinetic factor, inverse last stage, all in
//       registers on the positions the task read;
//   Z4  inverse z, first stage;  Z5 inverse cross DFT and store to HBM.
//   The tile is XOR-swizzled (column ^ 4 (z & 3)) so the z-row-major
//   accesses of Z1/Z5 and the column accesses of Z2-Z4 are conflict-free.
#include "kernels.cuh"

namespace ctap {

namespace {

// -------------------------------------------------------- small-angle kick
// exp(-i th) as a lifted rotation for |th| <= 0.5 (no half-turn reduction):
// p = -tan(-th/2), u = sin(-th) from odd Taylor series (own, |h| <= 0.25).
__device__ __forceinline__ void lift_small(float th, float &p, float &u)
{
    const float a = -th, a2 = a * a;
    float s = fmadd(a2, 2.75573192e-06f, -1.98412698e-04f);      // 1/9!, -1/7!
    s = fmadd(a2, s, 8.33333333e-03f);
    s = fmadd(a2, s, -1.66666667e-01f);
    u = fmadd(a2 * a, s, a);
    const float h = 0.5f * a, h2 = h * h;                        // tan h series
    float t = fmadd(h2, 8.86323552e-03f, 2.18694885e-02f);        // 1382/155925, 62/2835
    t = fmadd(h2, t, 5.39682540e-02f);                           // 17/315
    t = fmadd(h2, t, 1.33333333e-01f);                           // 2/15
    t = fmadd(h2, t, 3.33333333e-01f);                           // 1/3
    p = -fmadd(h2 * h, t, h);
}

template <class T>
__device__ __forceinline__ void kick_one(float2 &v, float th, int imag, int small)
{
    if (imag) {
        const float f = expf(-th);
        v.x *= f;
        v.y *= f;
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

template <int NQ> __device__ void block_sum(double (&acc)[NQ], double *out, int nthreads)
{
    __shared__ double red[32][NQ];
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
            double v = (lane < nthreads / 32) ? red[lane][q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) out[q] = v;
        }
    }
}

}  // namespace

// ======================================================================= XY
template <int NX, int LY, int RA, int RB, bool IN_MIXED, bool OUT_MIXED>
__global__ void __launch_bounds__(NX, 1) xy_fast_kernel(const XYArgs<float> a)
{
    static_assert(RA * RB == NX, "NX = RA RB");
    constexpr int NT = NX;
    constexpr int PITCH = NX + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    __shared__ float gtab[LY];
    __shared__ Lift<float> ytab[LY];

    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int z = blockIdx.x >> g.lgP, r = blockIdx.x & (g.P - 1);
    const long long pbase = (long long)z * g.plane;
    const float2 *src = a.src + pbase;
    float2 *dst = a.dst + pbase;
    const Lift<float> *wx = a.tw + g.fast_x_off;   // exp(-2 pi i e/NX), e < NX
    const int flags = a.flags;
    const Kick<float> &k = a.k;
    const bool kick = (flags & (XY_KICK_HALF | XY_KICK_FULL | XY_KICK_SPLIT)) != 0;

    // per-CTA y data of the potential factor
    if (t < LY) {
        const int y = r + t * g.P;
        if (k.form == VF_PRODUCT) gtab[t] = k.g[y];
        else if (k.form == VF_SEPARABLE)
            ytab[t] = ((flags & XY_KICK_FULL) ? k.sep_full : k.sep_half)[g.nx + y];
    }

    if constexpr (IN_MIXED) {
        // P1: inverse of the last x stage (Ns = RA, radix RB), from HBM
        constexpr int Q1 = LY * RA / NT;
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
            const int q = t + i * NT;
            const int j = q % RA, row = q / RA;
            const float2 *rowp = src + ((long long)(row * g.P + r) << g.lgnx);
            float2 v[RB];
            sfor<RB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v[brev(kk, RB)] = rowp[j + RA * kk];
            });
            dft_inv<RB, 0, 1, float>(v);
#pragma unroll
            for (int rr = 1; rr < RB; ++rr) lift_b<float>(v[rr], wx[j * rr]);
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) sm[row * PITCH + j + RA * rr] = v[rr];
        }
        __syncthreads();
        // P2: inverse of the first x stage (Ns = 1, radix RA)
        constexpr int Q2 = LY * RB / NT;
        float2 v2[Q2][RA];
#pragma unroll
        for (int i = 0; i < Q2; ++i) {
            const int q = t + i * NT;
            const int row = q % LY, j = q / LY;
            sfor<RA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v2[i][brev(kk, RA)] = sm[row * PITCH + j * RA + kk];
            });
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q2; ++i) {
            const int q = t + i * NT;
            const int row = q % LY, j = q / LY;
            dft_inv<RA, 0, 1, float>(v2[i]);
#pragma unroll
            for (int rr = 0; rr < RA; ++rr) sm[row * PITCH + j + RB * rr] = v2[i][rr];
        }
    } else {
        // natural rows straight into the tile
        for (int e = t; e < LY * NX; e += NT) {
            const int row = e / NX, x = e % NX;
            sm[row * PITCH + x] = src[((long long)(row * g.P + r) << g.lgnx) + x];
        }
    }
    __syncthreads();

    // P3: the y-line of column x = t in registers
    {
        const int x = t;
        float2 v[LY];
        if constexpr (IN_MIXED) {
            sfor<LY>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v[brev(kk, LY)] = sm[kk * PITCH + x];
            });
            dft_inv<LY, 0, 1, float>(v);
        } else {
#pragma unroll
            for (int j = 0; j < LY; ++j) v[j] = sm[j * PITCH + x];
        }
        if (flags & XY_RED_OBS) {
            double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            const double xq = g.box[0] + (double)x * g.dx;
            bool in[3] = {false, false, false};
            if (a.rd.xc)
                for (int q = 0; q < 3; ++q) in[q] = fabs(xq - a.rd.xc[q * g.nz + z]) < a.rd.hw;
            const double hz = (a.vform_obs == VF_PRODUCT) ? a.rd.H64[(long long)z * g.nx + x] : 0.0;
            const double vxz = (a.vform_obs == VF_SEPARABLE)
                                   ? a.rd.Vsep[x] + a.rd.Vsep[g.nx + g.ny + z] : 0.0;
#pragma unroll
            for (int j = 0; j < LY; ++j) {
                const int y = r + j * g.P;
                const double d = (double)v[j].x * v[j].x + (double)v[j].y * v[j].y;
                double V = 0.0;
                if (a.vform_obs == VF_DENSE) V = (double)k.Vd[pbase + ((long long)y << g.lgnx) + x];
                else if (a.vform_obs == VF_PRODUCT) V = a.rd.g64[y] * hz;
                else if (a.vform_obs == VF_SEPARABLE) V = vxz + a.rd.Vsep[g.nx + y];
                acc[0] += d;
                acc[1] += V * d;
                acc[2] += in[0] ? d : 0.0;
                acc[3] += in[1] ? d : 0.0;
                acc[4] += in[2] ? d : 0.0;
            }
            block_sum<5>(acc, a.partials + (long long)blockIdx.x * 5, NT);
        }
        if (kick) {
            const bool full = (flags & XY_KICK_FULL) != 0;
            const float tau = full ? k.tau_full : k.tau_half;
            double nacc[1] = {0.0};
            if (k.form == VF_SEPARABLE) {
                const Lift<float> *tb = full ? k.sep_full : k.sep_half;
                const Lift<float> lx = tb[x], lz = tb[g.nx + g.ny + z];
                const Lift<float> *th = k.sep_half;
#pragma unroll
                for (int j = 0; j < LY; ++j) {
                    const int y = r + j * g.P;
                    const Lift<float> ly = ytab[j];
                    if (k.imag) {
                        const float f = lx.f * ly.f * lz.f;
                        v[j].x *= f;
                        v[j].y *= f;
                    } else {
                        rot_f<float>(v[j], lx.p, lx.u);
                        rot_f<float>(v[j], ly.p, ly.u);
                        rot_f<float>(v[j], lz.p, lz.u);
                        const float s = lx.s * ly.s * lz.s;
                        v[j].x *= s;
                        v[j].y *= s;
                    }
                    if (flags & XY_RED_NORM)
                        nacc[0] += (double)v[j].x * v[j].x + (double)v[j].y * v[j].y;
                    if (flags & XY_STATE_OUT)
                        a.state_out[pbase + ((long long)y << g.lgnx) + x] = v[j];
                    if (flags & XY_KICK_SPLIT) {
                        const Lift<float> hx = th[x], hy = th[g.nx + y], hz2 = th[g.nx + g.ny + z];
                        if (k.imag) {
                            const float f = hx.f * hy.f * hz2.f;
                            v[j].x *= f;
                            v[j].y *= f;
                        } else {
                            rot_f<float>(v[j], hx.p, hx.u);
                            rot_f<float>(v[j], hy.p, hy.u);
                            rot_f<float>(v[j], hz2.p, hz2.u);
                            const float s = hx.s * hy.s * hz2.s;
                            v[j].x *= s;
                            v[j].y *= s;
                        }
                    }
                }
            } else {
                const int small = a.small_angle;
                const float hx = (k.form == VF_PRODUCT) ? k.H[(long long)z * g.nx + x] * tau : 0.f;
#pragma unroll
                for (int j = 0; j < LY; ++j) {
                    const int y = r + j * g.P;
                    const float th = (k.form == VF_PRODUCT)
                                         ? gtab[j] * hx
                                         : k.Vd[pbase + ((long long)y << g.lgnx) + x] * tau;
                    kick_one<float>(v[j], th, k.imag, small);
                    if (flags & XY_RED_NORM)
                        nacc[0] += (double)v[j].x * v[j].x + (double)v[j].y * v[j].y;
                    if (flags & XY_STATE_OUT)
                        a.state_out[pbase + ((long long)y << g.lgnx) + x] = v[j];
                    if (flags & XY_KICK_SPLIT) kick_one<float>(v[j], th, k.imag, small);
                }
            }
            if (flags & XY_RED_NORM) block_sum<1>(nacc, a.partials + blockIdx.x, NT);
        }
        if constexpr (OUT_MIXED) {
            dft_fwd<LY, 0, 1, float>(v);
            sfor<LY>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                sm[kk * PITCH + x] = v[brev(kk, LY)];
            });
        } else {
#pragma unroll
            for (int j = 0; j < LY; ++j) sm[j * PITCH + x] = v[j];
        }
    }
    __syncthreads();

    if constexpr (OUT_MIXED) {
        // P4: forward x, first stage (Ns = 1, radix RA)
        constexpr int Q4 = LY * RB / NT;
        float2 v4[Q4][RA];
#pragma unroll
        for (int i = 0; i < Q4; ++i) {
            const int q = t + i * NT;
            const int row = q % LY, j = q / LY;
#pragma unroll
            for (int rr = 0; rr < RA; ++rr) v4[i][rr] = sm[row * PITCH + j + RB * rr];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q4; ++i) {
            const int q = t + i * NT;
            const int row = q % LY, j = q / LY;
            dft_fwd<RA, 0, 1, float>(v4[i]);
            sfor<RA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                sm[row * PITCH + j * RA + kk] = v4[i][brev(kk, RA)];
            });
        }
        __syncthreads();
        // P5: forward x, last stage (Ns = RA, radix RB), straight to HBM
        constexpr int Q5 = LY * RA / NT;
#pragma unroll
        for (int i = 0; i < Q5; ++i) {
            const int q = t + i * NT;
            const int j = q % RA, row = q / RA;
            float2 v[RB];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) v[rr] = sm[row * PITCH + j + RA * rr];
#pragma unroll
            for (int rr = 1; rr < RB; ++rr) lift_f<float>(v[rr], wx[j * rr]);
            dft_fwd<RB, 0, 1, float>(v);
            float2 *rowp = dst + ((long long)(row * g.P + r) << g.lgnx);
            sfor<RB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                rowp[j + RA * kk] = v[brev(kk, RB)];
            });
        }
    } else {
        for (int e = t; e < LY * NX; e += NT) {
            const int row = e / NX, x = e % NX;
            dst[((long long)(row * g.P + r) << g.lgnx) + x] = sm[row * PITCH + x];
        }
    }
}

// ======================================================================== Z
template <int NZ, int ZA, int ZB, int P, int W>
__global__ void __launch_bounds__(512, 1) z_fast_kernel(const ZArgs<float> a)
{
    static_assert(ZA * ZB == NZ, "NZ = ZA ZB");
    constexpr int NT = 512;
    constexpr int C = P * W;
    static_assert(C * NZ == NT * 32, "tile of 32 points per thread");
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const Geom &g = a.g;
    const int t = threadIdx.x;
    const int kp = blockIdx.x >> g.nblk_lg, b = blockIdx.x & ((1 << g.nblk_lg) - 1);
    auto at = [](int zz, int col) {
        return zz * C + (col ^ (C >= 16 ? ((zz & 3) << 2) : 0));
    };
    const Lift<float> *wz = a.tw + g.fast_z_off;   // exp(-2 pi i e/NZ), e < NZ
    const Lift<float> *wc = a.tw + g.cross_off;    // exp(-2 pi i e/ny)
    const long long colbase = ((long long)(kp * P) << g.lgnx) + (b * W);

    Lift<float> cw[P];
#pragma unroll
    for (int rr = 1; rr < P; ++rr) cw[rr] = wc[(rr * kp) & (g.ny - 1)];

    // Z1: load P rows per (z, xo), forward cross DFT, write the tile
    {
        constexpr int Q = NZ * W / NT;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int xo = q % W, zz = q / W;
            const float2 *p = a.src + (long long)zz * g.plane + colbase + xo;
            float2 v[P];
#pragma unroll
            for (int rr = 0; rr < P; ++rr) v[rr] = p[(long long)rr << g.lgnx];
#pragma unroll
            for (int rr = 1; rr < P; ++rr) lift_f<float>(v[rr], cw[rr]);
            dft_fwd<P, 0, 1, float>(v);
            sfor<P>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                sm[at(zz, k2 * W + xo)] = v[brev(k2, P)];
            });
        }
    }
    __syncthreads();

    // Z2: forward z, first stage (Ns = 1, radix ZA)
    {
        constexpr int Q = C * ZB / NT;   // tasks (col, j < NZ/ZA = ZB)
        float2 v[Q > 0 ? Q : 1][ZA];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int col = q % C, j = q / C;
#pragma unroll
            for (int rr = 0; rr < ZA; ++rr) v[i][rr] = sm[at(j + ZB * rr, col)];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int col = q % C, j = q / C;
            dft_fwd<ZA, 0, 1, float>(v[i]);
            sfor<ZA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                sm[at(j * ZA + kk, col)] = v[i][brev(kk, ZA)];
            });
        }
    }
    __syncthreads();

    // Z3: forward last stage, kinetic factor (or energy reduction), inverse
    {
        constexpr int Q = C * ZA / NT;   // tasks (col, j < ZA)
        const float sc = a.inv_n * (a.scale ? (float)(*a.scale) : 1.0f);
        double acc[1] = {0.0};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int col = q % C, j = q / C;
            const int kx = b * W + (col % W);
            const int ky = kp + ((col / W) << g.lgLy);
            float2 v[ZB];
#pragma unroll
            for (int rr = 0; rr < ZB; ++rr) v[rr] = sm[at(j + ZA * rr, col)];
#pragma unroll
            for (int rr = 1; rr < ZB; ++rr) lift_f<float>(v[rr], wz[j * rr]);
            dft_fwd<ZB, 0, 1, float>(v);
            if (a.observe) {
                const double kxy = a.k2h[kx] + a.k2h[g.nx + ky];
                sfor<ZB>([&](auto kc) {
                    constexpr int kk = decltype(kc)::value;
                    const float2 u = v[brev(kk, ZB)];
                    acc[0] += (kxy + a.k2h[g.nx + g.ny + j + ZA * kk]) *
                              ((double)u.x * u.x + (double)u.y * u.y);
                });
                continue;
            }
            const Lift<float> ax = a.kin[kx], ay = a.kin[g.nx + ky];
            sfor<ZB>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                float2 &u = v[brev(kk, ZB)];
                const Lift<float> az = a.kin[g.nx + g.ny + j + ZA * kk];
                if (a.imag) {
                    const float f = ax.f * ay.f * az.f * sc;
                    u.x *= f;
                    u.y *= f;
                } else {
                    rot_f<float>(u, ax.p, ax.u);
                    rot_f<float>(u, ay.p, ay.u);
                    rot_f<float>(u, az.p, az.u);
                    const float s = ax.s * ay.s * az.s * sc;
                    u.x *= s;
                    u.y *= s;
                }
            });
            dft_inv<ZB, 0, 1, float>(v);
#pragma unroll
            for (int rr = 1; rr < ZB; ++rr) lift_b<float>(v[rr], wz[j * rr]);
#pragma unroll
            for (int rr = 0; rr < ZB; ++rr) sm[at(j + ZA * rr, col)] = v[rr];
        }
        if (a.observe) {
            block_sum<1>(acc, a.partials + blockIdx.x, NT);
            return;
        }
    }
    __syncthreads();

    // Z4: inverse z, first stage
    {
        constexpr int Q = C * ZB / NT;
        float2 v[Q > 0 ? Q : 1][ZA];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int col = q % C, j = q / C;
            sfor<ZA>([&](auto kc) {
                constexpr int kk = decltype(kc)::value;
                v[i][brev(kk, ZA)] = sm[at(j * ZA + kk, col)];
            });
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int col = q % C, j = q / C;
            dft_inv<ZA, 0, 1, float>(v[i]);
#pragma unroll
            for (int rr = 0; rr < ZA; ++rr) sm[at(j + ZB * rr, col)] = v[i][rr];
        }
    }
    __syncthreads();

    // Z5: inverse cross DFT and store
    {
        constexpr int Q = NZ * W / NT;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int q = t + i * NT;
            const int xo = q % W, zz = q / W;
            float2 v[P];
            sfor<P>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                v[brev(k2, P)] = sm[at(zz, k2 * W + xo)];
            });
            dft_inv<P, 0, 1, float>(v);
#pragma unroll
            for (int rr = 1; rr < P; ++rr) lift_b<float>(v[rr], cw[rr]);
            float2 *p = a.dst + (long long)zz * g.plane + colbase + xo;
#pragma unroll
            for (int rr = 0; rr < P; ++rr) p[(long long)rr << g.lgnx] = v[rr];
        }
    }
}

// ================================================================ dispatch
namespace {

template <int NX, int LY, int RA, int RB>
bool try_xy(const XYArgs<float> &a, cudaStream_t st)
{
    if (a.g.nx != NX || a.g.Ly != LY) return false;
    const bool in = (a.flags & XY_IN_MIXED) != 0, out = (a.flags & XY_OUT_MIXED) != 0;
    const size_t smem = (size_t)LY * (NX + 1) * sizeof(float2);
    static bool cfg = false;      // one flag for all four variants of this shape
    if (!cfg) {
        cudaFuncSetAttribute(xy_fast_kernel<NX, LY, RA, RB, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_fast_kernel<NX, LY, RA, RB, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_fast_kernel<NX, LY, RA, RB, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_fast_kernel<NX, LY, RA, RB, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    const int grid = xy_grid(a.g);
    if (in && out) xy_fast_kernel<NX, LY, RA, RB, true, true><<<grid, NX, smem, st>>>(a);
    else if (in) xy_fast_kernel<NX, LY, RA, RB, true, false><<<grid, NX, smem, st>>>(a);
    else if (out) xy_fast_kernel<NX, LY, RA, RB, false, true><<<grid, NX, smem, st>>>(a);
    else xy_fast_kernel<NX, LY, RA, RB, false, false><<<grid, NX, smem, st>>>(a);
    return true;
}

template <int NZ, int ZA, int ZB, int P, int W>
bool try_z(const ZArgs<float> &a, cudaStream_t st)
{
    if (a.g.nz != NZ || a.g.P != P || a.g.w != W) return false;
    const size_t smem = (size_t)NZ * P * W * sizeof(float2);
    static bool cfg = false;
    if (!cfg) {
        cudaFuncSetAttribute(z_fast_kernel<NZ, ZA, ZB, P, W>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    z_fast_kernel<NZ, ZA, ZB, P, W><<<z_grid(a.g), 512, smem, st>>>(a);
    return true;
}

}  // namespace

bool fast_xy_supported(int nx, int Ly)
{
    return (nx == 256 && Ly == 64) || (nx == 128 && Ly == 64) || (nx == 64 && Ly == 64);
}

bool fast_z_supported(int nz, int P, int w)
{
    return (nz == 1024 && ((P == 4 && w == 4) || (P == 1 && w == 16) || (P == 2 && w == 8))) ||
           (nz == 512 && ((P == 4 && w == 8) || (P == 2 && w == 16))) ||
           (nz == 256 && ((P == 4 && w == 16) || (P == 2 && w == 32) || (P == 1 && w == 64)));
}

bool launch_xy_fast(const XYArgs<float> &a, cudaStream_t st)
{
    return try_xy<256, 64, 16, 16>(a, st) || try_xy<128, 64, 16, 8>(a, st) ||
           try_xy<64, 64, 8, 8>(a, st);
}

bool launch_z_fast(const ZArgs<float> &a, cudaStream_t st)
{
    return try_z<1024, 32, 32, 4, 4>(a, st) || try_z<1024, 32, 32, 1, 16>(a, st) ||
           try_z<1024, 32, 32, 2, 8>(a, st) || try_z<512, 32, 16, 4, 8>(a, st) ||
           try_z<512, 32, 16, 2, 16>(a, st) || try_z<256, 16, 16, 4, 16>(a, st) ||
           try_z<256, 16, 16, 2, 32>(a, st) || try_z<256, 16, 16, 1, 64>(a, st);
}

}  // namespace ctap
