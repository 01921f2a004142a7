// kernels.cu -- XY and Z passes of the split-step propagation (Sec. IV),
// FP64-accumulated reductions and small helper kernels.
#include "kernels.cuh"

namespace ctap {


// -------------------------------------------------------------- reductions
// Block sum of NQ doubles, fixed order (warp shuffles, then warp 0): results
// are bitwise reproducible run to run.
template <int NQ> __device__ void block_sum_store(double (&acc)[NQ], double *out)
{
    __shared__ double red[kNT / 32][NQ];
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
            double v = (lane < kNT / 32) ? red[lane][q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) out[q] = v;
        }
    }
}

// ------------------------------------------------------------------ kicks
// psi <- exp(-i V tau) psi (real time) or exp(-V tau) psi (imaginary time)
template <class T>
__device__ __forceinline__ void kick_point(Cx<T> &v, const Kick<T> &k, const Geom &g, int x,
                                           int y, int z, int zl, bool full)
{
    // z: plane index over the batch (per-plane tables), zl: replica-local z
    if (k.form == VF_SEPARABLE) {
        const Lift<T> *t = full ? k.sep_full : k.sep_half;
        const Lift<T> a = t[x], b = t[g.nx + y], c = t[g.nx + g.ny + zl];
        if (k.imag) {
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
    } else {
        const T V = (k.form == VF_DENSE) ? k.Vd[((long long)z * g.ny + y) * g.nx + x]
                                         : k.g[y] * k.H[(long long)z * g.nx + x] +
                                               (k.vz ? k.vz[zl] : T(0));
        const T th = V * (full ? k.tau_full : k.tau_half);
        if (k.imag) {
            const T f = dexp(-th);
            v.x *= f;
            v.y *= f;
        } else {
            T p, u, s;
            if constexpr (std::is_same<T, df>::value) {
                if (fabsf(th.hi) <= 0.1f) {          // double-float series, no FP64
                    lift_small(th, p, u);
                    rot_f<T>(v, p, u);
                    return;
                }
                lift_from_angle(-th, p, u, s);
                rot_f<T>(v, p, u);
                v.x = sign_mul(v.x, s);
                v.y = sign_mul(v.y, s);
                return;
            }
            lift_from_angle(-th, p, u, s);
            rot_f<T>(v, p, u);
            v.x *= s;
            v.y *= s;
        }
    }
}

// --------------------------------------------------------------- XY pass
template <class T, int MAXV>
__global__ void __launch_bounds__(kNT, 1) xy_pass_kernel(const XYArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Cx<T> *sm = reinterpret_cast<Cx<T> *>(smraw);
    const Geom &g = a.g;
    const int z = blockIdx.x >> g.lgP, r = blockIdx.x & (g.P - 1);
    const int zl = z & (g.nz - 1);
    const long long pbase = (long long)z * g.plane;
    const int E = g.Ly << g.lgnx;
    const int flags = a.flags;

    for (int e = threadIdx.x; e < E; e += kNT) {
        const int j = e >> g.lgnx, x = e & (g.nx - 1);
        sm[j * g.pitchXY + x] = a.src[pbase + ((long long)(j * g.P + r) << g.lgnx) + x];
    }
    __syncthreads();

    if (flags & XY_RED_OBS) {
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int e = threadIdx.x; e < E; e += kNT) {
            const int j = e >> g.lgnx, x = e & (g.nx - 1), y = r + j * g.P;
            const Cx<T> v = sm[j * g.pitchXY + x];
            const double d = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            double V = 0.0;
            if (a.vform_obs == VF_DENSE) V = (double)a.k.Vd[(pbase + ((long long)y << g.lgnx)) + x];
            else if (a.vform_obs == VF_PRODUCT)
                V = a.rd.g64[y] * a.rd.H64[(long long)z * g.nx + x] + (a.rd.vz64 ? a.rd.vz64[zl] : 0.0);
            else if (a.vform_obs == VF_SEPARABLE)
                V = a.rd.Vsep[x] + a.rd.Vsep[g.nx + y] + a.rd.Vsep[g.nx + g.ny + zl];
            acc[0] += d;
            acc[1] += V * d;
            if (a.rd.xc) {
                const double xq = g.box[0] + (double)x * g.dx;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (fabs(xq - a.rd.xc[q * g.nz + zl]) < a.rd.hw) acc[2 + q] += d;
            }
        }
        block_sum_store<5>(acc, a.partials + (long long)blockIdx.x * 5);
        __syncthreads();
    }

    // adjoint gradient partial of one point: Im(conj(v) psi) g(y) D_j(z, x)
    double gacc[2] = {0.0, 0.0};
    auto grad_point = [&](const Cx<T> &v, int x, int y) {
        const Cx<T> q = static_cast<const Cx<T> *>(a.gd.psi)[pbase + ((long long)y << g.lgnx) + x];
        const double im = ((double)v.x * (double)q.y - (double)v.y * (double)q.x) * a.gd.g64[y];
        gacc[0] += im * a.gd.D1[(long long)z * g.nx + x];
        gacc[1] += im * a.gd.D3[(long long)z * g.nx + x];
    };
    if (flags & XY_GRAD_PRE) {
        for (int e = threadIdx.x; e < E; e += kNT) {
            const int j = e >> g.lgnx, x = e & (g.nx - 1);
            grad_point(sm[j * g.pitchXY + x], x, r + j * g.P);
        }
    }

    if (flags & XY_IN_MIXED) {
        axis_inv<MAXV, kNT, T>(sm, LineMap{g.lgLy, 0, g.pitchXY, 1}, g.lgLy, g.apx, a.tw);
        axis_inv<MAXV, kNT, T>(sm, LineMap{g.lgnx, 0, 1, g.pitchXY}, g.lgnx, g.apy, a.tw);
    }

    if (flags & (XY_KICK_HALF | XY_KICK_FULL | XY_KICK_SPLIT)) {
        double nacc[1] = {0.0};
        for (int e = threadIdx.x; e < E; e += kNT) {
            const int j = e >> g.lgnx, x = e & (g.nx - 1), y = r + j * g.P;
            Cx<T> v = sm[j * g.pitchXY + x];
            kick_point<T>(v, a.k, g, x, y, z, zl, (flags & XY_KICK_FULL) != 0);
            if (flags & XY_RED_NORM) nacc[0] += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            if (flags & XY_STATE_OUT)
                a.state_out[pbase + ((long long)y << g.lgnx) + x] = v;
            if (flags & XY_GRAD) grad_point(v, x, y);
            if (flags & XY_KICK_SPLIT) kick_point<T>(v, a.k, g, x, y, z, zl, false);
            sm[j * g.pitchXY + x] = v;
        }
        if (flags & XY_RED_NORM) block_sum_store<1>(nacc, a.partials + blockIdx.x);
        __syncthreads();
    }
    if (flags & (XY_GRAD | XY_GRAD_PRE)) {
        __shared__ double gtot[2];
        block_sum_store<2>(gacc, gtot);
        __syncthreads();
        if (threadIdx.x == 0) {
            a.gd.acc[2 * blockIdx.x] += a.gd.coef * gtot[0];
            a.gd.acc[2 * blockIdx.x + 1] += a.gd.coef * gtot[1];
        }
    }

    if (flags & XY_OUT_MIXED) {
        axis_fwd<MAXV, kNT, T>(sm, LineMap{g.lgnx, 0, 1, g.pitchXY}, g.lgnx, g.apy, a.tw);
        axis_fwd<MAXV, kNT, T>(sm, LineMap{g.lgLy, 0, g.pitchXY, 1}, g.lgLy, g.apx, a.tw);
    }

    for (int e = threadIdx.x; e < E; e += kNT) {
        const int j = e >> g.lgnx, x = e & (g.nx - 1);
        a.dst[pbase + ((long long)(j * g.P + r) << g.lgnx) + x] = sm[j * g.pitchXY + x];
    }
}

// ---------------------------------------------------------------- Z pass
// Load the tile (all z, rows k' P + r, columns b w .. b w + w - 1) and
// finish the forward y-transform: twiddle exp(-2 pi i r k'/ny), P-point DFT
// over the row classes r.  Result for ky = k' + Ly k2 goes to tile column
// k2 w + xo.
template <class T, int P>
__device__ __forceinline__ void z_load_cross(const ZArgs<T> &a, Cx<T> *sm, int kp, int b,
                                             long long roff)
{
    const Geom &g = a.g;
    const Lift<T> *W = a.tw + g.cross_off;
    const int ntask = g.nz << g.lgw;
    for (int t = threadIdx.x; t < ntask; t += kNT) {
        const int zz = t >> g.lgw, xo = t & (g.w - 1);
        const long long base = roff + (long long)zz * g.plane + ((long long)(kp * P) << g.lgnx) +
                               (b << g.lgw) + xo;
        Cx<T> v[P];
#pragma unroll
        for (int r = 0; r < P; ++r) v[r] = a.src[base + ((long long)r << g.lgnx)];
#pragma unroll
        for (int r = 1; r < P; ++r) lift_f<T>(v[r], W[(r * kp) & (g.ny - 1)]);
        dft_fwd<P, 0, 1, T>(v);
        sfor<P>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            sm[zz * g.pitchZ + (k2 << g.lgw) + xo] = v[brev(k2, P)];
        });
    }
}

// Exact mirror of z_load_cross, storing the rows back.
template <class T, int P>
__device__ __forceinline__ void z_store_cross(const ZArgs<T> &a, const Cx<T> *sm, int kp, int b,
                                              long long roff)
{
    const Geom &g = a.g;
    const Lift<T> *W = a.tw + g.cross_off;
    const int ntask = g.nz << g.lgw;
    for (int t = threadIdx.x; t < ntask; t += kNT) {
        const int zz = t >> g.lgw, xo = t & (g.w - 1);
        const long long base = roff + (long long)zz * g.plane + ((long long)(kp * P) << g.lgnx) +
                               (b << g.lgw) + xo;
        Cx<T> v[P];
        sfor<P>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            v[brev(k2, P)] = sm[zz * g.pitchZ + (k2 << g.lgw) + xo];
        });
        dft_inv<P, 0, 1, T>(v);
#pragma unroll
        for (int r = 1; r < P; ++r) lift_b<T>(v[r], W[(r * kp) & (g.ny - 1)]);
#pragma unroll
        for (int r = 0; r < P; ++r) a.dst[base + ((long long)r << g.lgnx)] = v[r];
    }
}

template <class T, int MAXV>
__global__ void __launch_bounds__(kNT, 1) z_pass_kernel(const ZArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Cx<T> *sm = reinterpret_cast<Cx<T> *>(smraw);
    const Geom &g = a.g;
    const int tl = blockIdx.x & ((1 << g.lgzt) - 1);          // tile within the replica
    const long long roff = (long long)(blockIdx.x >> g.lgzt) * g.rstride;
    const int kp = tl >> g.nblk_lg, b = tl & ((1 << g.nblk_lg) - 1);

    switch (g.P) {
    case 1: z_load_cross<T, 1>(a, sm, kp, b, roff); break;
    case 2: z_load_cross<T, 2>(a, sm, kp, b, roff); break;
    case 4: z_load_cross<T, 4>(a, sm, kp, b, roff); break;
    case 8: z_load_cross<T, 8>(a, sm, kp, b, roff); break;
    default: z_load_cross<T, 16>(a, sm, kp, b, roff); break;
    }
    __syncthreads();

    const LineMap lz{g.lgC, 0, 1, g.pitchZ};
    axis_fwd<MAXV, kNT, T>(sm, lz, g.lgC, g.apz, a.tw);

    const int E = g.nz << g.lgC;
    if (a.observe) {
        double acc[1] = {0.0};
        for (int e = threadIdx.x; e < E; e += kNT) {
            const int zz = e >> g.lgC, col = e & (g.C - 1);
            const int kx = (b << g.lgw) + (col & (g.w - 1));
            const int ky = kp + ((col >> g.lgw) << g.lgLy);
            const Cx<T> v = sm[zz * g.pitchZ + col];
            const double d = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            acc[0] += (a.k2h[kx] + a.k2h[g.nx + ky] + a.k2h[g.nx + g.ny + zz]) * d;
        }
        block_sum_store<1>(acc, a.partials + blockIdx.x);
        return;
    }

    const T sc = a.inv_n * (a.scale ? (T)(*a.scale) : T(1));
    for (int e = threadIdx.x; e < E; e += kNT) {
        const int zz = e >> g.lgC, col = e & (g.C - 1);
        const int kx = (b << g.lgw) + (col & (g.w - 1));
        const int ky = kp + ((col >> g.lgw) << g.lgLy);
        const Lift<T> ax = a.kin[kx], ay = a.kin[g.nx + ky], az = a.kin[g.nx + g.ny + zz];
        Cx<T> v = sm[zz * g.pitchZ + col];
        if (a.imag) {
            const T f = ax.f * ay.f * az.f * sc;
            v.x *= f;
            v.y *= f;
        } else {
            rot_f<T>(v, ax.p, ax.u);
            rot_f<T>(v, ay.p, ay.u);
            rot_f<T>(v, az.p, az.u);
            const T s = ax.s * ay.s * az.s * sc;
            v.x *= s;
            v.y *= s;
        }
        sm[zz * g.pitchZ + col] = v;
    }
    __syncthreads();

    axis_inv<MAXV, kNT, T>(sm, lz, g.lgC, g.apz, a.tw);

    switch (g.P) {
    case 1: z_store_cross<T, 1>(a, sm, kp, b, roff); break;
    case 2: z_store_cross<T, 2>(a, sm, kp, b, roff); break;
    case 4: z_store_cross<T, 4>(a, sm, kp, b, roff); break;
    case 8: z_store_cross<T, 8>(a, sm, kp, b, roff); break;
    default: z_store_cross<T, 16>(a, sm, kp, b, roff); break;
    }
}

// --------------------------------------------------------------- helpers
__global__ void reduce_partials_kernel(const double *p, int nblk, int nq, double *out)
{
    for (int q = 0; q < nq; ++q) {
        double acc[1] = {0.0};
        for (int i = threadIdx.x; i < nblk; i += kNT) acc[0] += p[(long long)i * nq + q];
        block_sum_store<1>(acc, out + q);
        __syncthreads();
    }
}

__global__ void norm_scale_kernel(const double *p, int nblk, double dV, double *scale)
{
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < nblk; i += kNT) acc[0] += p[i];
    __shared__ double tot;
    block_sum_store<1>(acc, &tot);
    __syncthreads();
    if (threadIdx.x == 0) scale[0] = 1.0 / sqrt(tot * dV);
}

template <class T> __global__ void scale_kernel(Cx<T> *psi, long long n, const double *scale)
{
    const T s = (T)scale[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        Cx<T> v = psi[i];
        v.x *= s;
        v.y *= s;
        psi[i] = v;
    }
}

template <class T>
__global__ void mask_kernel(const Cx<T> *psi, Cx<T> *lam, const Geom g, const double *xcj,
                            double hw, double *partials, long long chunk)
{
    const long long n = g.plane * g.nz;
    const long long i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double acc[1] = {0.0};
    for (long long i = i0 + threadIdx.x; i < i1; i += kNT) {
        const int x = (int)(i & (g.nx - 1));
        const int z = (int)(i >> (g.lgnx + g.lgny));
        const double xq = g.box[0] + (double)x * g.dx;
        Cx<T> v = psi[i];
        if (fabs(xq - xcj[z]) < hw) {
            acc[0] += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        } else {
            v.x = T(0);
            v.y = T(0);
        }
        lam[i] = v;
    }
    block_sum_store<1>(acc, partials + blockIdx.x);
}

// ------------------------------------------------- y-integrated density
// One thread per (z, x): sum over y in ascending order (deterministic).
template <class T>
__global__ void density_xz_kernel(const Cx<T> *psi, const Geom g, double dy, double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)g.batch * g.nz * g.nx) return;
    const int z = (int)(i >> g.lgnx), x = (int)(i & (g.nx - 1));
    const Cx<T> *p = psi + (long long)z * g.plane + x;
    double acc = 0.0;
    for (int y = 0; y < g.ny; ++y) {
        const Cx<T> v = p[(long long)y << g.lgnx];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    out[i] = acc * dy;
}

// ------------------------------------------------- atom-chip wire field
// V = vs |B| - voff on the grid, B = bias + the Biot-Savart field of thin
// straight segments (Sec. III, Eq. 4): for a segment A -> C carrying I, at P
// with a = P - A, c = P - C, l = C - A,
//     B = k I (l x a) / |l x a|^2 (l.a/|a| - l.c/|c|),   k = mu0/(4 pi).
// One thread per grid point, segments summed in input order (FP64).
__global__ void wire_potential_kernel(double *V, const Geom g, const double *seg, int nseg,
                                      double bx, double by, double bz, double k, double vs,
                                      double voff)
{
    const long long n = g.plane * g.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i & (g.nx - 1));
        const int y = (int)((i >> g.lgnx) & (g.ny - 1));
        const int z = (int)(i >> (g.lgnx + g.lgny));
        const double px = g.box[0] + x * (g.box[1] - g.box[0]) / g.nx;
        const double py = g.box[2] + y * (g.box[3] - g.box[2]) / g.ny;
        const double pz = g.box[4] + z * (g.box[5] - g.box[4]) / g.nz;
        double b0 = bx, b1 = by, b2 = bz;
        for (int m = 0; m < nseg; ++m) {
            const double *s = seg + 7 * m;
            const double lx = s[3] - s[0], ly = s[4] - s[1], lz = s[5] - s[2];
            const double ax = px - s[0], ay = py - s[1], az = pz - s[2];
            const double cx = px - s[3], cy = py - s[4], cz = pz - s[5];
            const double nx_ = ly * az - lz * ay, ny_ = lz * ax - lx * az, nz_ = lx * ay - ly * ax;
            const double n2 = nx_ * nx_ + ny_ * ny_ + nz_ * nz_;
            if (n2 == 0.0) continue;                        // on the segment's line
            const double ra = sqrt(ax * ax + ay * ay + az * az);
            const double rc = sqrt(cx * cx + cy * cy + cz * cz);
            const double f = k * s[6] * ((lx * ax + ly * ay + lz * az) / ra -
                                         (lx * cx + ly * cy + lz * cz) / rc) / n2;
            b0 += f * nx_;
            b1 += f * ny_;
            b2 += f * nz_;
        }
        V[i] = vs * sqrt(b0 * b0 + b1 * b1 + b2 * b2) - voff;
    }
}

void launch_wire_potential(double *V, const Geom &g, const double *seg, int nseg,
                           const double bias[3], double k, double vs, double voff, cudaStream_t st)
{
    wire_potential_kernel<<<148 * 8, 256, 0, st>>>(V, g, seg, nseg, bias[0], bias[1], bias[2], k,
                                                   vs, voff);
}

// ------------------------------------- complex128 <-> double-float storage
// In place: a complex128 value and its double-float form both take 16 bytes.
__global__ void c128_to_df_kernel(double2 *p, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = p[i];
        df2 w;
        w.x = df(v.x);
        w.y = df(v.y);
        reinterpret_cast<df2 *>(p)[i] = w;
    }
}
__global__ void df_to_c128_kernel(double2 *p, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const df2 w = reinterpret_cast<const df2 *>(p)[i];
        p[i] = make_double2(static_cast<double>(w.x), static_cast<double>(w.y));
    }
}
__global__ void c128_to_df_copy_kernel(const double2 *src, df2 *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        df2 w;
        w.x = df(v.x);
        w.y = df(v.y);
        dst[i] = w;
    }
}

void launch_c128_to_df(void *psi, long long n, cudaStream_t st)
{
    c128_to_df_kernel<<<1184, 256, 0, st>>>(static_cast<double2 *>(psi), n);
}
void launch_df_to_c128(void *psi, long long n, cudaStream_t st)
{
    df_to_c128_kernel<<<1184, 256, 0, st>>>(static_cast<double2 *>(psi), n);
}
void launch_c128_to_df_copy(const void *src, void *dst, long long n, cudaStream_t st)
{
    c128_to_df_copy_kernel<<<1184, 256, 0, st>>>(static_cast<const double2 *>(src),
                                                 static_cast<df2 *>(dst), n);
}

// -------------------------------------------------------------- launchers
int xy_grid(const Geom &g) { return g.batch * g.nz * g.P; }
int z_grid(const Geom &g) { return g.batch << g.lgzt; }
size_t xy_smem(const Geom &g, int esize) { return (size_t)g.Ly * g.pitchXY * esize; }
size_t z_smem(const Geom &g, int esize) { return (size_t)g.nz * g.pitchZ * esize; }
int mask_blocks(const Geom &g)
{
    const long long n = g.plane * g.nz;
    long long nb = (n + 8191) / 8192;
    return (int)(nb < 4096 ? nb : 4096);
}

template <class T> constexpr int maxv() { return sizeof(T) == 4 ? 32 : 16; }

template <class T> void launch_xy(const XYArgs<T> &a, cudaStream_t st)
{
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(xy_pass_kernel<T, maxv<T>()>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        configured = true;
    }
    xy_pass_kernel<T, maxv<T>()><<<xy_grid(a.g), kNT, xy_smem(a.g, sizeof(Cx<T>)), st>>>(a);
}

template <class T> void launch_z(const ZArgs<T> &a, cudaStream_t st)
{
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(z_pass_kernel<T, maxv<T>()>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        configured = true;
    }
    z_pass_kernel<T, maxv<T>()><<<z_grid(a.g), kNT, z_smem(a.g, sizeof(Cx<T>)), st>>>(a);
}

void launch_reduce(const double *partials, int nblk, int nq, double *out, cudaStream_t st)
{
    reduce_partials_kernel<<<1, kNT, 0, st>>>(partials, nblk, nq, out);
}

void launch_norm_scale(const double *partials, int nblk, double dV, double *scale,
                       cudaStream_t st)
{
    norm_scale_kernel<<<1, kNT, 0, st>>>(partials, nblk, dV, scale);
}

template <class T> void launch_scale(Cx<T> *psi, long long n, const double *scale, cudaStream_t st)
{
    long long nb = (n + kNT - 1) / kNT;
    scale_kernel<T><<<(int)(nb < 65535 ? nb : 65535), kNT, 0, st>>>(psi, n, scale);
}

template <class T>
void launch_mask(const Cx<T> *psi, Cx<T> *lam, const Geom &g, const double *xcj, double hw,
                 double *partials, int nblk, cudaStream_t st)
{
    const long long n = g.plane * g.nz;
    const long long chunk = (n + nblk - 1) / nblk;
    mask_kernel<T><<<nblk, kNT, 0, st>>>(psi, lam, g, xcj, hw, partials, chunk);
}


template <class T>
void launch_density_xz(const Cx<T> *psi, const Geom &g, double dy, double *out, cudaStream_t st)
{
    const long long n = (long long)g.batch * g.nz * g.nx;
    density_xz_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(psi, g, dy, out);
}

template void launch_density_xz<float>(const Cx<float> *, const Geom &, double, double *, cudaStream_t);
template void launch_density_xz<double>(const Cx<double> *, const Geom &, double, double *, cudaStream_t);
template void launch_xy<df>(const XYArgs<df> &, cudaStream_t);
template void launch_z<df>(const ZArgs<df> &, cudaStream_t);
template void launch_scale<df>(Cx<df> *, long long, const double *, cudaStream_t);
template void launch_xy<float>(const XYArgs<float> &, cudaStream_t);
template void launch_xy<double>(const XYArgs<double> &, cudaStream_t);
template void launch_z<float>(const ZArgs<float> &, cudaStream_t);
template void launch_z<double>(const ZArgs<double> &, cudaStream_t);
template void launch_scale<float>(Cx<float> *, long long, const double *, cudaStream_t);
template void launch_scale<double>(Cx<double> *, long long, const double *, cudaStream_t);
template void launch_mask<float>(const Cx<float> *, Cx<float> *, const Geom &, const double *,
                                 double, double *, int, cudaStream_t);
template void launch_mask<double>(const Cx<double> *, Cx<double> *, const Geom &, const double *,
                                  double, double *, int, cudaStream_t);

}  // namespace ctap
