// packed_passes.cu -- the steady complex64 passes in packed FP32 arithmetic.
//
// B300 (the sm_100 family) issues one instruction for a PAIR of FP32 adds,
// multiplies or fused multiply-adds (add/mul/fma.rn.f32x2): twice the FP32
// work per issue slot of the scalar forms, at the same FP32 pipe rate.  The
// specialised passes in fast_passes.cu are bound by instruction issue and
// shared-memory traffic, not by HBM, so the passes here hold the values of
// TWO transform lines per thread in structure-of-arrays form -- one FP32
// pair for the real parts, one for the imaginary parts -- and run every
// butterfly, lifted rotation and scaling on both lines with one packed
// instruction.  The multiplications by +-i inside the radix-2 butterflies
// become free (a swap of the two pairs and a choice of add or subtract).
//
// Same mathematics, HBM layout, tables and lifting scheme as the other
// passes (mixed representation between passes: natural kx, natural k',
// rows j P + r; every twiddle a three-shear rotation), so plans mix them
// freely; the results differ from the scalar passes by FP32 rounding only.
//
// Z pass (z_pk_kernel, complex64, nz = 1024, 16-column tiles of P = 4 row
// classes x W = 4 columns; the geometry of 256 x 256 planes):
//   z = 256 a + 16 b + c, kz = k0 + 4 k1 + 64 k2 (decimation in frequency)
//   A   cross twiddle + P-point DFT over the row classes (finishes ky), the
//       kinetic rotation of the column's (kx, ky) (constant along z), the
//       radix-4 DFT over a and the twiddle exp(-2 pi i b k0/64);
//   B   radix-16 DFT over b and the twiddle exp(-2 pi i c (k0 + 4 k1)/1024);
//   C   radix-16 DFT over c, the kz kinetic rotation with the sign, 1/N and
//       the (kx, ky) sign, then the exact mirror back;
//   B'  mirror of B;  A'  mirror of A (without the kinetic rotation), and
//       16-byte streaming stores.
// Each twiddle layer sits at the end of the phase that produces its inputs
// (and at the start of the mirror phase): the radix-4 phase needs only
// three table entries per task, and the middle phase none.
// A thread holds 16 values of each of two adjacent tile columns (32 complex
// values, 64 registers); 512 threads cover a tile per phase, 16 warps per
// SM.  The tile lives in the same ring of 128-row chunks as z_ring_kernel
// and the next tile's copies are issued between phases.
//
// XY pass (xy_pk_kernel, complex64, nx = 256, 64-row tiles): three register
// phases per direction (x = 16 x 16, y = 2 x 32) on 64 values per thread,
// 256 threads; 10 passes of a tile through shared memory against the 14 of
// the four-phase scalar passes (details at the kernel).
#include <algorithm>
#include <cstdlib>

#include "../../include/ctap.h"
#include "bounds.cuh"
#include "packed_passes.cuh"

namespace ctap {

namespace {

// ------------------------------------------------------------ pair arithmetic
__device__ __forceinline__ float2 pk(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
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

// Two complex values (one from each of two lines): x = (re_a, re_b),
// y = (im_a, im_b).
struct Q {
    float2 x, y;
};

__device__ __forceinline__ Q qadd(const Q &a, const Q &b) { return Q{add2(a.x, b.x), add2(a.y, b.y)}; }
__device__ __forceinline__ Q qsub(const Q &a, const Q &b) { return Q{sub2(a.x, b.x), sub2(a.y, b.y)}; }

// rotation of both values by the angles whose lifting coefficients are the
// pairs p = -tan(phi/2), u = sin(phi); qrot_b is its exact mirror
__device__ __forceinline__ void qrot_f(Q &v, float2 p, float2 u)
{
    v.x = fma2(p, v.y, v.x);
    v.y = fma2(u, v.x, v.y);
    v.x = fma2(p, v.y, v.x);
}
__device__ __forceinline__ void qrot_b(Q &v, float2 p, float2 u)
{
    const float2 mp = neg2(p), mu = neg2(u);
    v.x = fma2(mp, v.y, v.x);
    v.y = fma2(mu, v.x, v.y);
    v.x = fma2(mp, v.y, v.x);
}
__device__ __forceinline__ void qscale(Q &v, float2 s)
{
    v.x = mul2(s, v.x);
    v.y = mul2(s, v.y);
}
// a table twiddle (the same for both lines): s * rotate(phi), and its mirror
__device__ __forceinline__ void qlift_f(Q &v, const Lift<float> &w)
{
    qrot_f(v, pk(w.p), pk(w.u));
    qscale(v, pk(w.s));
}
__device__ __forceinline__ void qlift_b(Q &v, const Lift<float> &w)
{
    qscale(v, pk(w.s));
    qrot_b(v, pk(w.p), pk(w.u));
}

// Forward R-point DFT (exp(-2 pi i jk/R)) of v[OFF + k ST] on both lines,
// radix-2 decimation in frequency with the fixed rotations of RegTw; output
// frequency k lands in v[OFF + brev(k, R) ST].  The factor -i of a butterfly
// is taken before its rotation (the two commute), as a swap of the pairs.
template <int R, int OFF, int ST> __device__ __forceinline__ void qdft_fwd(Q *v)
{
    if constexpr (R > 1) {
        constexpr int H = R / 2;
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            const Q a = v[OFF + j * ST], b = v[OFF + (j + H) * ST];
            v[OFF + j * ST] = qadd(a, b);
            Q d;
            if constexpr (W::mode >= 2) {          // -i (a - b)
                d.x = sub2(a.y, b.y);
                d.y = sub2(b.x, a.x);
            } else {
                d = qsub(a, b);
            }
            if constexpr (W::mode == 1 || W::mode == 3) qrot_f(d, pk(float(W::p)), pk(float(W::u)));
            v[OFF + (j + H) * ST] = d;
        });
        qdft_fwd<H, OFF, ST>(v);
        qdft_fwd<H, OFF + H * ST, ST>(v);
    }
}

// Exact mirror of qdft_fwd: input in bit-reversed register order, output in
// natural order, R times the inverse DFT.
template <int R, int OFF, int ST> __device__ __forceinline__ void qdft_inv(Q *v)
{
    if constexpr (R > 1) {
        constexpr int H = R / 2;
        qdft_inv<H, OFF, ST>(v);
        qdft_inv<H, OFF + H * ST, ST>(v);
        sfor<H>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            using W = RegTw<R, j>;
            const Q a = v[OFF + j * ST];
            Q e = v[OFF + (j + H) * ST];
            if constexpr (W::mode == 1 || W::mode == 3) qrot_b(e, pk(float(W::p)), pk(float(W::u)));
            if constexpr (W::mode >= 2) {          // a +- i e
                v[OFF + j * ST] = Q{sub2(a.x, e.y), add2(a.y, e.x)};
                v[OFF + (j + H) * ST] = Q{add2(a.x, e.y), sub2(a.y, e.x)};
            } else {
                v[OFF + j * ST] = qadd(a, e);
                v[OFF + (j + H) * ST] = qsub(a, e);
            }
        });
    }
}

// shared-memory pieces: 16 bytes, two adjacent columns of one tile row.
// AoS (as copied from HBM): re0 im0 re1 im1.  SoA (after phase A): re0 re1
// im0 im1.
__device__ __forceinline__ Q ld_aos(const float2 *p)
{
    const float4 w = *reinterpret_cast<const float4 *>(p);
    return Q{make_float2(w.x, w.z), make_float2(w.y, w.w)};
}
__device__ __forceinline__ Q ld_soa(const float2 *p)
{
    const float4 w = *reinterpret_cast<const float4 *>(p);
    return Q{make_float2(w.x, w.y), make_float2(w.z, w.w)};
}
__device__ __forceinline__ void st_soa(float2 *p, const Q &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.x.x, v.x.y, v.y.x, v.y.y);
}

// Checked forms (bounds.cuh): off indexes float2 values of a buffer of lim
// values; a 16-byte access covers off and off + 1.  Unchecked in the normal
// build.
template <int SITE> __device__ __forceinline__ Q ld_aos_c(const float2 *b, int off, int lim)
{
    Q v{};
    if (CTAP_BOUNDS(SITE, off, lim - 1)) v = ld_aos(b + off);
    return v;
}
template <int SITE> __device__ __forceinline__ Q ld_soa_c(const float2 *b, int off, int lim)
{
    Q v{};
    if (CTAP_BOUNDS(SITE, off, lim - 1)) v = ld_soa(b + off);
    return v;
}
template <int SITE> __device__ __forceinline__ void st_soa_c(float2 *b, int off, int lim, const Q &v)
{
    if (CTAP_BOUNDS(SITE, off, lim - 1)) st_soa(b + off, v);
}
template <int SITE> __device__ __forceinline__ float4 ld4_c(const float2 *b, int off, int lim)
{
    float4 v{};
    if (CTAP_BOUNDS(SITE, off, lim - 1)) v = *reinterpret_cast<const float4 *>(b + off);
    return v;
}
template <int SITE> __device__ __forceinline__ void st4_c(float2 *b, int off, int lim, const float4 &v)
{
    if (CTAP_BOUNDS(SITE, off, lim - 1)) *reinterpret_cast<float4 *>(b + off) = v;
}
template <int SITE> __device__ __forceinline__ float2 ld2_c(const float2 *b, int off, int lim)
{
    float2 v{};
    if (CTAP_BOUNDS(SITE, off, lim)) v = b[off];
    return v;
}
template <int SITE> __device__ __forceinline__ void st2_c(float2 *b, int off, int lim, const float2 &v)
{
    if (CTAP_BOUNDS(SITE, off, lim)) b[off] = v;
}
// table entry e of a table of n entries
template <int SITE, class L> __device__ __forceinline__ L tab_c(const L *t, long long e, long long n)
{
    L v{};
    if (CTAP_BOUNDS(SITE, e, n)) v = t[e];
    return v;
}

// The thread index through an opaque move.  A mirror phase addresses the
// same shared-memory positions (and table entries) as its forward phase;
// taken from the plain index, the compiler keeps those values live from the
// forward phase through every phase in between, which overflows the
// 128-register budget of 512 threads into local memory.  The mirror phase
// phases that close the longest such spans (B' and A' in the Z pass, A' in
// the XY pass) take their index through this move instead: no spills
// (ptxas -v).
__device__ __forceinline__ int phase_tid()
{
    int t;
    asm volatile("mov.u32 %0, %1;" : "=r"(t) : "r"((int)threadIdx.x));
    return t;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int kZpkNT = 512;        // threads of the packed Z pass
constexpr int kZpkCHZ = 128;       // z-rows per ring chunk
constexpr int kZpkNRING = 12;      // ring chunks (a tile is eight)

}  // namespace

// =============================================================== Z (packed)
// Persistent: one CTA per SM walks over the tiles blockIdx.x + i gridDim.x.
// kin_xy: lifted rotations of exp(-i (kx^2 + ky^2) dt/2), [ny][nx] (FP64
// generated, rounded once).  Real time only.
__global__ void __launch_bounds__(kZpkNT, 1) z_pk_kernel(const ZArgs<float> a, int ntiles)
{
    constexpr int NZ = 1024, P = 4, W = 4, C = P * W, NT = kZpkNT;
    constexpr int CHZ = kZpkCHZ, NCH = NZ / CHZ, NRING = kZpkNRING, CHE = CHZ * C;
    using T = float;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *ring = reinterpret_cast<float2 *>(smraw);
    Lift<T> *wz = reinterpret_cast<Lift<T> *>(ring + NRING * CHE);   // exp(-2 pi i e/1024)
    Lift<T> *kz = wz + NZ;                                            // kz kinetic, s/N
    // per-tile tables, double buffered: [0..15] (kx, ky) kinetic rotation of
    // tile column k2 W + x (x fastest), [16..18] cross twiddles r = 1..3
    __shared__ Lift<T> tabs[2][C + P - 1];
    const Geom &g = a.g;
    const Lift<T> *kxy = static_cast<const Lift<T> *>(a.kin_xy);
    const int t0 = threadIdx.x;
    constexpr int RINGE = NRING * CHE;                 // float2 values in the ring
    [[maybe_unused]] const long long NTOT = (long long)g.batch * g.rstride;   // float2 values of psi
    const int G = gridDim.x;
    const int nmine = (ntiles - (int)blockIdx.x + G - 1) / G;
    const int nblk_mask = (1 << g.nblk_lg) - 1;

    auto slot_of = [](int i, int c) {
        int s = (i % 3) * NCH + c;
        s -= (s >= NRING) ? NRING : 0;
        s -= (s >= NRING) ? NRING : 0;
        return s;
    };
    // element offset of piece q (columns 2q, 2q + 1) of z-row zz in chunk slot
    // s.  Swizzle: the 32-byte group of a row class moves with z mod 4 and
    // its 16-byte halves swap with bit 2 of z.  A 16-byte shared access is
    // served eight lanes at a time; the eight lanes of phases A and A' are
    // four z-rows x two halves, of phases B and C and of the copies one
    // z-row's eight pieces: every group meets eight distinct bank groups.
    auto piece = [](int s, int zz, int q) {
        return s * CHE + (zz % CHZ) * C + 2 * (q ^ (((zz & 3) << 1) | ((zz >> 2) & 1)));
    };

    // asynchronous copy of chunks [c0, c1) of the i-th tile: thread t moves
    // piece (row class r, half h) of z-rows czl + 64 m of each chunk
    const int ch = t0 & 1, cr = (t0 >> 1) & (P - 1), czl = t0 >> 3;
    auto issue = [&](int i, int c0, int c1) {
        const int tile = blockIdx.x + i * G;
        const int tl = tile & ((1 << g.lgzt) - 1);
        const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
        long long so = (long long)(tile >> g.lgzt) * g.rstride + ((long long)(kp * P + cr) << g.lgnx) +
                       b * W + 2 * ch + (long long)(c0 * CHZ + czl) * g.plane;
        const long long zstep = (long long)(NT / 8) * g.plane;
        for (int c = c0; c < c1; ++c) {
            const int s = slot_of(i, c);
#pragma unroll
            for (int m = 0; m < CHZ / (NT / 8); ++m) {
                const int zz = c * CHZ + czl + m * (NT / 8);
                const int d = piece(s, zz, 2 * cr + ch);
                if (CTAP_BOUNDS(1, d, RINGE - 1) && CTAP_BOUNDS(2, so, NTOT - 1))
                    cp_async16(ring + d, a.src + so);
                so += zstep;
            }
        }
    };
    // per-tile tables: fetched from global memory into a register early in a
    // phase and stored to shared memory at its end, so the global latency
    // hides behind that phase's arithmetic (a direct global -> shared copy
    // at the top of a tile held the whole CTA at the next barrier)
    auto fetch_tabs = [&](int i) {
        Lift<T> v{};
        if (t0 < C + P - 1) {
            const int t = t0;
            const int tile = blockIdx.x + i * G;
            const int tl = tile & ((1 << g.lgzt) - 1);
            const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
            if (t < C) {
                const int kx = b * W + (t & (W - 1)), ky = kp + ((t / W) << g.lgLy);
                v = tab_c<3>(kxy, ((long long)ky << g.lgnx) + kx, (long long)g.nx * g.ny);
            } else {
                v = a.tw[g.cross_off + (((t - C + 1) * kp) & (g.ny - 1))];
            }
        }
        return v;
    };
    auto put_tabs = [&](int i, const Lift<T> &v) {
        if (t0 < C + P - 1) tabs[i & 1][t0] = v;
    };

    if (nmine > 0) {
        issue(0, 0, NCH);
        put_tabs(0, fetch_tabs(0));
    }
    cp_async_commit();
    for (int e = t0; e < NZ; e += NT) {
        wz[e] = a.tw[g.fast_z_off + e];
        Lift<T> k = a.kin[g.nx + g.ny + e];
        k.s *= a.inv_n;                      // 1/N of the unnormalised transforms
        kz[e] = k;
    }

    for (int i = 0; i < nmine; ++i) {
        const int tile = blockIdx.x + i * G;
        const int tl = tile & ((1 << g.lgzt) - 1);
        const int kp = tl >> g.nblk_lg, b = tl & nblk_mask;
        const long long colbase = (long long)(tile >> g.lgzt) * g.rstride +
                                  ((long long)(kp * P) << g.lgnx) + b * W;
        const bool more = i + 1 < nmine;
        cp_async_wait_all();
        __syncthreads();                               // tile i and its tables visible
        const Lift<T> *tb = tabs[i & 1];
        // ring slot of chunk c of tile i (computed, not indexed: a register
        // array indexed at run time would live in local memory)
        const int sbase = (i % 3) * NCH;
        auto sl = [sbase](int c) { const int s = sbase + c; return s >= NRING ? s - NRING : s; };

        // ---- A: cross DFT over r, (kx, ky) kinetic rotation, radix-4 over a
        {
            const int t = threadIdx.x;
            const int h = t & 1, zl = t >> 1;
            Lift<T> tw64[3];
#pragma unroll
            for (int k0 = 1; k0 < 4; ++k0) tw64[k0 - 1] = tab_c<16>(wz, 16 * (zl >> 4) * k0, NZ);
            Q v[4][4];                                 // [a -> k0][r -> k2y]
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) {
                const int zz = 256 * aa + zl;
#pragma unroll
                for (int r = 0; r < P; ++r) v[aa][r] = ld_aos_c<4>(ring, piece(sl(zz / CHZ), zz, 2 * r + h), RINGE);
            }
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) {
#pragma unroll
                for (int r = 1; r < P; ++r) qlift_f(v[aa][r], tb[C + r - 1]);
                qdft_fwd<4, 0, 1>(v[aa]);              // v[aa][brev(k2y)]
            }
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) {
                const Lift<T> &l0 = tb[k2 * W + 2 * h], &l1 = tb[k2 * W + 2 * h + 1];
                const float2 p = make_float2(l0.p, l1.p), u = make_float2(l0.u, l1.u);
                Q col[4];
#pragma unroll
                for (int aa = 0; aa < 4; ++aa) {
                    col[aa] = v[aa][brev(k2, 4)];
                    qrot_f(col[aa], p, u);
                }
                qdft_fwd<4, 0, 1>(col);                // col[brev(k0)]
#pragma unroll
                for (int k0 = 0; k0 < 4; ++k0) {
                    // twiddle of the next stage, exp(-2 pi i b k0/64), b = zl/16
                    if (k0 > 0) qlift_f(col[brev(k0, 4)], tw64[k0 - 1]);
                    const int zz = 256 * k0 + zl;
                    st_soa_c<5>(ring, piece(sl(zz / CHZ), zz, 2 * k2 + h), RINGE, col[brev(k0, 4)]);
                }
            }
        }
        if (more) issue(i + 1, 0, 1);
        __syncthreads();

        // ---- B: radix-16 over b, then the twiddle of the last stage,
        //      exp(-2 pi i c (k0 + 4 k1)/1024); the next tile's tables
        {
            const Lift<T> ntab = more ? fetch_tabs(i + 1) : Lift<T>{};
            const int t = threadIdx.x;
            const int q = t & 7, c = (t >> 3) & 15, k0 = t >> 7;
            Q v[16];
#pragma unroll
            for (int bb = 0; bb < 16; ++bb) {
                const int zz = 256 * k0 + 16 * bb + c;
                v[bb] = ld_soa_c<6>(ring, piece(sl(zz / CHZ), zz, q), RINGE);
            }
            qdft_fwd<16, 0, 1>(v);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                Q &w = v[brev(k1, 16)];
                qlift_f(w, tab_c<7>(wz, c * (k0 + 4 * k1), NZ));
                const int zz = 256 * k0 + 16 * k1 + c;
                st_soa_c<8>(ring, piece(sl(zz / CHZ), zz, q), RINGE, w);
            }
            if (more) put_tabs(i + 1, ntab);
        }
        if (more) issue(i + 1, 1, 2);
        __syncthreads();

        // ---- C: radix-16 over c, the kz kinetic factor, and back.  A warp
        //      spans four consecutive m (k0 fastest after the piece) so that
        //      its kinetic table reads fall on distinct banks.
        {
            const int t = threadIdx.x;
            const int q = t & 7, k0 = (t >> 3) & 3, k1 = t >> 5;
            const int m = k0 + 4 * k1;
            const int zr = 256 * k0 + 16 * k1;         // 16 consecutive rows, one chunk
            const int s = sl(zr / CHZ);
            // sign of the (kx, ky) rotation of the two columns
            const int k2y = q >> 1, x0 = 2 * (q & 1);
            const float2 sxy = make_float2(tb[k2y * W + x0].s, tb[k2y * W + x0 + 1].s);
            Q v[16];
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) v[cc] = ld_soa_c<9>(ring, piece(s, zr + cc, q), RINGE);
            qdft_fwd<16, 0, 1>(v);                     // v[brev(k2)]: kz = m + 64 k2
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const Lift<T> kk = tab_c<10>(kz, m + 64 * k2, NZ);
                Q &w = v[brev(k2, 16)];
                qrot_f(w, pk(kk.p), pk(kk.u));
                qscale(w, mul2(sxy, pk(kk.s)));
            }
            qdft_inv<16, 0, 1>(v);
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) st_soa_c<11>(ring, piece(s, zr + cc, q), RINGE, v[cc]);
        }
        if (more) issue(i + 1, 2, 3);
        __syncthreads();

        // ---- B': mirror of B
        {
            const int t = phase_tid();
            const int q = t & 7, c = (t >> 3) & 15, k0 = t >> 7;
            Q v[16];
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const int zz = 256 * k0 + 16 * k1 + c;
                Q w = ld_soa_c<12>(ring, piece(sl(zz / CHZ), zz, q), RINGE);
                qlift_b(w, tab_c<13>(wz, c * (k0 + 4 * k1), NZ));
                v[brev(k1, 16)] = w;
            }
            qdft_inv<16, 0, 1>(v);
#pragma unroll
            for (int bb = 0; bb < 16; ++bb) {
                const int zz = 256 * k0 + 16 * bb + c;
                st_soa_c<14>(ring, piece(sl(zz / CHZ), zz, q), RINGE, v[bb]);
            }
        }
        if (more) issue(i + 1, 3, 4);
        cp_async_commit();
        __syncthreads();

        // ---- A': read the task back (frees the tile's ring slots), mirror of A
        //      without the kinetic rotation, streaming stores.  Lanes 2l and
        //      2l + 1 hold the two 16-byte halves of one 32-byte row segment,
        //      so a warp store writes 16 whole sectors (with the halves in
        //      different warps it wrote 32 half sectors: 0.55 against 0.35 ms
        //      for the pass without its stores)
        {
            const int t = phase_tid();
            const int h = t & 1, zl = t >> 1;
            Q v[4][4];                                 // [k0][k2y] as stored
#pragma unroll
            for (int k0 = 0; k0 < 4; ++k0) {
                const int zz = 256 * k0 + zl;
#pragma unroll
                for (int k2 = 0; k2 < P; ++k2) v[k0][k2] = ld_soa_c<15>(ring, piece(sl(zz / CHZ), zz, 2 * k2 + h), RINGE);
            }
            Lift<T> cw[P];
#pragma unroll
            for (int r = 1; r < P; ++r) cw[r] = tb[C + r - 1];
            Lift<T> tw64[3];
#pragma unroll
            for (int k0 = 1; k0 < 4; ++k0) tw64[k0 - 1] = tab_c<16>(wz, 16 * (zl >> 4) * k0, NZ);
            __syncthreads();                           // every slot of tile i is free
            if (more) issue(i + 1, NCH / 2, NCH);
            cp_async_commit();
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) {
                Q col[4];
#pragma unroll
                for (int k0 = 0; k0 < 4; ++k0) {
                    col[brev(k0, 4)] = v[k0][k2];
                    if (k0 > 0) qlift_b(col[brev(k0, 4)], tw64[k0 - 1]);
                }
                qdft_inv<4, 0, 1>(col);                // col[a]
#pragma unroll
                for (int aa = 0; aa < 4; ++aa) v[aa][k2] = col[aa];
            }
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) {
                Q row[4];
#pragma unroll
                for (int k2 = 0; k2 < P; ++k2) row[brev(k2, 4)] = v[aa][k2];
                qdft_inv<4, 0, 1>(row);                // row[r]
#pragma unroll
                for (int r = 1; r < P; ++r) qlift_b(row[r], cw[r]);
                const int zz = 256 * aa + zl;
                const long long po = colbase + (long long)zz * g.plane + 2 * h;
#pragma unroll
                for (int r = 0; r < P; ++r) {
                    const long long o = po + ((long long)r << g.lgnx);
                    if (CTAP_BOUNDS(17, o, NTOT - 1))
                        __stcs(reinterpret_cast<float4 *>(a.dst + o),
                               make_float4(row[r].x.x, row[r].y.x, row[r].x.y, row[r].y.y));
                }
            }
        }
    }
    cp_async_wait_all();
}

namespace {

// potential factor exp(-i th) as lifting pairs for |th| <= 0.16 (TIER 2:
// series through the fifth order) or |th| <= 0.5 (TIER 1: through th^11 for
// p and th^9 for u), own odd Taylor series of tan(th/2) and -sin(th)
template <int TIER> __device__ __forceinline__ void qkick_coef(float2 th, float2 &p, float2 &u)
{
    const float2 t2 = mul2(th, th);
    if constexpr (TIER == 2) {
        // u = -sin th = th (-1 + t2/6 - t2^2/120), p = tan(th/2) = th (1/2 + t2/24 + t2^2/240)
        u = mul2(th, fma2(t2, fma2(t2, pk(-1.0f / 120.0f), pk(1.0f / 6.0f)), pk(-1.0f)));
        p = mul2(th, fma2(t2, fma2(t2, pk(1.0f / 240.0f), pk(1.0f / 24.0f)), pk(0.5f)));
    } else {
        float2 su = fma2(t2, pk(-1.0f / 362880.0f), pk(1.0f / 5040.0f));
        su = fma2(t2, su, pk(-1.0f / 120.0f));
        su = fma2(t2, su, pk(1.0f / 6.0f));
        u = mul2(th, fma2(t2, su, pk(-1.0f)));
        // tan(h), h = th/2: h + h^3/3 + 2h^5/15 + 17h^7/315 + 62h^9/2835 + 1382h^11/155925
        float2 sp = fma2(t2, pk(1382.0f / 155925.0f / 2048.0f), pk(62.0f / 2835.0f / 512.0f));
        sp = fma2(t2, sp, pk(17.0f / 315.0f / 128.0f));
        sp = fma2(t2, sp, pk(2.0f / 15.0f / 32.0f));
        sp = fma2(t2, sp, pk(1.0f / 3.0f / 8.0f));
        p = mul2(th, fma2(t2, sp, pk(0.5f)));
    }
}


}  // namespace

// ============================================================== XY (packed)
// Steady real-time XY pass (nx = 256, 64-row tiles, product or separable
// potential, merged half-kicks, in place), persistent with the ring of three 32-row
// half buffers of xy_ring_kernel, in three register phases per direction
// (the scalar passes take four), so a tile passes through shared memory 10
// times instead of 14:
//   x = 16 x1 + x2, kx = k1 + 16 k2 (as xy_ring_kernel); y = 2 j1 + j2 (j1 < 32),
//   k' = k1 + 32 k2 (k2 < 2)
//   A   inverse x, last stage (radix 16 over k2 for fixed k1, from the ring,
//       rows rw and rw + 32 paired), inverse twiddle exp(2 pi i x2 k1/256);
//   B   inverse x, first stage (radix 16 over the 16 contiguous positions of
//       one x2) and inverse y, last stage (radix 2 over the rows k1, k1 + 32)
//       with the inverse twiddle exp(2 pi i j2 k1/64);
//   C   inverse y, first stage (radix 32 over the 32 rows of one half buffer),
//       the potential factor, forward radix 32;
//   B', A' the mirrors (A' stores to HBM).
// 256 threads, 64 complex values (32 pairs) per thread in B and C, two
// 32-value tasks in A and A'.  Pairs: A and A' pair rows rw and rw + 32; B,
// C and B' pair positions p and p + 128 of one row, kept "split" in shared
// memory: the pair of real parts at position p, the pair of imaginary parts
// at position p + 128.
constexpr int kXpkNT = 256;

template <int TIER, bool SEP>
__global__ void __launch_bounds__(kXpkNT, 1) xy_pk_kernel(const XYArgs<float> a, int ntiles)
{
    constexpr int NX = 256, LY = 64, NT = kXpkNT;
    constexpr int PITCH = NX + 2;                // complex values per row (16-byte rows)
    constexpr int HR = LY / 2;                   // rows per half buffer
    constexpr int HB = HR * PITCH;               // complex values per half buffer
    constexpr int PPR = NX / 2;                  // 16-byte pieces per row
    constexpr int RPI = NT / PPR;                // rows per copy round (2)
    constexpr int NCR = HR / RPI;                // copy rounds per half (16)
    using T = float;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *bufs = reinterpret_cast<float2 *>(smraw);
    Lift<T> *wx = reinterpret_cast<Lift<T> *>(bufs + 3 * HB);   // [x2 16 + k1] = exp(-2 pi i k1 x2/256)
    Lift<T> *wy = wx + NX;                                      // exp(-2 pi i e/64)
    // angle of the kick at (x, y) of the tile's plane z: g(y) h(x) + thz
    // (product form) or h(x) + g(y) (separable form)
    __shared__ T gtab[2][LY];                    // product: g(y); separable: (Vy(y) + Vz(z)) tau
    __shared__ float2 htab[2][NX / 2];           // product: H(x, z) tau; separable: Vx(x) tau
    __shared__ T thzs[2];                        // product: Vz(z) tau

    const Geom &g = a.g;
    const Kick<T> &k = a.k;
    const int t0 = threadIdx.x;
    const int G = gridDim.x;
    const int nmine = (ntiles - (int)blockIdx.x + G - 1) / G;
    const T tau = k.tau_full;
    constexpr int BUFE = 3 * HB;
    [[maybe_unused]] const long long NTOT = (long long)g.batch * g.rstride;
    auto unswx = [](int q) { return q / 16 + 16 * (q % 16); };       // position -> x
    auto half_buf = [&](int i, int h) { return ((2 * i + h) % 3) * HB; };
    const int cpiece = t0 % PPR, crow = t0 / PPR;
    auto issue = [&](int i, int h, int m0, int m1) {
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        long long so = (long long)z * g.plane + ((long long)((h * HR + crow + RPI * m0) * g.P + r) << g.lgnx) +
                       2 * cpiece;
        int d = half_buf(i, h) + (crow + RPI * m0) * PITCH + 2 * cpiece;
        const long long rstep = (long long)(RPI * g.P) << g.lgnx;
        for (int m = m0; m < m1; ++m) {
            if (CTAP_BOUNDS(41, d, BUFE - 1) && CTAP_BOUNDS(42, so, NTOT - 1))
                cp_async16(bufs + d, a.src + so);
            so += rstep;
            d += RPI * PITCH;
        }
    };
    // per-tile tables (the row and column factors of the kick angle, the
    // z-only phase): fetched into registers early in phase B and stored to
    // shared memory at its end (the global latency hides behind B's
    // arithmetic).  Separable form: the angles are formed from the FP64 axis
    // potentials and rounded once.
    struct Tabs { float h0, h1, gy, vz; };
    auto fetch_tabs = [&](int i) {
        Tabs v{0.0f, 0.0f, 0.0f, 0.0f};
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        if constexpr (SEP) {
            const double *Vs = a.rd.Vsep;              // [nx | ny | nz]
            const long long nv = (long long)g.nx + g.ny + g.nz;
            const double td = (double)tau;
            if (t0 < LY)
                v.gy = (float)((tab_c<57>(Vs, g.nx + r + t0 * g.P, nv) +
                                tab_c<57>(Vs, g.nx + g.ny + (z & (g.nz - 1)), nv)) * td);
            if (t0 < NX / 2) {
                v.h0 = (float)(tab_c<58>(Vs, unswx(t0), nv) * td);
                v.h1 = (float)(tab_c<58>(Vs, unswx(t0 + NX / 2), nv) * td);
            }
        } else {
            if (t0 < LY) v.gy = tab_c<59>(k.g, r + t0 * g.P, g.ny);
            if (t0 < NX / 2) {
                const long long hz = (long long)z * g.nx, nh = (long long)g.batch * g.nz * g.nx;   // [batch][nz][nx]
                v.h0 = tab_c<60>(k.H, hz + unswx(t0), nh) * tau;
                v.h1 = tab_c<60>(k.H, hz + unswx(t0 + NX / 2), nh) * tau;
            }
            if (t0 == 0) v.vz = k.vz ? tab_c<61>(k.vz, z & (g.nz - 1), g.nz) * tau : T(0);
        }
        return v;
    };
    auto put_tabs = [&](int i, const Tabs &v) {
        if (t0 < LY) gtab[i & 1][t0] = v.gy;
        if (t0 < NX / 2) htab[i & 1][t0] = make_float2(v.h0, v.h1);
        if (t0 == 0) thzs[i & 1] = v.vz;
    };

    if (nmine > 0) {
        issue(0, 0, 0, NCR);
        issue(0, 1, 0, NCR);
        put_tabs(0, fetch_tabs(0));
    }
    cp_async_commit();
    for (int e = t0; e < NX + LY; e += NT)
        wx[e] = e < NX ? a.tw[g.fast_x_off + (e % 16) * (e / 16)] : a.tw[g.fast_y_off + e - NX];

    for (int i = 0; i < nmine; ++i) {
        const int tile = blockIdx.x + i * G;
        const int z = tile >> g.lgP, r = tile & (g.P - 1);
        const bool more = i + 1 < nmine;
        cp_async_wait_all();
        __syncthreads();
        const int o0 = half_buf(i, 0), o1 = half_buf(i, 1);

        // A: inverse x last stage on rows (rw, rw + 32); AoS in, position
        //    pairs (p, p + 128) out, split
#pragma unroll 1
        for (int s2 = 0; s2 < 2; ++s2) {
            const int q = threadIdx.x + NT * s2;
            const int k1 = q & 15, rw = q >> 4;
            const int pa = o0 + rw * PITCH + k1, pb = o1 + rw * PITCH + k1;
            Q v[16];
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const float2 ea = ld2_c<43>(bufs, pa + 16 * kk, BUFE), eb = ld2_c<43>(bufs, pb + 16 * kk, BUFE);
                v[brev(kk, 16)] = Q{make_float2(ea.x, eb.x), make_float2(ea.y, eb.y)};
            }
            qdft_inv<16, 0, 1>(v);
#pragma unroll
            for (int x2 = 1; x2 < 16; ++x2) qlift_b(v[x2], tab_c<44>(wx, x2 * 16 + k1, NX));
#pragma unroll
            for (int x2 = 0; x2 < 8; ++x2) {
                const Q &u = v[x2], &w = v[x2 + 8];
                st2_c<45>(bufs, pa + 16 * x2, BUFE, make_float2(u.x.x, w.x.x));
                st2_c<45>(bufs, pa + 16 * x2 + 128, BUFE, make_float2(u.y.x, w.y.x));
                st2_c<45>(bufs, pb + 16 * x2, BUFE, make_float2(u.x.y, w.x.y));
                st2_c<45>(bufs, pb + 16 * x2 + 128, BUFE, make_float2(u.y.y, w.y.y));
            }
        }
        if (more) issue(i + 1, 0, 0, 4);
        __syncthreads();

        // B: inverse x first stage (16 contiguous positions of x2 and of
        //    x2 + 8) and inverse y last stage (rows k1, k1 + 32), in place;
        //    the next tile's tables
        {
            const Tabs ntab = more ? fetch_tabs(i + 1) : Tabs{0.0f, 0.0f, 0.0f, 0.0f};
            const int t = threadIdx.x;
            const int k1 = t & 31, x2 = t >> 5;
            const int ra = o0 + k1 * PITCH + 16 * x2, rb = o1 + k1 * PITCH + 16 * x2;
            Q v[2][16];                                // [k2][x position]
#pragma unroll
            for (int m = 0; m < 16; m += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ro = h ? rb : ra;
                    const float4 xr = ld4_c<46>(bufs, ro + m, BUFE), xi = ld4_c<46>(bufs, ro + m + 128, BUFE);
                    v[h][brev(m, 16)] = Q{make_float2(xr.x, xr.y), make_float2(xi.x, xi.y)};
                    v[h][brev(m + 1, 16)] = Q{make_float2(xr.z, xr.w), make_float2(xi.z, xi.w)};
                }
            }
            qdft_inv<16, 0, 1>(v[0]);
            qdft_inv<16, 0, 1>(v[1]);
            const Lift<T> wyk = tab_c<47>(wy, k1, LY);
#pragma unroll
            for (int m = 0; m < 16; ++m) {             // radix 2 over k2, then exp(2 pi i j2 k1/64)
                const Q s0 = qadd(v[0][m], v[1][m]);
                Q s1 = qsub(v[0][m], v[1][m]);
                qlift_b(s1, wyk);
                v[0][m] = s0;
                v[1][m] = s1;
            }
#pragma unroll
            for (int m = 0; m < 16; m += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ro = h ? rb : ra;
                    st4_c<48>(bufs, ro + m, BUFE, make_float4(v[h][m].x.x, v[h][m].x.y, v[h][m + 1].x.x, v[h][m + 1].x.y));
                    st4_c<48>(bufs, ro + m + 128, BUFE, make_float4(v[h][m].y.x, v[h][m].y.y, v[h][m + 1].y.x, v[h][m + 1].y.y));
                }
            }
            if (more) put_tabs(i + 1, ntab);
        }
        if (more) issue(i + 1, 0, 4, 8);
        __syncthreads();

        // C: inverse y first stage (radix 32 over the rows of half buffer j2)
        //    -> potential factor -> forward radix 32, column pair (p, p + 128)
        {
            const int t = threadIdx.x;
            const int pp = t & 127, j2 = t >> 7;
            const int base = (j2 ? o1 : o0) + pp;
            const T *gt = gtab[i & 1];
            const T thz = thzs[i & 1];
            const float2 hx = htab[i & 1][pp];
            Q v[32];
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1)
                v[brev(k1, 32)] = Q{ld2_c<49>(bufs, base + k1 * PITCH, BUFE), ld2_c<49>(bufs, base + k1 * PITCH + 128, BUFE)};
            qdft_inv<32, 0, 1>(v);                     // v[j1]: real row j = 2 j1 + j2
#pragma unroll
            for (int j1 = 0; j1 < 32; ++j1) {
                float2 p, u;
                if constexpr (SEP)
                    qkick_coef<TIER>(add2(pk(gt[2 * j1 + j2]), hx), p, u);
                else
                    qkick_coef<TIER>(fma2(pk(gt[2 * j1 + j2]), hx, pk(thz)), p, u);
                qrot_f(v[j1], p, u);
            }
            qdft_fwd<32, 0, 1>(v);
#pragma unroll
            for (int k1 = 0; k1 < 32; ++k1) {
                st2_c<50>(bufs, base + k1 * PITCH, BUFE, v[brev(k1, 32)].x);
                st2_c<50>(bufs, base + k1 * PITCH + 128, BUFE, v[brev(k1, 32)].y);
            }
        }
        if (more) issue(i + 1, 0, 8, 12);
        __syncthreads();

        // B': mirror of B
        {
            const int t = threadIdx.x;
            const int k1 = t & 31, x2 = t >> 5;
            const int ra = o0 + k1 * PITCH + 16 * x2, rb = o1 + k1 * PITCH + 16 * x2;
            Q v[2][16];
#pragma unroll
            for (int m = 0; m < 16; m += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ro = h ? rb : ra;
                    const float4 xr = ld4_c<51>(bufs, ro + m, BUFE), xi = ld4_c<51>(bufs, ro + m + 128, BUFE);
                    v[h][m] = Q{make_float2(xr.x, xr.y), make_float2(xi.x, xi.y)};
                    v[h][m + 1] = Q{make_float2(xr.z, xr.w), make_float2(xi.z, xi.w)};
                }
            }
            const Lift<T> wyk = tab_c<52>(wy, k1, LY);
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                Q s1 = v[1][m];
                qlift_f(s1, wyk);
                const Q s0 = v[0][m];
                v[0][m] = qadd(s0, s1);
                v[1][m] = qsub(s0, s1);
            }
            qdft_fwd<16, 0, 1>(v[0]);
            qdft_fwd<16, 0, 1>(v[1]);
#pragma unroll
            for (int m = 0; m < 16; m += 2) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ro = h ? rb : ra;
                    const Q &e0 = v[h][brev(m, 16)], &e1 = v[h][brev(m + 1, 16)];
                    st4_c<53>(bufs, ro + m, BUFE, make_float4(e0.x.x, e0.x.y, e1.x.x, e1.x.y));
                    st4_c<53>(bufs, ro + m + 128, BUFE, make_float4(e0.y.x, e0.y.y, e1.y.x, e1.y.y));
                }
            }
        }
        if (more) issue(i + 1, 0, 12, 16);
        cp_async_commit();
        __syncthreads();

        // A': read both tasks back (frees both half buffers), then the mirror
        //     of A and the stores to HBM
        {
            const int t = phase_tid();
            Q v[2][16];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int q = t + NT * s2;
                const int k1 = q & 15, rw = q >> 4;
                const int pa = o0 + rw * PITCH + k1, pb = o1 + rw * PITCH + k1;
#pragma unroll
                for (int x2 = 0; x2 < 8; ++x2) {
                    const float2 ra = ld2_c<54>(bufs, pa + 16 * x2, BUFE), ia = ld2_c<54>(bufs, pa + 16 * x2 + 128, BUFE);
                    const float2 rb = ld2_c<54>(bufs, pb + 16 * x2, BUFE), ib = ld2_c<54>(bufs, pb + 16 * x2 + 128, BUFE);
                    v[s2][x2] = Q{make_float2(ra.x, rb.x), make_float2(ia.x, ib.x)};
                    v[s2][x2 + 8] = Q{make_float2(ra.y, rb.y), make_float2(ia.y, ib.y)};
                }
            }
            __syncthreads();                           // tile i's buffers are free
            if (more) issue(i + 1, 1, 0, NCR);
            cp_async_commit();
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {                // unrolled: v[s2] stays in registers
                const int q = t + NT * s2;
                const int k1 = q & 15, rw = q >> 4;
                Q w[16];
#pragma unroll
                for (int x2 = 0; x2 < 16; ++x2) w[x2] = v[s2][x2];
#pragma unroll
                for (int x2 = 1; x2 < 16; ++x2) qlift_f(w[x2], tab_c<55>(wx, x2 * 16 + k1, NX));
                qdft_fwd<16, 0, 1>(w);
                const long long oa = (long long)z * g.plane + ((long long)(rw * g.P + r) << g.lgnx) + k1;
                const long long ob = oa + ((long long)(HR * g.P) << g.lgnx);
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) {
                    const Q &e = w[brev(k2, 16)];
                    if (CTAP_BOUNDS(56, oa + 16 * k2, NTOT)) a.dst[oa + 16 * k2] = make_float2(e.x.x, e.y.x);
                    if (CTAP_BOUNDS(56, ob + 16 * k2, NTOT)) a.dst[ob + 16 * k2] = make_float2(e.x.y, e.y.y);
                }
            }
        }
    }
    cp_async_wait_all();
}

// ================================================================ dispatch
namespace {
int pk_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}
}  // namespace

bool packed_xy_supported(const Geom &g)
{
    return g.nx == 256 && g.Ly == 64;
}

bool launch_xy_packed(const XYArgs<float> &a, cudaStream_t st)
{
    const bool sep = a.k.form == VF_SEPARABLE && a.rd.Vsep;
    const bool hot = a.flags == (XY_IN_MIXED | XY_OUT_MIXED | XY_KICK_FULL) &&
                     (a.k.form == VF_PRODUCT || sep) && !a.k.imag && a.small_angle >= 1;
    if (!hot || !a.ring || a.src != a.dst || !packed_xy_supported(a.g)) return false;
    constexpr int HB = 32 * 258;
    constexpr size_t smem = 3 * HB * sizeof(float2) + (256 + 64) * sizeof(Lift<float>);
    static bool cfg = false;
    if (!cfg) {
        cudaFuncSetAttribute(xy_pk_kernel<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_pk_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_pk_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(xy_pk_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    const int ntiles = xy_grid(a.g);
    const int grid = std::min(ntiles, pk_sm_count());
    if (sep && a.small_angle == 2)
        xy_pk_kernel<2, true><<<grid, kXpkNT, smem, st>>>(a, ntiles);
    else if (sep)
        xy_pk_kernel<1, true><<<grid, kXpkNT, smem, st>>>(a, ntiles);
    else if (a.small_angle == 2)
        xy_pk_kernel<2, false><<<grid, kXpkNT, smem, st>>>(a, ntiles);
    else
        xy_pk_kernel<1, false><<<grid, kXpkNT, smem, st>>>(a, ntiles);
    return true;
}

}  // namespace ctap

// Record of the bounds-checked build (bounds.cuh): the checked kernels live
// in this file, so does their record.
extern "C" ctap_status ctap_debug_bounds(int clear, long long *out)
{
    if (!out) return CTAP_ERR_INVALID_ARG;
#ifdef CTAP_DEBUG_BOUNDS
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, g_ctap_bounds, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return CTAP_ERR_CUDA;
    }
    if (clear) {
        const unsigned long long zero = 0;
        if (cudaMemcpyToSymbol(g_ctap_bounds, &zero, sizeof zero) != cudaSuccess) {
            cudaGetLastError();
            return CTAP_ERR_CUDA;
        }
    }
    *out = (long long)v;
#else
    (void)clear;
    *out = -1;
#endif
    return CTAP_OK;
}

namespace ctap {

bool packed_z_supported(const Geom &g)
{
    return g.nz == 1024 && g.P == 4 && g.w == 4;
}

bool launch_z_packed(const ZArgs<float> &a, cudaStream_t st)
{
    if (!a.ring || a.observe || a.imag || a.scale || a.src != a.dst || !a.kin_xy ||
        !packed_z_supported(a.g))
        return false;
    constexpr size_t smem = (size_t)kZpkNRING * kZpkCHZ * 16 * sizeof(float2) +
                            2 * 1024 * sizeof(Lift<float>);
    static bool cfg = false;
    if (!cfg) {
        cudaFuncSetAttribute(z_pk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cfg = true;
    }
    const int ntiles = z_grid(a.g);
    z_pk_kernel<<<std::min(ntiles, pk_sm_count()), kZpkNT, smem, st>>>(a, ntiles);
    return true;
}

}  // namespace ctap
