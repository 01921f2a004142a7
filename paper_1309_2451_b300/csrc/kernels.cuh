// kernels.cuh -- argument blocks and launchers of the split-step passes.
//
// One Strang step (Sec. IV) is carried by two passes over psi in HBM:
//
//   XY pass, one CTA per (z-plane, row class r): the CTA holds the rows
//     y = r + P j (j < Ly = ny/P) of one plane.  It undoes the previous
//     step's forward x- and partial y-transforms, applies the potential
//     factor (both half-kicks merged), and redoes the forward transforms.
//     The y-transform is split by decimation: an Ly-point DFT over j inside
//     the CTA and a P-point "cross" DFT over the classes r done by the Z pass,
//     so no CTA ever needs a whole plane (a 256x256 complex64 plane is 512 KiB,
//     more than one SM's shared memory).
//   Z pass, one CTA per (k', block of w kx values): the CTA holds, for every z,
//     the P rows k' P + r and w columns: it finishes the y-transform (cross
//     DFT over r), runs the forward z-transform, applies the kinetic factor,
//     the inverse z-transform and the inverse cross DFT.
//
// Between passes psi lives in place, in the mixed representation
// (kx, k'-partial ky, z); rows keep their position (row j P + r of a plane).
#pragma once

#include "device_fft.cuh"

namespace ctap {

constexpr int kNT = 512;   // threads per pass CTA

enum VForm { VF_NONE = 0, VF_DENSE = 1, VF_SEPARABLE = 2, VF_PRODUCT = 3 };

enum XYFlags {
    XY_IN_MIXED = 1,      // input is in the mixed representation: inverse x, y first
    XY_OUT_MIXED = 2,     // forward y, x before storing
    XY_KICK_HALF = 4,     // one potential factor with tau = dt/2
    XY_KICK_FULL = 8,     // one potential factor with tau = dt (two merged halves)
    XY_KICK_SPLIT = 16,   // two factors of dt/2 with a reduction/state copy between
    XY_RED_NORM = 32,     // FP64 sum |psi|^2 after the first factor (imaginary time)
    XY_RED_OBS = 64,      // FP64 observables of the natural-layout input
    XY_STATE_OUT = 128,   // copy the state between the two half factors out
    XY_GRAD_PRE = 256,    // adjoint: gradient partials on the input (before any kick)
    XY_GRAD = 512         // adjoint: gradient partials after the first kick
};

// Adjoint gradient partials of one XY launch: for the state lambda held by
// the pass and the forward state psi (natural layout), per CTA
//   acc[cta][j] += coef * sum Im(conj(lambda) psi) g(y) D_j(z, x),  j = 1, 3.
struct GradData {
    const void *psi;          // forward state psi_m, natural layout
    const double *g64;        // [ny]
    const double *D1, *D3;    // [nz][nx]
    double *acc;              // [xy_grid][2]
    double coef;              // dt * w_m * dV
};

struct Geom {
    int nx, ny, nz, P, Ly, w, C;
    int lgnx, lgny, lgnz, lgP, lgLy, lgw, lgC;
    int pitchXY, pitchZ;
    int nblk_lg;            // log2(nx / w)
    long long plane;        // nx * ny
    double box[6];
    double dx;
    AxisPlan apx, apy, apz; // x: length nx; y: length Ly; z: length nz
    int cross_off;          // offset of the ny-entry table exp(-2 pi i e/ny)
    int fast_x_off;         // offset of exp(-2 pi i e/nx), e < nx (fast passes)
    int fast_z_off;         // offset of exp(-2 pi i e/nz), e < nz (fast passes)
    int fast_y_off;         // offset of exp(-2 pi i e/Ly), e < Ly (fast passes)
    // batched replicas: psi is [batch][nz][ny][nx]; the XY pass sees batch*nz
    // planes (plane index zall, replica-local z = zall mod nz), the Z pass
    // batch * 2^lgzt tiles (replica = tile >> lgzt)
    int batch;
    int lgzt;               // log2(Z tiles per replica) = lgLy + nblk_lg
    long long rstride;      // elements per replica = nz * plane
};

template <class T> struct Kick {
    int form;
    int imag;
    const T *Vd;              // dense, [nz][ny][nx]
    const T *g;               // product, [ny]
    const T *H;               // product, [nz][nx]
    const Lift<T> *sep_half;  // separable, [nx | ny | nz] for tau = dt/2
    const Lift<T> *sep_full;  // separable, tau = dt
    const T *vz;              // product form: additive z-only term Vz(z) [nz], or null
    T tau_half, tau_full;
};

// FP64 data for reductions (observables, norms, gradients)
struct RedData {
    const double *Vsep;       // [nx | ny | nz] for separable V
    const double *g64;        // [ny]
    const double *H64;        // [nz][nx]
    const double *vz64;       // product form: additive Vz(z) [nz], or null
    const double *xc;         // guide centres [3][nz] or null
    double hw;                // population half-width
    const double *k2h;        // k^2/2 per axis [nx | ny | nz]
};

template <class T> struct XYArgs {
    Geom g;
    const Lift<T> *tw;
    Kick<T> k;
    RedData rd;
    int vform_obs;            // V form for <V> (VF_*), dense uses k.Vd
    const Cx<T> *src;
    Cx<T> *dst;
    Cx<T> *state_out;         // XY_STATE_OUT target (natural layout) or null
    double *partials;         // per-CTA reduction results
    int flags;
    int small_angle;          // kick series tier: 0 any angle, 1 |V| dt <= 0.5, 2 (complex64) <= 0.16
    GradData gd;
    int ring;                 // 1: the persistent ring form may be used (in place only)
};

template <class T> struct ZArgs {
    Geom g;
    const Lift<T> *tw;
    const Lift<T> *kin;       // [nx | ny | nz] kinetic factors for this dt/mode
    int imag;
    T inv_n;                  // 1/N (transforms are unnormalised)
    const double *scale;      // lazy imaginary-time renormalisation, or null
    const Cx<T> *src;
    Cx<T> *dst;
    const double *k2h;        // for the kinetic-energy reduction
    double *partials;
    int observe;              // 1: forward only, reduce sum k^2/2 |psi_k|^2, no store
    int ring;                 // 1: the persistent ring form may be used (in place only)
    const void *kin_xy;       // Lift<T> of exp(-i (kx^2 + ky^2) dt/2) [ny][nx], or null
};

template <class T> void launch_xy(const XYArgs<T> &a, cudaStream_t st);
template <class T> void launch_z(const ZArgs<T> &a, cudaStream_t st);
int xy_grid(const Geom &g);
int z_grid(const Geom &g);
size_t xy_smem(const Geom &g, int esize);
size_t z_smem(const Geom &g, int esize);

// Deterministic fixed-order sum of nblk x nq partials; out[q] (device).
void launch_reduce(const double *partials, int nblk, int nq, double *out, cudaStream_t st);
// scale = 1/sqrt(sum partials * dV)  (imaginary-time renormalisation)
void launch_norm_scale(const double *partials, int nblk, double dV, double *scale,
                       cudaStream_t st);
template <class T> void launch_scale(Cx<T> *psi, long long n, const double *scale,
                                     cudaStream_t st);
// lambda = M psi on the region |x - xc(z)| < hw; per-CTA sum M |psi|^2.
template <class T> void launch_mask(const Cx<T> *psi, Cx<T> *lam, const Geom &g,
                                    const double *xcj, double hw, double *partials,
                                    int nblk, cudaStream_t st);
int mask_blocks(const Geom &g);
// out[z][x] = dy sum_y |psi(z, y, x)|^2 (FP64, fixed summation order)
template <class T> void launch_density_xz(const Cx<T> *psi, const Geom &g, double dy, double *out,
                                          cudaStream_t st);

// fast_passes.cu: specialised passes (same layout as the generic ones); the
// launchers return false when the geometry is not covered.  esize is the
// size of one complex value (8 or 16).
int fast_rows(int esize);
bool fast_xy_supported(int esize, int nx, int Ly);
bool fast_z_supported(int esize, int nz, int P, int w);
bool launch_xy_fast(const XYArgs<float> &a, cudaStream_t st);
bool launch_xy_fast(const XYArgs<double> &a, cudaStream_t st);
bool launch_xy_fast(const XYArgs<df> &a, cudaStream_t st);
bool launch_z_fast(const ZArgs<float> &a, cudaStream_t st);
bool launch_z_fast(const ZArgs<double> &a, cudaStream_t st);
bool launch_z_fast(const ZArgs<df> &a, cudaStream_t st);
// the double-float three-stage Z pass (z3_df_pass.cuh), one per tile
// geometry: 8, 4 or 2 row classes x 1, 2 or 4 columns (false: not this one)
bool launch_z3_df_p8(const ZArgs<df> &a, cudaStream_t st);
bool launch_z3_df_p4(const ZArgs<df> &a, cudaStream_t st);
bool launch_z3_df_p2(const ZArgs<df> &a, cudaStream_t st);

// V = vs |B| - voff on the grid ([nz][ny][nx], FP64, device) from thin
// current segments seg[7 m ..] = (A, C, I) and a uniform field bias
void launch_wire_potential(double *V, const Geom &g, const double *seg, int nseg,
                           const double bias[3], double k, double vs, double voff,
                           cudaStream_t st);

// complex128 psi <-> double-float storage (n complex values), in place or
// into a separate buffer
void launch_c128_to_df(void *psi, long long n, cudaStream_t st);
void launch_df_to_c128(void *psi, long long n, cudaStream_t st);
void launch_c128_to_df_copy(const void *src, void *dst, long long n, cudaStream_t st);

}  // namespace ctap
