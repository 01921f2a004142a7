/*
 * oracle.c -- plain, slow, FP64 CPU reference for the split-step hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What it computes (Morgan et al., "Coherent transport by adiabatic passage on
 * atom chips", Sec. IV): the three-dimensional time-dependent Schroedinger
 * equation (hbar = m = 1) advanced with the Fourier split-operator method,
 * written here in the symmetric (Strang) order
 *
 *     psi <- exp(-i V dt/2) psi                       (potential half-kick)
 *     psi <- F^-1 exp(-i |k|^2 dt/2) F psi            (kinetic step, k-space)
 *     psi <- exp(-i V dt/2) psi                       (potential half-kick)
 *
 * The paper states the per-step cost in transforms and pointwise complex
 * products but does not fix the order; the V/2-K-V/2 order is the reading
 * taken here.
 * The imaginary-time variant (used to find the transverse ground state,
 * which Sec. V obtains numerically without naming the method) replaces dt by
 * -i dtau, so every factor becomes real, and renormalises after each step.
 *
 * Conventions:
 *   arrays are [nz][ny][nx] with x fastest, complex128 interleaved (re, im);
 *   grid x_i = lo + i (hi - lo)/n, i = 0..n-1 (periodic, hi excluded);
 *   k_m = 2 pi m/(hi - lo), m in FFT order 0..n/2-1, -n/2..-1;
 *   forward DFT: sum_j a_j exp(-2 pi i j m/n), unnormalised;
 *   inverse DFT: (1/n) sum_m A_m exp(+2 pi i j m/n).
 *
 * The FFT is an iterative radix-2 decimation-in-time transform with a
 * bit-reversal permutation.  Every twiddle factor is evaluated directly with
 * cos/sin in FP64 (no recurrence).  OpenMP distributes independent lines.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ grids */

static double grid_x(int i, int n, double lo, double hi)
{
    return lo + (double)i * (hi - lo) / (double)n;
}

static double grid_k(int m, int n, double lo, double hi)
{
    int mm = (m < (n + 1) / 2) ? m : m - n;   /* FFT order; n = 1 gives 0 */
    if (n == 1) mm = 0;
    return 2.0 * ORC_PI * (double)mm / (hi - lo);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following calls (omp_set_num_threads): the timed CPU
 * baseline measures the oracle on one thread as well as on all host cores. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------- radix-2 FFT */

static int is_pow2(long n) { return n >= 1 && (n & (n - 1)) == 0; }

/* In-place radix-2 DIT FFT of one contiguous line of length n (power of 2).
 * dir = -1: forward (exp(-2 pi i jm/n)); dir = +1: inverse, scaled by 1/n.
 * w must hold n/2 precomputed factors w[j] = exp(dir 2 pi i j/n). */
static void fft_line(cplx *a, long n, int dir, const cplx *w)
{
    if (n < 2) return;
    /* bit-reversal permutation */
    for (long i = 1, j = 0; i < n; ++i) {
        long bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    /* butterflies: sub-transforms of length len combine two of length len/2 */
    for (long len = 2; len <= n; len <<= 1) {
        long half = len >> 1, step = n / len;
        for (long b = 0; b < n; b += len) {
            for (long j = 0; j < half; ++j) {
                cplx u = a[b + j];
                cplx t = w[j * step] * a[b + j + half];
                a[b + j] = u + t;
                a[b + j + half] = u - t;
            }
        }
    }
    if (dir > 0) {
        double s = 1.0 / (double)n;
        for (long i = 0; i < n; ++i) a[i] *= s;
    }
}

static cplx *twiddles(long n, int dir)
{
    long h = n / 2 > 0 ? n / 2 : 1;
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)h);
    for (long j = 0; j < h; ++j) {
        double ang = 2.0 * ORC_PI * (double)j / (double)n;
        w[j] = cos(ang) + (double)dir * sin(ang) * I;
    }
    return w;
}

/* Batched 1D FFT: `count` contiguous lines of length n. */
int orc_fft1d(double *data, long n, long count, int dir)
{
    if (!is_pow2(n) || (dir != 1 && dir != -1)) return -1;
    cplx *a = (cplx *)data;
    cplx *w = twiddles(n, dir);
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < count; ++c) fft_line(a + c * n, n, dir, w);
    free(w);
    return 0;
}

/* 3D FFT on [nz][ny][nx]: gather every line along each axis, transform it,
 * scatter it back. */
int orc_fft3d(double *data, int nx, int ny, int nz, int dir)
{
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz)) return -1;
    if (dir != 1 && dir != -1) return -1;
    cplx *a = (cplx *)data;
    const long sx = 1, sy = nx, sz = (long)nx * ny;
    const int n_ax[3] = {nx, ny, nz};
    const long s_ax[3] = {sx, sy, sz};
    for (int ax = 0; ax < 3; ++ax) {
        long n = n_ax[ax], st = s_ax[ax];
        if (n == 1) continue;
        long nlines = (long)nx * ny * nz / n;
        cplx *w = twiddles(n, dir);
        #pragma omp parallel
        {
            cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
            #pragma omp for schedule(static)
            for (long l = 0; l < nlines; ++l) {
                /* base offset of line l: enumerate the other two axes */
                long base;
                if (ax == 0)      base = l * nx;
                else if (ax == 1) base = (l / nx) * sz + (l % nx);
                else              base = l;
                for (long i = 0; i < n; ++i) line[i] = a[base + i * st];
                fft_line(line, n, dir, w);
                for (long i = 0; i < n; ++i) a[base + i * st] = line[i];
            }
            free(line);
        }
        free(w);
    }
    return 0;
}

/* ------------------------------------------------------------ split step */

static double cell_volume(int nx, int ny, int nz, const double *box)
{
    return (box[1] - box[0]) / nx * (box[3] - box[2]) / ny * (box[5] - box[4]) / nz;
}

static double sum_abs2(const cplx *a, long N)
{
    double s = 0.0;
    #pragma omp parallel for reduction(+:s) schedule(static)
    for (long i = 0; i < N; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* psi <- exp(-i V tau) psi  (real time) or exp(-V tau) psi (imaginary time) */
static void potential_factor(cplx *a, const double *V, long N, double tau, int imag)
{
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double th = V[i] * tau;
        if (imag) a[i] *= exp(-th);
        else      a[i] *= cos(th) - sin(th) * I;
    }
}

/* psihat <- exp(-i |k|^2 tau/2) psihat (real) or exp(-|k|^2 tau/2) psihat (imag) */
static void kinetic_factor(cplx *a, int nx, int ny, int nz, const double *box,
                           double tau, int imag)
{
    #pragma omp parallel for schedule(static)
    for (long iz = 0; iz < nz; ++iz) {
        double kz = grid_k((int)iz, nz, box[4], box[5]);
        for (int iy = 0; iy < ny; ++iy) {
            double ky = grid_k(iy, ny, box[2], box[3]);
            for (int ix = 0; ix < nx; ++ix) {
                double kx = grid_k(ix, nx, box[0], box[1]);
                double th = 0.5 * (kx * kx + ky * ky + kz * kz) * tau;
                long i = (iz * ny + iy) * (long)nx + ix;
                if (imag) a[i] *= exp(-th);
                else      a[i] *= cos(th) - sin(th) * I;
            }
        }
    }
}

/* nsteps Strang steps of size dt on psi (in place).  V is the dense
 * potential on the grid.  imag != 0: imaginary time with per-step
 * renormalisation so that sum |psi|^2 dV = 1.  Half-kicks are applied
 * separately (never merged across steps). */
int orc_step(double *psi, const double *V, int nx, int ny, int nz,
             const double *box, double dt, int nsteps, int imag)
{
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || nsteps < 0) return -1;
    cplx *a = (cplx *)psi;
    long N = (long)nx * ny * nz;
    double dV = cell_volume(nx, ny, nz, box);
    for (int s = 0; s < nsteps; ++s) {
        potential_factor(a, V, N, 0.5 * dt, imag);
        orc_fft3d(psi, nx, ny, nz, -1);
        kinetic_factor(a, nx, ny, nz, box, dt, imag);
        orc_fft3d(psi, nx, ny, nz, +1);
        potential_factor(a, V, N, 0.5 * dt, imag);
        if (imag) {
            double nrm = sqrt(sum_abs2(a, N) * dV);
            double inv = 1.0 / nrm;
            #pragma omp parallel for schedule(static)
            for (long i = 0; i < N; ++i) a[i] *= inv;
        }
    }
    return 0;
}

/* nsteps real-time steps of the other Strang ordering, K/2 V K/2 (the
 * kinetic factor split, the potential factor whole): per step
 * psihat = F psi; psihat *= exp(-i |k|^2 dt/4); psi = F^-1 psihat;
 * psi *= exp(-i V dt); psihat = F psi; psihat *= exp(-i |k|^2 dt/4);
 * psi = F^-1 psihat.  Sec. IV counts four transforms per step, which is this
 * ordering applied literally.  Nothing is merged across steps. */
int orc_step_kvk(double *psi, const double *V, int nx, int ny, int nz,
                 const double *box, double dt, int nsteps)
{
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || nsteps < 0) return -1;
    cplx *a = (cplx *)psi;
    long N = (long)nx * ny * nz;
    for (int s = 0; s < nsteps; ++s) {
        orc_fft3d(psi, nx, ny, nz, -1);
        kinetic_factor(a, nx, ny, nz, box, 0.5 * dt, 0);
        orc_fft3d(psi, nx, ny, nz, +1);
        potential_factor(a, V, N, dt, 0);
        orc_fft3d(psi, nx, ny, nz, -1);
        kinetic_factor(a, nx, ny, nz, box, 0.5 * dt, 0);
        orc_fft3d(psi, nx, ny, nz, +1);
    }
    return 0;
}

/* --------------------------------------------------------- observables */

/* out[0] = sum |psi|^2 dV                       (norm)
 * out[1] = <T> = sum_k (|k|^2/2) |F psi|^2 / (N sum |psi|^2)
 * out[2] = <V> = sum V |psi|^2 / sum |psi|^2
 * out[3+j] = sum_{|x - xc[j][z]| < hw} |psi|^2 dV, j = 0, 1, 2
 *            (population of guide j; xc is [3][nz], one centre per z-slice;
 *             the region spans every y).  Plain FP64 loops. */
int orc_observables(const double *psi, const double *V, int nx, int ny, int nz,
                    const double *box, const double *xc, double hw, double *out)
{
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz)) return -1;
    const cplx *a = (const cplx *)psi;
    long N = (long)nx * ny * nz;
    double dV = cell_volume(nx, ny, nz, box);
    double s2 = 0.0, sv = 0.0, p0 = 0.0, p1 = 0.0, p2 = 0.0;
    #pragma omp parallel for reduction(+:s2,sv,p0,p1,p2) schedule(static)
    for (long iz = 0; iz < nz; ++iz) {
        for (int iy = 0; iy < ny; ++iy) {
            for (int ix = 0; ix < nx; ++ix) {
                long i = (iz * ny + iy) * (long)nx + ix;
                double d = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
                s2 += d;
                if (V) sv += V[i] * d;
                if (xc) {
                    double x = grid_x(ix, nx, box[0], box[1]);
                    if (fabs(x - xc[0 * nz + iz]) < hw) p0 += d;
                    if (fabs(x - xc[1 * nz + iz]) < hw) p1 += d;
                    if (fabs(x - xc[2 * nz + iz]) < hw) p2 += d;
                }
            }
        }
    }
    cplx *b = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!b) return -2;
    memcpy(b, a, sizeof(cplx) * (size_t)N);
    orc_fft3d((double *)b, nx, ny, nz, -1);
    double sk = 0.0;
    #pragma omp parallel for reduction(+:sk) schedule(static)
    for (long iz = 0; iz < nz; ++iz) {
        double kz = grid_k((int)iz, nz, box[4], box[5]);
        for (int iy = 0; iy < ny; ++iy) {
            double ky = grid_k(iy, ny, box[2], box[3]);
            for (int ix = 0; ix < nx; ++ix) {
                double kx = grid_k(ix, nx, box[0], box[1]);
                long i = (iz * ny + iy) * (long)nx + ix;
                double d = creal(b[i]) * creal(b[i]) + cimag(b[i]) * cimag(b[i]);
                sk += 0.5 * (kx * kx + ky * ky + kz * kz) * d;
            }
        }
    }
    free(b);
    out[0] = s2 * dV;
    out[1] = (s2 > 0.0) ? sk / ((double)N * s2) : 0.0;
    out[2] = (s2 > 0.0) ? sv / s2 : 0.0;
    out[3] = p0 * dV;
    out[4] = p1 * dV;
    out[5] = p2 * dV;
    return 0;
}

/* ------------------------------------------------ three-guide potential */

/* V(x,y,z) = -V0 sum_{j=1..3} exp(-((x - x_j(z))^2 + y^2) / (2 s^2)),
 * with x_1 = x1z[z], x_2 = 0, x_3 = x3z[z]: three parallel Gaussian
 * waveguides whose separations vary along z (the spatial form of the
 * time-dependent couplings of Eq. (1)). */
/* ------------------------------------------------------ atom-chip wires */

/* Magnetic field of thin straight current segments plus a uniform field
 * (Sec. III, Eq. 4: the Biot-Savart law; a homogeneous bias field lifts the
 * minimum above the wire, Eq. 5, and a field along the wires removes the
 * zero).  For one straight segment from A to C carrying I, the line integral
 * of Eq. 4 evaluates in closed form: at perpendicular distance d from the
 * line through A and C,
 *     |B| = k I (cos t1 - cos t2) / d,   k = mu0 / (4 pi),
 * where t1, t2 are the angles between the direction A->C and the vectors
 * from A and from C to the point, and B points along (C - A) x (P - A).
 * seg[7 m .. 7 m + 6] = (Ax, Ay, Az, Cx, Cy, Cz, I); pts[3 i ..] the points;
 * B[3 i ..] receives bias + the sum over segments (segments in input
 * order).  A point on a segment's line (d = 0) gets no contribution from
 * that segment. */
int orc_wire_field(const double *pts, long npts, int nseg, const double *seg,
                   const double *bias, double k, double *B)
{
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < npts; ++i) {
        const double *P = pts + 3 * i;
        double b[3] = {bias[0], bias[1], bias[2]};
        for (int m = 0; m < nseg; ++m) {
            const double *A = seg + 7 * m, *C = A + 3;
            const double cur = A[6];
            double t[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
            const double len = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
            if (len == 0.0) continue;
            for (int q = 0; q < 3; ++q) t[q] /= len;
            const double pa[3] = {P[0] - A[0], P[1] - A[1], P[2] - A[2]};
            const double pc[3] = {P[0] - C[0], P[1] - C[1], P[2] - C[2]};
            const double along = pa[0] * t[0] + pa[1] * t[1] + pa[2] * t[2];
            double perp[3] = {pa[0] - along * t[0], pa[1] - along * t[1], pa[2] - along * t[2]};
            const double d = sqrt(perp[0] * perp[0] + perp[1] * perp[1] + perp[2] * perp[2]);
            if (d == 0.0) continue;
            const double ra = sqrt(pa[0] * pa[0] + pa[1] * pa[1] + pa[2] * pa[2]);
            const double rc = sqrt(pc[0] * pc[0] + pc[1] * pc[1] + pc[2] * pc[2]);
            const double cos1 = along / ra;
            const double cos2 = (pc[0] * t[0] + pc[1] * t[1] + pc[2] * t[2]) / rc;
            const double mag = k * cur * (cos1 - cos2) / d;
            /* direction: t x perp / d */
            const double n[3] = {(t[1] * perp[2] - t[2] * perp[1]) / d,
                                 (t[2] * perp[0] - t[0] * perp[2]) / d,
                                 (t[0] * perp[1] - t[1] * perp[0]) / d};
            for (int q = 0; q < 3; ++q) b[q] += mag * n[q];
        }
        B[3 * i] = b[0];
        B[3 * i + 1] = b[1];
        B[3 * i + 2] = b[2];
    }
    return 0;
}

int orc_ctap_potential(double *V, int nx, int ny, int nz, const double *box,
                       double V0, double s, const double *x1z, const double *x3z)
{
    double inv2s2 = 1.0 / (2.0 * s * s);
    #pragma omp parallel for schedule(static)
    for (long iz = 0; iz < nz; ++iz) {
        double c[3] = {x1z[iz], 0.0, x3z[iz]};
        for (int iy = 0; iy < ny; ++iy) {
            double y = grid_x(iy, ny, box[2], box[3]);
            for (int ix = 0; ix < nx; ++ix) {
                double x = grid_x(ix, nx, box[0], box[1]);
                double v = 0.0;
                for (int j = 0; j < 3; ++j) {
                    double dx = x - c[j];
                    v += exp(-(dx * dx + y * y) * inv2s2);
                }
                V[(iz * ny + iy) * (long)nx + ix] = -V0 * v;
            }
        }
    }
    return 0;
}

/* dV/dx_j for guide j in {0, 2} (the two moving outer guides):
 * -V0 exp(-((x - x_j)^2 + y^2)/(2 s^2)) (x - x_j)/s^2. */
int orc_ctap_dvdx(double *D, int nx, int ny, int nz, const double *box,
                  double V0, double s, const double *xjz)
{
    double inv2s2 = 1.0 / (2.0 * s * s);
    #pragma omp parallel for schedule(static)
    for (long iz = 0; iz < nz; ++iz) {
        double cj = xjz[iz];
        for (int iy = 0; iy < ny; ++iy) {
            double y = grid_x(iy, ny, box[2], box[3]);
            for (int ix = 0; ix < nx; ++ix) {
                double x = grid_x(ix, nx, box[0], box[1]);
                double dx = x - cj;
                D[(iz * ny + iy) * (long)nx + ix] =
                    -V0 * exp(-(dx * dx + y * y) * inv2s2) * dx / (s * s);
            }
        }
    }
    return 0;
}

/* ----------------------------------------------------------- adjoint */

/* Exact gradient of the discrete objective J = sum M |psi_N|^2 dV (M a real
 * mask, frozen) with respect to the potential, contracted with two
 * derivative fields W1 = dV/dx_1, W3 = dV/dx_3 and resolved per z-slice:
 *
 *   R_j(z) = dt sum_{n=0..N} w_n sum_{x,y} Im( conj(lambda_n) W_j psi_n ) dV,
 *   w_0 = w_N = 1, w_n = 2 otherwise,
 *   lambda_N = M psi_N,  lambda_n = S(-dt) lambda_{n+1},
 *
 * where S(dt) is one Strang step (S(-dt) is its adjoint because S is
 * unitary).  dJ/dc = sum_z B(z) R_j(z) then follows by the chain rule through
 * x_j(z).  Every forward state psi_0..psi_N is kept in memory (plain,
 * no checkpointing).  Returns J in *J_out. */
int orc_adjoint(const double *psi0, const double *V, int nx, int ny, int nz,
                const double *box, double dt, int nsteps, const double *mask,
                const double *W1, const double *W3,
                double *J_out, double *R1, double *R3)
{
    if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || nsteps < 1) return -1;
    long N = (long)nx * ny * nz;
    long plane = (long)nx * ny;
    double dV = cell_volume(nx, ny, nz, box);
    cplx *states = (cplx *)malloc(sizeof(cplx) * (size_t)N * (size_t)(nsteps + 1));
    cplx *lam = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    if (!states || !lam) { free(states); free(lam); return -2; }
    memcpy(states, psi0, sizeof(cplx) * (size_t)N);
    for (int n = 0; n < nsteps; ++n) {
        memcpy(states + (size_t)(n + 1) * N, states + (size_t)n * N, sizeof(cplx) * (size_t)N);
        orc_step((double *)(states + (size_t)(n + 1) * N), V, nx, ny, nz, box, dt, 1, 0);
    }
    const cplx *psiN = states + (size_t)nsteps * N;
    double J = 0.0;
    for (long i = 0; i < N; ++i) {
        J += mask[i] * (creal(psiN[i]) * creal(psiN[i]) + cimag(psiN[i]) * cimag(psiN[i]));
        lam[i] = mask[i] * psiN[i];
    }
    *J_out = J * dV;
    for (int z = 0; z < nz; ++z) { R1[z] = 0.0; R3[z] = 0.0; }
    for (int n = nsteps; n >= 0; --n) {
        const cplx *psi = states + (size_t)n * N;
        double wn = (n == 0 || n == nsteps) ? 1.0 : 2.0;
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z) {
            double a1 = 0.0, a3 = 0.0;
            for (long i = z * plane; i < (z + 1) * plane; ++i) {
                double im = cimag(conj(lam[i]) * psi[i]);
                a1 += im * W1[i];
                a3 += im * W3[i];
            }
            R1[z] += dt * wn * a1 * dV;
            R3[z] += dt * wn * a3 * dV;
        }
        if (n > 0) orc_step((double *)lam, V, nx, ny, nz, box, -dt, 1, 0);
    }
    free(states);
    free(lam);
    return 0;
}
