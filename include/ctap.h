/*
 * ctap.h -- C ABI of libctap, a single-GPU (B300, sm_103a) implementation of
 * the three-dimensional Fourier split-operator propagation used by
 * Morgan et al., "Coherent transport by adiabatic passage on atom chips".
 *
 * Physics and method (hbar = m = 1):
 *   i d psi/dt = (-(1/2) Laplacian + V(x,y,z)) psi               (Sec. IV)
 * advanced by symmetric (Strang) split steps
 *   psi <- exp(-i V dt/2) F^-1 exp(-i |k|^2 dt/2) F exp(-i V dt/2) psi
 * (the transforms and pointwise complex products of one step, Sec. IV),
 * and its imaginary-time variant (dt -> -i dtau, real factors, renormalised
 * every step) that prepares the guided transverse ground state used as the
 * initial state (Sec. V).
 *
 * Grid and layout conventions (every entry point):
 *   - psi is complex, interleaved (re, im), C order [nz][ny][nx] (x fastest);
 *     complex64 (float2) for CTAP_C64 plans, complex128 (double2) for
 *     CTAP_C128 plans.  psi is caller-owned DEVICE memory (e.g. a torch
 *     tensor), 16-byte aligned (32-byte for CTAP_C128).
 *   - box = {xmin, xmax, ymin, ymax, zmin, zmax}; grid point i of an axis with
 *     n points is lo + i (hi - lo)/n (periodic, hi excluded).
 *   - wavenumbers k = 2 pi m/(hi - lo), m in FFT order.
 *   - potentials given to the library are HOST arrays of FP64 and are copied;
 *     the caller keeps ownership.
 *
 * Sizes: every axis a power of two; nx, ny in [8, 1024], nz in [1, 1024];
 * the xy-plane is split into at most ny row classes so that one class fits in
 * a CTA's shared memory, and a z-line tile must hold all classes; shapes
 * outside that envelope return CTAP_ERR_UNSUPPORTED_SIZE (every shape with
 * nx*ny <= 65536 and nz <= 1024 is inside it).
 *
 * Errors: every call returns a ctap_status; no C++ exception crosses the ABI.
 * A plan is not thread-safe.  ctap_step is asynchronous on the plan's stream;
 * ctap_observables, ctap_adjoint, ctap_get_potential and ctap_sync
 * synchronise (with a host-side timeout, see ctap_set_timeout).
 */
#ifndef CTAP_H
#define CTAP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctap_plan *ctap_plan_t;          /* opaque, library-owned */

/* Precision of a plan.  CTAP_C64: complex64 psi, FP32 transforms.
 * CTAP_C128: complex128 psi, FP64 transforms.  CTAP_C128_DF: complex128 psi,
 * transforms in double-float arithmetic (pairs of FP32 numbers, about 48
 * significant bits; B300's FP32 rate is many times its FP64 rate): psi is
 * converted to the double-float form on entry to ctap_step and back on exit
 * (both forms take 16 bytes per value).  ctap_adjoint needs CTAP_C64 or
 * CTAP_C128. */
typedef enum { CTAP_C64 = 0, CTAP_C128 = 1, CTAP_C128_DF = 2 } ctap_dtype;
/* Time stepping of ctap_step: real time in the symmetric order V/2 K V/2
 * (the default), imaginary time in the same order, or real time in the
 * order K/2 V K/2 (the alternative Strang ordering). */
typedef enum { CTAP_REAL = 0, CTAP_IMAG = 1, CTAP_REAL_KVK = 2 } ctap_time;

typedef enum {
    CTAP_OK = 0,
    CTAP_ERR_INVALID_ARG = 1,       /* null pointer, bad enum, nsteps < 0 ... */
    CTAP_ERR_UNSUPPORTED_SIZE = 2,  /* grid outside the supported envelope    */
    CTAP_ERR_DTYPE = 3,             /* dtype mismatch                         */
    CTAP_ERR_NO_POTENTIAL = 4,      /* step/observables before set_potential  */
    CTAP_ERR_OOM = 5,               /* device allocation failed               */
    CTAP_ERR_CUDA = 6,              /* CUDA runtime error (see ctap_last_error)*/
    CTAP_ERR_TIMEOUT = 7,           /* host-side wait exceeded the timeout    */
    CTAP_ERR_NONFINITE = 8          /* a reduction produced NaN or Inf        */
} ctap_status;

/* Create a plan for an nx x ny x nz grid over `box` (6 doubles, host).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream); every launch
 * of the plan goes to it.  Builds the FP64-generated twiddle tables on the
 * host and uploads them.  *out receives the plan (NULL on error). */
ctap_status ctap_plan_create(int nx, int ny, int nz, const double *box,
                             ctap_dtype dtype, void *cuda_stream, ctap_plan_t *out);

/* Batched replicas (the analogue of the paper's parameter sweep, Fig. 6):
 * `batch` independent wave functions of the same grid in one psi buffer,
 * [batch][nz][ny][nx], advanced together by every ctap_step launch (small
 * grids fill the GPU).  Replicas differ only in their potential, which must
 * be in product form (ctap_set_potential_product: the same for all;
 * ctap_set_guides: the same for all; ctap_set_guides_batched: a middle-guide
 * depth per replica); ctap_add_potential_z applies to every replica.
 * ctap_observables returns 6 values per replica; ctap_density_xz and
 * ctap_get_potential cover all replicas.  Real time only (CTAP_IMAG,
 * ctap_set_guides_spline and ctap_adjoint need batch == 1 and return
 * CTAP_ERR_INVALID_ARG otherwise).  batch in [1, CTAP_MAX_BATCH];
 * ctap_plan_create is batch == 1. */
#define CTAP_MAX_BATCH 1024
ctap_status ctap_plan_create_batched(int nx, int ny, int nz, int batch, const double *box,
                                     ctap_dtype dtype, void *cuda_stream, ctap_plan_t *out);

/* Free every device and host resource of the plan (waits for its stream).
 * Passing NULL returns CTAP_ERR_INVALID_ARG. */
ctap_status ctap_plan_destroy(ctap_plan_t plan);

/* Potential, general form (Sec. III: any V(x,y,z) on the grid).
 * V: host FP64 [nz][ny][nx], copied.  Kept on the device in the plan's
 * precision (FP32 for CTAP_C64, FP64 for CTAP_C128). */
ctap_status ctap_set_potential(ctap_plan_t plan, const double *V);

/* Potential of an atom chip (Sec. III): thin straight current-carrying wire
 * segments (the Biot-Savart law, Eq. 4) plus a uniform field (the bias field
 * that lifts the minimum above the wires, Eq. 5, and the field along the
 * wires), V = v_per_field |B| - v_offset, evaluated on the device in FP64
 * and stored in the general (dense) form.  seg: host FP64 [nseg][7] rows
 * (Ax, Ay, Az, Cx, Cy, Cz, I) in grid units, current I from A to C;
 * bias: host FP64 [3]; mu0_over_4pi: the Biot-Savart constant in the
 * caller's units (field per current, times length); v_per_field converts
 * |B| to the plan's energy unit.  A grid point on a segment's line gets no
 * field from that segment.  nseg in [1, CTAP_MAX_SEGMENTS]; batch == 1. */
#define CTAP_MAX_SEGMENTS 65536
ctap_status ctap_set_potential_wires(ctap_plan_t plan, int nseg, const double *seg,
                                     const double *bias, double mu0_over_4pi,
                                     double v_per_field, double v_offset);

/* Potential, additively separable form V = Vx(x) + Vy(y) + Vz(z)
 * (e.g. the harmonic trap): three host FP64 arrays of nx, ny, nz values.
 * Phase factors are generated per axis in FP64 on the host. */
ctap_status ctap_set_potential_separable(ctap_plan_t plan, const double *Vx,
                                         const double *Vy, const double *Vz);

/* Potential, product form V = g(y) H(x,z): gy host FP64 [ny], Hxz host FP64
 * [nz][nx]. */
ctap_status ctap_set_potential_product(ctap_plan_t plan, const double *gy,
                                       const double *Hxz);

/* Three Gaussian waveguides (the stand-in for the chip guides of Sec. III
 * and Fig. 1-3): V = -V0 sum_j exp(-((x - x_j(z))^2 + y^2)/(2 s^2)) with
 * centres x1z[nz], 0, x3z[nz] (host FP64).  Stored in product form.  When
 * set_regions != 0 the population regions become |x - x_j(z)| < halfwidth
 * around these centres (otherwise the previous regions are kept: a frozen
 * mask).  Clears any spline controls. */
ctap_status ctap_set_guides(ctap_plan_t plan, double V0, double s,
                            const double *x1z, const double *x3z,
                            double halfwidth, int set_regions);

/* The guides of ctap_set_guides with the middle guide's depth scaled per
 * replica: replica b has V = -V0 (G_1 + mid_scale[b] G_2 + G_3) (the paper
 * sweeps the middle-wire current I_M, Fig. 6).  mid_scale: host FP64
 * [batch]. */
ctap_status ctap_set_guides_batched(ctap_plan_t plan, double V0, double s, const double *x1z,
                                    const double *x3z, const double *mid_scale,
                                    double halfwidth, int set_regions);

/* Same guides with x_1(z) = -d12(z), x_3(z) = +d23(z), where d12 and d23
 * are natural cubic splines through nknots knots (knots_z ascending, host)
 * with values c12[m], c23[m].  Required before ctap_adjoint.  nknots in
 * [2, 64]. */
ctap_status ctap_set_guides_spline(ctap_plan_t plan, double V0, double s, int nknots,
                                   const double *knots_z, const double *c12,
                                   const double *c23, double halfwidth, int set_regions);

/* Add a z-only term Vz(z) (host FP64 [nz]) to the potential the plan holds,
 * e.g. the longitudinal harmonic trap of Sec. III that drives the atom along
 * the guides and refocuses it at the far turning point.  For the product
 * form the term is kept separately (V = g(y) H(x,z) + Vz(z): one extra phase
 * per z-plane, no extra memory traffic); for the dense and separable forms it
 * is folded into the stored potential.  Calls accumulate; any ctap_set_*
 * call replaces the whole potential including this term.  The adjoint
 * gradient is unaffected (Vz does not depend on the guide controls).
 * Errors: CTAP_ERR_NO_POTENTIAL before a potential is set,
 * CTAP_ERR_INVALID_ARG for a null pointer or a non-finite value. */
ctap_status ctap_add_potential_z(ctap_plan_t plan, const double *Vz);

/* Copy the potential the plan holds, evaluated in FP64 on the grid, into V
 * (host, [batch][nz][ny][nx]).  For checking the potential builders. */
ctap_status ctap_get_potential(ctap_plan_t plan, double *V);

/* Advance psi (device, in place) by nsteps Strang steps of size dt.
 * mode CTAP_REAL: exp(-i V dt/2), exp(-i |k|^2 dt/2); CTAP_IMAG: real
 * factors exp(-V dt/2), exp(-|k|^2 dt/2) and renormalisation to
 * sum |psi|^2 dV = 1 after every step (Sec. V ground-state preparation);
 * CTAP_REAL_KVK: real time with the kinetic factor split instead,
 * exp(-i |k|^2 dt/4) exp(-i V dt) exp(-i |k|^2 dt/4) per step (the
 * ordering of Sec. IV's four transforms per step; consecutive kinetic
 * halves merge, so it costs the same two passes per step).
 * Asynchronous on the plan stream.  nsteps == 0 is a no-op. */
ctap_status ctap_step(ctap_plan_t plan, void *psi, int nsteps, double dt, ctap_time mode);

/* FP64-accumulated observables of psi (device, not modified), host out[6]
 * (out[6 batch] for a batched plan, replica b at out + 6 b):
 *   out[0] = sum |psi|^2 dV                    (norm)
 *   out[1] = <T>, out[2] = <V>                  (normalised expectations)
 *   out[3..5] = population of guides 1..3: sum over |x - x_j(z)| < halfwidth
 *               of |psi|^2 dV (Sec. V, Fig. 4); 0 without guide regions.
 * Synchronises.  Returns CTAP_ERR_NONFINITE if any value is NaN/Inf. */
ctap_status ctap_observables(ctap_plan_t plan, const void *psi, double *out);

/* Gradient of the final population of guide `guide` (1..3) after nsteps
 * real-time steps from psi0 (device, not modified) with respect to the
 * spline controls of ctap_set_guides_spline (not in the paper; the
 * differentiable form of the Fig. 4 observable).  Reverse conjugate-phase
 * sweep lambda_n = S(-dt) lambda_{n+1}, lambda_N = M psi_N, with forward
 * states recomputed from checkpoints taken every K steps.  The population
 * region and psi0 are held fixed.  Outputs (host): *J, grad[0..m-1] =
 * dJ/dc12, grad[m..2m-1] = dJ/dc23 (m = nknots).  Synchronises. */
ctap_status ctap_adjoint(ctap_plan_t plan, const void *psi0, int nsteps, double dt,
                         int K, int guide, double *J, double *grad);

/* Density integrated over y (Sec. V, Fig. 5): out[z][x] = sum_y |psi|^2 dy,
 * FP64 accumulated in a fixed order, psi device (not modified), out host
 * [batch][nz][nx].  Synchronises. */
ctap_status ctap_density_xz(ctap_plan_t plan, const void *psi, double *out);

/* Wait for the plan's stream; CTAP_ERR_TIMEOUT after timeout_ms
 * (timeout_ms <= 0: the plan's default, see ctap_set_timeout). */
ctap_status ctap_sync(ctap_plan_t plan, int timeout_ms);

/* Host-side timeout for every synchronising call (default 60000 ms). */
ctap_status ctap_set_timeout(ctap_plan_t plan, int timeout_ms);

/* Kernel launches the plan has issued so far (for accounting). */
ctap_status ctap_launch_count(ctap_plan_t plan, long long *count);

/* Per-pass timing with CUDA events on the plan stream.  When enabled, every
 * launch of ctap_step / ctap_observables is bracketed by events;
 * ctap_pass_times writes, per pass kind (0 steady XY pass, 1 Z pass, 2 every
 * other launch: prologue/epilogue/observe XY passes, reductions), the number
 * of launches and the summed milliseconds since the last call (synchronises).
 * Graph replay is disabled while profiling is on. */
ctap_status ctap_set_profiling(ctap_plan_t plan, int enable);
ctap_status ctap_pass_times(ctap_plan_t plan, long long counts[3], double ms[3]);

/* Pass geometry chosen for the plan: info[0] = P (row classes per plane),
 * info[1] = rows per XY tile, info[2] = columns per Z tile, info[3] = bytes
 * of one psi, info[4] = fast-pass mask (1: specialised XY pass, 2:
 * specialised Z pass, 4: the in-place Z pass runs as a persistent ring
 * kernel, 8: the steady in-place XY pass runs as a persistent ring kernel,
 * 16: the real-time Z ring runs in packed FP32-pair arithmetic, 32: the
 * steady XY ring runs in packed FP32-pair arithmetic).  Bits 8 and 32 depend
 * on the potential set: the scalar XY ring takes the product form, the
 * packed one the product and the separable forms; both also need a time
 * step with |V|max dt <= 0.5 (a larger kick angle takes the one-tile-per-CTA
 * pass with the general kick).  CTAP_NO_PACKED=1 in
 * the environment at plan creation keeps the scalar ring kernels,
 * CTAP_NO_RING=1 the one-tile-per-CTA passes. */
ctap_status ctap_plan_info(ctap_plan_t plan, long long info[5]);

/* Largest element count ctap_norm_noalloc accepts (2^27). */
#define CTAP_NOALLOC_MAX_ELEMENTS (16384LL * 8192LL)

/* sum |psi|^2 dV of n complex elements (the value ctap_observables returns
 * in out[0]) without allocating anything.  The paper has no counterpart:
 * this exists for callers that must not call cudaMalloc -- for example a
 * process whose device memory is already held by another framework's
 * caching allocator, or a latency-critical loop that cannot take
 * cudaMalloc's implicit device synchronisation.  No plan is needed.
 *   psi: device, complex64 (dtype CTAP_C64) or complex128 (CTAP_C128),
 *        interleaved, n elements, caller-owned; dV: cell volume;
 *   out: DEVICE pointer to one double, caller-owned, written
 *        asynchronously on cuda_stream (NULL = legacy default stream).
 * FP64 partial sums go to a fixed 64 KiB file-scope device array that
 * every GPU loading the library holds until the process exits.  Each call
 * made outside stream capture looks up that array's device address
 * (cudaGetSymbolAddress) on the current device, so the address stays valid
 * across a device reset; a call made during capture reuses the address of
 * the last call outside capture on that device, so make one call on each
 * device before any stream capture (a captured call with none fails with
 * CTAP_ERR_CUDA).  All calls share the array: calls that
 * overlap on the GPU (other streams or host threads) race on it, calls on
 * one stream are ordered.  Every slot a call reads is written by the same
 * call, so nothing needs clearing in between.
 * Errors: CTAP_ERR_INVALID_ARG (null pointer, n < 1, non-finite dV),
 * CTAP_ERR_DTYPE, CTAP_ERR_UNSUPPORTED_SIZE when n exceeds
 * CTAP_NOALLOC_MAX_ELEMENTS, CTAP_ERR_CUDA on a runtime error. */
ctap_status ctap_norm_noalloc(const void *psi, long long n, ctap_dtype dtype, double dV,
                              void *cuda_stream, double *out);

/* Arithmetic peaks of the current device, measured (not in the paper: the
 * denominators of the arithmetic rooflines the bench reports).  Runs three
 * FMA-bound probe kernels on cuda_stream (NULL = legacy default stream),
 * each timed with CUDA events after a warm-up launch, and writes host
 * out[0] = FP32 TFLOP/s with scalar FMA, out[1] = FP32 TFLOP/s with the
 * packed FP32-pair FMA (fma.rn.f32x2), out[2] = FP64 TFLOP/s (an FMA counts
 * two operations).  Synchronises; takes a few milliseconds.  Errors:
 * CTAP_ERR_INVALID_ARG (null out), CTAP_ERR_CUDA. */
ctap_status ctap_measure_fma_peaks(void *cuda_stream, double *out);

/* Record of the bounds-checked build (compiled with -DCTAP_DEBUG_BOUNDS;
 * not in the paper).  That build compares every shared-memory and HBM index
 * of the production passes with its buffer before the access; the first
 * violation is recorded and the access skipped (nothing traps).  *out = 0:
 * no violation since the last clear; > 0: check site << 48 | index of the
 * first violation; -1: a normal build without checks.  clear != 0 resets
 * the record.  Synchronises the device.  Errors: CTAP_ERR_INVALID_ARG (null
 * out), CTAP_ERR_CUDA. */
ctap_status ctap_debug_bounds(int clear, long long *out);

const char *ctap_status_string(ctap_status s);
const char *ctap_last_error(ctap_plan_t plan);   /* plan-local message; "" if none */
const char *ctap_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CTAP_H */
