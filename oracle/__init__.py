"""FP64 CPU oracle for the split-step Fourier hot path -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference leg may import this package.  The product (``paper_1309_2451_b300``)
never imports it and shares no code with it.

Everything arithmetic lives in ``oracle.c`` (plain C, FP64, own radix-2 FFT);
this module only marshals numpy arrays, except for the natural cubic spline
basis, which is written out here in numpy.

Paper: Morgan, O'Riordan, Crowley, O'Sullivan, Busch, "Coherent transport by
adiabatic passage on atom chips".  Sec. IV states the method (Fourier split
operator, FFT-based); Sec. V the initial state (transverse ground state of
the left guide, found numerically, times a longitudinal Gaussian) and the
observable (population of each guide versus time, Fig. 4).

Arrays are numpy complex128 of shape (nz, ny, nx) (x fastest).  ``box`` is
(xmin, xmax, ymin, ymax, zmin, zmax); grid points are lo + i (hi - lo)/n.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.orc_fft1d.argtypes = [_dp, ctypes.c_long, ctypes.c_long, ctypes.c_int]
        lib.orc_fft3d.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_step.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.orc_step_kvk.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                     ctypes.c_double, ctypes.c_int]
        lib.orc_observables.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        _dp, _dp, ctypes.c_double, _dp]
        lib.orc_ctap_potential.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                           ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.orc_ctap_dvdx.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                      ctypes.c_double, ctypes.c_double, _dp]
        lib.orc_adjoint.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                    ctypes.c_double, ctypes.c_int, _dp, _dp, _dp,
                                    _dp, _dp, _dp]
        lib.orc_wire_field.argtypes = [_dp, ctypes.c_long, ctypes.c_int, _dp, _dp,
                                       ctypes.c_double, _dp]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _box(box):
    b = _f64(box)
    if b.shape != (6,):
        raise ValueError("box must hold 6 numbers")
    return b


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def num_threads():
    """OpenMP threads the oracle uses (all host cores unless OMP_NUM_THREADS)."""
    return int(_load().orc_num_threads())


def set_num_threads(n):
    """OpenMP threads for the following oracle calls (timing only; the
    results do not depend on it: every parallel loop runs independent lines)."""
    _load().orc_set_num_threads(int(n))


# ------------------------------------------------------------------ grids

def grid_axis(n, lo, hi):
    """Periodic grid lo + i (hi - lo)/n, i = 0..n-1 (upper edge excluded)."""
    return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / n)


def k_axis(n, lo, hi):
    """Angular wavenumbers 2 pi m/(hi - lo), m in FFT order."""
    m = np.arange(n)
    m = np.where(m < (n + 1) // 2, m, m - n)
    if n == 1:
        m = np.zeros(1, dtype=np.int64)
    return 2.0 * np.pi * m / (hi - lo)


# --------------------------------------------------------------- transforms

def fft1d(a, direction):
    """Radix-2 FFT along the last axis.  direction -1 forward, +1 inverse (1/n)."""
    out = _c128(a).copy()
    n = out.shape[-1]
    _check(_load().orc_fft1d(_ptr(out.view(np.float64)), n, out.size // max(n, 1), direction),
           "fft1d")
    return out


def fft3d(psi, direction):
    """3D radix-2 FFT of a (nz, ny, nx) array.  direction -1 forward, +1 inverse."""
    out = _c128(psi).copy()
    nz, ny, nx = out.shape
    _check(_load().orc_fft3d(_ptr(out.view(np.float64)), nx, ny, nz, direction), "fft3d")
    return out


# --------------------------------------------------------------- split step

def step(psi, V, box, dt, nsteps, imag=False, order="VKV"):
    """nsteps Strang split steps of size dt; returns a new array.

    Sec. IV: Fourier split-operator method.  order "VKV" is V/2, K, V/2;
    order "KVK" is K/2, V, K/2 (real time only).  imag=True is the
    imaginary-time variant (real factors exp(-V dt/2), exp(-k^2 dt/2)) with
    renormalisation to sum |psi|^2 dV = 1 after every step (Sec. V obtains the
    transverse ground state numerically)."""
    out = _c128(psi).copy()
    nz, ny, nx = out.shape
    Vd = _f64(V)
    if Vd.shape != out.shape:
        raise ValueError("V must have the shape of psi")
    if order == "KVK":
        if imag:
            raise ValueError("the K/2 V K/2 ordering is real time only")
        _check(_load().orc_step_kvk(_ptr(out.view(np.float64)), _ptr(Vd), nx, ny, nz,
                                    _ptr(_box(box)), float(dt), int(nsteps)), "step_kvk")
        return out
    if order != "VKV":
        raise ValueError("order must be 'VKV' or 'KVK'")
    _check(_load().orc_step(_ptr(out.view(np.float64)), _ptr(Vd), nx, ny, nz, _ptr(_box(box)),
                            float(dt), int(nsteps), 1 if imag else 0), "step")
    return out


def density_xz(psi, box):
    """Density integrated over y, n(z, x) = sum_y |psi|^2 dy, in FP64: the
    quantity Fig. 5 shows in the x-z plane (Sec. V)."""
    a = _c128(psi)
    ny = a.shape[1]
    dy = (box[3] - box[2]) / ny
    return (a.real ** 2 + a.imag ** 2).sum(axis=1) * dy


def observables(psi, V, box, centres=None, halfwidth=1.5):
    """[norm, <T>, <V>, P_1, P_2, P_3] in FP64.

    norm = sum |psi|^2 dV; <T>, <V> are normalised expectation values (<T>
    from the spectrum of psi); P_j = sum over |x - x_j(z)| < halfwidth of
    |psi|^2 dV, the population of guide j (Sec. V, Fig. 4).  centres is a
    (3, nz) array of guide centres x_j(z)."""
    a = _c128(psi)
    nz, ny, nx = a.shape
    Vd = _f64(V) if V is not None else None
    xc = _f64(centres) if centres is not None else None
    if xc is not None and xc.shape != (3, nz):
        raise ValueError("centres must have shape (3, nz)")
    out = np.zeros(6)
    lib = _load()
    _check(lib.orc_observables(_ptr(a.view(np.float64)), _ptr(Vd) if Vd is not None else None,
                               nx, ny, nz, _ptr(_box(box)),
                               _ptr(xc) if xc is not None else None, float(halfwidth),
                               _ptr(out)), "observables")
    return out


# ------------------------------------------------------- guide potential

def ctap_potential(shape, box, V0, s, x1z, x3z):
    """Three Gaussian waveguides centred at x_1(z), 0, x_3(z):
    V = -V0 sum_j exp(-((x - x_j(z))^2 + y^2)/(2 s^2))."""
    nz, ny, nx = shape
    V = np.empty(shape)
    _check(_load().orc_ctap_potential(_ptr(V), nx, ny, nz, _ptr(_box(box)), float(V0), float(s),
                                      _ptr(_f64(x1z)), _ptr(_f64(x3z))), "ctap_potential")
    return V


def wire_field(points, segments, bias, k):
    """Magnetic field of thin straight current segments plus a uniform field
    (Sec. III, Eq. 4-5) at points (n, 3): segments (m, 7) rows
    (Ax, Ay, Az, Cx, Cy, Cz, I), bias (3,), k = mu0/(4 pi) in the caller's
    units.  Returns (n, 3)."""
    P = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    S = np.ascontiguousarray(segments, dtype=np.float64).reshape(-1, 7)
    out = np.zeros_like(P)
    _check(_load().orc_wire_field(_ptr(P), P.shape[0], S.shape[0], _ptr(S), _ptr(_f64(bias)),
                                  float(k), _ptr(out)), "wire_field")
    return out


def wire_potential(shape, box, segments, bias, k, v_per_field, v_offset=0.0):
    """Magnetic trapping potential V = v_per_field |B| - v_offset on the grid
    (Sec. III: the atom-chip waveguides)."""
    nz, ny, nx = shape
    x = grid_axis(nx, box[0], box[1])
    y = grid_axis(ny, box[2], box[3])
    z = grid_axis(nz, box[4], box[5])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    B = wire_field(pts, segments, bias, k)
    return (v_per_field * np.sqrt((B * B).sum(axis=1)) - v_offset).reshape(shape)


def ctap_dvdx(shape, box, V0, s, xjz):
    """dV/dx_j of one guide centred at x_j(z)."""
    nz, ny, nx = shape
    D = np.empty(shape)
    _check(_load().orc_ctap_dvdx(_ptr(D), nx, ny, nz, _ptr(_box(box)), float(V0), float(s),
                                 _ptr(_f64(xjz))), "ctap_dvdx")
    return D


def guide_mask(shape, box, xjz, halfwidth):
    """Indicator of |x - x_j(z)| < halfwidth (all y)."""
    nz, ny, nx = shape
    x = grid_axis(nx, box[0], box[1])
    m = (np.abs(x[None, :] - np.asarray(xjz, dtype=np.float64)[:, None]) < halfwidth)
    return np.broadcast_to(m[:, None, :], shape).astype(np.float64)


# ---------------------------------------------------------------- spline

def natural_spline_basis(knots, z):
    """Cardinal basis of the natural cubic interpolating spline.

    Returns B with shape (len(knots), len(z)) such that the natural spline
    through values c_m at the knots is sum_m c_m B[m](z).  Each column of the
    knot-value identity is interpolated: second derivatives M solve the usual
    tridiagonal continuity system with M_0 = M_last = 0.  Points outside the
    knot range use the nearest end interval's cubic."""
    t = np.asarray(knots, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    m = t.size
    h = np.diff(t)
    # system for interior second derivatives M_1..M_{m-2}
    A = np.zeros((m, m))
    A[0, 0] = 1.0
    A[-1, -1] = 1.0
    R = np.zeros((m, m))       # right-hand side for every unit data vector
    Y = np.eye(m)
    for i in range(1, m - 1):
        A[i, i - 1] = h[i - 1]
        A[i, i] = 2.0 * (h[i - 1] + h[i])
        A[i, i + 1] = h[i]
        R[i] = 6.0 * ((Y[i + 1] - Y[i]) / h[i] - (Y[i] - Y[i - 1]) / h[i - 1])
    M = np.linalg.solve(A, R)  # M[i, col]: second derivative at knot i for data e_col
    idx = np.clip(np.searchsorted(t, z, side="right") - 1, 0, m - 2)
    t0, t1, hh = t[idx], t[idx + 1], h[idx]
    a = (t1 - z)
    b = (z - t0)
    B = (M[idx] * (a ** 3)[:, None] / (6 * hh)[:, None]
         + M[idx + 1] * (b ** 3)[:, None] / (6 * hh)[:, None]
         + (Y[idx] / hh[:, None] - M[idx] * hh[:, None] / 6) * a[:, None]
         + (Y[idx + 1] / hh[:, None] - M[idx + 1] * hh[:, None] / 6) * b[:, None])
    return B.T.copy()


# ---------------------------------------------------------------- adjoint

def adjoint(psi0, V, box, dt, nsteps, mask, W1, W3):
    """J = sum mask |psi_N|^2 dV and the per-slice sensitivities
    R_j(z) = dt sum_n w_n sum_{x,y} Im(conj(lambda_n) W_j psi_n) dV (see
    oracle.c).  Returns (J, R1, R3)."""
    a = _c128(psi0)
    nz, ny, nx = a.shape
    R1 = np.zeros(nz)
    R3 = np.zeros(nz)
    J = np.zeros(1)
    _check(_load().orc_adjoint(_ptr(a.view(np.float64)), _ptr(_f64(V)), nx, ny, nz,
                               _ptr(_box(box)), float(dt), int(nsteps), _ptr(_f64(mask)),
                               _ptr(_f64(W1)), _ptr(_f64(W3)), _ptr(J), _ptr(R1), _ptr(R3)),
           "adjoint")
    return float(J[0]), R1, R3


def ctap_gradient(psi0, box, V0, s, knots, c12, c23, dt, nsteps, guide_index=2,
                  halfwidth=1.5):
    """Gradient of the final population of one guide with respect to the
    spline controls of d12(z) and d23(z) (x_1 = -d12, x_3 = +d23).

    The population region is the one at the given controls and is held fixed
    (frozen mask); psi0 is held fixed.  Returns (J, grad) with grad[:m] =
    dJ/dc12, grad[m:] = dJ/dc23."""
    nz, ny, nx = np.shape(psi0)
    shape = (nz, ny, nx)
    z = grid_axis(nz, box[4], box[5])
    B = natural_spline_basis(knots, z)
    d12 = np.asarray(c12, dtype=np.float64) @ B
    d23 = np.asarray(c23, dtype=np.float64) @ B
    x1, x3 = -d12, d23
    V = ctap_potential(shape, box, V0, s, x1, x3)
    centres = np.stack([x1, np.zeros(nz), x3])
    mask = guide_mask(shape, box, centres[guide_index], halfwidth)
    W1 = ctap_dvdx(shape, box, V0, s, x1)
    W3 = ctap_dvdx(shape, box, V0, s, x3)
    J, R1, R3 = adjoint(psi0, V, box, dt, nsteps, mask, W1, W3)
    # chain rule: dx_1/dc12_m = -B_m(z), dx_3/dc23_m = +B_m(z)
    g12 = -(B @ R1)
    g23 = B @ R3
    return J, np.concatenate([g12, g23])


def ctap_objective(psi0, box, V0, s, knots, c12, c23, dt, nsteps, mask):
    """J(c) = sum mask |psi_N|^2 dV for the potential built from spline
    controls (c12, c23), with a caller-supplied (frozen) mask."""
    nz, ny, nx = np.shape(psi0)
    z = grid_axis(nz, box[4], box[5])
    B = natural_spline_basis(knots, z)
    x1 = -(np.asarray(c12, dtype=np.float64) @ B)
    x3 = np.asarray(c23, dtype=np.float64) @ B
    V = ctap_potential((nz, ny, nx), box, V0, s, x1, x3)
    psiN = step(psi0, V, box, dt, nsteps)
    dv = (box[1] - box[0]) / nx * (box[3] - box[2]) / ny * (box[5] - box[4]) / nz
    return float(np.sum(mask * np.abs(psiN) ** 2) * dv)
