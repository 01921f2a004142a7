"""ctypes binding of libctap (include/ctap.h): argument marshalling only.

Every step of the propagation runs in the library's CUDA kernels; PyTorch
supplies device memory (psi is a CUDA tensor) and the stream.  There is no
CPU fallback: without the built library every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CTAP_LIB=debug selects the bounds-checked build (build.build(debug=True))
LIB_PATH = os.path.join(_HERE, "libctap_debug.so" if os.environ.get("CTAP_LIB") == "debug"
                        else "libctap.so")

CTAP_C64, CTAP_C128, CTAP_C128_DF = 0, 1, 2
CTAP_REAL, CTAP_IMAG, CTAP_REAL_KVK = 0, 1, 2
STATUS = ["ok", "invalid argument", "unsupported size", "dtype mismatch", "no potential",
          "out of memory", "CUDA error", "timeout", "non-finite result"]

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class CtapError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        name = STATUS[code] if 0 <= code < len(STATUS) else f"status {code}"
        super().__init__(f"ctap: {name}" + (f" ({msg})" if msg else ""))


def lib():
    """Load libctap.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libctap.so not built at {LIB_PATH}; run "
                           "paper_1309_2451_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "ctap_plan_create": [i, i, i, _dp, i, _vp, ctypes.POINTER(_vp)],
        "ctap_plan_create_batched": [i, i, i, i, _dp, i, _vp, ctypes.POINTER(_vp)],
        "ctap_set_guides_batched": [_vp, d, d, _dp, _dp, _dp, d, i],
        "ctap_set_potential_wires": [_vp, i, _dp, _dp, d, d, d],
        "ctap_plan_destroy": [_vp],
        "ctap_set_potential": [_vp, _dp],
        "ctap_set_potential_separable": [_vp, _dp, _dp, _dp],
        "ctap_set_potential_product": [_vp, _dp, _dp],
        "ctap_set_guides": [_vp, d, d, _dp, _dp, d, i],
        "ctap_set_guides_spline": [_vp, d, d, i, _dp, _dp, _dp, d, i],
        "ctap_get_potential": [_vp, _dp],
        "ctap_add_potential_z": [_vp, _dp],
        "ctap_density_xz": [_vp, _vp, _dp],
        "ctap_step": [_vp, _vp, i, d, i],
        "ctap_observables": [_vp, _vp, _dp],
        "ctap_adjoint": [_vp, _vp, i, d, i, i, _dp, _dp],
        "ctap_sync": [_vp, i],
        "ctap_set_timeout": [_vp, i],
        "ctap_launch_count": [_vp, ctypes.POINTER(ll)],
        "ctap_set_profiling": [_vp, i],
        "ctap_pass_times": [_vp, ctypes.POINTER(ll), _dp],
        "ctap_plan_info": [_vp, ctypes.POINTER(ll)],
        "ctap_norm_noalloc": [_vp, ll, i, d, _vp, _vp],
        "ctap_measure_fma_peaks": [_vp, _dp],
        "ctap_debug_bounds": [i, ctypes.POINTER(ll)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    for name in ("ctap_status_string", "ctap_version"):
        getattr(L, name).restype = ctypes.c_char_p
    L.ctap_status_string.argtypes = [ctypes.c_int]
    L.ctap_last_error.argtypes = [_vp]
    L.ctap_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    """Names of the functions the binding expects the library to export."""
    return ["ctap_plan_create", "ctap_plan_destroy", "ctap_set_potential",
            "ctap_set_potential_separable", "ctap_set_potential_product", "ctap_set_guides",
            "ctap_set_guides_spline", "ctap_get_potential", "ctap_step", "ctap_observables",
            "ctap_adjoint", "ctap_sync", "ctap_set_timeout", "ctap_launch_count",
            "ctap_set_profiling", "ctap_pass_times", "ctap_plan_info", "ctap_status_string",
            "ctap_last_error", "ctap_version", "ctap_norm_noalloc", "ctap_add_potential_z",
            "ctap_density_xz", "ctap_plan_create_batched", "ctap_set_guides_batched",
            "ctap_set_potential_wires", "ctap_measure_fma_peaks",
            "ctap_debug_bounds"]


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _p(a):
    return a.ctypes.data_as(_dp)


class Plan:
    """A split-step plan for psi of shape (nz, ny, nx) on `box`.

    dtype "c64" (FP32 bulk, FP64 tables and reductions) or "c128".  batch > 1
    makes a plan for `batch` independent replicas, psi of shape
    (batch, nz, ny, nx) (product-form potentials, real time)."""

    def __init__(self, shape, box, dtype="c64", stream=None, batch=1):
        import torch
        self._torch = torch
        nz, ny, nx = (int(s) for s in shape)
        self.shape = (nz, ny, nx)
        self.batch = int(batch)
        self.psi_shape = self.shape if self.batch == 1 else (self.batch,) + self.shape
        self.box = tuple(float(b) for b in box)
        # "c128df": complex128 psi, transforms in double-float (FP32-pair) arithmetic
        self.dtype = {"c64": CTAP_C64, "c128": CTAP_C128, "c128df": CTAP_C128_DF,
                      torch.complex64: CTAP_C64, torch.complex128: CTAP_C128}[dtype]
        self.torch_dtype = torch.complex64 if self.dtype == CTAP_C64 else torch.complex128
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _vp()
        self._h = None
        self._check(lib().ctap_plan_create_batched(nx, ny, nz, self.batch, _p(_f64(self.box, 6)),
                                                   self.dtype, _vp(stream.cuda_stream),
                                                   ctypes.byref(h)))
        self._h = h

    # ---------------------------------------------------------------- util
    def _check(self, rc):
        if rc != 0:
            msg = ""
            if getattr(self, "_h", None):
                msg = lib().ctap_last_error(self._h).decode()
            raise CtapError(rc, msg)

    def close(self):
        if self._h:
            lib().ctap_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _psi(self, psi):
        t = self._torch
        if not isinstance(psi, t.Tensor) or not psi.is_cuda:
            raise TypeError("psi must be a CUDA tensor")
        if psi.dtype != self.torch_dtype:
            raise CtapError(3, f"psi is {psi.dtype}, plan is {self.torch_dtype}")
        if tuple(psi.shape) != self.psi_shape or not psi.is_contiguous():
            raise ValueError(f"psi must be a contiguous {self.psi_shape} tensor")
        return _vp(psi.data_ptr())

    # ----------------------------------------------------------- potential
    def set_potential(self, V):
        self._check(lib().ctap_set_potential(self._h, _p(_f64(V, int(np.prod(self.psi_shape))))))

    def set_potential_wires(self, segments, bias, mu0_over_4pi, v_per_field, v_offset=0.0):
        """Atom-chip potential v_per_field |B| - v_offset from thin wire
        segments (rows A, C, I) and a uniform field (Sec. III, Eq. 4-5)."""
        seg = _f64(segments)
        if seg.size % 7:
            raise ValueError("segments must have 7 values per row")
        self._check(lib().ctap_set_potential_wires(self._h, seg.size // 7, _p(seg),
                                                   _p(_f64(bias, 3)), float(mu0_over_4pi),
                                                   float(v_per_field), float(v_offset)))

    def set_potential_separable(self, Vx, Vy, Vz):
        nz, ny, nx = self.shape
        self._check(lib().ctap_set_potential_separable(self._h, _p(_f64(Vx, nx)),
                                                       _p(_f64(Vy, ny)), _p(_f64(Vz, nz))))

    def set_potential_product(self, gy, Hxz):
        nz, ny, nx = self.shape
        self._check(lib().ctap_set_potential_product(self._h, _p(_f64(gy, ny)),
                                                     _p(_f64(Hxz, nz * nx))))

    def set_guides(self, V0, s, x1z, x3z, halfwidth=1.5, set_regions=True):
        nz = self.shape[0]
        self._check(lib().ctap_set_guides(self._h, float(V0), float(s), _p(_f64(x1z, nz)),
                                          _p(_f64(x3z, nz)), float(halfwidth),
                                          1 if set_regions else 0))

    def set_guides_batched(self, V0, s, x1z, x3z, mid_scale, halfwidth=1.5, set_regions=True):
        """Guides with the middle guide's depth scaled by mid_scale[b] in replica b."""
        nz = self.shape[0]
        self._check(lib().ctap_set_guides_batched(self._h, float(V0), float(s), _p(_f64(x1z, nz)),
                                                  _p(_f64(x3z, nz)), _p(_f64(mid_scale, self.batch)),
                                                  float(halfwidth), 1 if set_regions else 0))

    def set_guides_spline(self, V0, s, knots, c12, c23, halfwidth=1.5, set_regions=True):
        k = _f64(knots)
        self._check(lib().ctap_set_guides_spline(self._h, float(V0), float(s), k.size, _p(k),
                                                 _p(_f64(c12, k.size)), _p(_f64(c23, k.size)),
                                                 float(halfwidth), 1 if set_regions else 0))
        self.nknots = k.size

    def add_potential_z(self, Vz):
        """Add a z-only term Vz(z) (e.g. the longitudinal trap) to the potential."""
        self._check(lib().ctap_add_potential_z(self._h, _p(_f64(Vz, self.shape[0]))))

    def get_potential(self):
        V = np.empty(self.psi_shape)
        self._check(lib().ctap_get_potential(self._h, _p(V)))
        return V

    # ---------------------------------------------------------- propagation
    def step(self, psi, nsteps, dt, imag=False, order="VKV"):
        """order "VKV" (V/2 K V/2) or "KVK" (K/2 V K/2, real time only)."""
        if order == "KVK":
            if imag:
                raise ValueError("the K/2 V K/2 ordering is real time only")
            mode = CTAP_REAL_KVK
        elif order == "VKV":
            mode = CTAP_IMAG if imag else CTAP_REAL
        else:
            raise ValueError("order must be 'VKV' or 'KVK'")
        self._check(lib().ctap_step(self._h, self._psi(psi), int(nsteps), float(dt), mode))
        return psi

    def density_xz(self, psi):
        """sum_y |psi|^2 dy as an (nz, nx) FP64 array (Fig. 5)."""
        out = np.zeros((self.batch * self.shape[0], self.shape[2]))
        self._check(lib().ctap_density_xz(self._h, self._psi(psi), _p(out)))
        return out if self.batch == 1 else out.reshape(self.batch, self.shape[0], self.shape[2])

    def observables(self, psi):
        """[norm, <T>, <V>, P_1, P_2, P_3]; shape (batch, 6) for batched plans."""
        out = np.zeros(6 * self.batch)
        self._check(lib().ctap_observables(self._h, self._psi(psi), _p(out)))
        return out if self.batch == 1 else out.reshape(self.batch, 6)

    def adjoint(self, psi0, nsteps, dt, K=32, guide=3):
        m = getattr(self, "nknots", 0)
        J = np.zeros(1)
        grad = np.zeros(2 * max(m, 1))
        self._check(lib().ctap_adjoint(self._h, self._psi(psi0), int(nsteps), float(dt), int(K),
                                       int(guide), _p(J), _p(grad)))
        return float(J[0]), grad[:2 * m]

    def sync(self, timeout_ms=0):
        self._check(lib().ctap_sync(self._h, int(timeout_ms)))

    def set_timeout(self, ms):
        self._check(lib().ctap_set_timeout(self._h, int(ms)))

    @property
    def launch_count(self):
        c = ctypes.c_longlong()
        self._check(lib().ctap_launch_count(self._h, ctypes.byref(c)))
        return c.value

    def set_profiling(self, on=True):
        self._check(lib().ctap_set_profiling(self._h, 1 if on else 0))

    def pass_times(self):
        counts = (ctypes.c_longlong * 3)()
        ms = np.zeros(3)
        self._check(lib().ctap_pass_times(self._h, counts, _p(ms)))
        return list(counts), ms

    def info(self):
        out = (ctypes.c_longlong * 5)()
        self._check(lib().ctap_plan_info(self._h, out))
        keys = ("row_classes", "rows_per_xy_tile", "cols_per_z_tile", "psi_bytes", "fast_mask")
        return dict(zip(keys, list(out)))


def _adjoint_function():
    import torch

    class CtapAdjoint(torch.autograd.Function):
        """J(c12, c23) = final population of one guide after nsteps steps from
        psi0, for guide separations given by natural-spline controls.  The
        backward pass returns the adjoint gradient computed by libctap's reverse
        conjugate-phase sweep (checkpointed every K steps)."""

        @staticmethod
        def forward(ctx, c12, c23, plan, psi0, nsteps, dt, K, guide, V0, s, knots, halfwidth):
            plan.set_guides_spline(V0, s, knots, c12.detach().cpu().numpy(),
                                   c23.detach().cpu().numpy(), halfwidth, set_regions=True)
            J, grad = plan.adjoint(psi0, nsteps, dt, K, guide)
            m = len(knots)
            ctx.save_for_backward(torch.as_tensor(grad[:m], dtype=c12.dtype),
                                  torch.as_tensor(grad[m:], dtype=c23.dtype))
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            g12, g23 = ctx.saved_tensors
            return (gJ * g12, gJ * g23) + (None,) * 10

    return CtapAdjoint


_CtapAdjoint = None


def ctap_adjoint_apply(c12, c23, plan, psi0, nsteps, dt, K=32, guide=3, V0=20.0, s=1.0,
                       knots=None, halfwidth=1.5):
    """torch.autograd entry: returns J as a 0-d tensor differentiable in c12, c23."""
    global _CtapAdjoint
    if _CtapAdjoint is None:
        _CtapAdjoint = _adjoint_function()
    return _CtapAdjoint.apply(c12, c23, plan, psi0, nsteps, dt, K, guide, V0, s, knots,
                              halfwidth)


def debug_bounds(clear=True):
    """Record of the bounds-checked build: 0 (no violation), site << 48 |
    index of the first violation, or -1 for a build without checks."""
    v = ctypes.c_longlong()
    rc = lib().ctap_debug_bounds(1 if clear else 0, ctypes.byref(v))
    if rc != 0:
        raise CtapError(rc, "ctap_debug_bounds")
    return v.value


def measure_fma_peaks(stream=None):
    """Measured FP32 (scalar FMA), FP32 (packed pair FMA) and FP64 TFLOP/s of
    the current device (ctap_measure_fma_peaks)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    out = np.zeros(3)
    rc = lib().ctap_measure_fma_peaks(_vp(stream.cuda_stream), _p(out))
    if rc != 0:
        raise CtapError(rc, "ctap_measure_fma_peaks")
    return {"fp32_tflops": float(out[0]), "fp32x2_tflops": float(out[1]),
            "fp64_tflops": float(out[2])}


NOALLOC_MAX_ELEMENTS = 16384 * 8192


def norm_noalloc(psi, dV, out, stream=None):
    """sum |psi|^2 dV through ctap_norm_noalloc, which allocates nothing
    (for callers that must not call cudaMalloc).  psi: contiguous complex64
    or complex128 CUDA tensor; out: float64 CUDA tensor of one element,
    written asynchronously on `stream` (default: torch's current stream)."""
    import torch
    if psi.dtype not in (torch.complex64, torch.complex128) or not psi.is_cuda \
            or not psi.is_contiguous():
        raise TypeError("psi must be a contiguous complex CUDA tensor")
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
        raise TypeError("out must be a float64 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream()
    dtype = CTAP_C64 if psi.dtype == torch.complex64 else CTAP_C128
    rc = lib().ctap_norm_noalloc(_vp(psi.data_ptr()), psi.numel(), dtype, float(dV),
                                 _vp(stream.cuda_stream), _vp(out.data_ptr()))
    if rc != 0:
        raise CtapError(rc, "ctap_norm_noalloc")
    return out
