"""ctap_norm_noalloc: the norm reduction for callers that must not call
cudaMalloc (for example when another framework's caching allocator already
holds the device memory, or in a loop that cannot take cudaMalloc's implicit
device synchronisation).  Its partial sums live in a fixed device array
inside the library instead of plan-allocated scratch.

Checked through the C ABI against the existing entry point
(ctap_observables, out[0]) on two calls in a row -- the second on a smaller
state, so stale partial sums left by the first call would show -- with the
tolerances the observables tests use (1e-12 complex128, 1e-6 complex64).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1309_2451_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2451_b300 import build, ctap as c
    build.build()
    c.lib()
    return c


def _state(shape, seed, dtype):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    t = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(a).to("cuda", t)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-6)])
def test_norm_noalloc_matches_observables_on_two_calls(ctap, dtype, tol):
    box = wl.CTAP_BOX
    cases = [(256, 128, 64), (16, 32, 16)]           # 2^21 points, then 2^13
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed, shape in enumerate(cases):
        psi = _state(shape, seed, dtype)
        plan = ctap.Plan(shape, box, dtype)
        plan.set_potential(np.zeros(shape))
        ref = plan.observables(psi)[0]
        plan.close()
        ctap.norm_noalloc(psi, wl.cell_volume(shape, box), out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= tol * abs(ref), (shape, got, ref)


def test_norm_noalloc_rejects_oversize_and_bad_args(ctap):
    import ctypes
    lib = ctap.lib()
    psi = _state((8, 8, 8), 0, "c64")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    too_many = ctap.NOALLOC_MAX_ELEMENTS + 1
    # rejected from the size alone, before any launch
    assert lib.ctap_norm_noalloc(vp(psi.data_ptr()), too_many, 0, 1.0, None,
                                 vp(out.data_ptr())) == 2
    assert lib.ctap_norm_noalloc(None, 512, 0, 1.0, None, vp(out.data_ptr())) == 1
    assert lib.ctap_norm_noalloc(vp(psi.data_ptr()), 0, 0, 1.0, None, vp(out.data_ptr())) == 1
    assert lib.ctap_norm_noalloc(vp(psi.data_ptr()), 512, 5, 1.0, None, vp(out.data_ptr())) == 3
