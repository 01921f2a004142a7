"""GPU parity: libctap (through the C ABI) against the FP64 oracle.

Tolerances:
* complex128 path: relative L2 <= 1e-12 after 100 steps (and ~1e-13 for a
  few steps);
* complex64 path: relative L2 <= 1e-5 after 1000 steps with |norm drift| <
  1e-6; a few steps stay below 1e-6 (FP32 rounding, ~2^-24 per operation,
  times the depth of the transforms).
"""
import numpy as np
import pytest

import oracle
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(psi, dtype):
    t = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(np.ascontiguousarray(psi)).to(device="cuda", dtype=t)


def random_state(shape, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return a / np.linalg.norm(a)


def harmonic_plan(ctap, shape, box, dtype, form="separable"):
    plan = ctap.Plan(shape, box, dtype)
    vx, vy, vz = wl.harmonic_parts(shape, box)
    if form == "separable":
        plan.set_potential_separable(vx, vy, vz)
    elif form == "dense":
        plan.set_potential(wl.harmonic_dense(shape, box))
    return plan, wl.harmonic_dense(shape, box)


def guides_plan(ctap, shape, box, dtype):
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z)
    plan = ctap.Plan(shape, box, dtype)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    return plan, V, c


# ------------------------------------------------------------ transforms
SHAPES = [(8, 8, 8), (1, 8, 8), (1, 16, 64), (32, 16, 8), (64, 32, 16), (16, 8, 128),
          (2, 128, 128), (4, 128, 256), (2, 256, 256), (128, 8, 8), (1024, 8, 16)]


def max_kinetic_phase(shape, box, dt):
    kmax = [np.pi * n / (box[2 * a + 1] - box[2 * a]) for a, n in enumerate(shape[::-1])]
    return 0.5 * sum(k * k for k in kmax) * dt


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c64", 1e-6)])
def test_harmonic_steps_match_oracle(ctap, shape, dtype, tol):
    """Separable potential: covers every row-class split P (1..8), ragged
    tiles (nz = 1, 8-point axes, 1024-point z-lines) and both precisions.

    White noise fills the whole spectrum, where the kinetic phase k^2 dt/2
    reaches ~1500 rad on the 1024-point axis; both sides reduce that angle in
    FP64 with an absolute error ~ eps64 * theta, so the FP64 tolerance grows
    with theta_max (the FP32 tables are reduced in FP64 before rounding and
    do not)."""
    box = (-7.0, 9.0, -8.0, 8.0, -6.5, 6.5)
    dt, n = 0.05, 3
    plan, V = harmonic_plan(ctap, shape, box, dtype)
    psi0 = random_state(shape, 1)
    psi = to_dev(psi0, dtype)
    plan.step(psi, n, dt)
    ref = oracle.step(psi0, V, box, dt, n)
    if dtype == "c128":
        tol += 4 * n * 2.2e-16 * max_kinetic_phase(shape, box, dt)
    assert rel(psi.cpu().numpy(), ref) < tol, plan.info()


@pytest.mark.parametrize("form", ["dense", "separable"])
def test_potential_forms(ctap, form):
    shape, box = (16, 32, 64), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    plan, V = harmonic_plan(ctap, shape, box, "c128", form)
    psi0 = wl.coherent_state(shape, box, 2.0)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 20, 0.01)
    assert rel(psi.cpu().numpy(), oracle.step(psi0, V, box, 0.01, 20)) < 1e-13


def test_product_potential(ctap):
    shape, box = (16, 64, 32), (-6.0, 6.0, -5.0, 5.0, -4.0, 4.0)
    rng = np.random.default_rng(5)
    gy = 1.0 + 0.3 * rng.standard_normal(shape[1])
    H = -3.0 + rng.standard_normal((shape[0], shape[2]))
    plan = ctap.Plan(shape, box, "c128")
    plan.set_potential_product(gy, H)
    V = gy[None, :, None] * H[:, None, :]
    assert np.array_equal(plan.get_potential(), V)
    psi0 = random_state(shape, 2)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 10, 0.02)
    assert rel(psi.cpu().numpy(), oracle.step(psi0, V, box, 0.02, 10)) < 1e-13


def test_guides_potential_matches_oracle(ctap):
    shape, box = (64, 32, 64), wl.CTAP_BOX
    plan, V, _ = guides_plan(ctap, shape, box, "c128")
    assert np.max(np.abs(plan.get_potential() - V)) < 1e-12


def test_spline_guides_match_oracle_basis(ctap):
    shape, box = (256, 8, 16), wl.CTAP_BOX
    c12, c23 = wl.spline_controls()
    plan = ctap.Plan(shape, box, "c128")
    plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, wl.KNOTS_Z, c12, c23)
    z = wl.axis(shape[0], box[4], box[5])
    B = oracle.natural_spline_basis(wl.KNOTS_Z, z)
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, -(c12 @ B), c23 @ B)
    assert np.max(np.abs(plan.get_potential() - V)) < 1e-11


# -------------------------------------------------------- long real time
def test_ctap_c128_100_steps(ctap):
    """complex128 guides run: <= 1e-12 relative L2 after 100 steps."""
    shape, box = (128, 64, 64), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c128")
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=4) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, "c128")
    plan.step(psi, 100, 0.005)
    ref = oracle.step(psi0, V, box, 0.005, 100)
    assert rel(psi.cpu().numpy(), ref) < 1e-12


def test_ctap_c64_1000_steps_accuracy_and_norm(ctap):
    """complex64 bulk: <= 1e-5 after 1000 steps, norm drift < 1e-6."""
    shape, box = (64, 32, 32), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=7) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, "c64")
    n0 = plan.observables(psi)[0]
    plan.step(psi, 1000, 0.005)
    ref = oracle.step(psi0, V, box, 0.005, 1000)
    assert rel(psi.cpu().numpy().astype(complex), ref) < 1e-5
    assert abs(plan.observables(psi)[0] / n0 - 1.0) < 1e-6


# ----------------------------------------------------------- imaginary time
@pytest.mark.parametrize("n", [128, 256])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_imaginary_time_guide_ground_state(ctap, dtype, tol, n):
    """The transverse prep of the guide workloads: nz = 1 plane with guide 1
    only, 200 imaginary-time steps at dtau = 0.01, renormalised each step
    (n = 256: the plane of the 256x256x1024 workload)."""
    shape, box = (1, n, n), wl.CTAP_BOX
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    plan = ctap.Plan(shape, box, dtype)
    # guide 1 alone, V = -V0 exp(-y^2/2) exp(-(x - x1)^2/2), in product form
    y = wl.axis(n, box[2], box[3])
    x = wl.axis(n, box[0], box[1])
    gy = np.exp(-y ** 2 / 2)
    H = -wl.V0 * np.exp(-(x - xc) ** 2 / 2)[None, :]
    plan.set_potential_product(gy, H)
    V = gy[None, :, None] * H[:, None, :]
    psi0 = wl.guide_seed_2d((n, n), box, xc)
    psi = to_dev(psi0, dtype)
    plan.step(psi, 200, 0.01, imag=True)
    ref = oracle.step(psi0, V, box, 0.01, 200, imag=True)
    got = psi.cpu().numpy().astype(complex)
    assert rel(got, ref) < tol
    assert abs(np.sum(np.abs(got) ** 2) * wl.cell_volume(shape, box) - 1.0) < 10 * tol


# --------------------------------------------------------------- observables
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-6)])
def test_observables_match_oracle(ctap, dtype, tol):
    shape, box = (64, 64, 32), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, dtype)
    psi0 = wl.gaussian_sum(shape, (-8, 8, -4, 4, -30, 30), seed=2) \
        * np.exp(1j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, dtype)
    got = plan.observables(psi)
    ref = oracle.observables(psi.cpu().numpy().astype(complex), V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(got, ref, rtol=tol, atol=tol * 1e-3), (got, ref)


def test_observables_separable_and_dense(ctap):
    shape, box = (32, 16, 32), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    psi0 = wl.coherent_state(shape, box, 1.5)
    for form in ("separable", "dense"):
        plan, V = harmonic_plan(ctap, shape, box, "c128", form)
        got = plan.observables(to_dev(psi0, "c128"))
        ref = oracle.observables(psi0, V, box)
        assert np.allclose(got[:3], ref[:3], rtol=1e-12, atol=1e-15)
        assert np.all(got[3:] == 0.0)


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-6), ("c128", 1e-12)])
@pytest.mark.parametrize("shape", [(64, 64, 64), (256, 64, 256)])
def test_observables_separable_on_specialised_passes(ctap, shape, dtype, tol):
    """Observables of the harmonic (separable) potential on grids that take
    the specialised XY pass: the observe pass applies no kick and must not
    touch the kick tables (which the observables call does not build)."""
    box = (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    plan, V = harmonic_plan(ctap, shape, box, dtype)
    assert plan.info()["fast_mask"] & 1, plan.info()
    psi0 = wl.gaussian_sum(shape, box, seed=0)
    psi = to_dev(psi0, dtype)
    got = plan.observables(psi)
    ref = oracle.observables(psi.cpu().numpy().astype(complex), V, box)
    assert np.allclose(got[:3], ref[:3], rtol=tol, atol=tol * 1e-3), (got, ref)
    plan.step(psi, 5, 0.005)
    got = plan.observables(psi)
    ref = oracle.observables(psi.cpu().numpy().astype(complex), V, box)
    assert np.allclose(got[:3], ref[:3], rtol=tol, atol=tol * 1e-3), (got, ref)


# ------------------------------------------------------------------ adjoint
ADJ_SHAPE = (32, 16, 32)
ADJ_BOX = (-9.0, 9.0, -6.0, 6.0, -24.0, 24.0)
ADJ_KNOTS = np.linspace(-24.0, 24.0, 7)


def _adjoint_case():
    c12 = wl.separation(ADJ_KNOTS, wl.ZC_12, dmin=2.0, dmax=4.0, w=8.0)
    c23 = wl.separation(ADJ_KNOTS, wl.ZC_23, dmin=2.0, dmax=4.0, w=8.0)
    z = wl.axis(ADJ_SHAPE[0], ADJ_BOX[4], ADJ_BOX[5])
    x1 = -(c12 @ oracle.natural_spline_basis(ADJ_KNOTS, z))
    x, y, zz = wl.mesh(ADJ_SHAPE, ADJ_BOX)
    psi0 = np.exp(-((x - x1[:, None, None]) ** 2 + y ** 2) / 2.0 - (zz + 10.0) ** 2 / 18.0
                  + 2j * zz)
    return wl.normalise(psi0.astype(complex), ADJ_BOX), c12, c23


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-4)])
@pytest.mark.parametrize("K", [1, 7, 40])
def test_adjoint_matches_oracle_gradient(ctap, dtype, tol, K):
    psi0, c12, c23 = _adjoint_case()
    dt, n = 0.05, 40
    J_ref, g_ref = oracle.ctap_gradient(psi0, ADJ_BOX, 20.0, 1.0, ADJ_KNOTS, c12, c23, dt, n, 2)
    plan = ctap.Plan(ADJ_SHAPE, ADJ_BOX, dtype)
    plan.set_guides_spline(20.0, 1.0, ADJ_KNOTS, c12, c23, 1.5)
    J, g = plan.adjoint(to_dev(psi0, dtype), n, dt, K=K, guide=3)
    assert abs(J - J_ref) < tol * abs(J_ref)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) < tol * scale, (g, g_ref)


def test_adjoint_autograd_function(ctap):
    psi0, c12, c23 = _adjoint_case()
    plan = ctap.Plan(ADJ_SHAPE, ADJ_BOX, "c128")
    t12 = torch.tensor(c12, requires_grad=True)
    t23 = torch.tensor(c23, requires_grad=True)
    J = ctap.ctap_adjoint_apply(t12, t23, plan, to_dev(psi0, "c128"), 40, 0.05, K=8, guide=3,
                                V0=20.0, s=1.0, knots=ADJ_KNOTS)
    J.backward()
    _, g_ref = oracle.ctap_gradient(psi0, ADJ_BOX, 20.0, 1.0, ADJ_KNOTS, c12, c23, 0.05, 40, 2)
    got = np.concatenate([t12.grad.numpy(), t23.grad.numpy()])
    assert np.max(np.abs(got - g_ref)) < 1e-9 * np.max(np.abs(g_ref))


# ------------------------------------------------------------- edge cases
def test_zero_steps_is_identity_and_runs_are_deterministic(ctap):
    shape, box = (32, 64, 64), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    psi0 = to_dev(random_state(shape, 3), "c64")
    a = psi0.clone()
    plan.step(a, 0, 0.01)
    assert torch.equal(a, psi0)
    b = psi0.clone()
    plan.step(a, 17, 0.01)
    plan.step(b, 17, 0.01)
    assert torch.equal(a, b)
    assert np.array_equal(plan.observables(a), plan.observables(b))


def test_step_graphs_replay_bitwise_and_invalidate(ctap):
    """Repeated ctap_step calls on a non-default stream are captured once and
    replayed as a CUDA graph; the result must be bitwise that of the eager
    launches (legacy stream, no graphs), and a potential change after the
    capture must not leave a stale graph."""
    shape, box = (64, 64, 64), wl.CTAP_BOX
    z = wl.axis(64, box[4], box[5])
    c = wl.guide_centres(z)
    psi0 = to_dev(wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=13), "c64")
    side = torch.cuda.Stream()
    pg = ctap.Plan(shape, box, "c64", stream=side)
    pe = ctap.Plan(shape, box, "c64", stream=torch.cuda.default_stream())
    for p in (pg, pe):
        p.set_guides(wl.V0, 1.0, c[0], c[2], 1.5)
    a, b = psi0.clone(), psi0.clone()
    torch.cuda.synchronize()
    for _ in range(4):
        n0 = pg.launch_count
        pg.step(a, 5, 0.005)
        assert pg.launch_count - n0 == 11          # 2 n + 1 kernels, replayed or not
        pe.step(b, 5, 0.005)
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # change the potential: a captured graph must not survive
    pg.set_guides(wl.V0 * 0.5, 1.0, c[0], c[2], 1.5)
    pe.set_guides(wl.V0 * 0.5, 1.0, c[0], c[2], 1.5)
    for _ in range(3):
        pg.step(a, 5, 0.005)
        pe.step(b, 5, 0.005)
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_errors_are_reported(ctap):
    shape, box = (8, 8, 8), (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0)
    plan = ctap.Plan(shape, box, "c64")
    psi = to_dev(random_state(shape), "c64")
    with pytest.raises(ctap.CtapError) as e:
        plan.step(psi, 1, 0.1)
    assert e.value.code == 4                                   # no potential yet
    plan.set_potential(np.zeros(shape))
    with pytest.raises(ctap.CtapError) as e:
        plan.step(to_dev(random_state(shape), "c128"), 1, 0.1)
    assert e.value.code == 3                                   # dtype mismatch
    with pytest.raises(ctap.CtapError) as e:
        plan.adjoint(psi, 4, 0.1)
    assert e.value.code == 4                                   # adjoint without spline
    with pytest.raises(ctap.CtapError) as e:
        plan.set_potential(np.full(shape, np.nan))
    assert e.value.code == 1
    plan.sync(1000)


# ------------------------------------------------ specialised complex64 passes
FAST_SHAPES = [(256, 64, 64), (256, 128, 128), (512, 256, 256), (1024, 64, 256),
               (256, 256, 256), (8, 128, 256), (64, 64, 64)]


@pytest.mark.parametrize("shape", FAST_SHAPES)
def test_fast_and_generic_passes_match_oracle(ctap, shape, monkeypatch):
    """The specialised complex64 passes keep the generic passes' layout; both
    must match the oracle on the same input (guide potential, 3 steps)."""
    box = wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=5) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    assert plan.info()["fast_mask"] & 1, plan.info()
    psi = to_dev(psi0, "c64")
    plan.step(psi, 3, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 3)
    fast = psi.cpu().numpy().astype(complex)
    monkeypatch.setenv("CTAP_FORCE_GENERIC", "1")
    gplan, _, _ = guides_plan(ctap, shape, box, "c64")
    assert gplan.info()["fast_mask"] == 0
    psi = to_dev(psi0, "c64")
    gplan.step(psi, 3, 0.0025)
    gen = psi.cpu().numpy().astype(complex)
    assert rel(fast, ref) < 1e-6
    assert rel(gen, ref) < 1e-6
    obs_f = plan.observables(to_dev(psi0, "c64"))
    obs_g = gplan.observables(to_dev(psi0, "c64"))
    assert np.allclose(obs_f, obs_g, rtol=1e-6, atol=1e-9)


def test_persistent_z_ring_matches_plain_pass_and_oracle(ctap, monkeypatch):
    """The persistent Z passes (shared-memory ring refilled by asynchronous
    copies while the previous tile is transformed) run 1024-point z-lines
    with 4 row classes: the packed form (FP32-pair arithmetic, two columns
    per thread) by default, the scalar ring with CTAP_NO_PACKED=1 and the
    one-tile-per-CTA pass with CTAP_NO_RING=1.  All three must agree with
    each other and with the oracle."""
    shape, box = (1024, 256, 64), wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=15) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    ref = oracle.step(psi0, *guides_plan(ctap, shape, box, "c128")[1:2], box, 0.0025, 2)
    got = {}
    for env, mask in ((None, 23), ("CTAP_NO_PACKED", 7), ("CTAP_NO_RING", 3)):
        if env:
            monkeypatch.setenv(env, "1")
        plan, V, c = guides_plan(ctap, shape, box, "c64")
        info = plan.info()
        assert info["fast_mask"] == mask and info["row_classes"] == 4 and \
            info["cols_per_z_tile"] == 16, info
        psi = to_dev(psi0, "c64")
        plan.step(psi, 2, 0.0025)
        got[env] = psi.cpu().numpy().astype(complex)
        plan.close()
        if env:
            monkeypatch.delenv(env)
    assert rel(got[None], got["CTAP_NO_PACKED"]) < 1e-6
    assert rel(got["CTAP_NO_PACKED"], got["CTAP_NO_RING"]) < 1e-6
    for v in got.values():
        assert rel(v, ref) < 1e-6


def test_persistent_xy_ring_matches_plain_pass_and_oracle(ctap, monkeypatch):
    """The persistent XY passes (three 32-row half buffers, the next tile
    copied in while the current one is transformed) run the steady steps of
    256-wide complex64 planes with 64-row tiles: in packed FP32-pair
    arithmetic by default, in scalar arithmetic with CTAP_NO_PACKED=1, and
    one tile per CTA with CTAP_NO_RING=1.  1024 tiles over at most 148 CTAs
    exercise the prefetch.  All three must agree with each other and with
    the oracle."""
    shape, box = (256, 256, 256), wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=17) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    got = {}
    for env, bits in ((None, 41), ("CTAP_NO_PACKED", 9), ("CTAP_NO_RING", 1)):
        if env:
            monkeypatch.setenv(env, "1")
        plan, V, c = guides_plan(ctap, shape, box, "c64")
        assert plan.info()["fast_mask"] & 41 == bits, plan.info()
        psi = to_dev(psi0, "c64")
        plan.step(psi, 4, 0.0025)
        got[env] = psi.cpu().numpy().astype(complex)
        plan.close()
        if env:
            monkeypatch.delenv(env)
    ref = oracle.step(psi0, V, box, 0.0025, 4)
    assert rel(got[None], got["CTAP_NO_PACKED"]) < 1e-6
    assert rel(got["CTAP_NO_PACKED"], got["CTAP_NO_RING"]) < 1e-6
    for v in got.values():
        assert rel(v, ref) < 1e-6


@pytest.mark.parametrize("dt", [0.005, 0.001])
def test_separable_potential_on_packed_xy_pass(ctap, monkeypatch, dt):
    """The harmonic oscillator (separable potential, Sec. IV's test case) on
    256-wide planes with 64-row tiles runs its steady XY passes in the packed
    ring kernel, with the kick angle (Vx + Vy + Vz) dt formed per point from
    the FP64 axis potentials.  The scalar passes (CTAP_NO_PACKED=1) apply
    three table rotations per point instead.  On [-8, 8]^3, |V|max dt is 0.48
    at dt = 0.005 (the long kick series) and 0.096 at dt = 0.001 (the short
    one).  Both must agree with each other and with the oracle after 4 steps."""
    shape, box = (64, 256, 256), wl.HARMONIC_BOX
    x, y, _ = wl.mesh(shape, box)
    psi0 = wl.gaussian_sum(shape, box, seed=23) * np.exp(1j * (1.5 * x + y))
    got = {}
    for env, bits in ((None, 40), ("CTAP_NO_PACKED", 0)):
        if env:
            monkeypatch.setenv(env, "1")
        plan, V = harmonic_plan(ctap, shape, box, "c64")
        assert plan.info()["fast_mask"] & 40 == bits, plan.info()
        psi = to_dev(psi0, "c64")
        plan.step(psi, 4, dt)
        got[env] = psi.cpu().numpy().astype(complex)
        plan.close()
        if env:
            monkeypatch.delenv(env)
    ref = oracle.step(psi0, V, box, dt, 4)
    assert rel(got[None], got["CTAP_NO_PACKED"]) < 1e-6
    for v in got.values():
        assert rel(v, ref) < 1e-6


def test_separable_packed_xy_with_trap_term(ctap):
    """The separable oscillator plus an additive z-only term (the longitudinal
    trap form, Sec. III) on the packed XY pass: the term folds into the z
    axis potential, and |V|max for the series tier includes it."""
    shape, box = (64, 256, 256), wl.HARMONIC_BOX
    z = wl.axis(shape[0], box[4], box[5])
    extra = 0.5 * np.sin(0.7 * z)
    plan, V = harmonic_plan(ctap, shape, box, "c64")
    plan.add_potential_z(extra)
    V = V + extra[:, None, None]
    assert plan.info()["fast_mask"] & 40 == 40, plan.info()
    x, y, _ = wl.mesh(shape, box)
    psi0 = wl.gaussian_sum(shape, box, seed=24) * np.exp(1j * (x - 2.0 * y))
    psi = to_dev(psi0, "c64")
    plan.step(psi, 4, 0.005)
    assert rel(psi.cpu().numpy().astype(complex), oracle.step(psi0, V, box, 0.005, 4)) < 1e-6


def test_ring_with_16_byte_aligned_psi(ctap):
    """The persistent Z pass moves 16-byte pieces: a psi view that is 16- but
    not 32-byte aligned (row segments then straddle 32-byte sectors) gives
    the same result as an aligned one."""
    shape, box = (1024, 256, 64), wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=16)
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    psi = to_dev(psi0, "c64")
    plan.step(psi, 2, 0.0025)
    aligned = psi.cpu().numpy().astype(complex)
    n = int(np.prod(shape))
    buf = torch.zeros(n + 2, dtype=torch.complex64, device="cuda")
    view = buf[2:].view(shape)
    assert view.data_ptr() % 32 == 16
    view.copy_(to_dev(psi0, "c64"))
    plan.step(view, 2, 0.0025)
    assert rel(view.cpu().numpy().astype(complex), aligned) < 1e-6
    ref = oracle.step(psi0, V, box, 0.0025, 2)
    assert rel(aligned, ref) < 1e-6


FAST128_SHAPES = [(256, 128, 128), (256, 256, 256), (512, 256, 256), (1024, 128, 256),
                  (64, 64, 64), (16, 32, 128)]


@pytest.mark.parametrize("shape", FAST128_SHAPES)
def test_fast_passes_complex128_match_oracle(ctap, shape):
    """The specialised passes in FP64 (32-row XY classes, 8-column Z tiles)."""
    box = wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=6) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    plan, V, c = guides_plan(ctap, shape, box, "c128")
    assert plan.info()["fast_mask"] & 1, plan.info()
    psi = to_dev(psi0, "c128")
    plan.step(psi, 3, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 3)
    assert rel(psi.cpu().numpy(), ref) < 1e-13
    got = plan.observables(psi)
    ref_obs = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(got, ref_obs, rtol=1e-11, atol=1e-14)


def test_fast_passes_long_run(ctap):
    """300 steps on the specialised passes (fast XY and Z): relative L2
    < 1e-5 and |norm drift| < 1e-6 against the FP64 oracle."""
    shape, box = (256, 64, 64), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    assert plan.info()["fast_mask"] == 3
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=8) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, "c64")
    n0 = plan.observables(psi)[0]
    plan.step(psi, 300, 0.005)
    ref = oracle.step(psi0, V, box, 0.005, 300)
    assert rel(psi.cpu().numpy().astype(complex), ref) < 1e-5
    assert abs(plan.observables(psi)[0] / n0 - 1.0) < 1e-6


@pytest.mark.parametrize("imag", [False, True])
def test_fast_passes_imaginary_time_and_split(ctap, imag):
    """Imaginary time (split kick + FP64 norm) and the separable potential on
    the specialised passes."""
    shape, box = (256, 64, 64), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    plan, V = harmonic_plan(ctap, shape, box, "c64")
    assert plan.info()["fast_mask"] == 3
    psi0 = wl.gaussian_sum(shape, box, seed=9)
    psi = to_dev(psi0, "c64")
    plan.step(psi, 20, 0.02, imag=imag)
    ref = oracle.step(psi0, V, box, 0.02, 20, imag=imag)
    assert rel(psi.cpu().numpy().astype(complex), ref) < 2e-6


def test_misaligned_psi_uses_generic_passes(ctap):
    """A psi view 8 bytes off a 16-byte boundary cannot take the 16-byte
    vector accesses of the specialised passes; the result must not change."""
    shape, box = (256, 64, 64), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=12)
    n = int(np.prod(shape))
    buf = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
    psi = buf[1:].view(shape)
    assert psi.data_ptr() % 16 == 8
    psi.copy_(to_dev(psi0, "c64"))
    plan.step(psi, 3, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 3)
    assert rel(psi.cpu().numpy().astype(complex), ref) < 1e-6


# --------------------------------------------------- full size (bench shape)
@pytest.mark.slow
def test_full_size_c64_one_step_and_invariants(ctap):
    """256x256x1024 complex64 in the launch configuration bench.py times:
    three steps (prologue XY, the persistent Z and XY passes of the steady
    step, epilogue XY) element-wise against the oracle, then norm
    conservation and time reversibility over 20 steps (properties that hold
    at any size)."""
    shape, box = (1024, 256, 256), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    assert plan.info()["fast_mask"] & 12 == 12, plan.info()    # both ring passes
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=11) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, "c64")
    plan.step(psi, 3, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 3)
    got = psi.cpu().numpy().astype(complex)
    assert rel(got, ref) < 1e-6
    del ref
    # the FP64 reductions of the bench's observation step, and the
    # y-integrated density, on the same full-size state
    obs = plan.observables(psi)
    want = oracle.observables(got, V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(obs, want, rtol=1e-6, atol=1e-9), (obs, want)
    assert np.allclose(plan.density_xz(psi), oracle.density_xz(got, box), rtol=1e-12, atol=1e-300)
    del got
    n0 = plan.observables(psi)[0]
    start = psi.clone()
    plan.step(psi, 20, 0.0025)
    assert abs(plan.observables(psi)[0] / n0 - 1.0) < 1e-6
    plan.step(psi, 20, -0.0025)
    assert rel(psi.cpu().numpy().astype(complex), start.cpu().numpy().astype(complex)) < 1e-5


@pytest.mark.parametrize("dtype", ["c128", "c128df"])
def test_full_size_fp64_paths_match_oracle(ctap, dtype):
    """The FP64 (complex128) and double-float paths at the bench size,
    256x256x1024: two steps element-wise against the oracle at the FP64
    parity bound."""
    shape, box = (1024, 256, 256), wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, dtype)
    assert plan.info()["fast_mask"] & 3 == 3, plan.info()     # specialised XY and Z passes
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=12) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = to_dev(psi0, "c128")
    plan.step(psi, 2, 0.0025)
    got = psi.cpu().numpy()
    del psi
    plan.close()
    ref = oracle.step(psi0, V, box, 0.0025, 2)
    assert rel(got, ref) < 1e-12
