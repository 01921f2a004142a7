"""Long runs on the kernels the bench times, the C2 guide configuration end
to end, the adjoint at the size of the gradient workload, and a full
transfer through both coupling regions.

Accuracy targets of the complex64 path (FP32 transforms, FP64 tables and
reductions): relative L2 <= 1e-5 against FP64 after 1000 steps and a norm
that drifts by less than 1e-6.  The FP64 reference is the oracle itself
where it finishes in a minute or two; for the larger grids it is the
complex128 path of the library run from the same psi0, which is checked
against the oracle on the same grid over a shorter run (its own error,
~1e-13 per 100 steps, is many orders below the complex64 bound).
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


def host(psi):
    return psi.cpu().numpy().astype(complex)


def guides_plan(ctap, shape, box, dtype, order="counter"):
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z, order)
    plan = ctap.Plan(shape, box, dtype)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    return plan, V, c


def moving_packets(shape, box, seed):
    return wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=seed) \
        * np.exp(2j * wl.mesh(shape, box)[2])


# --------------------------------------------- the persistent (ring) passes
# (nz, ny, nx) -> the fast-pass bit the shape must select: 8 = the persistent
# XY pass (256-wide planes, 64-row tiles), 4 = the persistent Z pass
# (1024-point z-lines, 16-column tiles)
RING_CASES = [((64, 256, 256), 8), ((1024, 256, 64), 4)]


@pytest.mark.parametrize("shape,bit", RING_CASES)
def test_ring_passes_1000_steps_accuracy_and_norm(ctap, shape, bit):
    """1000 complex64 steps through the persistent XY or Z pass: relative L2
    <= 1e-5 against the complex128 run from the same psi0 and |norm drift|
    < 1e-6; the complex128 run itself matches the oracle to 1e-12 over the
    first 20 steps on the same grid."""
    box, dt = wl.CTAP_BOX, 0.005
    psi0 = moving_packets(shape, box, seed=21)
    p64, V, c = guides_plan(ctap, shape, box, "c64")
    assert p64.info()["fast_mask"] & bit, p64.info()
    p128, _, _ = guides_plan(ctap, shape, box, "c128")

    a = to_dev(psi0, "c128")
    p128.step(a, 20, dt)
    assert rel(host(a), oracle.step(psi0, V, box, dt, 20)) < 1e-12
    p128.step(a, 980, dt)
    ref = host(a)
    del a

    b = to_dev(psi0, "c64")
    n0 = p64.observables(b)[0]
    p64.step(b, 1000, dt)
    n1 = p64.observables(b)[0]
    assert rel(host(b), ref) < 1e-5
    assert abs(n1 / n0 - 1.0) < 1e-6


def test_separable_packed_xy_1000_steps_accuracy_and_norm(ctap):
    """The harmonic oscillator through the packed XY ring pass (separable
    kick: one angle (Vx + Vy + Vz) dt per point, long series at |V|max dt =
    0.48) for 1000 complex64 steps: relative L2 <= 1e-5 against complex128
    from the same psi0 and |norm drift| < 1e-6."""
    shape, box, dt = (64, 256, 256), wl.HARMONIC_BOX, 0.005
    vx, vy, vz = wl.harmonic_parts(shape, box)
    x, y, _ = wl.mesh(shape, box)
    psi0 = wl.gaussian_sum(shape, box, seed=25) * np.exp(1j * (1.5 * x - y))
    plans = {}
    for dtype in ("c64", "c128"):
        plans[dtype] = ctap.Plan(shape, box, dtype)
        plans[dtype].set_potential_separable(vx, vy, vz)
    assert plans["c64"].info()["fast_mask"] & 40 == 40, plans["c64"].info()
    a = to_dev(psi0, "c128")
    plans["c128"].step(a, 1000, dt)
    ref = host(a)
    del a
    b = to_dev(psi0, "c64")
    n0 = plans["c64"].observables(b)[0]
    plans["c64"].step(b, 1000, dt)
    n1 = plans["c64"].observables(b)[0]
    for p in plans.values():
        p.close()
    assert rel(host(b), ref) < 1e-5
    assert abs(n1 / n0 - 1.0) < 1e-6


def test_double_float_500_steps_against_complex128_full_size(ctap):
    """The double-float path at the bench size (its specialised XY and
    three-stage Z passes) for 500 steps from the moving packets: within
    1e-12 relative L2 of the native complex128 path (whose own error against
    the oracle is pinned above), norm conserved to the same bound."""
    shape, box, dt = (1024, 256, 256), wl.CTAP_BOX, 0.0025
    psi0 = moving_packets(shape, box, seed=27)
    out, norms = {}, {}
    for dtype in ("c128", "c128df"):
        plan, _, _ = guides_plan(ctap, shape, box, dtype)
        if dtype == "c128df":
            assert plan.info()["fast_mask"] & 3 == 3, plan.info()
        psi = to_dev(psi0, "c128")
        n0 = plan.observables(psi)[0]
        plan.step(psi, 500, dt)
        norms[dtype] = plan.observables(psi)[0] / n0 - 1.0
        out[dtype] = psi
        plan.close()
    a, b = out["c128df"], out["c128"]
    err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    assert err < 1e-12, err
    assert abs(norms["c128df"]) < 1e-12 and abs(norms["c128"]) < 1e-12, norms


# ------------------------------------------------------- C2 end to end
def c2_initial_state(shape, box):
    """The C2 initial state, prepared by the oracle: the guide-1 transverse
    ground state (200 imaginary-time steps at dtau = 0.01 on the nz = 1 plane
    holding guide 1 alone) times a z-Gaussian of width 4 at z = -40 with
    momentum 2 (Sec. V)."""
    nz, ny, nx = shape
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    y = wl.axis(ny, box[2], box[3])
    x = wl.axis(nx, box[0], box[1])
    gy = np.exp(-y ** 2 / 2)
    H = -wl.V0 * np.exp(-(x - xc) ** 2 / 2)[None, :]
    V2 = gy[None, :, None] * H[:, None, :]
    seed = wl.guide_seed_2d((ny, nx), box, xc)
    phi = oracle.step(seed, V2, box, 0.01, 200, imag=True)
    return seed, gy, H, phi, wl.packet_from_transverse(phi, nz, box)


@pytest.mark.slow
def test_c2_guides_config_end_to_end(ctap):
    """128x128x256 three-guide run: the imaginary-time preparation on the
    transverse plane, then complex128 within 1e-12 of the oracle after 100
    steps (and 1e-11 after 1000), complex64 within 1e-5 after 1000 steps
    with |norm drift| < 1e-6, and the guide populations of both paths
    against the oracle's after 1000 steps (Sec. V, Fig. 4)."""
    shape, box, dt = (256, 128, 128), wl.CTAP_BOX, 0.005
    seed, gy, H, phi, psi0 = c2_initial_state(shape, box)

    prep = ctap.Plan((1,) + shape[1:], box, "c128")
    prep.set_potential_product(gy, H)
    s = to_dev(seed, "c128")
    prep.step(s, 200, 0.01, imag=True)
    assert rel(s.cpu().numpy(), phi) < 1e-12

    p128, V, c = guides_plan(ctap, shape, box, "c128")
    p64, _, _ = guides_plan(ctap, shape, box, "c64")
    ref100 = oracle.step(psi0, V, box, dt, 100)
    ref1000 = oracle.step(ref100, V, box, dt, 900)
    obs_ref = oracle.observables(ref1000, V, box, c, wl.POP_HALFWIDTH)

    a = to_dev(psi0, "c128")
    p128.step(a, 100, dt)
    assert rel(a.cpu().numpy(), ref100) < 1e-12
    p128.step(a, 900, dt)
    assert rel(a.cpu().numpy(), ref1000) < 1e-11
    obs128 = p128.observables(a)
    assert np.allclose(obs128, obs_ref, rtol=1e-11, atol=1e-14), (obs128, obs_ref)

    b = to_dev(psi0, "c64")
    n0 = p64.observables(b)[0]
    p64.step(b, 1000, dt)
    obs64 = p64.observables(b)
    assert rel(host(b), ref1000) < 1e-5
    assert abs(obs64[0] / n0 - 1.0) < 1e-6
    # populations: absolute, on the scale of the normalised state
    assert np.max(np.abs(obs64[3:] - obs_ref[3:])) < 1e-5, (obs64, obs_ref)


# ---------------------------------------- FP64-grade complex64 reductions
@pytest.mark.parametrize("shape", [(64, 256, 256), (256, 128, 128)])
def test_complex64_observables_reach_fp64_accumulation(ctap, shape):
    """The complex64 reductions form the per-point products and short
    per-column partial sums in FP32 (the data carry 24 bits) and accumulate
    in FP64 from there.  On the same complex64 data the observables must
    agree with the oracle's per-point FP64 loops to 2e-8 of the norm (norm,
    populations; measured 1.9e-9 on 64x256x256, while an FP32 running sum
    over the grid would be off by ~1e-5); <V> weights FP32-rounded potential
    values (2e-8) and <T> passes through an FP32 forward transform (1e-7)."""
    box = wl.CTAP_BOX
    plan, V, c = guides_plan(ctap, shape, box, "c64")
    psi = to_dev(moving_packets(shape, box, seed=23), "c64")
    plan.step(psi, 10, 0.005)
    got = plan.observables(psi)
    want = oracle.observables(host(psi), V, box, c, wl.POP_HALFWIDTH)
    # norm and populations: absolute, on the scale of the norm
    for i in (0, 3, 4, 5):
        assert abs(got[i] - want[i]) <= 2e-8 * want[0], (i, got, want)
    # <V> weights FP32-rounded potential values, <T> an FP32 spectrum
    assert abs(got[2] - want[2]) <= 2e-8 * abs(want[2]), (got, want)
    assert abs(got[1] - want[1]) <= 1e-7 * abs(want[1]), (got, want)


# ------------------------------------------------ adjoint at C4's size
def c4_case(shape, box):
    c12, c23 = wl.spline_controls()
    _, _, _, _, psi0 = c2_initial_state(shape, box)
    return psi0, c12, c23


def seed_packet(shape, box):
    """The guide-1 seed Gaussian (not relaxed by imaginary time) times the
    z-packet: its overlap with guides 2 and 3 after 1000 steps is ~1e-4,
    well above the complex64 rounding floor."""
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    return wl.packet_from_transverse(wl.guide_seed_2d(shape[1:], box, xc), shape[0], box)


def fd_check(ctap, dtype, psi0, shape, box, n, dt, h=1e-3):
    """Adjoint gradient (dtype) of the final guide-3 population against
    central differences of complex128 forward runs with the population
    region and psi0 frozen, on numpy.random.default_rng(0).choice(32, 4)."""
    c12, c23 = wl.spline_controls()
    knots = np.asarray(wl.KNOTS_Z)
    pa = ctap.Plan(shape, box, dtype)
    pa.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, knots, c12, c23, wl.POP_HALFWIDTH)
    J, g = pa.adjoint(to_dev(psi0, dtype), n, dt, K=32, guide=3)
    pa.close()
    assert np.all(np.isfinite(g)) and J > 0.0
    p128 = ctap.Plan(shape, box, "c128")
    p128.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, knots, c12, c23, wl.POP_HALFWIDTH)
    base = to_dev(psi0, "c128")
    a = base.clone()
    p128.step(a, n, dt)
    J128 = p128.observables(a)[5]
    ctrl = np.concatenate([c12, c23])
    picks = np.random.default_rng(0).choice(32, 4, replace=False)
    scale = np.max(np.abs(g))
    errs = []
    for m in picks:
        Jpm = []
        for sgn in (1.0, -1.0):
            cc = ctrl.copy()
            cc[m] += sgn * h
            p128.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, knots, cc[:16], cc[16:],
                                   wl.POP_HALFWIDTH, set_regions=False)    # frozen region
            a = base.clone()
            p128.step(a, n, dt)
            Jpm.append(p128.observables(a)[5])
        gfd = (Jpm[0] - Jpm[1]) / (2 * h)
        errs.append((int(m), g[m], gfd, abs(g[m] - gfd) / max(abs(gfd), 1e-3 * scale)))
    p128.close()
    return J, J128, errs


@pytest.mark.slow
def test_adjoint_c4_against_central_differences_complex128(ctap):
    """The gradient workload exactly (128x128x256, the prepared guide-1
    state, 16 + 16 spline controls, 1000 steps at dt = 0.005, checkpoints
    every 32): the complex128 adjoint against central differences, relative
    error |g - g_fd| / max(|g_fd|, 1e-3 max|g|) <= 1e-4.  At t = 5 the
    packet has not reached the coupling regions and J is ~1e-10, below what
    complex64 resolves; the complex64 adjoint is checked on the test below."""
    shape, box = (256, 128, 128), wl.CTAP_BOX
    psi0 = c2_initial_state(shape, box)[4]
    J, J128, errs = fd_check(ctap, "c128", psi0, shape, box, 1000, 0.005)
    assert abs(J - J128) < 1e-10 * J128 + 1e-20
    for m, g, gfd, err in errs:
        assert err < 1e-4, (m, g, gfd, err)


@pytest.mark.slow
def test_adjoint_c4_size_complex64_against_central_differences(ctap):
    """The same size, controls, steps and checkpointing from the seed packet,
    whose guide-3 population after 1000 steps is ~1e-4: the complex128
    adjoint against central differences of complex128 runs within 1e-4 (as
    above), and the complex64 adjoint within 3e-4 of both (measured 1.3e-4
    on the dominant control, z = -36: FP32 rounding of psi and lambda
    against a gradient of ~4e-6)."""
    shape, box = (256, 128, 128), wl.CTAP_BOX
    psi0 = seed_packet(shape, box)
    J, J128, errs = fd_check(ctap, "c128", psi0, shape, box, 1000, 0.005)
    for m, g, gfd, err in errs:
        assert err < 1e-4, ("c128", m, g, gfd, err)
    J64, _, errs64 = fd_check(ctap, "c64", psi0, shape, box, 1000, 0.005)
    assert J64 > 1e-6 and abs(J64 - J128) < 1e-4 * J128
    scale = max(abs(g) for _, g, _, _ in errs)
    for (m, g, gfd, err), (_, g64, _, err64) in zip(errs, errs64):
        assert err64 < 3e-4, ("c64 vs fd", m, g64, gfd, err64)
        assert abs(g64 - g) < 3e-4 * max(abs(g), 1e-3 * scale), ("c64 vs c128", m, g64, g)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-4)])
def test_adjoint_c4_copy_against_oracle_gradient(ctap, dtype, tol):
    """The gradient workload on a 32x32x64 copy of its box with the same
    16 + 16 controls and 1000 steps: the library's adjoint against the
    oracle's FP64 adjoint (itself pinned to central differences)."""
    shape, box, dt, n = (64, 32, 32), wl.CTAP_BOX, 0.005, 1000
    psi0, c12, c23 = c4_case(shape, box)
    knots = np.asarray(wl.KNOTS_Z)
    J_ref, g_ref = oracle.ctap_gradient(psi0, box, wl.V0, wl.SIGMA_GUIDE, knots, c12, c23,
                                        dt, n, 2, wl.POP_HALFWIDTH)
    plan = ctap.Plan(shape, box, dtype)
    plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, knots, c12, c23, wl.POP_HALFWIDTH)
    J, g = plan.adjoint(to_dev(psi0, dtype), n, dt, K=32, guide=3)
    assert abs(J - J_ref) < tol * abs(J_ref)
    assert np.max(np.abs(g - g_ref)) < tol * np.max(np.abs(g_ref)), (g, g_ref)


def test_adjoint_rejects_checkpoints_beyond_device_memory(ctap):
    """Checkpoints of every step of a long run on the full grid would need
    far more than the device holds: the call must fail with an out-of-memory
    status before allocating, and the plan must keep working."""
    shape, box = (1024, 256, 256), wl.CTAP_BOX
    c12, c23 = wl.spline_controls()
    plan = ctap.Plan(shape, box, "c64")
    plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, wl.KNOTS_Z, c12, c23, wl.POP_HALFWIDTH)
    psi = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(ctap.CtapError) as e:
        plan.adjoint(psi, 100000, 0.0025, K=1, guide=3)
    assert e.value.code == 5
    plan.step(psi, 1, 0.0025)
    plan.sync()


# ------------------------------------------------ full transfer (Fig. 4)
def transfer_case(ctap, shape, box, order, dtype):
    """Guide-1 transverse state at rest at z = -40 in the guides plus the
    longitudinal trap omega^2 z^2/2, which carries it through both coupling
    regions to the far turning point z = +40 in half a period (Sec. III)."""
    nz, ny, nx = shape
    _, _, _, phi, _ = c2_initial_state(shape, box)
    psi0 = wl.packet_from_transverse(phi, nz, box, k0=0.0)
    plan, V, c = guides_plan(ctap, shape, box, dtype, order)
    z = wl.axis(nz, box[4], box[5])
    vz = wl.trap_z(z)
    plan.add_potential_z(vz)
    return plan, V + vz[:, None, None], c, psi0


@pytest.mark.parametrize("order", ["counter", "intuitive"])
def test_full_transfer_population_series(ctap, order):
    """Half a trap period (t = pi/omega) on a 32x32x256 grid in complex128:
    the guide populations every eighth of the run match the oracle's to
    1e-10, and the final state to 1e-10 relative L2."""
    shape, box = (256, 32, 32), wl.CTAP_BOX
    T = np.pi / wl.TRAP_OMEGA
    nobs, per = 8, 245
    dt = T / (nobs * per)
    plan, V, c, psi0 = transfer_case(ctap, shape, box, order, "c128")
    psi = to_dev(psi0, "c128")
    ref = psi0.copy()
    for k in range(nobs):
        plan.step(psi, per, dt)
        ref = oracle.step(ref, V, box, dt, per)
        got = plan.observables(psi)
        want = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
        assert np.max(np.abs(got[3:] - want[3:])) < 1e-10, (order, k, got, want)
    assert rel(psi.cpu().numpy(), ref) < 1e-10
