"""GPU parity of the paper-faithful variants against the FP64 oracle: the
K/2 V K/2 ordering, the longitudinal harmonic trap (an additive z-only term,
Sec. III), the intuitive guide arrangement (Fig. 4b) and the y-integrated
density (Fig. 5).  Same tolerances as the main parity tests."""
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


def guide_state(shape, box, seed):
    return wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=seed) \
        * np.exp(2j * wl.mesh(shape, box)[2])


def guides(ctap, shape, box, dtype, order="counter", trap=None):
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z, order)
    plan = ctap.Plan(shape, box, dtype)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    if trap is not None:
        vz = wl.trap_z(z, trap)
        plan.add_potential_z(vz)
        V = V + vz[:, None, None]
    return plan, V, c


# fast-path shapes (specialised passes) and a generic one (ragged 8-point axes)
SHAPES = [(256, 64, 64), (256, 128, 128), (64, 32, 16)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,tol", [("c64", 1e-6), ("c128", 1e-13)])
def test_kvk_ordering_matches_oracle(ctap, shape, dtype, tol):
    box = wl.CTAP_BOX
    plan, V, _ = guides(ctap, shape, box, dtype)
    psi0 = guide_state(shape, box, 21)
    psi = to_dev(psi0, dtype)
    plan.step(psi, 5, 0.02, order="KVK")
    ref = oracle.step(psi0, V, box, 0.02, 5, order="KVK")
    assert rel(psi.cpu().numpy().astype(complex), ref) < tol
    # the orderings differ at this dt by far more than the tolerance
    vkv = oracle.step(psi0, V, box, 0.02, 5)
    assert rel(ref, vkv) > 10 * tol


def test_kvk_graph_replay_matches_eager(ctap):
    """Repeated KVK calls on a side stream are captured and replayed; the
    capture is keyed on the ordering (a VKV call with the same arguments
    must not reuse it)."""
    shape, box = (256, 64, 64), wl.CTAP_BOX
    side = torch.cuda.Stream()
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z)
    psi0 = guide_state(shape, box, 22)
    pg = ctap.Plan(shape, box, "c64", stream=side)
    pg.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    pe = ctap.Plan(shape, box, "c64")
    pe.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    a, b = to_dev(psi0, "c64"), to_dev(psi0, "c64")
    with torch.cuda.stream(side):
        for _ in range(3):
            pg.step(a, 4, 0.0025, order="KVK")
        pg.step(a, 4, 0.0025)
    for _ in range(3):
        pe.step(b, 4, 0.0025, order="KVK")
    pe.step(b, 4, 0.0025)
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(256, 64, 64), (64, 32, 16)])
@pytest.mark.parametrize("dtype,tol", [("c64", 1e-6), ("c128", 1e-13)])
def test_trap_term_matches_oracle(ctap, shape, dtype, tol):
    """Guides plus the longitudinal trap, product form + z-only term, against
    the oracle's dense V; observables (<V> includes the trap) too."""
    box = wl.CTAP_BOX
    plan, V, c = guides(ctap, shape, box, dtype, trap=wl.TRAP_OMEGA)
    assert np.allclose(plan.get_potential(), V, rtol=1e-14, atol=1e-12)
    psi0 = guide_state(shape, box, 23)
    psi = to_dev(psi0, dtype)
    plan.step(psi, 6, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 6)
    assert rel(psi.cpu().numpy().astype(complex), ref) < tol
    got = plan.observables(psi)
    want = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(got, want, rtol=1e-5 if dtype == "c64" else 1e-11, atol=1e-9)


@pytest.mark.parametrize("form", ["dense", "separable"])
def test_trap_term_on_dense_and_separable_forms(ctap, form):
    shape, box = (32, 16, 16), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    vx, vy, vz = wl.harmonic_parts(shape, box)
    z = wl.axis(shape[0], box[4], box[5])
    extra = 0.3 * np.sin(z)
    plan = ctap.Plan(shape, box, "c128")
    if form == "dense":
        plan.set_potential(wl.harmonic_dense(shape, box))
    else:
        plan.set_potential_separable(vx, vy, vz)
    plan.add_potential_z(extra)
    V = wl.harmonic_dense(shape, box) + extra[:, None, None]
    assert np.allclose(plan.get_potential(), V, rtol=1e-14, atol=1e-13)
    psi0 = wl.gaussian_sum(shape, box, seed=24)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 10, 0.01)
    assert rel(psi.cpu().numpy(), oracle.step(psi0, V, box, 0.01, 10)) < 1e-13


def test_trap_requires_a_potential(ctap):
    plan = ctap.Plan((8, 8, 8), (-1, 1, -1, 1, -1, 1), "c64")
    with pytest.raises(ctap.CtapError) as e:
        plan.add_potential_z(np.zeros(8))
    assert e.value.code == 4
    plan.set_potential(np.zeros((8, 8, 8)))
    with pytest.raises(ctap.CtapError) as e:
        plan.add_potential_z(np.full(8, np.nan))
    assert e.value.code == 1


@pytest.mark.parametrize("dtype,tol", [("c64", 1e-6), ("c128", 1e-13)])
def test_intuitive_arrangement_matches_oracle(ctap, dtype, tol):
    shape, box = (256, 64, 64), wl.CTAP_BOX
    plan, V, c = guides(ctap, shape, box, dtype, order="intuitive")
    psi0 = guide_state(shape, box, 25)
    psi = to_dev(psi0, dtype)
    plan.step(psi, 5, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, 5)
    assert rel(psi.cpu().numpy().astype(complex), ref) < tol


@pytest.mark.parametrize("shape", [(256, 64, 64), (1024, 256, 64), (8, 8, 8)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_density_xz_matches_oracle(ctap, shape, dtype):
    box = wl.CTAP_BOX
    psi0 = guide_state(shape, box, 26)
    plan = ctap.Plan(shape, box, dtype)
    psi = to_dev(psi0, dtype)
    got = plan.density_xz(psi)
    want = oracle.density_xz(psi.cpu().numpy().astype(complex), box)
    assert got.shape == (shape[0], shape[2])
    # FP64 accumulation of the stored values: only summation order differs
    assert np.allclose(got, want, rtol=1e-12, atol=1e-300)
    # deterministic
    assert np.array_equal(got, plan.density_xz(psi))


# --------------------------------------------------- batched replicas (N3)
BATCH_SHAPES = [(256, 64, 64), (64, 32, 16), (1024, 256, 64)]


# complex128 on the two smaller shapes; the 1024-point z-lines in complex64
# (the persistent Z pass over replica tiles)
BATCH_CASES = [(s, d) for s in BATCH_SHAPES for d in ("c64", "c128")
               if not (d == "c128" and s[0] == 1024)]


@pytest.mark.parametrize("shape,dtype", BATCH_CASES)
def test_batched_replicas_match_separate_plans_and_oracle(ctap, shape, dtype):
    """Three replicas with different middle-guide depths (the Fig. 6 sweep
    variable) advanced by one batched plan: each equals its own unbatched
    plan bitwise (same kernels per replica) and the oracle with that
    replica's potential; observables per replica match."""
    box = wl.CTAP_BOX
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z)
    mids = [0.8, 1.0, 1.25]
    B = len(mids)
    psis = np.stack([guide_state(shape, box, 30 + b) for b in range(B)])
    plan = ctap.Plan(shape, box, dtype, batch=B)
    plan.set_guides_batched(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], mids, wl.POP_HALFWIDTH)
    plan.add_potential_z(wl.trap_z(z))
    psi = to_dev(psis, dtype)
    plan.step(psi, 4, 0.0025)
    got = psi.cpu().numpy()
    obs = plan.observables(psi)
    assert obs.shape == (B, 6)
    Vall = plan.get_potential()
    nsteps_oracle = 4 if shape[0] < 1024 else 1
    for b, m in enumerate(mids):
        single = ctap.Plan(shape, box, dtype)
        single.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
        G2 = np.exp(-wl.axis(shape[2], box[0], box[1]) ** 2 / (2 * wl.SIGMA_GUIDE ** 2))
        gy = np.exp(-wl.axis(shape[1], box[2], box[3]) ** 2 / (2 * wl.SIGMA_GUIDE ** 2))
        V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2]) \
            + wl.V0 * (1.0 - m) * gy[None, :, None] * G2[None, None, :] \
            + wl.trap_z(z)[:, None, None]
        assert np.allclose(Vall[b], V, rtol=1e-13, atol=1e-12)
        if m == 1.0:
            single.add_potential_z(wl.trap_z(z))
            s1 = to_dev(psis[b], dtype)
            single.step(s1, 4, 0.0025)
            assert np.array_equal(s1.cpu().numpy(), got[b])
        if nsteps_oracle == 4:
            ref = oracle.step(psis[b], V, box, 0.0025, 4)
            assert rel(got[b].astype(complex), ref) < (1e-6 if dtype == "c64" else 1e-13)
            want = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
            assert np.allclose(obs[b], want, rtol=1e-5 if dtype == "c64" else 1e-11, atol=1e-9)
    dens = plan.density_xz(psi)
    assert dens.shape == (B, shape[0], shape[2])
    for b in range(B):
        assert np.allclose(dens[b], oracle.density_xz(got[b].astype(complex), box), rtol=1e-12,
                           atol=1e-300)


def test_batched_plan_restrictions(ctap):
    shape, box = (16, 16, 16), wl.CTAP_BOX
    plan = ctap.Plan(shape, box, "c64", batch=2)
    with pytest.raises(ctap.CtapError) as e:
        plan.set_potential(np.zeros((2,) + shape))
    assert e.value.code == 1
    with pytest.raises(ctap.CtapError) as e:
        plan.set_potential_separable(np.zeros(16), np.zeros(16), np.zeros(16))
    assert e.value.code == 1
    z = wl.axis(16, box[4], box[5])
    c = wl.guide_centres(z)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    psi = to_dev(np.zeros((2,) + shape, complex), "c64")
    with pytest.raises(ctap.CtapError) as e:
        plan.step(psi, 1, 0.01, imag=True)
    assert e.value.code == 1
    with pytest.raises(ctap.CtapError) as e:
        plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, wl.KNOTS_Z, *wl.spline_controls())
    assert e.value.code == 1
    with pytest.raises(ValueError):
        plan.step(to_dev(np.zeros(shape, complex), "c64"), 1, 0.01)


# ---------------------------------------- double-float complex128 path (N1)
@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 32, 16), (256, 64, 64)])
def test_double_float_path_matches_oracle(ctap, shape):
    """Complex128 psi with double-float transforms: harmonic oscillator,
    100 steps (the complex128 target is 1e-12 relative L2)."""
    box = (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    vx, vy, vz = wl.harmonic_parts(shape, box)
    psi0 = wl.gaussian_sum(shape, box, seed=40)
    plan = ctap.Plan(shape, box, "c128df")
    plan.set_potential(wl.harmonic_dense(shape, box))
    psi = to_dev(psi0, "c128")
    plan.step(psi, 100, 0.005)
    ref = oracle.step(psi0, wl.harmonic_dense(shape, box), box, 0.005, 100)
    err = rel(psi.cpu().numpy(), ref)
    assert err < 1e-12, err
    # far better than complex64 on the same run
    p64 = ctap.Plan(shape, box, "c64")
    p64.set_potential(wl.harmonic_dense(shape, box))
    q = to_dev(psi0, "c64")
    p64.step(q, 100, 0.005)
    assert rel(q.cpu().numpy().astype(complex), ref) > 100 * err


@pytest.mark.parametrize("order", ["VKV", "KVK"])
def test_double_float_guides_and_observables(ctap, order):
    shape, box = (256, 64, 64), wl.CTAP_BOX
    plan, V, c = guides(ctap, shape, box, "c128df", trap=wl.TRAP_OMEGA)
    psi0 = guide_state(shape, box, 41)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 20, 0.0025, order=order)
    ref = oracle.step(psi0, V, box, 0.0025, 20, order=order)
    assert rel(psi.cpu().numpy(), ref) < 1e-12
    got = plan.observables(psi)
    want = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-14)


# (nz, ny, nx), row classes, steps: 1024-point z-lines on 256-wide planes take
# the three-stage double-float Z pass, here with 4 and 2 row classes per Z
# tile (2 and 4 columns); the 8-class geometry is the full 256x256x1024 size
# (tests/test_gpu_parity.py::test_full_size_fp64_paths_match_oracle)
DF_Z3_CASES = [((1024, 128, 256), 4, 3), ((1024, 64, 256), 2, 40)]


@pytest.mark.parametrize("shape,row_classes,steps", DF_Z3_CASES)
def test_double_float_three_stage_z_pass(ctap, shape, row_classes, steps):
    """The double-float Z pass for 1024-point z-lines (16 x 4 x 16 register
    stages) in each of its tile geometries: guides with the longitudinal
    trap, moving packets, against the oracle at the complex128 target; the
    observables (their kinetic sum takes the generic Z pass) against the
    oracle's."""
    box = wl.CTAP_BOX
    plan, V, c = guides(ctap, shape, box, "c128df", trap=wl.TRAP_OMEGA)
    info = plan.info()
    assert info["fast_mask"] & 2 and info["row_classes"] == row_classes and \
        info["cols_per_z_tile"] == 8, info
    psi0 = guide_state(shape, box, 43)
    psi = to_dev(psi0, "c128")
    plan.step(psi, steps, 0.0025)
    ref = oracle.step(psi0, V, box, 0.0025, steps)
    assert rel(psi.cpu().numpy(), ref) < 1e-12
    got = plan.observables(psi)
    want = oracle.observables(ref, V, box, c, wl.POP_HALFWIDTH)
    assert np.allclose(got, want, rtol=1e-11, atol=1e-14)


def test_double_float_three_stage_z_pass_imaginary_time(ctap):
    """Imaginary time through the three-stage double-float Z pass (the decay
    factors of the kinetic step with the per-step renormalisation scale
    folded in): guides, 1024-point z-lines, against the oracle."""
    shape, box = (1024, 64, 256), wl.CTAP_BOX
    plan, V, c = guides(ctap, shape, box, "c128df")
    assert plan.info()["fast_mask"] & 2, plan.info()
    psi0 = guide_state(shape, box, 44)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 10, 0.01, imag=True)
    ref = oracle.step(psi0, V, box, 0.01, 10, imag=True)
    assert rel(psi.cpu().numpy(), ref) < 1e-12


def test_double_float_imaginary_time(ctap):
    shape, box = (32, 32, 32), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    vx, vy, vz = wl.harmonic_parts(shape, box)
    plan = ctap.Plan(shape, box, "c128df")
    plan.set_potential_separable(vx, vy, vz)
    psi0 = wl.gaussian_sum(shape, box, seed=42)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 20, 0.02, imag=True)
    ref = oracle.step(psi0, wl.harmonic_dense(shape, box), box, 0.02, 20, imag=True)
    assert rel(psi.cpu().numpy(), ref) < 1e-12


def test_double_float_adjoint_is_rejected(ctap):
    shape, box = (16, 16, 16), wl.CTAP_BOX
    plan = ctap.Plan(shape, box, "c128df")
    plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, wl.KNOTS_Z, *wl.spline_controls())
    with pytest.raises(ctap.CtapError) as e:
        plan.adjoint(to_dev(np.zeros(shape, complex), "c128"), 4, 0.01)
    assert e.value.code == 3


# --------------------------------------------- atom-chip wire potential (N4)
@pytest.mark.parametrize("shape", [(64, 32, 64), (128, 16, 32)])
def test_wire_potential_matches_oracle(ctap, shape):
    """Biot-Savart field of the three chip wires plus the bias fields, built
    on the device, against the oracle; then steps on it (complex128)."""
    box = (-10.0, 10.0, 0.5, 4.5, 0.0, 1000.0)
    seg = wl.chip_wires(48)
    bias = wl.chip_bias()
    k = wl.CHIP["mu0_over_4pi"]
    vpf, voff = 0.5, 0.5 * wl.CHIP["B_ip"]
    plan = ctap.Plan(shape, box, "c128")
    plan.set_potential_wires(seg, bias, k, vpf, voff)
    got = plan.get_potential()
    want = oracle.wire_potential(shape, box, seg, bias, k, vpf, voff)
    assert rel(got, want) < 1e-13
    x, y, z = wl.mesh(shape, box)
    psi0 = wl.normalise(np.exp(-x ** 2 / 8.0 - (y - 2.5) ** 2 / 1.0 - (z - 500.0) ** 2 / 7200.0
                               + 0.05j * z), box)
    psi = to_dev(psi0, "c128")
    plan.step(psi, 5, 0.01)
    assert rel(psi.cpu().numpy(), oracle.step(psi0, want, box, 0.01, 5)) < 1e-12


def test_wire_potential_rejects_bad_input(ctap):
    plan = ctap.Plan((8, 8, 8), (-1, 1, -1, 1, -1, 1), "c64")
    with pytest.raises(ctap.CtapError) as e:
        plan.set_potential_wires(np.full((1, 7), np.nan), [0, 0, 0], 1.0, 1.0)
    assert e.value.code == 1
    with pytest.raises(ValueError):
        plan.set_potential_wires(np.zeros(6), [0, 0, 0], 1.0, 1.0)
