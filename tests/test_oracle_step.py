"""Pins for the oracle's split step (Sec. IV, Fourier split-operator method).

Each pin is independent of the oracle: exact discrete Gaussian trajectories,
the continuum coherent state, the imaginary-time oscillator fixed point,
unitarity, time reversibility and second-order convergence in dt.
"""
import numpy as np
import pytest

from gaussian_exact import Gauss1D, coherent_1d, product3
from paper_1309_2451_b300 import workloads as wl


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def grids(shape, box):
    nz, ny, nx = shape
    return wl.axis(nx, box[0], box[1]), wl.axis(ny, box[2], box[3]), wl.axis(nz, box[4], box[5])


def test_free_gaussian_is_exact_for_any_dt(orc):
    """V = 0: the split step is exact; a moving packet spreads as the
    closed-form Gaussian (Fourier transform of exp(-i k^2 t/2))."""
    shape, box = (64, 64, 64), (-16.0, 16.0, -16.0, 16.0, -16.0, 16.0)
    x, y, z = grids(shape, box)
    gx, gy, gz = Gauss1D.packet(1.0, -2.0, 1.0), Gauss1D.packet(1.2, 0.0, -0.5), \
        Gauss1D.packet(0.9, 1.0, 0.0)
    psi0 = product3(gx, gy, gz, x, y, z)
    V = np.zeros(shape)
    psi = orc.step(psi0, V, box, 0.5, 4)          # big steps: still exact
    for g in (gx, gy, gz):
        g.drift(2.0)
    ref = product3(gx, gy, gz, x, y, z)
    assert rel(psi, ref) < 1e-10


def test_harmonic_matches_exact_discrete_strang(orc):
    """V = |r|^2/2: the oracle must follow the exact discrete Strang
    trajectory of a displaced Gaussian, global phase included."""
    shape = (64, 64, 128)
    box = (-14.0, 14.0, -10.0, 10.0, -10.0, 10.0)
    x, y, z = grids(shape, box)
    V = (0.5 * (x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2))
    gx = Gauss1D.displaced_ground(2.0, 0.5)
    gy = Gauss1D.displaced_ground(0.0, 0.0)
    gz = Gauss1D.displaced_ground(-1.0, 0.0)
    psi0 = product3(gx, gy, gz, x, y, z)
    dt, n = 0.05, 40
    psi = orc.step(psi0, V, box, dt, n)
    for g in (gx, gy, gz):
        g.strang_ho(dt, n)
    ref = product3(gx, gy, gz, x, y, z)
    assert rel(psi, ref) < 1e-11


def test_harmonic_coherent_state_second_order(orc):
    """Against the continuum coherent state the error is O(dt^2): halving dt
    quarters it (harmonic_tiny workload's physics, 32^3 on [-8,8]^3 grid
    family)."""
    shape, box = (32, 32, 64), (-10.0, 10.0, -8.0, 8.0, -8.0, 8.0)
    x, y, z = grids(shape, box)
    V = wl.harmonic_dense(shape, box)
    psi0 = product3(lambda q: coherent_1d(q, 0.0, 2.0), lambda q: coherent_1d(q, 0.0, 0.0),
                    lambda q: coherent_1d(q, 0.0, 0.0), x, y, z)
    T = 1.0
    errs = []
    for dt in (0.04, 0.02, 0.01):
        psi = orc.step(psi0, V, box, dt, int(round(T / dt)))
        ref = product3(lambda q: coherent_1d(q, T, 2.0), lambda q: coherent_1d(q, T, 0.0),
                       lambda q: coherent_1d(q, T, 0.0), x, y, z)
        errs.append(rel(psi, ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2, errs
    assert errs[1] < 2e-3


def test_coherent_state_tiny_workload(orc):
    """harmonic_tiny: 32^3 on [-8,8]^3, coherent state x0 = 2, dt = 0.01, 100
    steps.  Centroid follows (x0 cos t); the deviation from the continuum is
    the O(dt^2) splitting error plus the grid's aliasing."""
    w = wl.WORKLOADS["harmonic_tiny"]
    x, y, z = grids(w.shape, w.box)
    psi0 = wl.coherent_state(w.shape, w.box, 2.0)
    V = wl.harmonic_dense(w.shape, w.box)
    psi = orc.step(psi0, V, w.box, w.dt, w.steps)
    t = w.dt * w.steps
    ref = product3(lambda q: coherent_1d(q, t, 2.0), lambda q: coherent_1d(q, t, 0.0),
                   lambda q: coherent_1d(q, t, 0.0), x, y, z)
    assert rel(psi, ref) < 1e-4
    dens = np.abs(psi) ** 2
    xc = np.sum(dens * x[None, None, :]) / np.sum(dens)
    assert abs(xc - 2.0 * np.cos(t)) < 1e-5


def test_imaginary_time_oscillator_fixed_point(orc):
    """Imaginary-time Strang steps converge to exp(-a r^2/2) with
    a = sqrt(1 + dtau^2/4) exactly (fixed point of the Gaussian map), whose
    energy is (3/4)(a + 1/a) = 3/2 + O(dtau^4)."""
    shape, box = (32, 32, 32), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    x, y, z = grids(shape, box)
    V = wl.harmonic_dense(shape, box)
    psi0 = product3(Gauss1D.packet(0.4, 0.3), Gauss1D.packet(0.6), Gauss1D.packet(0.5, -0.2),
                    x, y, z)
    dtau = 0.2
    psi = orc.step(psi0, V, box, dtau, 150, imag=True)
    a = np.sqrt(1.0 + dtau * dtau / 4.0)
    g = Gauss1D(a, 0.0, 0.25 * np.log(a / np.pi))
    ref = product3(g, g, g, x, y, z)
    assert rel(psi, ref) < 1e-10
    obs = orc.observables(psi, V, box)
    assert abs(obs[0] - 1.0) < 1e-12
    assert abs(obs[1] + obs[2] - 0.75 * (a + 1.0 / a)) < 1e-10
    # and the discrete energy is 3/2 to O(dtau^4)
    assert abs(obs[1] + obs[2] - 1.5) < dtau ** 4


def test_imaginary_time_follows_exact_trajectory(orc):
    """Before convergence: each imaginary-time step maps Gaussians to
    Gaussians; compare after 5 steps (normalised)."""
    shape, box = (32, 32, 32), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    x, y, z = grids(shape, box)
    V = wl.harmonic_dense(shape, box)
    gs = [Gauss1D.packet(0.8, 0.5), Gauss1D.packet(1.0), Gauss1D.packet(0.9, -0.4)]
    psi0 = product3(*gs, x, y, z)
    psi = orc.step(psi0, V, box, 0.1, 5, imag=True)
    for g in gs:
        g.strang_ho(0.1, 5, imag=True)
    ref = wl.normalise(product3(*gs, x, y, z), box)
    assert rel(psi, ref) < 1e-11


def _ctap_case(shape=(64, 32, 32)):
    box = wl.CTAP_BOX
    nz = shape[0]
    z = wl.axis(nz, box[4], box[5])
    c = wl.guide_centres(z)
    import oracle
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    psi = wl.gaussian_sum(shape, (-10, 10, -10, 10, -40, 40), seed=3)
    psi = psi * np.exp(1j * 0.7 * wl.mesh(shape, box)[2])
    return psi.astype(complex), V, box


def test_unitarity_real_time(orc):
    psi0, V, box = _ctap_case()
    psi = orc.step(psi0, V, box, 0.01, 100)
    n0 = np.sum(np.abs(psi0) ** 2)
    assert abs(np.sum(np.abs(psi) ** 2) - n0) < 1e-13 * n0


def test_time_reversibility(orc):
    """S(-dt) S(dt) = identity for the symmetric splitting."""
    psi0, V, box = _ctap_case()
    psi = orc.step(psi0, V, box, 0.01, 100)
    back = orc.step(psi, V, box, -0.01, 100)
    assert rel(back, psi0) < 1e-13


def test_zero_steps_is_identity(orc):
    psi0, V, box = _ctap_case((8, 8, 8))
    assert np.array_equal(orc.step(psi0, V, box, 0.01, 0), psi0)


def test_thread_count_does_not_change_results(orc):
    """The parallel loops of the oracle run independent lines, so one thread
    and all host cores give bitwise the same state (the timed CPU baseline
    uses both)."""
    psi0, V, box = _ctap_case()
    cores = orc.num_threads()
    many = orc.step(psi0, V, box, 0.01, 5)
    orc.set_num_threads(1)
    try:
        assert orc.num_threads() == 1
        one = orc.step(psi0, V, box, 0.01, 5)
    finally:
        orc.set_num_threads(cores)
    assert orc.num_threads() == cores
    assert np.array_equal(one, many)
