"""Pins for the oracle's paper-faithful variants: the K/2 V K/2 ordering of
the split step (Sec. IV counts four transforms per step), the longitudinal
harmonic trap added to the guides (Sec. III) and the y-integrated density
of Fig. 5.  Each pin is independent of the oracle's own arithmetic."""
import numpy as np

from gaussian_exact import Gauss1D, product3
from paper_1309_2451_b300 import workloads as wl


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def grids(shape, box):
    nz, ny, nx = shape
    return wl.axis(nx, box[0], box[1]), wl.axis(ny, box[2], box[3]), wl.axis(nz, box[4], box[5])


def test_kvk_harmonic_matches_exact_discrete_trajectory(orc):
    """V = |r|^2/2 with the kinetic factor split: the exact discrete
    trajectory is drift dt/2, kick dt, drift dt/2 per step (Gaussian
    parameter recursion, phase included)."""
    shape = (64, 64, 128)
    box = (-14.0, 14.0, -10.0, 10.0, -10.0, 10.0)
    x, y, z = grids(shape, box)
    V = 0.5 * (x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)
    gx = Gauss1D.displaced_ground(2.0, 0.5)
    gy = Gauss1D.displaced_ground(0.0, 0.0)
    gz = Gauss1D.displaced_ground(-1.0, 0.0)
    psi0 = product3(gx, gy, gz, x, y, z)
    dt, n = 0.05, 40
    psi = orc.step(psi0, V, box, dt, n, order="KVK")
    for g in (gx, gy, gz):
        g.strang_ho_kvk(dt, n)
    ref = product3(gx, gy, gz, x, y, z)
    assert rel(psi, ref) < 1e-11
    # and it is a different trajectory from V/2 K V/2 at this dt
    vkv = orc.step(psi0, V, box, dt, n)
    assert rel(psi, vkv) > 1e-4


def test_kvk_free_particle_is_exact(orc):
    """V = 0: both orderings are the exact free propagator."""
    shape, box = (64, 64, 64), (-16.0, 16.0, -16.0, 16.0, -16.0, 16.0)
    x, y, z = grids(shape, box)
    gx, gy, gz = Gauss1D.packet(1.0, -2.0, 1.0), Gauss1D.packet(1.2, 0.0, -0.5), \
        Gauss1D.packet(0.9, 1.0, 0.0)
    psi0 = product3(gx, gy, gz, x, y, z)
    psi = orc.step(psi0, np.zeros(shape), box, 0.4, 5, order="KVK")
    for g in (gx, gy, gz):
        g.drift(2.0)
    assert rel(psi, product3(gx, gy, gz, x, y, z)) < 1e-10


def test_trap_z_shifts_oscillator_phase_only(orc):
    """A z-only term ω²z²/2 added to the guide potential acts on the z
    factor alone: for V = (x² + y²)/2 + ω²z²/2 and a Gaussian in z with
    width 1/sqrt(ω), the z factor follows the exact discrete Strang
    trajectory of the oscillator of frequency ω (rescaled recursion)."""
    w = 0.5
    shape = (128, 64, 64)
    box = (-8.0, 8.0, -8.0, 8.0, -20.0, 20.0)
    x, y, z = grids(shape, box)
    V = 0.5 * (x[None, None, :] ** 2 + y[None, :, None] ** 2) + wl.trap_z(z, w)[:, None, None]
    gx, gy = Gauss1D.displaced_ground(1.0, 0.0), Gauss1D.displaced_ground(0.0, 0.3)
    # oscillator of frequency w in z: q = sqrt(w) z maps it to the unit oscillator
    # with time scaled by w; a Gaussian exp(-A z^2/2 + B z + C) in z is the unit
    # oscillator's Gaussian with A' = A/w, B' = B/sqrt(w) and the same C up to
    # the normalisation constant ln(w)/4.
    gq = Gauss1D.displaced_ground(2.0, 0.0)
    dt, n = 0.1, 30
    sq = np.sqrt(w)
    psi0 = product3(gx, gy, Gauss1D(gq.A * w, gq.B * sq, gq.C), x, y, z)
    psi = orc.step(psi0, V, box, dt, n)
    gx.strang_ho(dt, n)
    gy.strang_ho(dt, n)
    gq.strang_ho(w * dt, n)
    ref = product3(gx, gy, Gauss1D(gq.A * w, gq.B * sq, gq.C), x, y, z)
    assert rel(psi, ref) < 1e-10


def test_guide_orders_mirror_each_other():
    """The intuitive arrangement exchanges the two separation profiles."""
    z = wl.axis(64, -60.0, 60.0)
    c = wl.guide_centres(z, "counter")
    i = wl.guide_centres(z, "intuitive")
    assert np.allclose(i[0], -c[2]) and np.allclose(i[2], -c[0])
    # intuitive: the left-middle gap is smallest before the middle-right gap
    assert z[np.argmin(-i[0])] < z[np.argmin(i[2])]
    assert z[np.argmin(c[2])] < z[np.argmin(-c[0])]


def test_density_xz_of_gaussian_closed_form(orc):
    """n(z, x) = sum_y |psi|^2 dy of a product Gaussian: the y-integral of
    exp(-y^2/s^2) is s sqrt(pi) (the grid sum converges spectrally)."""
    shape, box = (16, 64, 32), (-6.0, 6.0, -10.0, 10.0, -4.0, 4.0)
    x, y, z = grids(shape, box)
    s = 1.3
    fx = np.exp(-(x - 0.5) ** 2 / 2.0)
    fz = np.exp(-z ** 2 / 3.0)
    psi = fz[:, None, None] * np.exp(-y ** 2 / (2 * s * s))[None, :, None] * fx[None, None, :] \
        * np.exp(0.7j * x)[None, None, :]
    n = orc.density_xz(psi, box)
    ref = (fz ** 2)[:, None] * (fx ** 2)[None, :] * s * np.sqrt(np.pi)
    assert n.shape == (shape[0], shape[2])
    assert np.allclose(n, ref, rtol=1e-12, atol=1e-15)
