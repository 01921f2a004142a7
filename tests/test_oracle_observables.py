"""Pins for the oracle's observables, guide potential and spline basis.

Observables (Sec. V, Fig. 4: population of each guide versus time; norm and
energy as diagnostics) are pinned by states whose values are known exactly;
the three-guide potential by its structural properties; the spline basis by
scipy's natural cubic spline.
"""
import numpy as np
import pytest
import scipy.interpolate

from paper_1309_2451_b300 import workloads as wl


def test_norm_and_energy_of_oscillator_ground_state(orc):
    shape, box = (32, 32, 32), (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)
    psi = wl.coherent_state(shape, box, 0.0)
    V = wl.harmonic_dense(shape, box)
    obs = orc.observables(psi, V, box)
    assert abs(obs[0] - 1.0) < 1e-12          # normalised Gaussian
    assert abs(obs[1] - 0.75) < 1e-10         # <T> = 3/4
    assert abs(obs[2] - 0.75) < 1e-10         # <V> = 3/4


def test_kinetic_energy_of_plane_wave(orc):
    """A grid plane wave exp(i k.r) has <T> = |k|^2/2 exactly."""
    shape, box = (16, 8, 32), (-4.0, 4.0, -2.0, 6.0, 0.0, 3.0)
    x, y, z = wl.mesh(shape, box)
    kx, ky, kz = 2 * np.pi * 3 / 8.0, -2 * np.pi * 2 / 8.0, 2 * np.pi * 5 / 3.0
    psi = np.exp(1j * (kx * x + ky * y + kz * z)) * np.ones(shape)
    obs = orc.observables(psi, np.full(shape, -2.5), box)
    assert abs(obs[1] - 0.5 * (kx * kx + ky * ky + kz * kz)) < 1e-10
    assert abs(obs[2] + 2.5) < 1e-14
    assert abs(obs[0] - 8.0 * 8.0 * 3.0) < 1e-10   # |psi|^2 = 1 over the box volume


def test_populations_count_grid_points(orc):
    """|psi|^2 = 1 on a grid whose x-points are the integers -16..15 (dV = 1);
    each guide region |x - c| < 1.5 (strict) then holds a countable number of
    x-points per slice: 3 for an integer or quarter-offset centre, 2 for a
    half-integer centre (both ends c +- 1.5 are grid points and excluded)."""
    shape, box = (4, 2, 32), (-16.0, 16.0, 0.0, 2.0, 0.0, 4.0)   # dV = 1
    psi = np.ones(shape, dtype=complex)
    centres = np.array([[-5.25, -5.25, 2.0, 2.0],
                        [0.0, 0.5, 0.5, 0.0],
                        [3.5, 7.75, 10.0, 3.5]])
    # x-points per slice, region (c - 1.5, c + 1.5):
    # c=-5.25 -> {-6,-5,-4}; c=2 -> {1,2,3}; c=0 -> {-1,0,1}; c=0.5 -> {0,1};
    # c=3.5 -> {3,4}; c=7.75 -> {7,8,9}; c=10 -> {9,10,11}; ny = 2 rows each
    expect = [2 * (3 + 3 + 3 + 3), 2 * (3 + 2 + 2 + 3), 2 * (2 + 3 + 3 + 2)]
    obs = orc.observables(psi, np.zeros(shape), box, centres, 1.5)
    assert np.allclose(obs[3:], expect, rtol=0, atol=1e-12)
    assert abs(obs[0] - psi.size) < 1e-12


def test_population_of_gaussian_in_guide(orc):
    """Density pi^(-3/2) exp(-x^2-y^2-z^2) centred on a guide: the region
    |x| < 1.5 holds erf(1.5) of it (grid boundaries at midpoints)."""
    shape, box = (64, 64, 128), (-12.0, 12.0, -8.0, 8.0, -8.0, 8.0)
    dx = 24.0 / 128
    psi = wl.coherent_state(shape, box, 0.0)
    c = np.zeros((3, 64))
    c[0] -= 6.0 + dx / 2
    c[2] += 6.0 + dx / 2
    obs = orc.observables(psi, None, box, c, 1.5 + dx / 2)
    from math import erf
    assert abs(obs[4] - erf(1.5 + dx / 2)) < 1e-3
    assert abs(obs[3] - obs[5]) < 1e-14
    assert obs[3] < 1e-6


# ---------------------------------------------------------------- potential

def _centres(nz, box):
    return wl.guide_centres(wl.axis(nz, box[4], box[5]))


def test_potential_product_structure_and_symmetry(orc):
    shape, box = (16, 32, 64), wl.CTAP_BOX
    c = _centres(16, box)
    V = orc.ctap_potential(shape, box, 20.0, 1.0, c[0], c[2])
    y = wl.axis(32, box[2], box[3])
    iy0 = 16                                   # y = 0
    ratio = V / V[:, iy0:iy0 + 1, :]
    assert np.allclose(ratio, np.exp(-y ** 2 / 2.0)[None, :, None], rtol=1e-13, atol=0)
    # mirror symmetry when the outer guides are placed symmetrically
    Vs = orc.ctap_potential((4, 8, 64), (-12.0, 12.0, -1, 1, 0, 1), 20.0, 1.0,
                            -np.full(4, 4.0), np.full(4, 4.0))
    # x grid -12 + 24 i/64: x -> -x maps index i to 64 - i (i >= 1)
    assert np.allclose(Vs[:, :, 1:], Vs[:, :, :0:-1], rtol=1e-14, atol=1e-14)


def test_potential_depth_and_curvature_at_guide(orc):
    """Guides at -6, 0, 6: V(0, 0) = -V0 (1 + 2 e^{-18/s^2}) at the middle
    guide, and the transverse curvature there is
    V0/s^2 - 2 V0 e^{-18/s^2} (36/s^4 - 1/s^2)."""
    nx = 1024
    box = (-12.0, 12.0, -1.0, 1.0, 0.0, 1.0)
    s = 1.25
    V = orc.ctap_potential((1, 2, nx), box, 20.0, s, np.array([-6.0]), np.array([6.0]))
    i0 = nx // 2                                # x = 0
    e = np.exp(-36.0 / (2 * s * s))
    assert abs(V[0, 1, i0] - (-20.0 * (1 + 2 * e))) < 1e-12
    h = 24.0 / nx
    f = V[0, 1, i0 - 2:i0 + 3]
    curv = (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)
    expect = 20.0 / s ** 2 - 2 * 20.0 * e * (36.0 / s ** 4 - 1.0 / s ** 2)
    assert abs(curv - expect) < 1e-6


def test_dvdx_matches_finite_difference_of_potential(orc):
    """dV/dx_j from the oracle equals the central difference of the
    potential builder with respect to the guide centre."""
    shape, box = (8, 16, 32), wl.CTAP_BOX
    c = _centres(8, box)
    eps = 1e-6
    for j in (0, 2):
        cp, cm = c.copy(), c.copy()
        cp[j] += eps
        cm[j] -= eps
        Vp = orc.ctap_potential(shape, box, 20.0, 1.0, cp[0], cp[2])
        Vm = orc.ctap_potential(shape, box, 20.0, 1.0, cm[0], cm[2])
        fd = (Vp - Vm) / (2 * eps)
        D = orc.ctap_dvdx(shape, box, 20.0, 1.0, c[j])
        assert np.max(np.abs(D - fd)) < 1e-7


# ---------------------------------------------------------------- spline

def test_spline_basis_matches_scipy_natural_spline(orc):
    knots = np.array(wl.KNOTS_Z)
    z = np.linspace(-60, 60, 257)[:-1]
    B = orc.natural_spline_basis(knots, z)
    rng = np.random.default_rng(0)
    for _ in range(3):
        c = rng.standard_normal(knots.size)
        ref = scipy.interpolate.CubicSpline(knots, c, bc_type="natural")(z)
        assert np.max(np.abs(c @ B - ref)) < 1e-12


def test_spline_basis_is_cardinal_and_reproduces_lines(orc):
    knots = np.array(wl.KNOTS_Z)
    B = orc.natural_spline_basis(knots, knots)
    assert np.max(np.abs(B - np.eye(knots.size))) < 1e-13
    z = np.linspace(-60, 59.5, 300)
    Bz = orc.natural_spline_basis(knots, z)
    assert np.max(np.abs((3.0 - 0.25 * knots) @ Bz - (3.0 - 0.25 * z))) < 1e-12
