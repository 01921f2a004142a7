"""Pin for the oracle's adjoint gradient: central finite differences of the
oracle's own forward objective (frozen initial state and frozen population
region).  The adjoint (reverse conjugate-phase sweep) is not in the paper; it
differentiates the final population of a guide (Sec. V, Fig. 4 observable)
with respect to the guide-separation profile.
"""
import numpy as np
import pytest

from paper_1309_2451_b300 import workloads as wl

SHAPE = (32, 16, 32)
BOX = (-9.0, 9.0, -6.0, 6.0, -24.0, 24.0)
KNOTS = np.linspace(-24.0, 24.0, 7)


def _setup(orc, guide_index):
    nz, ny, nx = SHAPE
    c12 = wl.separation(KNOTS, wl.ZC_12, dmin=2.0, dmax=4.0, w=8.0)
    c23 = wl.separation(KNOTS, wl.ZC_23, dmin=2.0, dmax=4.0, w=8.0)
    z = wl.axis(nz, BOX[4], BOX[5])
    B = orc.natural_spline_basis(KNOTS, z)
    x1 = -(c12 @ B)
    x, y, zz = wl.mesh(SHAPE, BOX)
    psi0 = np.exp(-((x - x1[:, None, None]) ** 2 + y ** 2) / 2.0 - (zz + 10.0) ** 2 / 18.0
                  + 2j * zz)
    psi0 = wl.normalise(psi0.astype(complex), BOX)
    centres = np.stack([x1, np.zeros(nz), c23 @ B])
    mask = orc.guide_mask(SHAPE, BOX, centres[guide_index], 1.5)
    return psi0, c12, c23, mask


@pytest.mark.parametrize("guide_index", [1, 2])
def test_adjoint_gradient_matches_central_differences(orc, guide_index):
    dt, n = 0.05, 40
    psi0, c12, c23, mask = _setup(orc, guide_index)
    J, g = orc.ctap_gradient(psi0, BOX, 20.0, 1.0, KNOTS, c12, c23, dt, n, guide_index)
    J0 = orc.ctap_objective(psi0, BOX, 20.0, 1.0, KNOTS, c12, c23, dt, n, mask)
    assert abs(J - J0) < 1e-14
    assert J > 1e-4
    h = 1e-4
    m = KNOTS.size
    scale = np.max(np.abs(g))
    assert scale > 1e-4
    for idx in (1, 2, 3, m + 2, m + 3, m + 4):
        cp12, cp23, cm12, cm23 = c12.copy(), c23.copy(), c12.copy(), c23.copy()
        if idx < m:
            cp12[idx] += h
            cm12[idx] -= h
        else:
            cp23[idx - m] += h
            cm23[idx - m] -= h
        Jp = orc.ctap_objective(psi0, BOX, 20.0, 1.0, KNOTS, cp12, cp23, dt, n, mask)
        Jm = orc.ctap_objective(psi0, BOX, 20.0, 1.0, KNOTS, cm12, cm23, dt, n, mask)
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[idx] - fd) < 1e-6 * scale + 1e-6 * abs(fd), (idx, g[idx], fd)


def test_adjoint_per_slice_sensitivity(orc):
    """R_3(z) is dJ/dx_3(z) for a shift of the guide centre in one slice."""
    dt, n = 0.05, 30
    psi0, c12, c23, mask = _setup(orc, 2)
    nz = SHAPE[0]
    z = wl.axis(nz, BOX[4], BOX[5])
    B = orc.natural_spline_basis(KNOTS, z)
    x1, x3 = -(c12 @ B), c23 @ B
    V = orc.ctap_potential(SHAPE, BOX, 20.0, 1.0, x1, x3)
    W1 = orc.ctap_dvdx(SHAPE, BOX, 20.0, 1.0, x1)
    W3 = orc.ctap_dvdx(SHAPE, BOX, 20.0, 1.0, x3)
    J, R1, R3 = orc.adjoint(psi0, V, BOX, dt, n, mask, W1, W3)
    dv = wl.cell_volume(SHAPE, BOX)
    h = 1e-5
    for iz in (8, 12, 16):
        for which, R in ((0, R1), (2, R3)):
            res = []
            for sgn in (1, -1):
                xa, xb = x1.copy(), x3.copy()
                (xa if which == 0 else xb)[iz] += sgn * h
                Vp = orc.ctap_potential(SHAPE, BOX, 20.0, 1.0, xa, xb)
                res.append(np.sum(mask * np.abs(orc.step(psi0, Vp, BOX, dt, n)) ** 2) * dv)
            fd = (res[0] - res[1]) / (2 * h)
            assert abs(R[iz] - fd) < 1e-6 * np.max(np.abs(R)) + 1e-5 * abs(fd), (iz, which, R[iz], fd)
