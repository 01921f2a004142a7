"""Pins for the oracle's atom-chip field (Sec. III, Eq. 4-5): thin straight
current segments (the Biot-Savart law) plus uniform fields.  Pinned against
textbook closed forms and a direct quadrature of the Biot-Savart integral."""
import numpy as np

K = 1.0      # mu0/(4 pi) in these units


def test_long_wire_field_is_2kI_over_d(orc):
    seg = [[0.0, 0.0, -1e7, 0.0, 0.0, 1e7, 0.7]]
    rng = np.random.default_rng(3)
    pts = rng.uniform(-3, 3, size=(50, 3))
    B = orc.wire_field(pts, seg, [0, 0, 0], K)
    d = np.hypot(pts[:, 0], pts[:, 1])
    assert np.allclose(np.linalg.norm(B, axis=1), 2 * K * 0.7 / d, rtol=1e-10)
    # direction z x r_perp (right-hand rule)
    rp = np.stack([pts[:, 0], pts[:, 1], 0 * pts[:, 0]], axis=1)
    want = np.cross([0.0, 0.0, 1.0], rp) / (d ** 2)[:, None] * 2 * K * 0.7
    assert np.allclose(B, want, rtol=1e-9, atol=1e-12)


def test_bias_lifts_the_zero_to_r0(orc):
    """Eq. 5: a wire along z on the chip and a bias field B_b orthogonal to
    it: the total field vanishes at height r0 = mu0 I/(2 pi B_b) = 2 k I/B_b."""
    I, Bb = 0.1, 0.14
    seg = [[0.0, 0.0, -1e7, 0.0, 0.0, 1e7, I]]
    r0 = 2 * K * I / Bb
    ys = np.linspace(0.2, 4.0, 1901)
    pts = np.stack([0 * ys, ys, 0 * ys], axis=1)
    B = orc.wire_field(pts, seg, [Bb, 0.0, 0.0], K)
    mag = np.linalg.norm(B, axis=1)
    assert abs(ys[np.argmin(mag)] - r0) < 2e-3
    at = orc.wire_field([[0.0, r0, 0.0]], seg, [Bb, 0.0, 0.0], K)
    assert np.linalg.norm(at) < 1e-12


def test_square_loop_centre(orc):
    """Centre of a square loop of side a: |B| = 2 sqrt(2) mu0 I/(pi a)."""
    a, I = 2.0, 1.3
    c = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    seg = []
    for i in range(4):
        (x0, y0), (x1, y1) = c[i], c[(i + 1) % 4]
        seg.append([x0 * a / 2, y0 * a / 2, 0.0, x1 * a / 2, y1 * a / 2, 0.0, I])
    B = orc.wire_field([[0.0, 0.0, 0.0]], seg, [0, 0, 0], K)
    mu0 = 4 * np.pi * K
    assert np.allclose(np.abs(B[0]), [0, 0, 2 * np.sqrt(2) * mu0 * I / (np.pi * a)], rtol=1e-12)


def test_bent_wire_matches_biot_savart_quadrature(orc):
    """A kinked wire (two segments) against the line integral of Eq. 4,
    B = k I sum dl x r / |r|^3, by the midpoint rule on 200000 elements."""
    I = 0.4
    A, Bk, C = np.array([0.0, -1.0, -3.0]), np.array([0.5, -1.0, 0.0]), np.array([-0.2, -1.0, 2.5])
    seg = [list(A) + list(Bk) + [I], list(Bk) + list(C) + [I]]
    pts = np.array([[0.3, 0.5, 0.1], [-1.0, 0.2, 1.7], [2.0, -0.5, -1.0]])
    got = orc.wire_field(pts, seg, [0, 0, 0], K)
    want = np.zeros_like(pts)
    n = 200000
    for P0, P1 in ((A, Bk), (Bk, C)):
        t = (np.arange(n) + 0.5) / n
        mid = P0[None, :] + t[:, None] * (P1 - P0)[None, :]
        dl = (P1 - P0) / n
        for i, p in enumerate(pts):
            r = p[None, :] - mid
            want[i] += K * I * np.sum(np.cross(dl[None, :], r) / np.linalg.norm(r, axis=1)[:, None] ** 3,
                                      axis=0)
    assert np.allclose(got, want, rtol=1e-8, atol=1e-12)


def test_wire_potential_is_scaled_field_magnitude(orc):
    shape, box = (4, 8, 8), (-2.0, 2.0, 0.5, 2.5, -1.0, 1.0)
    seg = [[0.0, 0.0, -50.0, 0.0, 0.0, 50.0, 0.2]]
    V = orc.wire_potential(shape, box, seg, [0.1, 0.0, 0.3], K, 5.0, 1.5)
    x = orc.grid_axis(8, -2.0, 2.0)
    y = orc.grid_axis(8, 0.5, 2.5)
    B = orc.wire_field([[x[3], y[5], orc.grid_axis(4, -1.0, 1.0)[2]]], seg, [0.1, 0.0, 0.3], K)
    assert np.isclose(V[2, 5, 3], 5.0 * np.linalg.norm(B) - 1.5, rtol=1e-14)


def test_paper_chip_parameters_trap_height(orc):
    """The paper's chip (Sec. III, captions of Fig. 2-3, stored with
    citations in golden/paper_chip_parameters.json), in SI units: a long wire
    with I = 0.1 A under B_b = 140 x 10^-4 T has its field zero at Eq. 5's
    r0 = mu0 I/(2 pi B_b) = 1.43 um, inside the 4 um the paper simulates above
    the chip; the reduced middle current 0.07 A lowers it by the same ratio.
    The oracle's segment sum must put the minimum there; and the process time
    is half a period of the 5 Hz longitudinal trap."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_chip_parameters.json")
    p = json.load(open(path))
    k = p["mu0_over_4pi_SI"]["value"]
    Bb = p["bias_field_T"]["value"]
    height = p["height_above_chip_m"]["value"]
    for key in ("wire_current_outer_A", "wire_current_middle_reduced_A"):
        I = p[key]["value"]
        r0 = 2 * k * I / Bb
        assert 0.0 < r0 < height
        seg = [[0.0, 0.0, -1.0, 0.0, 0.0, 1.0, I]]            # 2 m wire: long against um
        ys = np.linspace(0.05e-6, height, 3951)
        pts = np.stack([0 * ys, ys, 0 * ys], axis=1)
        mag = np.linalg.norm(orc.wire_field(pts, seg, [Bb, 0.0, 0.0], k), axis=1)
        assert abs(ys[np.argmin(mag)] - r0) < 1.5e-9
        # the bias is orthogonal to the wire; B_ip along the wire only adds
        # a constant |B| floor, the minimum stays at r0
        Bip = p["applied_field_T"]["value"]
        mag2 = np.linalg.norm(orc.wire_field(pts, seg, [Bb, 0.0, Bip], k), axis=1)
        assert ys[np.argmin(mag2)] == ys[np.argmin(mag)]
        assert abs(mag2.min() - Bip) < 1e-3 * Bip
    assert abs(p["wire_current_middle_reduced_A"]["value"] / p["wire_current_outer_A"]["value"] - 0.7) < 1e-12
    f = p["longitudinal_trap_hz"]["value"]
    assert abs(0.5 / f - p["process_time_s"]["value"]) < 1e-12
