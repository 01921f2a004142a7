"""Seeded synthetic inputs shared by the CUDA path, the tests and bench.py.

Holds none of the split-step arithmetic: only grids for evaluating initial
states, the initial states themselves, the guide-separation profiles and the
workload definitions.  Both the CUDA library and the CPU oracle build their
own potentials, phases and transforms from these parameters.

Workloads (hbar = m = 1, arrays shaped (nz, ny, nx), x fastest):

* ``harmonic_tiny``   32^3 on [-8,8]^3, V = |r|^2/2, coherent state displaced
                      to x0 = 2, dt = 0.01, 100 real-time steps.
* ``ctap_fp64``       128x128x256 on [-12,12]^2 x [-60,60], three Gaussian
                      guides (V0 = 20, s = 1), counter-intuitive separation
                      profiles; guide-1 transverse ground state (imaginary
                      time, 200 steps) times a z-Gaussian (width 4 at z = -40,
                      momentum 2); 2000 real-time steps at dt = 0.005.
* ``ctap_large``      the same family on 256x256x1024, 4000 steps at dt = 0.0025.
* ``ctap_adjoint``    128x128x256 complex64, 16+16 natural-spline controls of the
                      two separation profiles, 1000 steps at dt = 0.005.
* ``sweep``           harmonic and guide potentials at 64^3 ... 256x256x1024,
                      500 steps at dt = 0.005, psi0 a normalised sum of 4 random
                      Gaussians (centres in [-4,4]^3, widths in [0.8,2]).

The guide model stands in for the paper's Biot-Savart atom-chip field
(Sec. III, Eq. 4-5): three waveguides whose separations shrink and grow along
the propagation axis z, the spatial version of the couplings in Eq. (1); the
middle-to-right pair approaches first (counter-intuitive order, Sec. II).
"""
from dataclasses import dataclass, field

import numpy as np

CTAP_BOX = (-12.0, 12.0, -12.0, 12.0, -60.0, 60.0)
HARMONIC_BOX = (-8.0, 8.0, -8.0, 8.0, -8.0, 8.0)

# separation profile d(z) = dmin + (dmax - dmin)(1 - exp(-(z - zc)^2/(2 w^2)))
PROFILE = dict(dmin=2.5, dmax=6.0, w=12.0)
ZC_12 = 10.0     # left-middle pair approaches second
ZC_23 = -10.0    # middle-right pair approaches first (counter-intuitive)
V0 = 20.0
SIGMA_GUIDE = 1.0
POP_HALFWIDTH = 1.5
KNOTS_Z = tuple(-60.0 + 8.0 * m for m in range(16))
# longitudinal trap: a packet released at rest at z = -40 reaches the far
# turning point z = +40 after half a period pi/omega, with peak momentum
# 40 omega = 3.2 (resolved by nz >= 256 on the 120-long box)
TRAP_OMEGA = 0.08


def axis(n, lo, hi):
    """Periodic grid lo + i (hi - lo)/n (upper edge excluded)."""
    return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / n)


def mesh(shape, box):
    nz, ny, nx = shape
    z = axis(nz, box[4], box[5])[:, None, None]
    y = axis(ny, box[2], box[3])[None, :, None]
    x = axis(nx, box[0], box[1])[None, None, :]
    return x, y, z


def cell_volume(shape, box):
    nz, ny, nx = shape
    return (box[1] - box[0]) / nx * (box[3] - box[2]) / ny * (box[5] - box[4]) / nz


def normalise(psi, box):
    n = np.sqrt(np.sum(np.abs(psi) ** 2) * cell_volume(psi.shape, box))
    return psi / n


def separation(z, zc, dmin=PROFILE["dmin"], dmax=PROFILE["dmax"], w=PROFILE["w"]):
    """Analytic guide separation d(z)."""
    z = np.asarray(z, dtype=np.float64)
    return dmin + (dmax - dmin) * (1.0 - np.exp(-(z - zc) ** 2 / (2.0 * w * w)))


def guide_centres(z, order="counter"):
    """x_1(z) = -d12(z), x_2 = 0, x_3(z) = +d23(z) as a (3, nz) array.

    order "counter": the middle-right pair approaches first (counter-intuitive
    sequence, Fig. 4a); order "intuitive": the two profiles are exchanged, so
    the left-middle pair approaches first (Fig. 4b)."""
    z = np.asarray(z, dtype=np.float64)
    if order == "counter":
        zc12, zc23 = ZC_12, ZC_23
    elif order == "intuitive":
        zc12, zc23 = ZC_23, ZC_12
    else:
        raise ValueError("order must be 'counter' or 'intuitive'")
    return np.stack([-separation(z, zc12), np.zeros_like(z), separation(z, zc23)])


# Atom-chip wires (Sec. III, Fig. 1-3 captions): lengths in um, fields in
# gauss, currents in A.  mu0/(4 pi) = 1e-7 T m/A = 1e3 G um/A.
CHIP = dict(mu0_over_4pi=1.0e3, I_outer=0.1, I_mid=0.07, B_bias=140.0, B_ip=300.0,
            sep_far=7.0, sep_near=4.3, straight=50.0, length=1000.0, width=12.0)


def chip_wires(nseg=64, order="counter", zc=(600.0, 400.0), w=120.0, **kw):
    """Three wires on the chip surface (the plane y = 0) running along z over
    the chip length: polylines of nseg straight segments each, rows
    (Ax, Ay, Az, Cx, Cy, Cz, I).  The gaps to the middle wire shrink from
    sep_far to sep_near as Gaussian dips centred at zc = (left, right); the
    left wire stays straight over the first `straight` um (the asymmetry of
    Fig. 2).  The paper gives these numbers but not the wire curves: the dip
    profile is this stand-in's choice.  order "intuitive" exchanges the two
    dips."""
    c = dict(CHIP, **kw)
    zl, zr = zc if order == "counter" else zc[::-1]
    z = np.linspace(0.0, c["length"], nseg + 1)

    def gap(zz, z0):
        return c["sep_far"] - (c["sep_far"] - c["sep_near"]) * np.exp(-(zz - z0) ** 2 / (2 * w * w))

    xl = -gap(z, zl)
    xl[z <= c["straight"]] = -c["sep_far"]
    xr = gap(z, zr)
    rows = []
    for xs, cur in ((xl, c["I_outer"]), (np.zeros_like(z), c["I_mid"]), (xr, c["I_outer"])):
        for i in range(nseg):
            rows.append([xs[i], 0.0, z[i], xs[i + 1], 0.0, z[i + 1], cur])
    return np.array(rows)


def chip_bias(**kw):
    """Uniform field: the bias along x (in the chip plane, across the wires)
    and the field along the wires (z)."""
    c = dict(CHIP, **kw)
    return np.array([c["B_bias"], 0.0, c["B_ip"]])


def trap_z(z, omega=TRAP_OMEGA, zc=0.0):
    """Longitudinal harmonic trap omega^2 (z - zc)^2 / 2 centred on the chip
    (Sec. III: it accelerates the atom along the guides and refocuses it at
    the far turning point)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * omega * omega * (z - zc) ** 2


def spline_controls():
    """Nominal natural-spline controls: the analytic separations at the knots."""
    k = np.asarray(KNOTS_Z)
    return separation(k, ZC_12), separation(k, ZC_23)


# ------------------------------------------------------------ initial states

def coherent_state(shape, box, x0=2.0):
    """pi^(-3/4) exp(-((x - x0)^2 + y^2 + z^2)/2): the 3D oscillator ground
    state displaced along x."""
    x, y, z = mesh(shape, box)
    return (np.pi ** -0.75 * np.exp(-((x - x0) ** 2 + y ** 2 + z ** 2) / 2.0)).astype(np.complex128)


def gaussian_sum(shape, box, seed=0, count=4, lo=-4.0, hi=4.0, wmin=0.8, wmax=2.0):
    """Normalised real sum of `count` Gaussians, centres ~ U[lo,hi]^3 and
    widths ~ U[wmin,wmax] drawn from numpy.random.default_rng(seed) in FP64."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(lo, hi, size=(count, 3))
    widths = rng.uniform(wmin, wmax, size=count)
    x, y, z = mesh(shape, box)
    psi = np.zeros(shape, dtype=np.complex128)
    for (cx, cy, cz), w in zip(centres, widths):
        psi += np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2.0 * w * w))
    return normalise(psi, box)


def guide_seed_2d(shape2d, box, xc):
    """exp(-((x - xc)^2 + y^2)/2) on a (1, ny, nx) plane: the starting guess of
    the imaginary-time search for the guide-1 transverse ground state."""
    ny, nx = shape2d
    x = axis(nx, box[0], box[1])[None, None, :]
    y = axis(ny, box[2], box[3])[None, :, None]
    return np.exp(-((x - xc) ** 2 + y ** 2) / 2.0).astype(np.complex128) * np.ones((1, ny, nx))


def packet_from_transverse(phi_xy, nz, box, z0=-40.0, width=4.0, k0=2.0):
    """psi0 = phi(x,y) exp(-(z - z0)^2/(2 width^2)) exp(i k0 z), normalised."""
    z = axis(nz, box[4], box[5])[:, None, None]
    psi = phi_xy.reshape(1, *phi_xy.shape[-2:]) * np.exp(-(z - z0) ** 2 / (2.0 * width ** 2)) \
        * np.exp(1j * k0 * z)
    return normalise(psi.astype(np.complex128), box)


# ------------------------------------------------------------ potentials

def harmonic_parts(shape, box):
    """Separable oscillator V = Vx(x) + Vy(y) + Vz(z), each q^2/2."""
    nz, ny, nx = shape
    return (0.5 * axis(nx, box[0], box[1]) ** 2,
            0.5 * axis(ny, box[2], box[3]) ** 2,
            0.5 * axis(nz, box[4], box[5]) ** 2)


def harmonic_dense(shape, box):
    vx, vy, vz = harmonic_parts(shape, box)
    return vz[:, None, None] + vy[None, :, None] + vx[None, None, :]


# ------------------------------------------------------------ workloads

@dataclass(frozen=True)
class Workload:
    name: str
    shape: tuple           # (nz, ny, nx)
    box: tuple
    dtype: str             # "c64" or "c128"
    dt: float
    steps: int
    potential: str         # "harmonic" or "ctap"
    extra: dict = field(default_factory=dict)

    @property
    def points(self):
        nz, ny, nx = self.shape
        return nz * ny * nx


WORKLOADS = {
    "harmonic_tiny": Workload("harmonic_tiny", (32, 32, 32), HARMONIC_BOX, "c128", 0.01, 100,
                              "harmonic", {"x0": 2.0}),
    "ctap_fp64": Workload("ctap_fp64", (256, 128, 128), CTAP_BOX, "c128", 0.005, 2000, "ctap",
                          {"imag_steps": 200, "imag_dt": 0.01}),
    "ctap_large": Workload("ctap_large", (1024, 256, 256), CTAP_BOX, "c64", 0.0025, 4000, "ctap",
                           {"imag_steps": 200, "imag_dt": 0.01}),
    "ctap_adjoint": Workload("ctap_adjoint", (256, 128, 128), CTAP_BOX, "c64", 0.005, 1000, "ctap",
                             {"checkpoint_every": 32}),
}

SWEEP_SHAPES = [(64, 64, 64), (128, 128, 128), (256, 256, 256), (512, 256, 256),
                (1024, 256, 256), (1024, 64, 256)]
