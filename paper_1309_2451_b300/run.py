"""Propagate a three-guide workload and print its observables.

    python -m paper_1309_2451_b300.run --grid 256 256 1024 --dtype c64 \
        --steps 200 --every 50 --dt 0.0025 [--imag-prep 200]

Grid sizes are given as nx ny nz.  The initial state is the guide-1 seed
(optionally refined by --imag-prep imaginary-time steps on an nz = 1 plane,
the transverse ground state of Sec. V) times a z-packet at z = -40 with
momentum --k0 (default 2).  --order intuitive exchanges the two separation
profiles (Fig. 4b); --trap adds the longitudinal harmonic trap of Sec. III,
which carries a packet released at rest at z = -40 through both coupling
regions to z = +40 in half a trap period (the full transfer of Fig. 4:
--k0 0 --trap --steps 15708 --dt 0.0025).  Every --every steps the FP64
observables (norm, <T>, <V>, guide populations) are printed as one JSON
line.
"""
import argparse
import json
import time

import numpy as np


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--grid", type=int, nargs=3, default=[128, 128, 256])
    p.add_argument("--dtype", choices=["c64", "c128", "c128df"], default="c64")
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--every", type=int, default=50)
    p.add_argument("--dt", type=float, default=0.005)
    p.add_argument("--imag-prep", type=int, default=0)
    p.add_argument("--order", choices=["counter", "intuitive"], default="counter")
    p.add_argument("--trap", action="store_true",
                   help="add the longitudinal trap omega^2 z^2/2 (Sec. III)")
    p.add_argument("--k0", type=float, default=2.0, help="initial z-momentum of the packet")
    a = p.parse_args(argv)

    import torch

    from . import build, ctap, workloads as wl
    build.build()
    nx, ny, nz = a.grid
    box = wl.CTAP_BOX
    z = wl.axis(nz, box[4], box[5])
    c = wl.guide_centres(z, a.order)
    xc = float(wl.guide_centres(np.array([-40.0]), a.order)[0, 0])
    phi = wl.guide_seed_2d((ny, nx), box, xc)
    tdt = torch.complex64 if a.dtype == "c64" else torch.complex128
    if a.imag_prep > 0:
        prep = ctap.Plan((1, ny, nx), box, a.dtype)
        y = wl.axis(ny, box[2], box[3])
        x = wl.axis(nx, box[0], box[1])
        prep.set_potential_product(np.exp(-y ** 2 / 2.0),
                                   -wl.V0 * np.exp(-(x - xc) ** 2 / 2.0)[None, :])
        t = torch.from_numpy(phi).to("cuda", tdt)
        prep.step(t, a.imag_prep, 0.01, imag=True)
        phi = t.cpu().numpy().astype(np.complex128)
        prep.close()
    psi = torch.from_numpy(wl.packet_from_transverse(phi, nz, box, k0=a.k0)).to("cuda", tdt)
    plan = ctap.Plan((nz, ny, nx), box, a.dtype)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    if a.trap:
        plan.add_potential_z(wl.trap_z(z))
    done = 0
    t0 = time.perf_counter()
    while done < a.steps:
        n = min(a.every, a.steps - done)
        plan.step(psi, n, a.dt)
        done += n
        obs = plan.observables(psi)
        print(json.dumps({"step": done, "t": done * a.dt, "norm": obs[0], "T": obs[1],
                          "V": obs[2], "P": list(obs[3:]),
                          "wall_s": time.perf_counter() - t0}), flush=True)
    plan.close()


if __name__ == "__main__":
    main()
