"""The bounds-checked build (libctap_debug.so, -DCTAP_DEBUG_BOUNDS): every
shared-memory and HBM index of the packed persistent passes is checked
before the access, a violation is recorded and the access skipped (nothing
traps).  Steps through both packed passes (guide potential; the XY pass
also with the separable oscillator) run in a child process on the checked
library: no violation may be recorded, and the result must equal
the normal library's (the checks change no arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1309_2451_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1309_2451_b300 import ctap, workloads as wl
out = {}
cases = [(s, "guides") for s in ((64, 256, 256), (1024, 256, 64), (1024, 256, 256))]
for shape, pot in cases + [((64, 256, 256), "harmonic")]:
    plan = ctap.Plan(shape, wl.CTAP_BOX if pot == "guides" else wl.HARMONIC_BOX, "c64")
    if pot == "guides":
        box = wl.CTAP_BOX
        c = wl.guide_centres(wl.axis(shape[0], box[4], box[5]))
        plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    else:
        box = wl.HARMONIC_BOX
        plan.set_potential_separable(*wl.harmonic_parts(shape, box))
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -6, 6), seed=31) \
        * np.exp(2j * wl.mesh(shape, box)[2])
    psi = torch.from_numpy(psi0).to("cuda", torch.complex64)
    plan.step(psi, 4, 0.0025)
    plan.sync()
    out[str(shape) + pot] = {"mask": plan.info()["fast_mask"], "bounds": ctap.debug_bounds(),
                       "sum": psi.abs().double().sum().item(),
                       "l2": torch.linalg.vector_norm(psi.to(torch.complex128)).item(),
                       "first": [psi.flatten()[1234567 % psi.numel()].real.item()]}
    plan.close()
print(json.dumps(out))
"""


def run_child(lib):
    env = dict(os.environ, CTAP_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_records_no_violation_and_matches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2451_b300 import build
    build.build(debug=True)
    checked = run_child("debug")
    normal = run_child("normal")
    for key, rec in checked.items():
        assert rec["mask"] & 48, (key, rec)             # a packed pass ran
        assert rec["bounds"] == 0, (key, hex(rec["bounds"]))
        assert normal[key]["bounds"] == -1               # the normal build has no checks
        assert rec["sum"] == normal[key]["sum"] and rec["l2"] == normal[key]["l2"], (key, rec, normal[key])
