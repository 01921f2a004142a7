"""Failure reporting and checkpoint/resume through the C ABI.

None of these tests faults, traps or hangs the GPU.  The failures are made on
the host: a deadline shorter than the queued work (ctap_sync returns
CTAP_ERR_TIMEOUT and the plan stays usable), a NaN planted in psi (the FP64
reductions report CTAP_ERR_NONFINITE), and the library's host-side fault
injector (CTAP_FAULT_INJECT=alloc:N / launch:N fails the N-th allocation or
launch before it reaches the GPU), run in a child process because the
injector reads its setting once per process.

Checkpoint/resume: a run stopped after N steps, copied to the host and
restarted from that copy on a fresh plan continues bit for bit as the run
that was never stopped (the kernels are deterministic: fixed-order
reductions, no atomics).  Splitting a run into two calls differs from one
call only by rounding: one call merges the two half-kicks at the seam into
one full kick.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1309_2451_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE = 5, 6, 7, 8


@pytest.fixture(scope="module")
def ctap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2451_b300 import build, ctap as c
    build.build()
    c.lib()
    return c


def guides_plan(ctap, shape, box, dtype):
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z)
    plan = ctap.Plan(shape, box, dtype)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    return plan, c


def packet(shape, seed):
    box = wl.CTAP_BOX
    return wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=seed) \
        * np.exp(2j * wl.mesh(shape, box)[2])


def to_dev(psi, dtype):
    t = torch.complex64 if dtype == "c64" else torch.complex128
    return torch.from_numpy(np.ascontiguousarray(psi)).to(device="cuda", dtype=t)


def test_sync_deadline_reports_timeout_and_plan_stays_usable(ctap):
    """A 1 ms deadline on ~0.2 s of queued steps returns CTAP_ERR_TIMEOUT;
    a later wait with room finishes, and the plan still computes."""
    shape, box = (1024, 256, 256), wl.CTAP_BOX
    plan, _ = guides_plan(ctap, shape, box, "c64")
    psi = to_dev(packet(shape, 3), "c64")
    norm0 = plan.observables(psi)[0]
    plan.step(psi, 1, 0.0025)
    plan.sync(60000)
    plan.step(psi, 200, 0.0025)
    with pytest.raises(ctap.CtapError) as e:
        plan.sync(1)
    assert e.value.code == ERR_TIMEOUT
    plan.sync(60000)
    obs = plan.observables(psi)
    assert np.all(np.isfinite(obs)) and abs(obs[0] - norm0) < 1e-5 * norm0
    plan.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_nonfinite_state_is_reported(ctap, dtype):
    """One NaN in psi makes the FP64 reductions return CTAP_ERR_NONFINITE
    instead of a silent NaN; the plan then works on a finite state."""
    shape, box = (64, 32, 32), wl.CTAP_BOX
    plan, _ = guides_plan(ctap, shape, box, dtype)
    bad = packet(shape, 4)
    bad[17, 5, 9] = np.nan
    with pytest.raises(ctap.CtapError) as e:
        plan.observables(to_dev(bad, dtype))
    assert e.value.code == ERR_NONFINITE
    obs = plan.observables(to_dev(packet(shape, 4), dtype))
    assert np.all(np.isfinite(obs))
    plan.close()


_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1309_2451_b300 import ctap, workloads as wl
shape, box = (64, 32, 32), wl.CTAP_BOX
z = wl.axis(shape[0], box[4], box[5])
c = wl.guide_centres(z)
psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=2)
results = []
for attempt in range(2):
    try:
        plan = ctap.Plan(shape, box, "c128")
        plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
        psi = torch.from_numpy(psi0).to("cuda")
        plan.step(psi, 4, 0.0025)
        obs = plan.observables(psi)
        plan.close()
        results.append({"ok": True, "norm": float(obs[0])})
    except ctap.CtapError as e:
        results.append({"ok": False, "code": e.code, "msg": str(e)})
print(json.dumps(results))
"""


@pytest.mark.parametrize("inject,code,msg", [("alloc:2", ERR_OOM, "out of memory"),
                                             ("launch:3", ERR_CUDA, "CUDA error")])
def test_host_fault_injection(ctap, inject, code, msg):
    """The N-th allocation or launch fails on the host with the right status;
    the next attempt in the same process runs normally."""
    env = dict(os.environ, CTAP_FAULT_INJECT=inject)
    out = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert not res[0]["ok"] and res[0]["code"] == code, res[0]
    assert msg in res[0]["msg"], res[0]     # status name, e.g. "out of memory"
    if "(" in res[0]["msg"]:                # plan-local detail, when a plan existed
        assert "injected" in res[0]["msg"], res[0]
    shape, box = (64, 32, 32), wl.CTAP_BOX
    psi0 = wl.gaussian_sum(shape, (-6, 6, -6, 6, -40, 40), seed=2)
    norm0 = float(np.sum(np.abs(psi0) ** 2) * wl.cell_volume(shape, box))
    assert res[1]["ok"] and abs(res[1]["norm"] - norm0) < 1e-10 * norm0, (res[1], norm0)


@pytest.mark.parametrize("dtype,shape,tol", [("c128", (64, 32, 32), 1e-12),
                                             ("c64", (64, 256, 256), 1e-5)])
def test_checkpoint_resume_is_bitwise(ctap, dtype, shape, tol):
    """Stop after N steps, keep a host copy, resume on a fresh plan: the
    result equals the uninterrupted two-call run bit for bit, and the
    one-call run of 2N steps to rounding; both match the oracle."""
    box, n, dt = wl.CTAP_BOX, 6, 0.0025
    psi0 = packet(shape, 7)
    plan, c = guides_plan(ctap, shape, box, dtype)
    psi = to_dev(psi0, dtype)
    plan.step(psi, n, dt)
    checkpoint = psi.cpu().numpy().copy()
    plan.step(psi, n, dt)
    straight = psi.cpu().numpy()

    fresh, _ = guides_plan(ctap, shape, box, dtype)
    psi = to_dev(checkpoint, dtype)
    fresh.step(psi, n, dt)
    resumed = psi.cpu().numpy()
    assert np.array_equal(resumed, straight)

    psi = to_dev(psi0, dtype)
    fresh.step(psi, 2 * n, dt)
    one_call = psi.cpu().numpy().astype(complex)
    V = oracle.ctap_potential(shape, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    ref = oracle.step(psi0, V, box, dt, 2 * n)
    for got in (straight.astype(complex), one_call):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    plan.close()
    fresh.close()
