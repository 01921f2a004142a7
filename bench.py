#!/usr/bin/env python
"""Benchmark: 3D split-step steps/s and HBM roofline at 256x256x1024.

One bench step = one observation interval of the propagation: SPLIT Strang
steps of the three-guide workload (ctap_step) followed by the FP64
observables (norm, energies, guide populations; ctap_observables), the
paper's per-interval record (Sec. V, Fig. 4).  `value` counts split steps per
second, whole job.  The FP32 path (complex64 with FP64 tables and
reductions) is the headline; the FP64 path (complex128) is timed on the same
workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun): the
propagation does not shard without all-to-all transposes, so the multi-GPU
mode is a replica sweep, as in the paper's concurrent runs on a second card.
--impl reference times the FP64 CPU oracle (the test reference) on the
host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "3D split-step steps/s and HBM roofline % at 256x256x1024, FP32 vs FP64 path"
SHAPE = (1024, 256, 256)
DT = 0.0025
SPLIT = 50                 # split steps per bench step (one observation interval)
SPLIT_FP64 = 4
FP64_NOMINAL_TFLOPS = 1.25  # nominal B300 FP64 rate (used only if the probe fails)
ACC_STEPS = 500            # split steps of the complex64-vs-complex128 accuracy run
# size x precision sweep: (nz, ny, nx); the paper's 256x64x1024 grid last
SWEEP_SHAPES = [(64, 64, 64), (128, 128, 128), (256, 256, 256), (512, 256, 256),
                (1024, 256, 256), (1024, 64, 256)]
SWEEP_STEPS = 500          # split steps of each complex64-vs-complex128 comparison
SWEEP_DT = 0.005
L2_BYTES = 126 * 2 ** 20


def pass_flops_per_point(shape, P):
    """Algorithmic flops per point of one steady pass: 5 n log2 n per complex
    FFT of length n (radix-2 count; forward and inverse), 6 per complex
    product (the potential or kinetic factor).  XY: x over nx, partial y over
    ny/P; Z: cross over P, z over nz."""
    import math
    nz, ny, nx = shape
    xy = 2 * 5 * (math.log2(nx) + math.log2(ny // P)) + 6
    z = 2 * 5 * (math.log2(P) + math.log2(nz)) + 6
    return xy, z
KERNEL_SOURCES = ["device_fft.cuh", "kernels.cuh", "kernels.cu", "fast_passes.cu",
                  "packed_passes.cu"]


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--no-sweep", action="store_true")
    return p.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(ms, e2e_value, steps, world, reduce):
    """Whole-job numbers of a replica run: the step time is the slowest
    rank's, `value` counts the split steps of all ranks, the e2e rate is the
    slowest rank's times the number of ranks.  reduce(x, "max"|"min") combines
    a float over ranks (identity for one rank)."""
    ms_max = reduce(ms, "max")
    e2e_total = reduce(e2e_value, "min") * world
    value = steps * SPLIT * world / (ms_max / 1000.0)
    return ms_max, value, e2e_total


def make_reduce(dist, torch, device):
    def reduce(x, op):
        if dist is None:
            return float(x)
        t = torch.tensor([float(x)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.MIN)
        return float(t.item())
    return reduce


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1309_2451_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_hash") != kernel_hash():
            return None
        return d.get(kind)
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the
    timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def build_plan(ctap, wl, dtype, stream):
    box = wl.CTAP_BOX
    z = wl.axis(SHAPE[0], box[4], box[5])
    c = wl.guide_centres(z)
    plan = ctap.Plan(SHAPE, box, dtype, stream=stream)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    return plan


def initial_state(wl, dtype_t, torch, device):
    """Guide-1 transverse ground state (imaginary time on the nz = 1 plane is
    skipped here: the bench times propagation) approximated by the seed
    Gaussian, times the z-packet; seeded and synthetic."""
    box = wl.CTAP_BOX
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    phi = wl.guide_seed_2d(SHAPE[1:], box, xc)
    psi = wl.packet_from_transverse(phi, SHAPE[0], box)
    return torch.from_numpy(psi).to(device=device, dtype=dtype_t)


def time_path(ctap, wl, torch, dtype, split, steps, warmup, device, stream, profile=True,
              barrier=None):
    """W untimed warm-up bench steps, then exactly K timed ones, bracketed by
    barrier() (all ranks) and a device synchronisation on both sides."""
    plan = build_plan(ctap, wl, dtype, stream)
    t = torch.complex64 if dtype == "c64" else torch.complex128
    psi = initial_state(wl, t, torch, device)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.step(psi, split, DT)
            plan.observables(psi)
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    plan.set_profiling(profile)
    plan.pass_times()
    launches0 = plan.launch_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    obs = None
    with Clocks(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            plan.step(psi, split, DT)
            obs = plan.observables(psi)
        e1.record(stream)
        torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    ms = e0.elapsed_time(e1)
    launches = plan.launch_count - launches0
    counts, pms = plan.pass_times()
    plan.set_profiling(False)
    return dict(plan=plan, psi=psi, ms=ms, launches=launches, counts=counts, pass_ms=pms,
                obs=obs, clocks=clk.summary())


def time_e2e(ctap, wl, torch, steps, device, stream, plan):
    """Same metric through the public API with host buffers: every bench
    step copies psi from pinned host memory, propagates, and reads the
    observables back.  The copy of step n+1 runs on a second stream into a
    second device buffer while step n computes (double buffering), so the
    link and the passes overlap as they would in a production loop."""
    host = initial_state(wl, torch.complex64, torch, "cpu").pin_memory()
    bufs = [torch.empty(SHAPE, dtype=torch.complex64, device=device) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=device)
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    for b in bufs:                                  # warm-up (graphs for both buffers)
        with torch.cuda.stream(stream):
            b.copy_(host, non_blocking=True)
            plan.step(b, SPLIT, DT)
            plan.step(b, SPLIT, DT)
            plan.observables(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(copy_stream):
        bufs[0].copy_(host, non_blocking=True)
        copied[0].record(copy_stream)
    for i in range(steps):
        cur, nxt = i % 2, (i + 1) % 2
        if i + 1 < steps:
            with torch.cuda.stream(copy_stream):
                if i >= 1:
                    copy_stream.wait_event(done[nxt])
                bufs[nxt].copy_(host, non_blocking=True)
                copied[nxt].record(copy_stream)
        with torch.cuda.stream(stream):
            stream.wait_event(copied[cur])
            plan.step(bufs[cur], SPLIT, DT)
            plan.observables(bufs[cur])     # synchronising D2H of 6 doubles
            done[cur].record(stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(value=steps * SPLIT / dt, unit="steps/s",
                h2d_bytes_per_step=int(host.numel() * host.element_size()),
                d2h_bytes_per_step=6 * 8,
                overlap="H2D copy of step n+1 on a second stream during step n")


def time_variants(torch, wl, device, stream, plan, psi, reps=4):
    """The paper-faithful variants on the bench workload, CUDA events on the
    plan stream: the K/2 V K/2 ordering, the guides plus the longitudinal
    trap term, and the y-integrated density of Fig. 5."""
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        with torch.cuda.stream(stream):
            fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: plan.step(psi, SPLIT, DT, order="KVK"))
    out["kvk_order"] = {"steps_per_s": SPLIT * 1000.0 / ms, "ms_per_step": ms / SPLIT}
    z = wl.axis(SHAPE[0], wl.CTAP_BOX[4], wl.CTAP_BOX[5])
    plan.add_potential_z(wl.trap_z(z))
    ms = timed(lambda: plan.step(psi, SPLIT, DT))
    out["guides_plus_trap"] = {"steps_per_s": SPLIT * 1000.0 / ms, "ms_per_step": ms / SPLIT}
    c = wl.guide_centres(z)
    plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)   # back to the bench V
    t0 = time.perf_counter()
    for _ in range(reps):
        plan.density_xz(psi)
    out["density_xz"] = {"ms_per_call_with_copy": 1000.0 * (time.perf_counter() - t0) / reps,
                         "bytes_read": int(np.prod(SHAPE)) * 8}
    # atom-chip potential from 3 x 64 wire segments on the full grid (device
    # FP64 Biot-Savart sum, then stored as the dense form)
    from paper_1309_2451_b300 import ctap
    chip = ctap.Plan(SHAPE, (-10.0, 10.0, 0.5, 4.5, 0.0, 1000.0), "c64", stream=stream)
    seg = wl.chip_wires(64)
    t0 = time.perf_counter()
    chip.set_potential_wires(seg, wl.chip_bias(), wl.CHIP["mu0_over_4pi"], 0.5, 0.5 * wl.CHIP["B_ip"])
    out["wire_potential_build"] = {"s": time.perf_counter() - t0, "segments": int(seg.shape[0]),
                                   "points": int(np.prod(SHAPE))}
    chip.close()
    return out


def time_batched(torch, wl, device, stream, B=16, shape=(128, 64, 64), steps=200):
    """The parameter sweep of Fig. 6 as batched replicas: B middle-guide
    depths on a small grid advanced by one batched plan, against the same B
    runs one plan at a time (replica-steps per second)."""
    box = wl.CTAP_BOX
    z = wl.axis(shape[0], box[4], box[5])
    c = wl.guide_centres(z)
    mids = np.linspace(0.8, 1.2, B)
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    one = wl.packet_from_transverse(wl.guide_seed_2d(shape[1:], box, xc), shape[0], box)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bp = ctap_mod().Plan(shape, box, "c64", stream=stream, batch=B)
    bp.set_guides_batched(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], mids, wl.POP_HALFWIDTH)
    psi = torch.from_numpy(np.stack([one] * B)).to(device, torch.complex64)
    with torch.cuda.stream(stream):
        bp.step(psi, steps, DT)
        bp.step(psi, steps, DT)
        e0.record(stream)
        bp.step(psi, steps, DT)
        e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    plans, psis = [], []
    for m in mids:
        p1 = ctap_mod().Plan(shape, box, "c64", stream=stream, batch=1)
        p1.set_guides_batched(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], [m], wl.POP_HALFWIDTH)
        plans.append(p1)
        psis.append(torch.from_numpy(one).to(device, torch.complex64))
    with torch.cuda.stream(stream):
        for p1, q in zip(plans, psis):
            p1.step(q, steps, DT)
            p1.step(q, steps, DT)
        e0.record(stream)
        for p1, q in zip(plans, psis):
            p1.step(q, steps, DT)
        e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    return {"grid": list(shape[::-1]), "replicas": B, "steps": steps,
            "batched_replica_steps_per_s": B * steps * 1000.0 / ms_b,
            "sequential_replica_steps_per_s": B * steps * 1000.0 / ms_s,
            "speedup": ms_s / ms_b}


def ctap_mod():
    from paper_1309_2451_b300 import ctap
    return ctap


def time_cufft(torch, device, stream, plan, steps=20):
    """Comparison step in the paper's own design (Sec. IV): a library 3D FFT
    (torch.fft, i.e. cuFFT) and separate elementwise phase multiplies, on the
    same complex64 workload, half-kicks merged as in the fused path.  Not the
    product path: it only puts the fused two-pass step in context."""
    nz, ny, nx = SHAPE
    N = nz * ny * nx
    box = plan.box
    V = torch.from_numpy(plan.get_potential()).to(device)
    k = [2.0 * np.pi * np.fft.fftfreq(n, d=(box[2 * a + 1] - box[2 * a]) / n)
         for a, n in ((2, nz), (1, ny), (0, nx))]
    kz, ky, kx = (torch.from_numpy(v).to(device) for v in k)
    k2h = 0.5 * (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    PK = (torch.exp(-1j * k2h * DT) / N).to(torch.complex64)
    PV = torch.exp(-1j * V * DT).to(torch.complex64)
    del V, k2h
    dims = (0, 1, 2)

    def one(psi):
        psi = torch.fft.fftn(psi, dim=dims, norm="backward")
        psi.mul_(PK)
        psi = torch.fft.ifftn(psi, dim=dims, norm="forward")
        return psi.mul_(PV)

    with torch.cuda.stream(stream):
        psi = torch.randn(SHAPE, dtype=torch.complex64, device=device)
        for _ in range(3):
            psi = one(psi)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            psi = one(psi)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del PK, PV, psi
    torch.cuda.empty_cache()
    return {"steps_per_s": 1000.0 / ms, "ms_per_step": ms, "steps": steps,
            "design": "torch.fft (cuFFT) 3D C2C forward + inverse and two elementwise "
                      "phase multiplies per step, complex64, merged half-kicks"}


def time_rows(ctap, wl, torch, device, stream):
    """The hot-path rows outside the headline loop, each timed once with CUDA
    events: imaginary-time preparation of the guide-1 transverse state
    (256x256 plane, 200 steps) and the adjoint gradient of the final guide-3
    population w.r.t. 32 spline controls (128x128x256 complex64, 1000 steps,
    checkpoints every 32)."""
    out = {}
    box = wl.CTAP_BOX
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # a5: imaginary time on the nz = 1 plane
    prep = ctap.Plan((1, 256, 256), box, "c64", stream=stream)
    y = wl.axis(256, box[2], box[3])
    x = wl.axis(256, box[0], box[1])
    prep.set_potential_product(np.exp(-y ** 2 / 2.0), -wl.V0 * np.exp(-(x - xc) ** 2 / 2.0)[None, :])
    phi = torch.from_numpy(wl.guide_seed_2d((256, 256), box, xc)).to(device, torch.complex64)
    with torch.cuda.stream(stream):
        prep.step(phi.clone(), 10, 0.01, imag=True)
        torch.cuda.synchronize()
        e0.record(stream)
        prep.step(phi, 200, 0.01, imag=True)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["imag_prep_256x256"] = {"steps": 200, "ms": ms, "steps_per_s": 200 / (ms * 1e-3)}
    # a7: adjoint gradient on the adjoint workload
    shape = (256, 128, 128)
    plan = ctap.Plan(shape, box, "c64", stream=stream)
    c12, c23 = wl.spline_controls()
    plan.set_guides_spline(wl.V0, wl.SIGMA_GUIDE, wl.KNOTS_Z, c12, c23, wl.POP_HALFWIDTH)
    phi128 = wl.guide_seed_2d((128, 128), box, xc)
    psi0 = torch.from_numpy(wl.packet_from_transverse(phi128, shape[0], box)).to(device, torch.complex64)
    with torch.cuda.stream(stream):
        plan.adjoint(psi0, 64, 0.005, K=32, guide=3)           # warm-up
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        J, grad = plan.adjoint(psi0, 1000, 0.005, K=32, guide=3)
    el = time.perf_counter() - t0
    out["adjoint_128x128x256"] = {"steps": 1000, "checkpoint_every": 32, "s": el,
                                  "forward_equiv_steps_per_s": 1000 / el, "J": J,
                                  "grad_norm": float(np.linalg.norm(grad))}
    prep.close()
    plan.close()
    return out


def rel_l2(torch, a, b):
    """||a - b|| / ||b|| on the device, in FP64."""
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def norm_dv(torch, psi, dV):
    return float(torch.sum(psi.to(torch.complex128).abs() ** 2)) * dV


def accuracy_c64_vs_c128(ctap, wl, torch, device, stream, steps=ACC_STEPS):
    """The accuracy the complex64 speed is quoted at: complex64 and
    complex128 runs of the bench workload from the same psi0 for the same
    number of split steps; relative L2 of the complex64 state against the
    complex128 one and the norm drift of each."""
    out = {"steps": steps, "dt": DT}
    states = {}
    for dtype, t in (("c64", torch.complex64), ("c128", torch.complex128)):
        plan = build_plan(ctap, wl, dtype, stream)
        psi = initial_state(wl, t, torch, device)
        n0 = plan.observables(psi)[0]
        with torch.cuda.stream(stream):
            plan.step(psi, steps, DT)
        obs = plan.observables(psi)
        out[f"norm_drift_{dtype}"] = float(obs[0] / n0 - 1.0)
        out[f"populations_{dtype}"] = [float(x) for x in obs[3:]]
        states[dtype] = psi
        plan.close()
    out["rel_l2_c64_vs_c128"] = rel_l2(torch, states["c64"], states["c128"])
    del states
    torch.cuda.empty_cache()
    return out


def sweep_case(wl, shape, potential):
    """Box, potential setter and psi0 of one sweep point: the harmonic
    oscillator on [-8,8]^3 or the three guides on the guide box; psi0 a
    normalised sum of 4 Gaussians, centres U[-4,4]^3, widths U[0.8,2],
    numpy.random.default_rng(0)."""
    if potential == "harmonic":
        box = wl.HARMONIC_BOX

        def setup(plan):
            plan.set_potential_separable(*wl.harmonic_parts(shape, box))
    else:
        box = wl.CTAP_BOX
        c = wl.guide_centres(wl.axis(shape[0], box[4], box[5]))

        def setup(plan):
            plan.set_guides(wl.V0, wl.SIGMA_GUIDE, c[0], c[2], wl.POP_HALFWIDTH)
    return box, setup, wl.gaussian_sum(shape, box, seed=0)


def time_sweep(ctap, wl, torch, device, stream, hbm, steps=SWEEP_STEPS):
    """Size x precision sweep (harmonic and guide potentials, complex64 and
    complex128): split steps per second (CUDA events, graph replay), design
    HBM bytes per second (32 B per point and step for complex64, 64 B for
    complex128) and its fraction of the measured copy bandwidth where psi
    does not fit in L2, and the relative L2 of complex64 against complex128
    after `steps` steps from the same psi0."""
    rows = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for shape in SWEEP_SHAPES:
        npts = int(np.prod(shape))
        for potential in ("ctap", "harmonic"):
            box, setup, psi0 = sweep_case(wl, shape, potential)
            row = {"grid": list(shape[::-1]), "potential": potential, "steps": steps,
                   "dt": SWEEP_DT}
            finals = {}
            for dtype, t, esize in (("c64", torch.complex64, 8), ("c128", torch.complex128, 16)):
                plan = ctap.Plan(shape, box, dtype, stream=stream)
                setup(plan)
                psi = torch.from_numpy(psi0).to(device, t)
                n0 = plan.observables(psi)[0]
                with torch.cuda.stream(stream):
                    plan.step(psi, steps, SWEEP_DT)     # the accuracy run
                n1 = plan.observables(psi)[0]           # synchronises the plan stream
                finals[dtype] = psi.clone()
                nt = 100 if dtype == "c64" else 20
                with torch.cuda.stream(stream):
                    plan.step(psi, nt, SWEEP_DT)
                    plan.step(psi, nt, SWEEP_DT)        # graph captured here
                    e0.record(stream)
                    plan.step(psi, nt, SWEEP_DT)
                    e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / nt
                gbps = 4 * npts * esize / (ms * 1e-3) / 1e9
                row[dtype] = {"steps_per_s": 1000.0 / ms, "ms_per_step": ms,
                              "point_updates_per_s": npts * 1000.0 / ms, "design_GBps": gbps,
                              "hbm_frac": gbps / hbm if npts * esize > L2_BYTES else None,
                              "norm_drift": float(n1 / n0 - 1.0),
                              "fast_mask": plan.info()["fast_mask"]}
                plan.close()
                del psi
            row["rel_l2_c64_vs_c128"] = rel_l2(torch, finals["c64"], finals["c128"])
            row["fp32_speedup"] = row["c64"]["steps_per_s"] / row["c128"]["steps_per_s"]
            rows.append(row)
            del finals
            torch.cuda.empty_cache()
    return rows



def cpu_baseline_leg(ctap, wl, torch, device, stream, seconds_cap=30.0, sweep=True):
    """The FP64 oracle, as it stands, on the host cores.  Timed: split steps
    of the full 256x256x1024 workload, as many as fit in about
    `seconds_cap`; the oracle's seconds per step at every sweep point (its 3
    parity steps; 100 more at the grids of at most 128^3), and on one thread
    at 128^3.  The oracle's own results then anchor the GPU paths: the
    relative L2 of the complex64 and complex128 states after the same steps
    from the same psi0, and after 3 steps at every sweep point."""
    import oracle
    box = wl.CTAP_BOX
    z = wl.axis(SHAPE[0], box[4], box[5])
    c = wl.guide_centres(z)
    V = oracle.ctap_potential(SHAPE, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    psi0 = wl.packet_from_transverse(wl.guide_seed_2d(SHAPE[1:], box, xc), SHAPE[0], box)
    psi = psi0
    n, t_total = 0, 0.0
    while t_total < seconds_cap and n < 10:
        t0 = time.perf_counter()
        psi = oracle.step(psi, V, box, DT, 1)
        t_total += time.perf_counter() - t0
        n += 1
        if n == 1 and t_total > seconds_cap / 2:
            break
    base = {"value": n / t_total, "unit": "steps/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} FP64 split step(s) of the 256x256x1024 three-guide workload "
                      f"({t_total:.1f} s, OpenMP over lines)"}
    ref = torch.from_numpy(psi).to(device)
    del psi, V
    parity = {"steps": n, "workload": "ctap_large, the bench psi0"}
    for dtype, t in (("c64", torch.complex64), ("c128", torch.complex128)):
        plan = build_plan(ctap, wl, dtype, stream)
        g = torch.from_numpy(psi0).to(device, t)
        with torch.cuda.stream(stream):
            plan.step(g, n, DT)
        torch.cuda.synchronize()
        parity[dtype] = rel_l2(torch, g, ref)
        plan.close()
        del g
    del ref
    torch.cuda.empty_cache()
    sweep_parity = []
    if sweep:
        for shape in SWEEP_SHAPES:
            for potential in ("ctap", "harmonic"):
                sbox, setup, p0 = sweep_case(wl, shape, potential)
                if potential == "harmonic":
                    Vs = wl.harmonic_dense(shape, sbox)
                else:
                    cz = wl.guide_centres(wl.axis(shape[0], sbox[4], sbox[5]))
                    Vs = oracle.ctap_potential(shape, sbox, wl.V0, wl.SIGMA_GUIDE, cz[0], cz[2])
                t0 = time.perf_counter()
                r = torch.from_numpy(oracle.step(p0, Vs, sbox, SWEEP_DT, 3)).to(device)
                row = {"grid": list(shape[::-1]), "potential": potential, "steps": 3,
                       "oracle_s_per_step": (time.perf_counter() - t0) / 3,
                       "oracle_threads": oracle.num_threads()}
                if np.prod(shape) <= 128 ** 3:
                    t0 = time.perf_counter()
                    oracle.step(p0, Vs, sbox, SWEEP_DT, 100)
                    row["oracle_s_per_step_100"] = (time.perf_counter() - t0) / 100
                if np.prod(shape) == 128 ** 3 and potential == "ctap":
                    cores = oracle.num_threads()
                    oracle.set_num_threads(1)
                    t0 = time.perf_counter()
                    oracle.step(p0, Vs, sbox, SWEEP_DT, 3)
                    row["oracle_s_per_step_1_thread"] = (time.perf_counter() - t0) / 3
                    oracle.set_num_threads(cores)
                del Vs
                for dtype, t in (("c64", torch.complex64), ("c128", torch.complex128)):
                    plan = ctap.Plan(shape, sbox, dtype, stream=stream)
                    setup(plan)
                    g = torch.from_numpy(p0).to(device, t)
                    with torch.cuda.stream(stream):
                        plan.step(g, 3, SWEEP_DT)
                    torch.cuda.synchronize()
                    row[dtype] = rel_l2(torch, g, r)
                    plan.close()
                    del g
                sweep_parity.append(row)
                del r
                torch.cuda.empty_cache()
    return base, parity, sweep_parity


def run_reference(a):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    from paper_1309_2451_b300 import workloads as wl
    box = wl.CTAP_BOX
    z = wl.axis(SHAPE[0], box[4], box[5])
    c = wl.guide_centres(z)
    V = oracle.ctap_potential(SHAPE, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    psi = wl.packet_from_transverse(wl.guide_seed_2d(SHAPE[1:], box, xc), SHAPE[0], box)
    # each bench step is a bounded sample of the workload: one FP64 split step
    for _ in range(a.warmup):
        psi = oracle.step(psi, V, box, DT, 1)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        psi = oracle.step(psi, V, box, DT, 1)
    el = time.perf_counter() - t0
    v = a.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1000.0 * el / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ctap_large: 256x256x1024 three-guide split step",
                       "grid": list(SHAPE[::-1]), "dt": DT,
                       "bench_step": "one FP64 split step (the oracle, bounded sample)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{a.steps} FP64 split steps of the full workload"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dominant_pass(plan, counts, pms):
    """(kind, kernel name, average ms) of the pass with the larger share."""
    kind = 0 if pms[0] >= pms[1] else 1
    fast = plan.info()["fast_mask"]
    if kind == 0:
        name = ("xy_pk_kernel" if fast & 32 else "xy_ring_kernel" if fast & 8 else
                "xy_fast_kernel" if fast & 1 else "xy_pass_kernel")
    else:
        name = ("z_pk_kernel" if fast & 16 else "z_ring_kernel" if fast & 4 else
                "z_fast_kernel" if fast & 2 else "z_pass_kernel")
    return kind, name, pms[kind] / max(counts[kind], 1)


def run_ours(a):
    import torch
    from paper_1309_2451_b300 import build, ctap, workloads as wl
    rank, world, local = dist_info()
    build.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.Stream(device=device)
    reduce = make_reduce(dist, torch, device)
    barrier = dist.barrier if dist is not None else None

    # the headline: profiling off, so repeated ctap_step calls replay a graph
    res = time_path(ctap, wl, torch, "c64", SPLIT, a.steps, a.warmup, device, stream,
                    profile=False, barrier=barrier)
    # the per-pass breakdown of the same loop: per-launch CUDA events recorded
    # by the library on its stream (graph replay off while they are on)
    prof = time_path(ctap, wl, torch, "c64", SPLIT, min(a.steps, 5), 1, device, stream,
                     profile=True, barrier=barrier)

    N = int(np.prod(SHAPE))
    esize = 8
    hbm, peak_kind = peaks()
    counts, pms = prof["counts"], prof["pass_ms"]
    kind, name, avg_ms = dominant_pass(prof["plan"], counts, pms)
    bytes_launch = 2 * N * esize       # one read and one write of psi
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": recorded_traffic(name),
                "kernel": name, "peak_kind": peak_kind,
                "step_design_GBps": 4 * N * esize * a.steps * SPLIT / (res["ms"] * 1e-3) / 1e9}
    passes = {"xy_ms_per_launch": pms[0] / max(counts[0], 1),
              "z_ms_per_launch": pms[1] / max(counts[1], 1),
              "launches": list(counts), "ms_total": [float(x) for x in pms],
              "timed_bench_steps": min(a.steps, 5),
              "note": "separate profiled run of the same loop (graph replay off)"}
    prof["plan"].close()
    del prof

    extra = {}
    if rank == 0:
        try:
            extra["fma_peaks"] = dict(ctap.measure_fma_peaks(stream), unit="TFLOP/s",
                                      how="CUDA events, FMA-bound probe kernels (ctap_measure_fma_peaks)")
        except Exception as e:   # the probe is reported, never fatal
            extra["fma_peaks"] = {"error": str(e)}
    fp64_peak = extra.get("fma_peaks", {}).get("fp64_tflops")
    if rank == 0 and not a.no_fp64:
        n64 = max(2, a.steps // 10)
        r64 = time_path(ctap, wl, torch, "c128", SPLIT_FP64, n64, 1, device, stream,
                        profile=False)
        ms64 = r64["ms"] / (n64 * SPLIT_FP64)
        r64["plan"].close()
        p64 = time_path(ctap, wl, torch, "c128", SPLIT_FP64, 2, 1, device, stream, profile=True)
        k64, name64, avg64 = dominant_pass(p64["plan"], p64["counts"], p64["pass_ms"])
        ach64 = 2 * N * 16 / (avg64 * 1e-3) / 1e9
        P64 = p64["plan"].info()["row_classes"]
        fxy, fz = pass_flops_per_point(SHAPE, P64)
        tflops = (fxy if k64 == 0 else fz) * N / (avg64 * 1e-3) / 1e12
        peak64 = fp64_peak if fp64_peak else FP64_NOMINAL_TFLOPS
        extra["fp64_path"] = {
            "steps_per_s": 1000.0 / ms64, "ms_per_step": ms64,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak64,
                         "unit": "TFLOP/s", "frac": tflops / peak64,
                         "peak_kind": "measured FP64 FMA rate (ctap_measure_fma_peaks)"
                                      if fp64_peak else "nominal FP64 (profiling recipe)",
                         "kernel": name64.replace("_kernel", "_kernel<double>"),
                         "flops_per_point": fxy if k64 == 0 else fz,
                         "flop_count": "radix-2 5 n log2 n per transform + 6 per factor"},
            "hbm_frac_of_dominant_kernel": ach64 / hbm,
            "fp32_speedup": (1000.0 / (res["ms"] / (a.steps * SPLIT))) / (1000.0 / ms64),
            "dtype": "f64", "obs": [float(x) for x in p64["obs"]]}
        p64["plan"].close()
        del r64, p64
        extra["fp64_path"]["fp32_speedup_accuracy"] = accuracy_c64_vs_c128(ctap, wl, torch, device,
                                                                            stream)
        rdf = time_path(ctap, wl, torch, "c128df", SPLIT_FP64, max(2, a.steps // 10), 1, device,
                        stream, profile=False)
        msdf = rdf["ms"] / (max(2, a.steps // 10) * SPLIT_FP64)
        extra["fp64_df_path"] = {
            "steps_per_s": 1000.0 / msdf, "ms_per_step": msdf,
            "arithmetic": "double-float (FP32 pairs, ~48-bit significands) on complex128 psi",
            "speedup_over_fp64": ms64 / msdf,
            "obs": [float(x) for x in rdf["obs"]]}
        rdf["plan"].close()
        del rdf
    if rank == 0 and not a.no_extras:
        extra["rows"] = time_rows(ctap, wl, torch, device, stream)
        extra["variants"] = time_variants(torch, wl, device, stream, res["plan"], res["psi"])
        extra["variants"]["batched_sweep"] = time_batched(torch, wl, device, stream)
        extra["cufft_comparison"] = time_cufft(torch, device, stream, res["plan"])
    if rank == 0 and not a.no_sweep:
        extra["sweep"] = time_sweep(ctap, wl, torch, device, stream, hbm)
    if rank == 0 and not a.no_extras:
        base, parity, sweep_parity = cpu_baseline_leg(ctap, wl, torch, device, stream,
                                                      sweep=not a.no_sweep)
        extra["cpu_baseline"] = base
        extra["rel_l2_vs_oracle"] = parity
        if sweep_parity:
            extra["sweep_rel_l2_vs_oracle"] = sweep_parity
    e2e = time_e2e(ctap, wl, torch, max(3, a.steps // 4), device, stream, res["plan"])
    ms, value, e2e["value"] = combine_ranks(res["ms"], e2e["value"], a.steps, world, reduce)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "ctap_large: 256x256x1024 three-guide Strang split step, "
                                       "complex64 bulk, FP64 tables and reductions",
                           "grid": list(SHAPE[::-1]), "dt": DT,
                           "split_steps_per_bench_step": SPLIT,
                           "bench_step": f"{SPLIT} split steps + FP64 observables",
                           "l2": "inputs larger than L2 (psi = 512 MiB)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline,
                "passes": passes,
                "clocks": res["clocks"],
                "gpu_launches": res["launches"] * world,
                "e2e": e2e,
                "point_updates_per_s": value * N,
                "observables": [float(x) for x in res["obs"]]}
        line.update({k: v for k, v in extra.items() if k != "cpu_baseline"})
        if "cpu_baseline" in extra:
            line["cpu_baseline"] = extra["cpu_baseline"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
