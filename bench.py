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
FP64_PEAK_TFLOPS = 1.25    # nominal B300 FP64 rate (no measured figure on this machine)


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
KERNEL_SOURCES = ["device_fft.cuh", "kernels.cuh", "kernels.cu", "fast_passes.cu"]


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-extras", action="store_true")
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


def cpu_baseline(seconds_cap=30.0):
    """The FP64 oracle, as it stands, on the host cores: split steps of the
    full 256x256x1024 workload, as many as fit in about `seconds_cap`."""
    import oracle
    from paper_1309_2451_b300 import workloads as wl
    box = wl.CTAP_BOX
    z = wl.axis(SHAPE[0], box[4], box[5])
    c = wl.guide_centres(z)
    V = oracle.ctap_potential(SHAPE, box, wl.V0, wl.SIGMA_GUIDE, c[0], c[2])
    xc = float(wl.guide_centres(np.array([-40.0]))[0, 0])
    psi = wl.packet_from_transverse(wl.guide_seed_2d(SHAPE[1:], box, xc), SHAPE[0], box)
    n, t_total = 0, 0.0
    while t_total < seconds_cap and n < 10:
        t0 = time.perf_counter()
        psi = oracle.step(psi, V, box, DT, 1)
        t_total += time.perf_counter() - t0
        n += 1
        if n == 1 and t_total > seconds_cap / 2:
            break
    return {"value": n / t_total, "unit": "steps/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n} FP64 split step(s) of the 256x256x1024 three-guide workload "
                      f"({t_total:.1f} s, OpenMP over lines)"}


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

    res = time_path(ctap, wl, torch, "c64", SPLIT, a.steps, a.warmup, device, stream,
                    barrier=dist.barrier if dist is not None else None)

    N = int(np.prod(SHAPE))
    esize = 8
    hbm, peak_kind = peaks()
    counts, pms = res["counts"], res["pass_ms"]
    kind = 0 if pms[0] >= pms[1] else 1
    fast = res["plan"].info()["fast_mask"]
    name = (("xy_ring_kernel" if fast & 8 else ("xy_fast_kernel" if fast & 1 else "xy_pass_kernel"))
            if kind == 0
            else ("z_ring_kernel" if fast & 4 else ("z_fast_kernel" if fast & 2 else "z_pass_kernel")))
    avg_ms = pms[kind] / max(counts[kind], 1)
    bytes_launch = 2 * N * esize       # one read and one write of psi
    achieved = bytes_launch / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": recorded_traffic(name),
                "kernel": name, "peak_kind": peak_kind,
                "step_design_GBps": 4 * N * esize * a.steps * SPLIT / (res["ms"] * 1e-3) / 1e9}

    extra = {}
    if rank == 0 and not a.no_fp64:
        r64 = time_path(ctap, wl, torch, "c128", SPLIT_FP64, max(2, a.steps // 10), 1, device,
                        stream)
        ms64 = r64["ms"] / (max(2, a.steps // 10) * SPLIT_FP64)
        c64, p64 = r64["counts"], r64["pass_ms"]
        k64 = 0 if p64[0] >= p64[1] else 1
        avg64 = p64[k64] / max(c64[k64], 1)
        ach64 = 2 * N * 16 / (avg64 * 1e-3) / 1e9
        P64 = r64["plan"].info()["row_classes"]
        fxy, fz = pass_flops_per_point(SHAPE, P64)
        tflops = (fxy if k64 == 0 else fz) * N / (avg64 * 1e-3) / 1e12
        fast64 = r64["plan"].info()["fast_mask"]
        extra["fp64_path"] = {
            "steps_per_s": 1000.0 / ms64, "ms_per_step": ms64,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": tflops / FP64_PEAK_TFLOPS,
                         "peak_kind": "nominal FP64 (profiling recipe)",
                         "kernel": ("xy_" if k64 == 0 else "z_") + ("fast" if fast64 else "pass")
                                   + "_kernel<double>",
                         "flops_per_point": fxy if k64 == 0 else fz},
            "hbm_frac_of_dominant_kernel": ach64 / hbm,
            "fp32_speedup": (1000.0 / (res["ms"] / (a.steps * SPLIT))) / (1000.0 / ms64),
            "dtype": "f64", "obs": [float(x) for x in r64["obs"]]}
        del r64
        rdf = time_path(ctap, wl, torch, "c128df", SPLIT_FP64, max(2, a.steps // 10), 1, device,
                        stream)
        msdf = rdf["ms"] / (max(2, a.steps // 10) * SPLIT_FP64)
        extra["fp64_df_path"] = {
            "steps_per_s": 1000.0 / msdf, "ms_per_step": msdf,
            "arithmetic": "double-float (FP32 pairs, ~48-bit significands) on complex128 psi",
            "speedup_over_fp64": ms64 / msdf,
            "obs": [float(x) for x in rdf["obs"]]}
        del rdf
    if rank == 0 and not a.no_extras:
        extra["rows"] = time_rows(ctap, wl, torch, device, stream)
        extra["variants"] = time_variants(torch, wl, device, stream, res["plan"], res["psi"])
        extra["variants"]["batched_sweep"] = time_batched(torch, wl, device, stream)
        extra["cufft_comparison"] = time_cufft(torch, device, stream, res["plan"])
        extra["cpu_baseline"] = cpu_baseline()
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
