"""Benchmark: FISTA iterations per second of the one-step reconstruction.

One step = one FISTA iteration (Algorithm 1) of the whole hot path on the
medium workload (64x64 scan, 64 depths, T=256, 15x15 lateral support,
40 pulses in 4 cycles of 10, 2 species, 10 inner TV iterations): switching
map P, acoustic forward A with the folded residual, adjoint A^T, P^T with
the gradient step, the FGP TV prox, the l1/nonnegativity prox and the
momentum update.  Inputs are synthetic and seeded (tube phantom, transducer
kernel, 20 dB noise) and resident in HBM before the timed region.

The default arithmetic is the refined solve: A / A^T on the tensor cores in
BF16 applied to the iterate increments, with the gradient recomputed exactly
(two-term BF16 split) every 25 iterations.  The same run times the plain
FP32 solve (CUDA-core FMA) on the same problem and reports the relative
difference of the two objectives after the same number of iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl swopt|reference]
                       [--precision fp32|bf16|bf16x3] [--refine R]
For N > 1 it is launched by torch.distributed.run, one rank per GPU; each rank
solves its own independent problem (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "medium_64x64x64_T256_k15_N40_P2"
METRIC = "FISTA iterations/s"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _smi_id(device) -> str:
    """nvidia-smi --id for a torch device: its PCI bus id when torch exposes
    it, else the physical index from CUDA_VISIBLE_DEVICES."""
    import torch
    props = torch.cuda.get_device_properties(device)
    dom = getattr(props, "pci_domain_id", None)
    bus = getattr(props, "pci_bus_id", None)
    dv = getattr(props, "pci_device_id", None)
    if bus is not None and dom is not None and dv is not None:
        return f"{dom:08X}:{bus:02X}:{dv:02X}.0"
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    idx = device.index or 0
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if idx < len(ids):
            return ids[idx]
    return str(idx)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("operator_simt.cu", "operator_tc.cu", "swopt_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2510_23739_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_name: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_name}_{workload}.txt")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*(\w+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != _kernel_source_hash():
        return None
    return float(m_bytes.group(1))


def workload_problem(name: str, kernel: str = "aperture"):
    """The named workload; the paper-literal kernel runs on the matched time
    grid (c dt = dz) that its construction assumes."""
    prob = synth.workload(name)
    if kernel == "semicircle":
        prob = synth.small_variant(prob, dt_us=synth.matched_time_grid(prob.geom).dt_us)
    return prob


def semicircle_args(g):
    """Arguments of the paper-literal kernel for geometry g: 3D half-sphere
    masks, lateral pitch in depth pitches, the focus at the middle depth and
    at the middle time sample, the synthetic SPR image and impulse response."""
    return (g.Z, g.k, g.T, 3, g.dx_mm / g.dz_mm, (g.Z - 1) / 2.0, g.T // 2,
            synth.spr_image(g, seed=0), synth.eir_taps(g))


def make_problem(prob, seed: int, device, kernel: str = "aperture"):
    """Seeded synthetic inputs on the device: kernel, phantom, measurements."""
    import torch
    import paper_2510_23739_gb300 as sw

    g = prob.geom
    if kernel == "semicircle":
        K = sw.semicircle_kernel(*semicircle_args(g))
    else:
        K = synth.transducer_kernel(g, seed=0)
    op = sw.Operator(g, K, prob.sw)
    c_true = torch.tensor(synth.tube_phantom(g, prob.tubes, seed=seed,
                                             per_species=prob.tubes_per_species),
                          dtype=torch.float32, device=device)
    clean = op.forward(c_true)
    # noise power from the full clean signal (FP64 on the device)
    sigma = math.sqrt(float(clean.double().pow(2).mean()) / 10 ** (prob.snr_db / 10))
    noise = torch.tensor(synth.gaussian(g.y_shape(), seed + 1000), dtype=torch.float32,
                         device=device)
    y = clean + sigma * noise
    del noise, clean
    return op, K, c_true, y


def run_swopt(args, rank, world, device):
    import torch
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    op, K, c_true, y = make_problem(prob, seed=rank, device=device, kernel=args.kernel)
    if args.precision != "fp32":
        op.set_precision(args.precision)
    L = op.lipschitz(100)
    alpha = 1.0 / L
    refine = dict(refine_every=args.refine, refine_precision=args.refine_precision)
    params = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                            inner_iters=prob.inner, max_iters=args.steps, **refine)
    stream = torch.cuda.current_stream()
    op.fista_init(y, params)
    for _ in range(args.warmup):
        op.fista_step(1)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    op.profile(True)
    op.profile_read(0)
    op.profile_read(1)
    launches0 = op.launch_count()
    clocks = ClockSampler(_smi_id(device))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    # a profiler that starts with profiling off (ncu --profile-from-start off)
    # sees the timed steps only
    torch.cuda.profiler.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # evict the working set from L2 between timed steps
        starts[i].record(stream)
        op.fista_step(1)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = op.launch_count() - launches0
    op.profile(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    kinfo = [op.profile_read(0), op.profile_read(1)]
    kinfo_ref = [op.profile_read(2), op.profile_read(3)]
    c_final = op.fista_get().clone()
    issued = [op.issued_flops(0), op.issued_flops(1)]
    avg = [ki["total_ms"] / max(ki["launches"], 1) for ki in kinfo]
    dom = 0 if avg[0] >= avg[1] else 1
    flops = kinfo[dom]["flops_per_launch"]

    # e2e: a user call with host buffers (pinned), copies inside the timed region
    y_host = y.cpu().pin_memory()
    c_host = torch.empty(op.c_shape, dtype=torch.float32).pin_memory()
    e2e_params = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                                inner_iters=prob.inner, max_iters=args.steps, **refine)
    y_dev = torch.empty_like(y)
    c_dev = torch.empty(op.c_shape, dtype=torch.float32, device=device)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    y_dev.copy_(y_host, non_blocking=True)
    op.fista_init(y_dev, e2e_params)
    op.fista_step(args.steps)
    op.fista_get(c_dev)
    c_host.copy_(c_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    result = {"total_ms": total_ms, "wall_s": wall, "dom": dom, "avg_ms": avg, "flops": flops,
              "launches": launches, "clocks": clk, "e2e_ms": e2e_ms,
              "h2d": y_host.numel() * 4, "d2h": c_host.numel() * 4, "info": op.info(),
              "kinfo": kinfo, "kinfo_ref": kinfo_ref, "issued": issued}
    op.close()

    # the plain FP32 solve on the same problem and step: time and objective
    # after the same number of iterations (warm-up + timed)
    if args.precision != "fp32" or args.refine > 0:
        ref = sw.Operator(g, K, prob.sw)
        fp = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                            inner_iters=prob.inner, max_iters=args.warmup + args.steps)
        ref.fista_init(y, fp)
        ref.fista_step(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        ref.fista_step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fp32_ms = e0.elapsed_time(e1) / args.steps
        c32 = ref.fista_get()
        F32, _ = ref.objective(c32, y, prob.lam_l1, prob.lam_tv)
        Fme, _ = ref.objective(c_final, y, prob.lam_l1, prob.lam_tv)
        ref.close()
        result["fp32"] = {"ms_per_step": fp32_ms, "F_fp32": F32, "F": Fme,
                          "iters": args.warmup + args.steps,
                          "c_rel_diff": float((c_final - c32).norm() / c32.norm())}
    return result


def run_two_step(args, device):
    """The two-step approach (per-pulse acoustic inversion with TV, then
    unmixing with l1 + TV; swopt_two_step) against the one-step solve on the
    same data, both FP32 with `steps` FISTA iterations per solve and steps
    from the power iteration computed before the timed region."""
    import torch
    from dataclasses import replace
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    op, K, c_true, y = make_problem(prob, seed=0, device=device, kernel=args.kernel)
    g1 = replace(g, N=1, P=1, pulses_per_cycle=1)
    s1 = synth.Switching((0.0,), (0.0,), (1.0,), 0.0)
    op1 = sw.Operator(g1, K, s1)
    eye = np.zeros((g.Z, 1, 1, g.Z))
    for j in range(g.Z):
        eye[j, 0, 0, j] = 1.0
    op2 = sw.Operator(replace(g, T=g.Z, k=1), eye, prob.sw)
    a0, a1, a2 = (1.0 / o.lipschitz(100) for o in (op, op1, op2))
    op1.close()
    op2.close()
    iters = args.steps
    acoustic = sw.SolveParams(step=a1, lambda_l1=0.0, lambda_tv=prob.lam_tv,
                              inner_iters=prob.inner, max_iters=iters)
    unmixing = sw.SolveParams(step=a2, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                              inner_iters=prob.inner, max_iters=iters)
    one = sw.SolveParams(step=a0, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                         inner_iters=prob.inner, max_iters=iters)
    stream = torch.cuda.current_stream()
    sw.two_step(g, K, prob.sw, y, replace_iters(acoustic, 2), replace_iters(unmixing, 2))
    op.solve(y, replace_iters(one, 2))
    times = {}
    for name, fn in (("two_step", lambda: sw.two_step(g, K, prob.sw, y, acoustic, unmixing)),
                     ("one_step", lambda: op.solve(y, one))):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1)
        if name == "two_step":
            c2 = out[0]
        else:
            c1 = out[0]
    ct = c_true.double()
    err = {k: float((v.double() - ct).norm() / ct.norm()) for k, v in (("two_step", c2),
                                                                       ("one_step", c1))}
    print(json.dumps({
        "metric": "two-step reconstruction time", "value": times["two_step"], "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": iters, "dtype": "f32",
        "data": "synthetic (seeded tube phantom, transducer kernel, 20 dB noise)",
        "config": {"workload": args.workload, "kernel": args.kernel,
                   "iterations_per_solve": iters, "pulses": g.N},
        "one_step_ms_same_iterations": times["one_step"],
        "relative_error_vs_phantom": err}), flush=True)


def run_prox_joint(args, device):
    """The prox of the full R3 with its lambda_3 term (swopt_prox_joint) on
    the workload's volume and pulses: time per call of `inner` dual
    iterations, CUDA events over `steps` calls after `warmup`, inputs larger
    than L2."""
    import torch
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    K = synth.transducer_kernel(g, seed=0)
    op = sw.Operator(g, K, prob.sw)
    z = torch.tensor(synth.gaussian(g.c_shape(), 5), dtype=torch.float32, device=device) + 0.5
    lam_tv, lam_l1, lam_b, alpha, inner = prob.lam_tv, prob.lam_l1, prob.lam_tv, 0.5, prob.inner
    # a dual step below 1/||L||^2 (|S| <= 2 here); the time does not depend on it
    step2 = 1.0 / (12 * lam_tv ** 2 + lam_l1 ** 2 + 12 * lam_b ** 2 * g.N * 4.0)
    out = torch.empty_like(z)
    for _ in range(args.warmup):
        op.prox_joint(z, alpha, lam_tv, lam_l1, lam_b, inner, step2, out=out)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        op.prox_joint(z, alpha, lam_tv, lam_l1, lam_b, inner, step2, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    L = g.Y * g.X * g.Z
    nu = (4 * g.P + 3 * g.N) * L
    # per dual iteration: L^T reads the momentum duals and z, writes w; the
    # update reads w (and neighbours), reads and writes u and r
    bytes_iter = 4 * (nu + 2 * g.P * L) + 4 * (g.P * L + 4 * nu)
    print(json.dumps({
        "metric": "joint prox time (full R3, lambda_3 term)", "value": ms, "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32", "data": "synthetic (seeded Gaussian input)",
        "config": {"workload": args.workload, "inner_iters": inner, "pulses": g.N,
                   "species": g.P, "dual_values": nu},
        "algorithmic_gb_per_s": bytes_iter * inner / (ms * 1e-3) / 1e9}), flush=True)


def replace_iters(params, iters):
    import copy
    p = copy.copy(params)
    p.max_iters = iters
    return p


def run_batch(args, device):
    """Sixteen independent problems of uneven size (scan 32^2..128^2, depths
    48-128, T 128-512, 20-80 pulses, 2-3 species, supports 11-31; seeded):
    aggregate FISTA iterations per second of the batched step (one CUDA graph
    per iteration, a stream per problem) against the same problems stepped
    one after another at the same precision, and against plain FP32 one after
    another (a few iterations per problem, the per-iteration cost being
    constant)."""
    import torch
    import paper_2510_23739_gb300 as sw

    probs = synth.batch_shapes(16, 0)
    ops, ys, params = [], [], []
    refine = dict(refine_every=args.refine, refine_precision=args.refine_precision)
    for i, prob in enumerate(probs):
        op, K, c_true, y = make_problem(prob, seed=i, device=device)
        op.set_precision(args.precision)
        L = op.lipschitz(50)
        prm = sw.SolveParams(step=1.0 / L, lambda_l1=1e-3, lambda_tv=1e-3, inner_iters=10,
                             max_iters=args.warmup + args.steps, **refine)
        op.fista_init(y, prm)
        ops.append(op)
        ys.append(y)
        params.append(prm)
        del c_true
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    batch = sw.Batch(ops)
    batch.step(args.warmup)
    launches0 = ops[0].launch_count()
    clocks = ClockSampler(_smi_id(device))
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    batch_ms = e0.elapsed_time(e1)
    launches = ops[0].launch_count() - launches0
    batch.close()
    # the same problems one after another (each handle's own graph)
    for op, y, prm in zip(ops, ys, params):
        op.fista_init(y, prm)
        op.fista_step(args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    for op in ops:
        op.fista_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    # plain FP32, one after another
    fp32_ms = 0.0
    fp32_iters = 2
    for op, y, prm in zip(ops, ys, params):
        op.set_precision("fp32")
        p32 = sw.SolveParams(step=prm.step, lambda_l1=prm.lambda_l1, lambda_tv=prm.lambda_tv,
                             inner_iters=prm.inner_iters, max_iters=fp32_iters + 1)
        op.fista_init(y, p32)
        op.fista_step(1)
        torch.cuda.synchronize()
        e0.record(stream)
        op.fista_step(fp32_iters)
        e1.record(stream)
        torch.cuda.synchronize()
        fp32_ms += e0.elapsed_time(e1) / fp32_iters
        op.check_device()
        op.close()
    n = len(probs)
    value = n * args.steps / (batch_ms / 1e3)
    line = {
        "metric": "aggregate FISTA iterations/s (16 uneven problems)", "value": value,
        "unit": "it/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": batch_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.precision + (f" + refinement (exact {args.refine_precision} gradient every "
                                   f"{args.refine} iterations)" if args.refine > 0 else ""),
        "data": "synthetic (seeded tube phantoms, transducer kernels, 20 dB noise)",
        "config": {"workload": "batch16_uneven (synth.batch_shapes(16, 0))",
                   "l2": "working set larger than L2 (no flush)",
                   "problems": [f"{p.geom.X}x{p.geom.Y}x{p.geom.Z} T{p.geom.T} k{p.geom.k} "
                                f"N{p.geom.N} P{p.geom.P}" for p in probs]},
        "sequential_same_precision_it_s": n * args.steps / (seq_ms / 1e3),
        "sequential_fp32_plain_it_s": n / (fp32_ms / 1e3),
        "speedup_vs_sequential_fp32": value / (n / (fp32_ms / 1e3)),
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def combine_ranks(total_ms: float, e2e_ms: float, steps: int, world: int, device=None):
    """Replicas (one independent problem per rank): the slowest rank's timed
    region and end-to-end time decide, and the whole-job throughput counts
    every rank's iterations.  Returns (total_ms, e2e_ms, it/s, e2e it/s)."""
    if world > 1:
        import torch
        t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms, e2e_ms = float(t[0]), float(t[1])
    return (total_ms, e2e_ms, world * steps / (total_ms / 1e3), world * steps / (e2e_ms / 1e3))


def cpu_oracle_iteration_ms(prob, sample_pulses: int, kernel: str = "aperture"):
    """Time the FP64 oracle on a bounded sample of one FISTA iteration and
    extrapolate to the full workload: forward + adjoint on `sample_pulses`
    pulses (the per-pulse work is identical), the TV/l1 prox on the full
    volume."""
    import oracle
    from dataclasses import replace

    g = prob.geom
    if kernel == "semicircle":
        K = oracle.semicircle_kernel(*semicircle_args(g))
    else:
        K = synth.transducer_kernel(g, seed=0)
    gs = replace(g, N=sample_pulses)
    c = synth.tube_phantom(g, prob.tubes, seed=0)
    y = synth.gaussian(gs.y_shape(), 7) * 0.01
    t0 = time.perf_counter()
    yy = oracle.forward(gs, prob.sw, K, c)
    t1 = time.perf_counter()
    oracle.adjoint(gs, prob.sw, K, yy - y)
    t2 = time.perf_counter()
    oracle.prox(c, 1e-3, prob.lam_l1, prob.lam_tv, prob.inner)
    t3 = time.perf_counter()
    scale = g.N / sample_pulses
    ms = ((t1 - t0) + (t2 - t1)) * scale * 1e3 + (t3 - t2) * 1e3
    sample = (f"forward+adjoint on {sample_pulses} of {g.N} pulses, extrapolated x{scale:g}; "
              f"TV+l1 prox ({prob.inner} inner) on the full volume")
    return ms, sample, oracle.num_threads()


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, each step a bounded sample of
    one FISTA iteration extrapolated to the full workload."""
    prob = workload_problem(args.workload, args.kernel)
    times = []
    sample = ""
    cores = 1
    for i in range(args.warmup + args.steps):
        ms, sample, cores = cpu_oracle_iteration_ms(prob, args.ref_sample_pulses, args.kernel)
        if i >= args.warmup:
            times.append(ms)
    ms = sum(times) / len(times)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "it/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "kernel": args.kernel,
                       "impl": "FP64 CPU oracle (plain C, OpenMP)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "it/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="swopt", choices=["swopt", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--method", default="one-step", choices=["one-step", "two-step", "prox-joint"],
                    help="two-step: time swopt_two_step against the one-step solve (FP32); "
                         "prox-joint: time the prox of the full R3 (lambda_3 term)")
    ap.add_argument("--kernel", default="aperture", choices=["aperture", "semicircle"],
                    help="per-depth kernel: the aperture-point transducer model, or the "
                         "paper-literal SPR on discrete half spheres (matched time grid)")
    ap.add_argument("--refine", type=int, default=None,
                    help="refined solve: exact gradient every R iterations (0: off; "
                         "default 25 for bf16, else 0)")
    ap.add_argument("--refine-precision", default="bf16x3", choices=["fp32", "bf16x3"])
    ap.add_argument("--cpu-sample-pulses", type=int, default=2)
    ap.add_argument("--ref-sample-pulses", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.refine is None:
        args.refine = 25 if args.precision == "bf16" else 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)

    import paper_2510_23739_gb300 as sw
    sw.lib()
    if args.method == "prox-joint":
        if rank == 0:
            run_prox_joint(args, device)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.method == "two-step":
        if rank == 0:
            run_two_step(args, device)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "batch16":
        if rank == 0:
            run_batch(args, device)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    res = run_swopt(args, rank, world, device)

    total_ms, e2e_ms, value, e2e_value = combine_ranks(res["total_ms"], res["e2e_ms"],
                                                       args.steps, world, device)

    if rank == 0:
        peaks, peak_src = _peaks()
        ms_step = total_ms / args.steps
        dom = res["dom"]
        avg_ms = res["avg_ms"][dom]
        achieved = res["flops"] / (avg_ms * 1e-3) / 1e12
        clk = res["clocks"]
        issued_tflops = res["issued"][dom] / (avg_ms * 1e-3) / 1e12
        if args.precision == "fp32":
            # FP32 FMA on the CUDA cores: 152 SMs x 128 lanes x 2 FLOP x max SM clock
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound, peak_note = "alu", f"FP32 FMA peak at {peaks.get('sm_max_mhz', 2070.0):g} MHz"
        elif args.precision == "bf16":
            peak = peaks["bf16_tflops_sustained"]
            bound, peak_note = "tensor", f"bf16 dense sustained ({peak_src})"
        else:
            # each useful multiply-add costs 3 BF16 multiply-adds (two-term split)
            nprod = 3
            peak = peaks["bf16_tflops_sustained"] / nprod
            bound, peak_note = "tensor", f"bf16 dense sustained / {nprod} products ({peak_src})"
        kname = ["A_forward", "AT_adjoint"][dom]
        traffic = _profiled_traffic(kname, args.workload) if args.kernel == "aperture" else None
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            ms_cpu, sample, cores = cpu_oracle_iteration_ms(
                workload_problem(args.workload, args.kernel), args.cpu_sample_pulses, args.kernel)
            cpu = {"value": 1000.0 / ms_cpu, "unit": "it/s", "cores": cores, "kind": "oracle",
                   "sample": sample}
        line = {
            "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3 (2-term split)"}[
                args.precision] + (f" + refinement (exact {args.refine_precision} gradient every "
                                   f"{args.refine} iterations)" if args.refine > 0 else ""),
            "data": "synthetic (seeded tube phantom, transducer kernel, 20 dB noise)",
            "config": {"workload": args.workload, "kernel": args.kernel,
                       "precision": args.precision,
                       "refine_every": args.refine,
                       "refine_precision": args.refine_precision if args.refine > 0 else None,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "time_window": res["info"], "inner_iters": 10},
            "roofline": {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "avg_launch_ms": avg_ms, "flops_per_launch": res["flops"],
                         "peak_source": peak_note, "issued_tflops": issued_tflops,
                         "issued_frac_of_bf16_peak": issued_tflops / peaks["bf16_tflops_sustained"],
                         "other_kernel_avg_ms": res["avg_ms"][1 - dom]},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "it/s",
                    "h2d_bytes_per_step": res["h2d"] / args.steps,
                    "d2h_bytes_per_step": res["d2h"] / args.steps,
                    "note": "one swopt solve of `steps` iterations from pinned host y to host c"},
            "gpu_launches": res["launches"],
            "clocks": clk,
        }
        if args.refine > 0:
            kr = res["kinfo_ref"]
            line["roofline"]["resync_avg_launch_ms"] = [
                k["total_ms"] / k["launches"] if k["launches"] else None for k in kr]
        if "fp32" in res:
            f = res["fp32"]
            line["precision_path"] = {
                "fp32_plain_it_s": 1000.0 / f["ms_per_step"],
                "speedup_vs_fp32_plain": (value / world) / (1000.0 / f["ms_per_step"]),
                "objective_rel_diff_vs_fp32": abs(f["F"] - f["F_fp32"]) / abs(f["F_fp32"]),
                "iterate_rel_diff_vs_fp32": f["c_rel_diff"],
                "iterations_compared": f["iters"],
                "note": "same problem, step and iteration count; plain FP32 = CUDA-core FMA "
                        "operators, objectives both evaluated in FP32 with FP64 sums"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
