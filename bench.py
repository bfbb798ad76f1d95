"""Benchmark: FISTA iterations per second of the one-step reconstruction.

One step = one FISTA iteration (Algorithm 1) of the whole hot path on the
large workload (128x128 scan, 96 depths, T=512, 31x31 lateral support, 60
pulses in 6 cycles of 10, 3 species, 10 inner TV iterations): switching map
P, acoustic forward A with the folded residual, adjoint A^T, P^T with the
gradient step, the FGP TV prox, the l1/nonnegativity prox and the momentum
update.  Inputs are synthetic and seeded (tube phantom, transducer kernel,
20 dB noise) and resident in HBM before the timed region.

The default arithmetic is the refined solve: A / A^T on the tensor cores in
BF16 applied to the iterate increments, with the gradient recomputed exactly
(two-term BF16 split) every 25 iterations or sooner, when the relative steps
taken on increments since the last exact gradient add up to 0.1 (decided on
the GPU).  Timed iterations are taken in the solve's steady phase, after
`--presolve` untimed iterations; the first iterations (where most gradients
are exact) are timed separately and reported as `early_phase`, and `e2e`
times a whole solve from host measurements to host concentrations.  The same
run reports the operators' error against the FP64 oracle on sampled outputs,
the plain FP32 solve's speed, and the difference from an FP32-class (two-term
BF16) solve after the same iteration count.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl swopt|reference]
                       [--workload NAME] [--precision fp32|bf16|bf16x3|bf16x6|fp8]
                       [--refine R] [--refine-budget B] [--presolve I]
                       [--method one-step|two-step|prox-joint|prox-sweep|prox-tv|objective-gap]
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

WORKLOAD = "large_128x128x96_T512_k31_N60_P3"
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
    for name in ("operator_tc.cu", "swopt_internal.cuh"):
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


def schedule_params(args):
    """The refined solve's settings of this run (empty for an unrefined solve)."""
    if args.refine <= 0:
        return {}
    return {"refine_every": args.refine, "refine_precision": args.refine_precision,
            "refine_budget": args.refine_budget}


def sampled_operator_error(op, prob, K, c, seed: int, rows: int = 24, entries: int = 48):
    """Relative L2 error of H c and H^T w against the FP64 oracle on sampled
    outputs: `rows` measurement rows (n, y, x, all t) and `entries` adjoint
    entries (p, y, x, j), each an independent sum evaluated by the oracle."""
    import torch
    import oracle

    g = prob.geom
    rng = np.random.default_rng(seed)
    nyx = np.stack([rng.integers(0, g.N, rows), rng.integers(0, g.Y, rows),
                    rng.integers(0, g.X, rows)], axis=1)
    c_host = c.double().cpu().numpy()
    y_gpu = op.forward(c)
    got = y_gpu[nyx[:, 0], nyx[:, 1], nyx[:, 2], :].double().cpu().numpy()
    del y_gpu
    ref = oracle.forward_at(g, prob.sw, K, c_host, nyx)
    e_fwd = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # w ~ N(0,1) on the first cycle of pulses (every switching state), zero
    # on the rest: the host array stays small where it is zero
    ncyc = min(g.N, g.pulses_per_cycle)
    w_host = np.zeros(g.y_shape())
    w_host[:ncyc] = synth.gaussian((ncyc, g.Y, g.X, g.T), seed + 1)
    w = torch.zeros(g.y_shape(), dtype=torch.float32, device=c.device)
    w[:ncyc] = torch.tensor(w_host[:ncyc], dtype=torch.float32, device=c.device)
    w_host[:ncyc] = w[:ncyc].double().cpu().numpy()  # the values the GPU sees
    pyxj = np.stack([rng.integers(0, g.P, entries), rng.integers(0, g.Y, entries),
                     rng.integers(0, g.X, entries), rng.integers(0, g.Z, entries)], axis=1)
    gt = op.adjoint(w)
    got_a = gt[pyxj[:, 0], pyxj[:, 1], pyxj[:, 2], pyxj[:, 3]].double().cpu().numpy()
    ref_a = oracle.adjoint_at(g, prob.sw, K, w_host, pyxj)
    del w, gt, w_host
    e_adj = float(np.linalg.norm(got_a - ref_a) / np.linalg.norm(ref_a))
    return {"A": e_fwd, "AT": e_adj, "sample": f"{rows} rows (n,y,x,:) of H c and {entries} "
            f"entries (p,y,x,j) of H^T w, w ~ N(0,1) on the first {ncyc} pulses, 0 after"}


def run_swopt(args, rank, world, device):
    import torch
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    op, K, c_true, y = make_problem(prob, seed=rank, device=device, kernel=args.kernel)
    if args.precision != "fp32":
        op.set_precision(args.precision)
    L = op.lipschitz(args.power_iters)
    alpha = 1.0 / L
    refine = schedule_params(args)
    total_iters = args.presolve + args.warmup + args.steps
    params = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                            inner_iters=prob.inner, max_iters=total_iters, **refine)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    op.fista_init(y, params)
    early = None
    if args.presolve >= 2:
        # the first iterations of the solve (the graph of an iteration kind is
        # captured at its first step: iteration 1 stays outside the timing)
        op.fista_step(1)
        n_early = min(args.presolve, 25) - 1
        torch.cuda.synchronize()
        e0.record(stream)
        op.fista_step(n_early)
        e1.record(stream)
        torch.cuda.synchronize()
        early = {"iterations": f"2..{n_early + 1}", "ms_per_iteration":
                 e0.elapsed_time(e1) / n_early,
                 "exact_gradients": op.refine_stats()[1] if refine else None}
        op.fista_step(args.presolve - 1 - n_early)
    else:
        op.fista_step(args.presolve)
    op.fista_step(args.warmup)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    op.profile(True)
    for kid in range(4):
        op.profile_read(kid)
    launches0 = op.launch_count()
    it0, rs0 = op.refine_stats()
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
    it1, rs1 = op.refine_stats()
    op.profile(False)
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    kinfo = [op.profile_read(k) for k in range(4)]
    c_final = op.fista_get().clone()
    issued = [op.issued_flops(0), op.issued_flops(1)]
    avg = [ki["total_ms"] / ki["launches"] if ki["launches"] else 0.0 for ki in kinfo]
    # the dominant contraction of the timed iterations: the slower of A / A^T
    # at the handle's precision (the increments), or at the resync precision
    # when no increment ran
    cand = [0, 1] if kinfo[0]["launches"] and kinfo[1]["launches"] else [2, 3]
    dom = max(cand, key=lambda k: avg[k])
    flops = kinfo[dom]["flops_per_launch"]
    op_err = None
    if rank == 0 and not args.no_oracle_check:
        op_err = {args.precision: sampled_operator_error(op, prob, K, c_true, 21)}
        if refine and args.refine_precision != args.precision:
            op.set_precision(args.refine_precision)
            op_err[args.refine_precision] = sampled_operator_error(op, prob, K, c_true, 21)
    info = op.info()
    op.close()

    # e2e: a user's whole solve through the public API from pinned host
    # measurements to host concentrations, copies inside the timed region
    y_host = y.cpu().pin_memory()
    c_host = torch.empty(tuple(c_final.shape), dtype=torch.float32).pin_memory()
    op2 = sw.Operator(g, K, prob.sw)
    if args.precision != "fp32":
        op2.set_precision(args.precision)
    y_dev = torch.empty_like(y)
    c_dev = torch.empty(tuple(c_final.shape), dtype=torch.float32, device=device)
    # build the operators and capture the graphs once, outside the timed region
    op2.fista_init(y, params)
    op2.fista_step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    y_dev.copy_(y_host, non_blocking=True)
    op2.fista_init(y_dev, params)
    op2.fista_step(total_iters)
    op2.fista_get(c_dev)
    c_host.copy_(c_dev, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    op2.close()

    result = {"total_ms": total_ms, "wall_s": wall, "dom": dom, "avg_ms": avg, "flops": flops,
              "launches": launches, "clocks": clk, "e2e_ms": e2e_ms, "e2e_iters": total_iters,
              "h2d": y_host.numel() * 4, "d2h": c_host.numel() * 4, "info": info,
              "kinfo": kinfo, "issued": issued, "early": early, "op_err": op_err,
              "timed_iters": (it0 + 1, it1), "timed_resyncs": rs1 - rs0}

    # the plain FP32 solve's speed on the same problem and step, and an
    # FP32-class solve (two-term BF16, every gradient exact) after the same
    # number of iterations as the refined one
    if rank == 0 and (args.precision != "fp32" or refine):
        ref = sw.Operator(g, K, prob.sw)
        fp = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                            inner_iters=prob.inner, max_iters=args.fp32_iters + 1)
        ref.fista_init(y, fp)
        ref.fista_step(1)
        torch.cuda.synchronize()
        e0.record(stream)
        ref.fista_step(args.fp32_iters)
        e1.record(stream)
        torch.cuda.synchronize()
        fp32_ms = e0.elapsed_time(e1) / args.fp32_iters
        ref.set_precision("bf16x3")
        full = sw.SolveParams(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv,
                              inner_iters=prob.inner, max_iters=total_iters)
        ref.fista_init(y, full)
        ref.fista_step(total_iters)
        c32 = ref.fista_get()
        torch.cuda.synchronize()
        ref.set_precision("fp32")
        F32, _ = ref.objective(c32, y, prob.lam_l1, prob.lam_tv)
        Fme, _ = ref.objective(c_final, y, prob.lam_l1, prob.lam_tv)
        ref.close()
        result["fp32"] = {"ms_per_step": fp32_ms, "F_ref": F32, "F": Fme,
                          "iters": total_iters,
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
    the workload's volume and switching states: time per call of `inner` dual
    iterations, CUDA events over `steps` calls after `warmup`.  Per dual
    iteration (one dual per switching state, nd = 4 P + 3 Q volumes): L^T
    reads the momentum duals and z and writes w (nd + 2 P volumes); the update
    reads w, reads and writes u and r (4 nd + P volumes).  The duals of the
    large workload (P = 3, Q = 10) are 42 volumes of 6.3 MB, twice L2 per
    array."""
    import torch
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    K = synth.transducer_kernel(g, seed=0)
    op = sw.Operator(g, K, prob.sw)
    z = torch.tensor(synth.gaussian(g.c_shape(), 5), dtype=torch.float32, device=device) + 0.5
    lam_tv, lam_l1, lam_b, alpha, inner = prob.lam_tv, prob.lam_l1, prob.lam_tv, 0.5, prob.inner
    step2 = 1.0 / op.prox_joint_step_bound(lam_tv, lam_l1, lam_b)
    out = torch.empty_like(z)
    for _ in range(args.warmup):
        op.prox_joint(z, alpha, lam_tv, lam_l1, lam_b, inner, step2, out=out)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(_smi_id(device))
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(args.steps):
        op.prox_joint(z, alpha, lam_tv, lam_l1, lam_b, inner, step2, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    op.check_device()
    states = op.info()["states"]
    op.close()
    ms = e0.elapsed_time(e1) / args.steps
    L = g.Y * g.X * g.Z
    nd = 4 * g.P + 3 * states
    bytes_iter = 4.0 * L * ((nd + 2 * g.P) + (4 * nd + g.P))
    gbs = bytes_iter * inner / (ms * 1e-3) / 1e9
    peaks, src = _peaks()
    print(json.dumps({
        "metric": "joint prox algorithmic HBM throughput (full R3, lambda_3 term)",
        "value": gbs, "unit": "GB/s", "higher_is_better": True, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "dtype": "f32", "data": "synthetic (seeded Gaussian input)",
        "config": {"workload": args.workload, "inner_iters": inner, "pulses": g.N,
                   "species": g.P, "switching_states": states, "dual_volumes": nd,
                   "l2": "dual arrays about 2x L2 each (no flush)"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                     "bytes_per_dual_iter": bytes_iter, "peak_source": f"HBM copy ({src})"},
        "clocks": clk}), flush=True)


def run_prox_tv(args, device):
    """The TV prox (Algorithm 2, the workload's inner iteration count) alone on
    the workload's volume [P][Y][X][Z] (the large workload: 3 x 128 x 128 x
    96, 57 MB per dual array, beyond L2 together): time per call, and GB/s of
    algorithmic traffic at 52 B per element and inner iteration (read z, r and
    the previous u, three components each; write u and r) against the HBM
    copy peak.  The kernel also moves x between its two phases (72 B)."""
    import torch
    import paper_2510_23739_gb300 as sw

    prob = synth.workload(args.workload)
    g = synth.small_variant(prob, T=8, k=1).geom
    K = np.zeros(g.k_shape())
    K[:, 0, 0, 0] = 1.0
    op = sw.Operator(g, K, prob.sw)
    gen = torch.Generator(device=device)
    gen.manual_seed(7)
    z = 0.1 * torch.randn(g.c_shape(), generator=gen, device=device, dtype=torch.float32)
    x = torch.empty_like(z)
    tau, inner = 0.02, prob.inner
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        op.prox_tv(z, tau, inner, out=x)
    clocks = ClockSampler(_smi_id(device))
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(args.steps):
        op.prox_tv(z, tau, inner, out=x)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    op.check_device()
    op.close()
    ms = e0.elapsed_time(e1) / args.steps
    n = z.numel()
    gbs = 52.0 * n * inner / (ms * 1e-3) / 1e9
    peaks, src = _peaks()
    print(json.dumps({
        "metric": "TV prox algorithmic HBM throughput", "value": gbs, "unit": "GB/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "dtype": "f32", "data": "synthetic (seeded Gaussian volume)",
        "config": {"workload": args.workload, "volume": list(g.c_shape()), "inner_iters": inner,
                   "l2": "dual arrays 3 x 19 MB per component block, 190 MB in all (no flush)"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                     "moved_gb_per_s": 72.0 * n * inner / (ms * 1e-3) / 1e9,
                     "peak_source": f"HBM copy ({src})"},
        "clocks": clk}), flush=True)


def run_prox_sweep(args, device):
    """The proximal maps alone on a volume far beyond L2: 2 species x 1024 x
    512 x 256 (1.07 GB per array, about 8x L2).  The TV prox (Algorithm 2,
    10 inner iterations, the cooperative global-memory kernel) is charged 52
    algorithmic bytes per element and inner iteration (read z, r and the
    previous u, three components each; write u and r), the l1 prox 8 bytes
    per element (read and write in place); GB/s against the HBM copy peak."""
    import torch
    import paper_2510_23739_gb300 as sw
    from synth import Geometry, Switching

    g = Geometry(X=512, Y=1024, Z=256, T=8, N=1, P=2, k=1, pulses_per_cycle=1)
    K = np.zeros(g.k_shape())
    K[:, 0, 0, 0] = 1.0
    op = sw.Operator(g, K, Switching((0.0, 0.0), (0.0, 0.0), (1.0, 1.0), 0.0))
    gen = torch.Generator(device=device)
    gen.manual_seed(5)
    z = 0.1 * torch.randn(g.c_shape(), generator=gen, device=device, dtype=torch.float32)
    x = torch.empty_like(z)
    tau, inner = 0.02, 10
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        op.prox_tv(z, tau, inner, out=x)
        op.prox_l1(x, 1e-3)
    clocks = ClockSampler(_smi_id(device))
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.profiler.start()
    ev[0].record(stream)
    for _ in range(args.steps):
        op.prox_tv(z, tau, inner, out=x)
    ev[1].record(stream)
    ev[2].record(stream)
    for _ in range(args.steps):
        op.prox_l1(x, 1e-3)
    ev[3].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    op.check_device()
    op.close()
    n = z.numel()
    tv_ms = ev[0].elapsed_time(ev[1]) / args.steps
    l1_ms = ev[2].elapsed_time(ev[3]) / args.steps
    peaks, src = _peaks()
    tv_gbs = 52.0 * n * inner / (tv_ms * 1e-3) / 1e9
    l1_gbs = 8.0 * n / (l1_ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "TV prox algorithmic HBM throughput", "value": tv_gbs, "unit": "GB/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32", "data": "synthetic (seeded Gaussian volume)",
        "config": {"workload": "prox_sweep_2x1024x512x256", "inner_iters": inner,
                   "bytes_per_array": 4 * n, "l2": "arrays about 8x L2 (no flush)"},
        "roofline": {"bound": "hbm", "achieved": tv_gbs, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": tv_gbs / peaks["hbm_gbs"], "traffic": None,
                     "avg_launch_ms": tv_ms, "peak_source": f"HBM copy ({src})"},
        "prox_l1": {"ms": l1_ms, "gb_per_s": l1_gbs, "frac": l1_gbs / peaks["hbm_gbs"]},
        "clocks": clk}), flush=True)



def _gap_trace(op, ev_op, y, params, iters, every, stream):
    """Step a FISTA solve for `iters` iterations; every `every` iterations
    read the iterate and evaluate F on the FP32 evaluator handle.  Returns
    [(iteration, solve ms so far, F)]: the solve time is the CUDA-event time
    of the FISTA steps alone, the evaluations stay outside it."""
    import torch
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    op.fista_init(y, params)
    trace, done, ms = [], 0, 0.0
    c = None
    while done < iters:
        n = min(every, iters - done)
        torch.cuda.synchronize()
        s0.record(stream)
        op.fista_step(n)
        s1.record(stream)
        torch.cuda.synchronize()
        ms += s0.elapsed_time(s1)
        done += n
        c = op.fista_get(c)
        F, _ = ev_op.objective(c, y, params.lambda_l1, params.lambda_tv)
        trace.append((done, ms, F))
    return trace


def run_objective_gap(args, device):
    """Time to a relative objective gap (F(c_k) - F*)/F* of the one-step
    problem (Eq. one-step, l1 + TV) on the workload: the refined BF16 solve
    (the bench default), the FP32-class solve (two-term BF16, every gradient
    exact), plain BF16 and, with `--gap-fp32-iters`, plain FP32 on the CUDA
    cores.  F is evaluated every `--gap-every` iterations in
    FP32 (CUDA-core operator, FP64 sums) on a separate handle; F* is the
    lowest F seen in any run (the FP32-class solve runs `--gap-ref-iters`
    iterations, twice the compared runs' length by default)."""
    import torch
    import paper_2510_23739_gb300 as sw

    prob = workload_problem(args.workload, args.kernel)
    g = prob.geom
    op, K, c_true, y = make_problem(prob, seed=0, device=device, kernel=args.kernel)
    L = op.lipschitz(args.power_iters)
    alpha = 1.0 / L
    ev_op = sw.Operator(g, K, prob.sw)  # FP32 evaluator
    stream = torch.cuda.current_stream()
    iters, every = args.gap_iters, args.gap_every
    ref_iters = args.gap_ref_iters or 2 * iters
    base = dict(step=alpha, lambda_l1=prob.lam_l1, lambda_tv=prob.lam_tv, inner_iters=prob.inner)
    runs = {}
    clocks = ClockSampler(_smi_id(device))
    clocks.start()
    op.set_precision("bf16")
    runs["refined_bf16"] = _gap_trace(
        op, ev_op, y, sw.SolveParams(max_iters=iters, refine_every=25, refine_precision="bf16x3",
                                     refine_budget=0.1, **base), iters, every, stream)
    plain = args.gap_plain_iters or iters
    runs["plain_bf16"] = _gap_trace(op, ev_op, y, sw.SolveParams(max_iters=plain, **base),
                                    plain, every, stream)
    if args.gap_fp32_iters:
        op.set_precision("fp32")
        runs["plain_fp32"] = _gap_trace(op, ev_op, y,
                                        sw.SolveParams(max_iters=args.gap_fp32_iters, **base),
                                        args.gap_fp32_iters, every, stream)
    op.set_precision("bf16x3")
    runs["fp32_class_bf16x3"] = _gap_trace(op, ev_op, y, sw.SolveParams(max_iters=ref_iters,
                                                                        **base),
                                           ref_iters, every, stream)
    clk = clocks.stop()
    op.check_device()
    op.close()
    ev_op.close()
    Fstar = min(F for tr in runs.values() for _, _, F in tr)
    levels = (1e-3, 1e-4, 1e-5)
    out = {}
    for name, tr in runs.items():
        reach = {}
        for lv in levels:
            hit = next(((it, ms) for it, ms, F in tr if (F - Fstar) / abs(Fstar) <= lv), None)
            reach[f"{lv:g}"] = ({"iterations": hit[0], "seconds": hit[1] / 1e3}
                                if hit else None)
        last_it, last_ms, last_F = tr[-1]
        out[name] = {"reached": reach, "final_gap": (last_F - Fstar) / abs(Fstar),
                     "iterations": last_it, "ms_per_iteration": last_ms / last_it,
                     "trace_every_4th": [(it, round(ms, 1), (F - Fstar) / abs(Fstar))
                                         for it, ms, F in tr[::4]]}
    me_t = out["refined_bf16"]["reached"]["1e-05"]

    def speedup(name):
        ref_t = out[name]["reached"]["1e-05"] if name in out else None
        return (ref_t["seconds"] / me_t["seconds"]) if ref_t and me_t else None
    print(json.dumps({
        "metric": "seconds to 1e-5 relative objective gap, refined BF16 solve",
        "value": me_t["seconds"] if me_t else None, "unit": "s", "higher_is_better": False,
        "n_gpus": 1, "dtype": "bf16 + refinement (bf16x3 resync)",
        "data": "synthetic (seeded tube phantom, transducer kernel, 20 dB noise)",
        "config": {"workload": args.workload, "kernel": args.kernel, "eval_every": every,
                   "compared_iterations": iters, "reference_iterations": ref_iters,
                   "plain_bf16_iterations": plain,
                   "objective_evaluator": "FP32 CUDA-core operator, FP64 sums"},
        "F_star": Fstar, "speedup_vs_fp32_class_to_1e-5": speedup("fp32_class_bf16x3"),
        "speedup_vs_plain_fp32_to_1e-5": speedup("plain_fp32"), "runs": out,
        "clocks": clk}), flush=True)


def replace_iters(params, iters):
    import copy
    p = copy.copy(params)
    p.max_iters = iters
    return p


def run_batch(args, device):
    """Sixteen independent problems of uneven size (scan 32^2..128^2, depths
    48-128, T 128-512, 20-80 pulses, 2-3 species, supports 11-31; seeded):
    aggregate FISTA iterations per second of the batched step (one CUDA graph
    per iteration, a stream per problem) against the same batch with the
    contractions as shared persistent launches over all problems' tile-states,
    the same problems stepped one after another at the same precision, and
    plain FP32 one after another (a few iterations per problem, the
    per-iteration cost being constant)."""
    import torch
    import paper_2510_23739_gb300 as sw

    probs = synth.batch_shapes(16, 0)
    ops, ys, params = [], [], []
    refine = schedule_params(args)
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
    torch.cuda.profiler.start()
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    batch_ms = e0.elapsed_time(e1)
    launches = ops[0].launch_count() - launches0
    batch.close()
    # the same batch with the contractions as shared launches over all problems
    for op, y, prm in zip(ops, ys, params):
        op.fista_init(y, prm)
    batch = sw.Batch(ops, shared=True)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    shared_ms = e0.elapsed_time(e1)
    shared = batch.shared_in_use()
    shared_launches = batch.contraction_launches()
    batch.close()
    # the same problems one after another (each handle's own graph)
    for op, y, prm in zip(ops, ys, params):
        op.fista_init(y, prm)
        op.fista_step(args.warmup)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    e0.record(stream)
    for op in ops:
        op.fista_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
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
        "shared_launch_it_s": n * args.steps / (shared_ms / 1e3) if shared else None,
        "shared_launch_contractions_per_path": shared_launches,
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


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    return platform.processor() or platform.machine()


_ORACLE_INPUTS = {}


def _oracle_inputs(prob, kernel: str):
    """Kernel, iterate and a full measurement-sized array for the oracle
    (cached per workload; the measurement array is the data the adjoint
    reads)."""
    key = (prob.name, kernel)
    if key not in _ORACLE_INPUTS:
        import oracle
        g = prob.geom
        K = (oracle.semicircle_kernel(*semicircle_args(g)) if kernel == "semicircle"
             else synth.transducer_kernel(g, seed=0))
        c = synth.tube_phantom(g, prob.tubes, seed=0)
        # the sums' cost does not depend on the values: a constant array of
        # the measurements' size stands in for them (drawing 5e8 Gaussian
        # numbers would cost more than the sample timed)
        y = np.full(g.y_shape(), 0.01)
        _ORACLE_INPUTS[key] = (K, c, y)
    return _ORACLE_INPUTS[key]


def oracle_iteration_sample(prob, frac_fwd: float, frac_adj: float, kernel: str = "aperture",
                            prox: bool = True):
    """The FP64 oracle on a bounded sample of one FISTA iteration,
    extrapolated to the whole iteration: H on a fraction `frac_fwd` of the
    measurement rows (n, y, x, all t), H^T on a fraction `frac_adj` of the
    concentration entries (p, y, x, j), each scaled by the inverse fraction
    (every row / entry is a sum of the same length), plus the TV + l1 prox of
    one species' volume scaled by the species count (the species' proxes are
    independent and equal in cost).  Returns (ms per iteration, description,
    threads)."""
    import oracle

    g = prob.geom
    K, c, y = _oracle_inputs(prob, kernel)
    rng = np.random.default_rng(3)
    n_rows = g.N * g.Y * g.X
    n_ent = g.P * g.Y * g.X * g.Z
    rf = max(1, int(round(frac_fwd * n_rows)))
    ra = max(1, int(round(frac_adj * n_ent)))
    nyx = np.stack([rng.integers(0, g.N, rf), rng.integers(0, g.Y, rf),
                    rng.integers(0, g.X, rf)], axis=1)
    pyxj = np.stack([rng.integers(0, g.P, ra), rng.integers(0, g.Y, ra),
                     rng.integers(0, g.X, ra), rng.integers(0, g.Z, ra)], axis=1)
    t0 = time.perf_counter()
    oracle.forward_at(g, prob.sw, K, c, nyx)
    t1 = time.perf_counter()
    oracle.adjoint_at(g, prob.sw, K, y, pyxj)
    t2 = time.perf_counter()
    if prox:
        oracle.prox(c[:1], 1e-3, prob.lam_l1, prob.lam_tv, prob.inner)
    t3 = time.perf_counter()
    ms = ((t1 - t0) * n_rows / rf + (t2 - t1) * n_ent / ra + (t3 - t2) * g.P) * 1e3
    sample = (f"extrapolated: H on {rf} of {n_rows} measurement rows ({100.0 * rf / n_rows:.3g}%), "
              f"H^T on {ra} of {n_ent} entries ({100.0 * ra / n_ent:.3g}%), each scaled to all; "
              + (f"TV+l1 prox ({prob.inner} inner) of one species x {g.P}" if prox else "no prox"))
    return ms, sample, oracle.num_threads()


def cpu_baseline(prob, kernel: str, frac_fwd: float, frac_adj: float):
    """The oracle's FISTA iteration rate on the host cores (all threads), its
    single-thread rate on a smaller sample, and the CPU model."""
    import oracle

    ms, sample, cores = oracle_iteration_sample(prob, frac_fwd, frac_adj, kernel)
    oracle.set_threads(1)
    try:
        ms1, sample1, _ = oracle_iteration_sample(prob, frac_fwd / 32, frac_adj / 32, kernel)
    finally:
        oracle.set_threads(cores)
    return {"value": 1000.0 / ms, "unit": "it/s", "cores": cores, "kind": "oracle",
            "sample": sample, "cpu_model": cpu_model(),
            "single_thread": {"value": 1000.0 / ms1, "unit": "it/s", "sample": sample1}}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, each step a bounded sample of
    one FISTA iteration extrapolated to the whole workload."""
    prob = workload_problem(args.workload, args.kernel)
    times = []
    sample = ""
    cores = 1
    for i in range(args.warmup + args.steps):
        ms, sample, cores = oracle_iteration_sample(prob, args.ref_frac_fwd, args.ref_frac_adj,
                                                    args.kernel)
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
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: one resync period of the refined solve, "
                         "refine_every iterations, else 20)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="swopt", choices=["swopt", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="bf16",
                    choices=["fp32", "bf16", "bf16x3", "bf16x6", "fp8"])
    ap.add_argument("--method", default="one-step",
                    choices=["one-step", "two-step", "prox-joint", "prox-sweep", "prox-tv",
                             "objective-gap"],
                    help="two-step: time swopt_two_step against the one-step solve (FP32); "
                         "prox-joint: time the prox of the full R3 (lambda_3 term); "
                         "prox-sweep: the TV and l1 proxes on a volume 8x larger than L2; "
                         "prox-tv: the TV prox on the workload's volume; "
                         "objective-gap: time to a relative objective gap per precision")
    ap.add_argument("--kernel", default="aperture", choices=["aperture", "semicircle"],
                    help="per-depth kernel: the aperture-point transducer model, or the "
                         "paper-literal SPR on discrete half spheres (matched time grid)")
    ap.add_argument("--refine", type=int, default=None,
                    help="refined solve: exact gradient at least every R iterations (0: off; "
                         "default 25 for bf16, else 0)")
    ap.add_argument("--refine-precision", default="bf16x3", choices=["fp32", "bf16x3", "bf16x6"])
    ap.add_argument("--refine-budget", type=float, default=None,
                    help="refined solve: also resync when the relative steps since the last "
                         "exact gradient add up to this (0: off; default 0.1)")
    ap.add_argument("--presolve", type=int, default=None,
                    help="untimed FISTA iterations before the warm-up (the timed iterations "
                         "are taken in the solve's steady phase; default 200 for the refined "
                         "solve, else 0)")
    ap.add_argument("--power-iters", type=int, default=50)
    ap.add_argument("--fp32-iters", type=int, default=2,
                    help="iterations timed for the plain FP32 speed comparison")
    ap.add_argument("--cpu-frac-fwd", type=float, default=None,
                    help="fraction of H rows the CPU baseline evaluates (default 1%%, 0.2%% on "
                         "the large workload)")
    ap.add_argument("--cpu-frac-adj", type=float, default=None,
                    help="fraction of H^T entries the CPU baseline evaluates (default 1%%, "
                         "0.05%% on the large workload)")
    ap.add_argument("--ref-frac-fwd", type=float, default=None)
    ap.add_argument("--ref-frac-adj", type=float, default=None)
    ap.add_argument("--gap-iters", type=int, default=3000,
                    help="objective-gap: iterations of the compared solves")
    ap.add_argument("--gap-every", type=int, default=50,
                    help="objective-gap: iterations between objective evaluations")
    ap.add_argument("--gap-ref-iters", type=int, default=0,
                    help="objective-gap: iterations of the FP32-class solve (default 2x)")
    ap.add_argument("--gap-fp32-iters", type=int, default=0,
                    help="objective-gap: iterations of a plain FP32 (CUDA-core) solve (0: none)")
    ap.add_argument("--gap-plain-iters", type=int, default=0,
                    help="objective-gap: iterations of the plain BF16 solve (default: "
                         "--gap-iters)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.refine is None:
        args.refine = 25 if args.precision == "bf16" else 0
    if args.steps is None:
        # a whole resync period: the timed iterations hold the schedule's average
        # share of exact gradients
        args.steps = args.refine if args.refine > 0 and args.method == "one-step" else 20
    if args.refine_budget is None:
        args.refine_budget = 0.1 if args.refine > 0 else 0.0
    if args.presolve is None:
        args.presolve = 200 if args.refine > 0 else 0
    large = args.workload.startswith("large")
    if args.cpu_frac_fwd is None:
        args.cpu_frac_fwd = 0.002 if large else 0.01
    if args.cpu_frac_adj is None:
        args.cpu_frac_adj = 0.0005 if large else 0.01
    if args.ref_frac_fwd is None:
        args.ref_frac_fwd = 0.0002 if large else 0.002
    if args.ref_frac_adj is None:
        args.ref_frac_adj = 0.00005 if large else 0.002

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
    single = {"prox-joint": run_prox_joint, "two-step": run_two_step,
              "prox-sweep": run_prox_sweep, "prox-tv": run_prox_tv,
              "objective-gap": run_objective_gap}
    if args.method in single or args.workload == "batch16":
        if rank == 0:
            (run_batch if args.workload == "batch16" else single[args.method])(args, device)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    res = run_swopt(args, rank, world, device)

    total_ms, e2e_ms, value, _ = combine_ranks(res["total_ms"], res["e2e_ms"], args.steps, world,
                                               device)
    e2e_value = world * res["e2e_iters"] / (e2e_ms / 1e3)

    if rank == 0:
        peaks, peak_src = _peaks()
        ms_step = total_ms / args.steps
        dom = res["dom"]
        avg_ms = res["avg_ms"][dom]
        achieved = res["flops"] / (avg_ms * 1e-3) / 1e12
        clk = res["clocks"]
        prec_dom = args.precision if dom < 2 else args.refine_precision
        issued_tflops = res["issued"][dom % 2] / (avg_ms * 1e-3) / 1e12 if dom < 2 else None
        if prec_dom == "fp32":
            # FP32 FMA on the CUDA cores: 152 SMs x 128 lanes x 2 FLOP x max SM clock
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound, peak_note = "alu", f"FP32 FMA peak at {peaks.get('sm_max_mhz', 2070.0):g} MHz"
        elif prec_dom == "bf16":
            peak = peaks["bf16_tflops"]
            bound, peak_note = "tensor", f"bf16 dense burst ({peak_src})"
        elif prec_dom == "fp8":
            # the measured BF16 burst times the nominal FP8 / BF16 ratio (4.5 / 2.25)
            peak = peaks["bf16_tflops"] * 2
            bound, peak_note = "tensor", f"bf16 dense burst x 2, nominal fp8 ratio ({peak_src})"
        elif prec_dom == "bf16x6":
            # each useful multiply-add costs 6 BF16 multiply-adds (three-term split)
            peak = peaks["bf16_tflops"] / 6
            bound, peak_note = "tensor", f"bf16 dense burst / 6 products ({peak_src})"
        else:
            # each useful multiply-add costs 3 BF16 multiply-adds (two-term split)
            peak = peaks["bf16_tflops"] / 3
            bound, peak_note = "tensor", f"bf16 dense burst / 3 products ({peak_src})"
        kname = ["A_forward", "AT_adjoint"][dom % 2]
        traffic = _profiled_traffic(kname, args.workload) if args.kernel == "aperture" else None
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(workload_problem(args.workload, args.kernel), args.kernel,
                               args.cpu_frac_fwd, args.cpu_frac_adj)
        refine = schedule_params(args)
        t0_, t1_ = res["timed_iters"]
        line = {
            "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3 (2-term split)",
                      "bf16x6": "bf16x6 (3-term split)",
                      "fp8": "fp8 e4m3 (per-depth equilibration)"}[args.precision] + (f" + refinement (exact {args.refine_precision} gradient at "
                                   f"least every {args.refine} iterations, budget "
                                   f"{args.refine_budget:g})" if refine else ""),
            "data": "synthetic (seeded tube phantom, transducer kernel, 20 dB noise)",
            "config": {"workload": args.workload, "kernel": args.kernel,
                       "precision": args.precision, **refine,
                       "timed_iterations": f"{t0_}..{t1_} of the solve ({args.presolve} "
                                           f"untimed before the {args.warmup} warm-up)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "time_window": res["info"], "inner_iters": 10},
            "roofline": {"bound": bound, "kernel": kname + ("" if dom < 2 else " (resync)"),
                         "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "avg_launch_ms": avg_ms, "flops_per_launch": res["flops"],
                         "peak_source": peak_note,
                         "frac_of_sustained": achieved / (peak * peaks["bf16_tflops_sustained"]
                                                          / peaks["bf16_tflops"])
                         if bound == "tensor" else None,
                         "issued_tflops": issued_tflops,
                         # every executed MMA against the BF16 (FP8: 2x) dense rate
                         "issued_frac_of_peak": (issued_tflops / (peaks["bf16_tflops"] *
                                                                  (2 if prec_dom == "fp8" else 1))
                                                 if issued_tflops else None),
                         "kernel_avg_ms": {"A": res["avg_ms"][0], "AT": res["avg_ms"][1],
                                           "A_resync": res["avg_ms"][2],
                                           "AT_resync": res["avg_ms"][3]},
                         "kernel_launches": {k: res["kinfo"][i]["launches"] for i, k in
                                             enumerate(["A", "AT", "A_resync", "AT_resync"])}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "it/s",
                    "h2d_bytes_per_step": res["h2d"] / res["e2e_iters"],
                    "d2h_bytes_per_step": res["d2h"] / res["e2e_iters"],
                    "note": f"one whole swopt solve of {res['e2e_iters']} iterations (set-up, "
                            f"early phase included) from pinned host y to host c"},
            "gpu_launches": res["launches"],
            "clocks": clk,
            "early_phase": res["early"],
        }
        if refine:
            line["refinement"] = {"exact_gradients_in_timed_iterations": res["timed_resyncs"],
                                  "timed_iterations": args.steps}
        if res["op_err"]:
            line["operator_error_vs_fp64_oracle"] = res["op_err"]
        if "fp32" in res:
            f = res["fp32"]
            line["precision_path"] = {
                "fp32_plain_it_s": 1000.0 / f["ms_per_step"],
                "speedup_vs_fp32_plain": (value / world) / (1000.0 / f["ms_per_step"]),
                "objective_rel_diff_vs_bf16x3_solve": abs(f["F"] - f["F_ref"]) / abs(f["F_ref"]),
                "iterate_rel_diff_vs_bf16x3_solve": f["c_rel_diff"],
                "iterations_compared": f["iters"],
                "note": "plain FP32 = CUDA-core FMA operators (speed); the comparison solve "
                        "runs every gradient exactly in two-term BF16 (FP32-class) for the "
                        "same iterations; objectives both evaluated with the FP32 operator "
                        "and FP64 sums"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
