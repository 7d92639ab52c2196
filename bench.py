#!/usr/bin/env python
"""Benchmark of the fJOFC in-sample hot path on GB300.

One step = one ``fjofc_embed`` call on the m=2, n=5000, d=3 workload (float32 Delta,
200 Guttman transforms or relative stress change < 1e-7), i.e. every row of the hot path:
the closed-form W^-1 set-up on the host, then one persistent kernel that runs every pass
(fused all-pairs tiles, W^-1 mix/centring/stress, device-side stopping test).  Inputs are resident in HBM when the timed
region starts.  The upper triangles of Delta that a pass reads (100 MB) fit in L2, so L2
is flushed (256 MB write) before every timed step, outside that step's CUDA events.

Output: one JSON line (rank 0).  ``value`` = Guttman pair-updates/s summed over all
ranks, with pair-updates per transform = m*C(n,2) + C(m,2)*n (the distances of
Remark faststress).  Extra keys: roofline of the all-pairs kernel (algorithmic bytes of
the upper triangles of Delta / measured device time of the kernel, against the measured
HBM copy bandwidth), the CPU oracle timed on a bounded sample, an end-to-end figure
through the public API with host buffers, clocks sampled during the timed region.

``--impl reference`` times the float64 CPU oracle (the dense Algorithm 1) instead, on a
bounded sample of the same workload; with several ranks only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(k=1, m=2, n=5000, d=3, max_iter=200, tol=1e-7, tol_mode="relative")
CPU_SAMPLE = dict(n=1000, iters=30)


def aggregate_ranks(dist, device, elapsed_ms, work):
    """Whole-job figures of independent replicas: the slowest rank's time (max over
    ranks) and the work of all ranks (sum).  ``dist`` None: one process."""
    if dist is None:
        return float(elapsed_ms), float(work)
    import torch
    t = torch.tensor([float(elapsed_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], device=device, dtype=torch.float64)
    dist.all_reduce(w)
    return float(t.item()), float(w.item())


def pairs_per_transform(m, n):
    return m * n * (n - 1) // 2 + (m * (m - 1) // 2) * n


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in ("paper_1502_03391_gb300/csrc/k_guttman_pass.cuh", "paper_1502_03391_gb300/csrc/fjofc_device.cuh",
                "paper_1502_03391_gb300/csrc/k_embed_persistent.cuh", "paper_1502_03391_gb300/csrc/k_apply_common.cuh",
                "paper_1502_03391_gb300/csrc/kp_d01_04.cu"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the all-pairs kernel from the committed ncu summary, if it
    was captured on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "k_embed_persistent_workload1.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    msha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    mtr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not msha or not mtr or msha.group(1) != kernel_source_sha():
        return None
    return float(mtr.group(1))


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- oracle arm

def oracle_rate(n, iters, seed_rep=0):
    """Pair-updates/s of the float64 dense oracle (Algorithm 1 with pinv) on a workload-1
    shaped sample of n objects."""
    import numpy as np
    import synthetic
    from oracle import fjofc_oracle as O
    prob = synthetic.make_insample(WORKLOAD["k"], n=n, rep=seed_rep)
    t0 = time.perf_counter()
    res = O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=iters)
    dt = time.perf_counter() - t0
    return pairs_per_transform(WORKLOAD["m"], n) * res.iters / dt, dt


# transforms of the float64 C Algorithm 2 timed per step (a bounded sample of the
# workload's 200)
CPU_TRANSFORMS = 20
# transforms of the cpu_baseline leg: the whole workload (200), a few seconds on the host
CPU_BASELINE_TRANSFORMS = 200


def cpu_fjofc_rate(deltas, W, X0, transforms):
    """Pair-updates/s of the float64 C Algorithm 2 (oracle/fjofc_cpu.c, every host core)
    on the full workload: ``transforms`` Guttman transforms from X0."""
    from oracle import fjofc_cpu as C
    m, n = len(deltas), deltas[0].shape[0]
    t0 = time.perf_counter()
    _, it, _ = C.cpu_embed(deltas, W, X0, transforms)
    dt = time.perf_counter() - t0
    return pairs_per_transform(m, n) * it / dt, dt, C.threads()


def host_problem():
    """Workload 1 on the host in float64 (Delta rounded to float32 first, as the device
    path stores it)."""
    import numpy as np
    import synthetic
    prob = synthetic.make_insample(WORKLOAD["k"])
    deltas = [np.asarray(D, np.float32).astype(np.float64) for D in prob.deltas]
    return prob, deltas, np.asarray(prob.X0, np.float32).astype(np.float64)


def run_reference(args, rank, world):
    if rank != 0:
        return
    prob, deltas, X0 = host_problem()
    from oracle import fjofc_cpu as C
    C.build()
    for _ in range(args.warmup):
        cpu_fjofc_rate(deltas, prob.W, X0, 1)
    times = []
    threads = 1
    for _ in range(args.steps):
        _, dt, threads = cpu_fjofc_rate(deltas, prob.W, X0, CPU_TRANSFORMS)
        times.append(dt)
    m, n = WORKLOAD["m"], WORKLOAD["n"]
    value = args.steps * CPU_TRANSFORMS * pairs_per_transform(m, n) / sum(times)
    sample = (f"float64 Algorithm 2 in C (oracle/fjofc_cpu.c, OpenMP on {threads} threads) on the full workload "
              f"(m={m}, n={n}, d={WORKLOAD['d']}), {CPU_TRANSFORMS} of its 200 transforms per step")
    line = {
        "impl": "reference", "metric": "Guttman pair-updates/s", "value": value, "unit": "pair-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "insample-m2-n5000-d3", "sample": sample, "m": m, "n": n, "d": WORKLOAD["d"],
                   "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": "pair-updates/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "pair-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm

def make_device_problem(torch, fj, seed_rep, device):
    import numpy as np
    import synthetic
    prob = synthetic.make_insample(WORKLOAD["k"], rep=seed_rep, with_deltas=False)
    deltas = []
    for Fi in prob.F:
        buf = fj.empty_delta(prob.spec.n, torch.float32, device)
        buf.copy_(synthetic.torch_distances(Fi, device, torch.float32))
        deltas.append(buf)
    X0 = torch.as_tensor(np.asarray(prob.X0, np.float32), device=device).contiguous()
    return prob, deltas, X0


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj

    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    m, n, d = WORKLOAD["m"], WORKLOAD["n"], WORKLOAD["d"]
    prob, deltas, X0 = make_device_problem(torch, fj, rank, device)
    X = torch.empty_like(X0)
    stream = torch.cuda.current_stream(device)

    def step(profile=True):
        X.copy_(X0)
        return fj.embed(deltas, prob.W, X, max_iter=WORKLOAD["max_iter"], tol=WORKLOAD["tol"],
                        tol_mode=WORKLOAD["tol_mode"], history=False, profile=2 if profile else 0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # Delta's upper triangles (the bytes a pass reads, 100 MB) fit in L2: flush L2 before
    # every timed step by writing a 256 MB buffer, outside the step's own events
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    iters, ms_pass, passes, launches = 0, 0.0, 0, 0
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        barrier()
        for s_i in range(args.steps):
            flush.fill_(float(s_i))
            step_ev[s_i][0].record(stream)
            r = step()
            step_ev[s_i][1].record(stream)
            iters += r.iters
            ms_pass += r.ms_pass
            passes += r.passes
            launches += r.launches
        barrier()
    elapsed_ms, total_iters = aggregate_ranks(dist, device, sum(a.elapsed_time(b) for a, b in step_ev), iters)
    ppt = pairs_per_transform(m, n)
    value = ppt * total_iters / (elapsed_ms / 1e3)

    # roofline of the dominant kernel, the persistent loop kernel (one launch per step):
    # algorithmic bytes = the strict upper triangles of Delta, once per all-pairs pass
    alg_bytes = m * n * (n - 1) // 2 * 4
    passes_per_launch = passes / max(args.steps, 1)
    avg_launch_ms = ms_pass / max(args.steps, 1)
    alg_per_launch = alg_bytes * passes_per_launch
    achieved = alg_per_launch / (avg_launch_ms / 1e3) / 1e9
    peaks, src = measured_peaks()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(),
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6.8 TB/s",
            "kernel": "k_embed_persistent<3,float> (all passes of one fjofc_embed call)",
            "algorithmic_bytes_per_launch": alg_per_launch, "algorithmic_bytes_per_pass": alg_bytes,
            "passes_per_launch": passes_per_launch, "avg_launch_ms": avg_launch_ms, "launches_timed": args.steps}

    # end to end through the public API with host buffers (pinned): Delta and X0 in, X and
    # the stress out, every step
    e2e = None
    if not args.no_e2e:
        hostD = [dd.cpu().pin_memory() for dd in deltas]
        hostX0 = X0.cpu().pin_memory()
        hostX = torch.empty_like(hostX0).pin_memory()
        devD = [torch.empty_like(dd) for dd in deltas]
        for _ in range(2):
            for a, b in zip(devD, hostD):
                a.copy_(b, non_blocking=True)
            X.copy_(hostX0, non_blocking=True)
            fj.embed(devD, prob.W, X, max_iter=WORKLOAD["max_iter"], tol=WORKLOAD["tol"], tol_mode=WORKLOAD["tol_mode"],
                     history=False)
            hostX.copy_(X, non_blocking=True)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it2 = 0
        for _ in range(args.steps):
            for a, b in zip(devD, hostD):
                a.copy_(b, non_blocking=True)
            X.copy_(hostX0, non_blocking=True)
            r = fj.embed(devD, prob.W, X, max_iter=WORKLOAD["max_iter"], tol=WORKLOAD["tol"],
                         tol_mode=WORKLOAD["tol_mode"], history=False)
            hostX.copy_(X, non_blocking=True)
            it2 += r.iters
        e1.record(stream)
        barrier()
        ems, it2 = aggregate_ranks(dist, device, e0.elapsed_time(e1), it2)
        h2d = sum(dd.numel() * dd.element_size() for dd in hostD) + hostX0.numel() * 4
        e2e = {"value": ppt * it2 / (ems / 1e3), "unit": "pair-updates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(hostX.numel() * 4 + 8 + 4)}

    cpu = cpu_dense = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        hostD = [dd.double().cpu().numpy() for dd in deltas]         # the same float32 inputs
        v, dt, thr = cpu_fjofc_rate(hostD, prob.W, X0.double().cpu().numpy(), CPU_BASELINE_TRANSFORMS)
        cpu = {"value": v, "unit": "pair-updates/s", "cores": thr, "kind": "oracle",
               "sample": f"float64 Algorithm 2 in C (oracle/fjofc_cpu.c, OpenMP) on the same inputs (m={m}, n={n}, "
                         f"d={d}), all {CPU_BASELINE_TRANSFORMS} transforms of the workload, {dt:.1f} s",
               "same_config": True}
        del hostD
        v, dt = oracle_rate(CPU_SAMPLE["n"], CPU_SAMPLE["iters"])
        cpu_dense = {"value": v, "unit": "pair-updates/s", "cores": os.cpu_count(), "kind": "oracle",
                     "sample": f"dense float64 Algorithm 1 (pinv + dense B(X)) on n={CPU_SAMPLE['n']} objects of the "
                               f"same generator (mn={2 * CPU_SAMPLE['n']}), {CPU_SAMPLE['iters']} transforms, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": "Guttman pair-updates/s", "value": value, "unit": "pair-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "insample-m2-n5000-d3: fjofc_embed, float32 Delta, 200 transforms or relative "
                                   "stress change < 1e-7", "m": m, "n": n, "d": d,
                       "transforms_per_step": total_iters / args.steps / world,
                       "l2": "L2 flushed before every timed step (256 MB write outside the step's events); "
                             "Delta 200 MB stored, 100 MB (upper triangles) read per pass",
                       "parallelism": f"{world} independent replica(s)"},
            "hbm_gbs_step": alg_bytes * total_iters / (elapsed_ms / 1e3) / 1e9,
            "roofline": roof, "cpu_baseline": cpu, "cpu_dense_oracle": cpu_dense, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------- other forms

ALU_LANES_PER_SM = 128          # float32 lanes per SM (4 sub-partitions x 32)


def alu_peak(sm_mhz):
    """float32 lane-operations per second: SMs x 128 lanes x SM clock (FMA counted once)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * ALU_LANES_PER_SM * sm_mhz * 1e6, sms


def _timed(torch, stream, fn, steps, flush):
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    outs = []
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        outs.append(fn())
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs], outs


def run_precision(args, rank, world, local_rank):
    """m=3, n=20000, d=10: the float32-Delta path against float16 and bfloat16 storage (Delta
    divided by s_l = max(Delta_l)/2^10), each iterated to relative stress change < 1e-7 (at
    most 300 transforms) from the same X0; every final configuration is re-scored with the
    float32 Delta.  value = pair-updates/s of the float16 path."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    prob = synthetic.make_insample(2, rep=rank, with_deltas=False, n=args.n or None)
    m, n, d = prob.spec.m, prob.spec.n, prob.spec.d
    cap = args.max_iter or 300
    dev = {"f32": [], "f16": [], "bf16": []}
    scales = {"f32": None, "f16": [], "bf16": []}
    for Fi in prob.F:
        full = synthetic.torch_distances(Fi, device, torch.float32)
        s = float(full.max().item()) / 1024.0
        for key, dt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
            buf = fj.empty_delta(n, dt, device)
            buf.copy_(full if key == "f32" else (full / s).to(dt))
            dev[key].append(buf)
            if key != "f32":
                scales[key].append(s)
        del full
    X0 = torch.as_tensor(np.asarray(prob.X0, np.float32), device=device)
    X = torch.empty_like(X0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    ppt = pairs_per_transform(m, n)
    forms = {}
    with ClockSampler(local_rank) as clk:
        for key in ("f32", "f16", "bf16"):
            def step():
                X.copy_(X0)
                return fj.embed(dev[key], prob.W, X, max_iter=cap, tol=1e-7, tol_mode="relative", history=False,
                                delta_scale=scales[key], profile=2)
            for _ in range(args.warmup):
                step()
            ms, outs = _timed(torch, stream, step, args.steps, flush)
            final = fj.stress(dev["f32"], prob.W, X)
            iters = sum(r.iters for r in outs)
            forms[key] = {"ms_to_tol": sum(ms) / len(ms), "transforms": iters / len(outs),
                          "pair_updates_per_s": ppt * iters / (sum(ms) / 1e3),
                          "kernel_ms": sum(r.ms_pass for r in outs) / len(outs),
                          "final_stress_f32_delta": final, "stress_own_delta": outs[-1].stress}
    clocks = clk.summary()
    ref = forms["f32"]["final_stress_f32_delta"]
    for key in forms:
        forms[key]["final_stress_rel_to_f32"] = (forms[key]["final_stress_f32_delta"] - ref) / ref
    f16 = forms["f16"]
    passes = f16["transforms"] + 1
    ops = (4 * d + 3) * m * n * (n - 1) / 2 * passes
    peak, sms = alu_peak(clocks["sm_max_mhz"] or 2070.0)
    achieved = ops / (f16["kernel_ms"] / 1e3)
    peaks, src = measured_peaks()
    bytes_pass = m * n * (n - 1) // 2 * 2
    if rank == 0:
        line = {
            "metric": "Guttman pair-updates/s", "value": f16["pair_updates_per_s"], "unit": "pair-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f16["ms_to_tol"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 Delta, f32 math",
            "data": "synthetic",
            "config": {"workload": "precision-m3-n20000-d10: fjofc_embed to relative stress change < 1e-7 "
                                   "(max 300), Delta float16 / bfloat16 / float32", "m": m, "n": n, "d": d,
                       "l2": "L2 flushed before every timed step"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T lane-op/s",
                         "frac": achieved / peak,
                         "peak_source": f"{sms} SMs x 128 float32 lanes x {clocks['sm_max_mhz'] or 2070.0} MHz",
                         "ops_per_pair": 4 * d + 3, "kernel": "k_embed_persistent<10,__half>",
                         "hbm_achieved_gbs": bytes_pass * passes / (f16["kernel_ms"] / 1e3) / 1e9,
                         "hbm_peak_gbs": peaks["hbm_gbs"], "traffic": None},
            "forms": forms, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def run_relaxed(args, rank, world, local_rank):
    """Relaxed updates on the in-sample workload m=2, n=5000, d=3 (float32 Delta): the plain
    Guttman transform (relax 1) against relax 1.9 and 2.0, each iterated from the same X0 to
    a relative stress change < 1e-6 (at most 3000 transforms).  value = time to that
    tolerance with relax 1.9 (lower is better); every form's final stress is reported."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    m, n, d = WORKLOAD["m"], WORKLOAD["n"], WORKLOAD["d"]
    prob, deltas, X0 = make_device_problem(torch, fj, rank, device)
    X = torch.empty_like(X0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    cap, tol = args.max_iter or 3000, 1e-6
    forms = {}
    with ClockSampler(local_rank) as clk:
        for relax in (1.0, 1.9, 2.0):
            def step():
                X.copy_(X0)
                return fj.embed(deltas, prob.W, X, max_iter=cap, tol=tol, tol_mode="relative", history=False,
                                relax=relax, profile=2)
            for _ in range(args.warmup):
                step()
            ms, outs = _timed(torch, stream, step, args.steps, flush)
            iters = sum(r.iters for r in outs) / len(outs)
            forms[str(relax)] = {"ms_to_tol": sum(ms) / len(ms), "transforms": iters,
                                 "final_stress": outs[-1].stress, "status": outs[-1].status,
                                 "us_per_pass": 1e3 * sum(r.ms_pass for r in outs) / sum(r.passes for r in outs)}
    base = forms["1.0"]
    for key in forms:
        forms[key]["speedup_vs_plain"] = base["ms_to_tol"] / forms[key]["ms_to_tol"]
        forms[key]["final_stress_rel_to_plain"] = (forms[key]["final_stress"] - base["final_stress"]) / base["final_stress"]
    if rank == 0:
        line = {
            "metric": "time to relative stress change < 1e-6", "value": forms["1.9"]["ms_to_tol"], "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms["1.9"]["ms_to_tol"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "relaxed-m2-n5000-d3: fjofc_embed with relax 1 / 1.9 / 2 to relative stress "
                                   f"change < {tol} (max {cap})", "m": m, "n": n, "d": d,
                       "l2": "L2 flushed before every timed step"},
            "forms": forms, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_paper(args, rank, world, local_rank):
    """The paper's run-time experiment (Sec. 4.3), synthetic from its own generator
    (Y ~ N((5,5), I_2), modality i = Y + U(-z/50, z/50) jitter, Delta_i its distances;
    Eq. W with w = 0.5, d = 2, X0 seeded N(0, I)): time per Guttman transform of
    fjofc_embed (100 transforms per call) for m = 2..6 at n = 400 and for n = 200..1000
    at m = 3, beside the float64 dense Algorithm 1 of the oracle (JOFC with an explicit
    pseudoinverse, timed per transform after its pinv, on the host cores; 3 transforms).
    value = GPU transforms per second at m = 6, n = 400."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    rows = []
    cases = [(m, 400) for m in (2, 3, 4, 5, 6)] + [(3, n) for n in (200, 600, 800, 1000)]
    with ClockSampler(local_rank) as clk:
        for m, n in cases:
            deltas = synthetic.paper_jitter_modalities(n=n, m=m, dim=2, seed=4300 + 10 * m + n)
            W = synthetic.weights_matrix(m, 1.0, 0.5)
            X0n = np.random.default_rng(4400 + m + n).standard_normal((m * n, 2))
            dev = [fj.to_device_delta(D) for D in deltas]
            X0 = torch.as_tensor(np.asarray(X0n, np.float32), device=device)
            X = torch.empty_like(X0)

            def step():
                X.copy_(X0)
                return fj.embed(dev, W, X, max_iter=100, history=False, profile=2)
            for _ in range(args.warmup):
                step()
            ms, outs = _timed(torch, stream, step, args.steps, flush)
            us_gpu = 1e3 * sum(ms) / sum(r.iters for r in outs)
            us_kernel = 1e3 * sum(r.ms_pass for r in outs) / sum(r.passes for r in outs)
            # Algorithm 2's initialisation (classical MDS + Procrustes) on the device
            fj.init_cmds(dev, 2, X=X)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, init_iters = fj.init_cmds(dev, 2, X=X)
            torch.cuda.synchronize()
            init_ms = (time.perf_counter() - t0) * 1e3
            row = {"m": m, "n": n, "gpu_us_per_transform": us_gpu, "kernel_us_per_pass": us_kernel,
                   "init_ms": init_ms, "init_subspace_iterations": init_iters}
            if rank == 0 and not args.no_cpu_baseline:
                from oracle import fjofc_oracle as O
                Wo = O.omnibus_weights(W, n)
                Do = O.omnibus_dissimilarity(deltas)
                Lp = O.pseudoinverse(O.laplacian(Wo))
                Xc = X0n.copy()
                t0 = time.perf_counter()
                for _ in range(3):
                    Xc = O.guttman_step(Xc, Lp, Wo, Do)
                row["oracle_ms_per_transform"] = (time.perf_counter() - t0) / 3 * 1e3
                row["oracle_over_gpu"] = row["oracle_ms_per_transform"] * 1e3 / us_gpu
                t0 = time.perf_counter()
                X0_ref = O.initial_configuration(deltas, 2)
                row["oracle_init_ms"] = (time.perf_counter() - t0) * 1e3
                row["init_rel_diff_to_oracle"] = float(np.linalg.norm(X.cpu().numpy() - X0_ref) / np.linalg.norm(X0_ref))
            rows.append(row)
    if rank == 0:
        top = [r for r in rows if r["m"] == 6][0]
        line = {
            "metric": "Guttman transforms/s (paper-shaped workload, m=6, n=400, d=2)",
            "value": 1e6 / top["gpu_us_per_transform"], "unit": "transforms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["gpu_us_per_transform"] * 100 / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (the paper's Sec. 4.3 generator)",
            "config": {"workload": "paper-4.3: m = 2..6 at n = 400 and n = 200..1000 at m = 3, d = 2, Eq. W "
                                   "w = 0.5, 100 transforms per call", "cpu_cores": os.cpu_count()},
            "cases": rows, "clocks": clk.summary(),
            "paper_context": "the paper's per-iteration JOFC/fJOFC ratios (serial CPU): 2.86-10.71 for m = 2..6, "
                             "2.10-12.63 for n = 200..1000",
        }
        print(json.dumps(line), flush=True)


def _loglog_slope(xs, ys):
    """Least-squares slope of log(y) against log(x) (None for fewer than two sizes)."""
    import numpy as np
    if len(set(xs)) < 2:
        return None
    return float(np.polyfit(np.log(np.asarray(xs, float)), np.log(np.asarray(ys, float)), 1)[0])


def held_out_rows(m, n):
    """Mask over the m*n modality-major rows of a configuration: False at the last
    object (row j*n + n-1) of every modality j."""
    import numpy as np
    keep = np.ones(m * n, dtype=bool)
    keep[n - 1::n] = False
    return keep


def procrustes_rotation(A, B):
    """The orthogonal R minimising ||A R - B||_F (from the SVD of A'B)."""
    import numpy as np
    U, _, Vt = np.linalg.svd(np.asarray(A, np.float64).T @ np.asarray(B, np.float64))
    return U @ Vt


def run_paper_oos(args, rank, world, local_rank):
    """The paper's out-of-sample experiment (Sec. 4.4) with its Sec. 4.3 generator in three
    dimensions (d = 3, Eq. W with w = 0.5): Algorithm 2 in-sample (fjofc_init_cmds, then
    fjofc_embed) on all n objects and on the first n - 1, then the n-th object's m views
    out-of-sample against the (n-1)-object configuration (fjofc_oos, k = 1, seeded
    N(0, I) start).  Every solve runs to the paper's normalised tolerance (decrease of
    sigma / #pairs below 1e-6, Remark eps).  The paper varies m = 10..30 at n = 200 and
    n = 200..600 at m = 10; here m = 2..30 at n = 200 and n = 200..600 at m = 10.  Reports
    the in-sample and out-of-sample times, the residual
    of Table 2 (sum over modalities of |X^(i)[n] - y_i|) as computed and after the
    orthogonal Procrustes fit of the (n-1)-object configuration onto the full one (the
    paper does not say how the two frames are matched), the out-of-sample result against
    the oracle's closed-form loop run for the same number of iterations from the same
    start, and log-log slopes of time over m and n.  value = out-of-sample embeddings
    per second at m = 10, n = 600."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    d, tol, mode = 3, 1e-6, "abs_normalized"
    cap = args.max_iter or 2000
    cases = [(m, 200) for m in (2, 4, 6, 8, 10, 15, 20, 25, 30)] + [(10, n) for n in (300, 400, 500, 600)]
    if args.paper_case:
        cases = [tuple(int(v) for v in args.paper_case.split(","))]
    rows = []
    with ClockSampler(local_rank) as clk:
        for m, n in cases:
            deltas = synthetic.paper_jitter_modalities(n=n, m=m, dim=3, seed=4500 + 10 * m + n)
            W = synthetic.weights_matrix(m, 1.0, 0.5)
            y0 = np.random.default_rng(4700 + m + n).standard_normal((1, m, d)).astype(np.float32)
            keep = held_out_rows(m, n)
            full = [fj.to_device_delta(D) for D in deltas]
            part = [fj.to_device_delta(np.ascontiguousarray(D[:n - 1, :n - 1])) for D in deltas]
            dnew = fj.empty_oos_delta(1, m, n - 1, torch.float32, device)
            for j in range(m):
                dnew[0, j].copy_(torch.as_tensor(deltas[j][n - 1, :n - 1].astype(np.float32), device=device))
            Y0 = torch.as_tensor(y0, device=device)
            Xf = torch.empty((m * n, d), dtype=torch.float32, device=device)
            Xp = torch.empty((m * (n - 1), d), dtype=torch.float32, device=device)
            Y = torch.empty_like(Y0)
            it_oos = torch.zeros(1, dtype=torch.int32, device=device)

            def step_full():
                fj.init_cmds(full, d, X=Xf)
                return fj.embed(full, W, Xf, max_iter=cap, tol=tol, tol_mode=mode, history=False).iters

            def step_part():
                fj.init_cmds(part, d, X=Xp)
                return fj.embed(part, W, Xp, max_iter=cap, tol=tol, tol_mode=mode, history=False).iters

            def step_oos():
                Y.copy_(Y0)
                fj.oos(Xp, dnew, W, Y, max_iter=cap, tol=tol, tol_mode=mode, iters_out=it_oos)
                return 0

            for fn in (step_full, step_part, step_oos):
                for _ in range(args.warmup):
                    fn()
            ms_full, it_full = _timed(torch, stream, step_full, args.steps, flush)
            ms_part, it_part = _timed(torch, stream, step_part, args.steps, flush)
            ms_oos, _ = _timed(torch, stream, step_oos, args.steps, flush)
            k_oos = int(it_oos.item())
            Xf_h = Xf.cpu().numpy().astype(np.float64).reshape(m, n, d)
            Xp_h = Xp.cpu().numpy().astype(np.float64)
            Y_h = Y.cpu().numpy().astype(np.float64)[0]
            Xk = Xf_h.reshape(m * n, d)[keep]
            R = procrustes_rotation(Xp_h, Xk)           # Xp R ~ Xf without object n
            row = {"m": m, "n": n,
                   "insample_ms": float(np.median(ms_full)), "insample_transforms": int(it_full[-1]),
                   "insample_minus_one_ms": float(np.median(ms_part)), "insample_minus_one_transforms": int(it_part[-1]),
                   "oos_ms": float(np.median(ms_oos)), "oos_iterations": k_oos,
                   "table2_residual": float(np.linalg.norm(Xf_h[:, n - 1, :] - Y_h, axis=1).sum()),
                   "table2_residual_aligned": float(np.linalg.norm(Xf_h[:, n - 1, :] - Y_h @ R, axis=1).sum()),
                   "insample_frames_rel_diff": float(np.linalg.norm(Xp_h @ R - Xk) / np.linalg.norm(Xk)),
                   "config_rms": float(np.sqrt(np.mean(np.sum(Xf_h ** 2, axis=2))))}
            row["insample_us_per_transform"] = 1e3 * row["insample_ms"] / max(row["insample_transforms"], 1)
            row["oos_us_per_iteration"] = 1e3 * row["oos_ms"] / max(k_oos, 1)
            if rank == 0 and not args.no_cpu_baseline:
                from oracle import fjofc_oracle as O
                dn = np.stack([deltas[j][n - 1, :n - 1].astype(np.float32).astype(np.float64) for j in range(m)])
                t0 = time.perf_counter()
                ref = O.oos_embed_closed_form(Xp_h, dn, y0[0].astype(np.float64), W, max_iter=k_oos)
                row["oracle_oos_ms"] = (time.perf_counter() - t0) * 1e3
                row["oos_rel_diff_to_oracle"] = float(np.linalg.norm(Y_h - ref.y) / np.linalg.norm(ref.y))
            rows.append(row)
    if rank == 0:
        by_m = [r for r in rows if r["n"] == 200] or rows
        by_n = [r for r in rows if r["m"] == 10] or rows
        slopes = {}
        for key in ("insample_ms", "insample_us_per_transform", "oos_ms", "oos_us_per_iteration"):
            slopes[key] = {"over_m_at_n200": _loglog_slope([r["m"] for r in by_m], [r[key] for r in by_m]),
                           "over_n_at_m10": _loglog_slope([r["n"] for r in by_n], [r[key] for r in by_n])}
        top = by_n[-1]
        line = {
            "metric": "out-of-sample embeddings/s (one held-out object, paper-shaped, m=10, n=600, d=3)",
            "value": 1e3 / top["oos_ms"], "unit": "objects/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["oos_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (the paper's Sec. 4.3 generator, 3-dimensional)",
            "config": {"workload": "paper-4.4: m = 2..30 at n = 200 and n = 200..600 at m = 10, d = 3, Eq. W "
                                   "w = 0.5, Algorithm 2 (classical MDS start), every solve to normalised "
                                   "stress decrease < 1e-6",
                       "cpu_cores": os.cpu_count()},
            "cases": rows, "loglog_slopes": slopes, "clocks": clk.summary(),
            "paper_context": "the paper reports in-sample time growing quadratically and out-of-sample time "
                             "linearly in m and n (serial CPU, Sec. 4.4)",
        }
        print(json.dumps(line), flush=True)


def run_oos(args, rank, world, local_rank):
    """Out-of-sample batch: the m=2, n=10000, d=5 in-sample configuration (200 transforms or
    relative change < 1e-7), then 100000 new objects (float32 dissimilarities to all
    in-sample objects in both modalities, 8 GB) from the standard init, each iterated to its
    own relative stress change < 1e-6 (at most 500).  value = (object, in-sample point)
    pair-updates per second: sum over objects of iterations x m n / time."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    prob = synthetic.make_insample(4, rep=rank, with_deltas=False)
    m, n, d = prob.spec.m, prob.spec.n, prob.spec.d
    deltas = []
    for Fi in prob.F:
        buf = fj.empty_delta(n, torch.float32, device)
        buf.copy_(synthetic.torch_distances(Fi, device, torch.float32))
        deltas.append(buf)
    X = torch.as_tensor(np.asarray(prob.X0, np.float32), device=device)
    fj.embed(deltas, prob.W, X, max_iter=200, tol=1e-7, tol_mode="relative", history=False)
    del deltas
    k = args.k or 100000
    F_new, _, Y0 = synthetic.make_oos_objects(prob, k, stream=2, with_deltas=False)
    dnew = fj.empty_oos_delta(k, m, n, torch.float32, device)
    for j in range(m):
        dnew[:, j, :].copy_(synthetic.torch_distances(F_new[j], device, torch.float32, G=prob.F[j]))
    Y0t = torch.as_tensor(np.asarray(Y0, np.float32), device=device).contiguous()
    Y = torch.empty_like(Y0t)
    iters = torch.zeros(k, dtype=torch.int32, device=device)
    sout = torch.zeros(k, dtype=torch.float64, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def step():
        Y.copy_(Y0t)
        fj.oos(X, dnew, prob.W, Y, max_iter=500, tol=1e-6, tol_mode="relative", iters_out=iters, stress_out=sout)
        return int(iters.sum().item())

    for _ in range(args.warmup):
        step()
    with ClockSampler(local_rank) as clk:
        ms, outs = _timed(torch, stream, step, args.steps, flush)
    clocks = clk.summary()
    total_obj_iters = sum(outs)
    secs = sum(ms) / 1e3
    value = total_obj_iters * m * n / secs
    peaks, src = measured_peaks()
    alg_bytes = total_obj_iters * m * n * 4
    peak, sms = alu_peak(clocks["sm_max_mhz"] or 2070.0)
    ops = total_obj_iters * m * n * (4 * d + 8)
    if rank == 0:
        it = iters.cpu().numpy()
        line = {
            "metric": "OOS (object, point) pair-updates/s", "value": value, "unit": "pair-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "oos-m2-n10000-d5: fjofc_oos on 100000 new objects from the standard init, "
                                   "per-object relative stress change < 1e-6 (max 500)", "k": k, "m": m, "n": n,
                       "d": d, "l2": "delta_new 8 GB > L2; L2 flushed before every timed step"},
            "iterations": {"mean": float(it.mean()), "max": int(it.max()), "min": int(it.min())},
            "roofline": {"bound": "alu", "achieved": ops / secs / 1e12, "peak": peak / 1e12, "unit": "T lane-op/s",
                         "frac": ops / secs / peak, "ops_per_pair": 4 * d + 8, "kernel": "k_oos_solve<5,float>",
                         "hbm_algorithmic_gbs": alg_bytes / secs / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                         "traffic": None},
            "mean_final_stress": float(sout.mean().item()), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def run_learned(args, rank, world, local_rank):
    """Learned warm start on the out-of-sample workload: the m=2, n=10000, d=5 configuration,
    a 512-512 GELU network (m*d outputs) trained on the method's own solutions for 20000
    held-out objects, then 100000 test objects solved to relative stress change < 1e-6
    from (a) the standard start and (b) the network's start with the per-object fallback.
    Timed per step: (a) the solve; (b) features + network + fallback choice + solve.
    value = object-solves per second of (b)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    from paper_1502_03391_gb300 import learned as L
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    prob = synthetic.make_insample(4, rep=rank, with_deltas=False)
    m, n, d = prob.spec.m, prob.spec.n, prob.spec.d
    deltas = []
    for Fi in prob.F:
        buf = fj.empty_delta(n, torch.float32, device)
        buf.copy_(synthetic.torch_distances(Fi, device, torch.float32))
        deltas.append(buf)
    X = torch.as_tensor(np.asarray(prob.X0, np.float32), device=device)
    fj.embed(deltas, prob.W, X, max_iter=200, tol=1e-7, tol_mode="relative", history=False)
    inv_mean = [float(n * (n - 1)) / float(D.double().sum().item()) for D in deltas]
    del deltas
    lm = L.choose_landmarks(n, 256, seed=1)

    def objects(count, stream_id):
        F_new, _, Y0 = synthetic.make_oos_objects(prob, count, stream=stream_id, with_deltas=False)
        dn = fj.empty_oos_delta(count, m, n, torch.float32, device)
        for j in range(m):
            dn[:, j, :].copy_(synthetic.torch_distances(F_new[j], device, torch.float32, G=prob.F[j]))
        return dn, torch.as_tensor(np.asarray(Y0, np.float32), device=device).contiguous()

    def solve(dn, Y, it, st):
        fj.oos(X, dn, prob.W, Y, max_iter=500, tol=1e-6, tol_mode="relative", iters_out=it, stress_out=st)

    ntr, kte = 20000, args.k or 100000
    dtr, Ytr = objects(ntr, 1)
    itr = torch.zeros(ntr, dtype=torch.int32, device=device)
    str_ = torch.zeros(ntr, dtype=torch.float64, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solve(dtr, Ytr, itr, str_)            # the training targets: the method's own solutions
    torch.cuda.synchronize()
    targets_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    net = L.WarmStartMLP(m * len(lm), 512, m * d, seed=3, device=device)
    xtr = L.features(dtr, lm, inv_mean)
    hist = net.train(xtr, Ytr.reshape(ntr, m * d).contiguous(), epochs=40, batch=256, lr=1e-3, seed=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del dtr, xtr
    dte, Y0 = objects(kte, 2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    it = torch.zeros(kte, dtype=torch.int32, device=device)
    st = torch.zeros(kte, dtype=torch.float64, device=device)
    Y = torch.empty_like(Y0)
    res = {}

    def plain():
        Y.copy_(Y0)
        solve(dte, Y, it, st)

    def warm():
        ws = net.warm_start(X, dte, prob.W, Y0, lm, inv_mean)
        Y.copy_(ws.Y)
        solve(dte, Y, it, st)
        return ws

    with ClockSampler(local_rank) as clk:
        for name, fn in (("standard", plain), ("learned", warm)):
            for _ in range(args.warmup):
                fn()
            ms, outs = _timed(torch, stream, fn, args.steps, flush)
            res[name] = {"ms": sum(ms) / len(ms), "mean_iterations": float(it.double().mean().item()),
                         "max_iterations": int(it.max().item()), "mean_final_stress": float(st.mean().item())}
            if name == "learned":
                res[name]["warm_start_kept"] = float(outs[-1].used_warm.double().mean().item())
    clocks = clk.summary()
    ratio = res["learned"]["mean_final_stress"] / res["standard"]["mean_final_stress"] - 1.0
    if rank == 0:
        line = {
            "metric": "out-of-sample object solves/s (learned warm start)", "value": kte / (res["learned"]["ms"] / 1e3),
            "unit": "objects/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["learned"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (float16 network inputs)", "data": "synthetic",
            "config": {"workload": "learned-oos-m2-n10000-d5: 100000 new objects to relative stress change < 1e-6, "
                                   "network 512-512-512-10 GELU trained on 20000 held-out objects' solutions",
                       "k": kte, "m": m, "n": n, "d": d, "landmarks": len(lm), "train_objects": ntr,
                       "l2": "delta_new 8 GB > L2; L2 flushed before every timed step"},
            "forms": res, "speedup_vs_standard": res["standard"]["ms"] / res["learned"]["ms"],
            "final_stress_rel_to_standard": ratio, "train_seconds": train_s, "targets_seconds": targets_s,
            "one_batch_ms_including_training": res["learned"]["ms"] + 1e3 * (train_s + targets_s),
            "batches_to_recover_training": (1e3 * (train_s + targets_s)) / max(res["standard"]["ms"] - res["learned"]["ms"],
                                                                                1e-9),
            "train_loss_first_last": [float(hist[0]), float(hist[-1])], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local_rank):
    """256 independent problems, n ~ U[100, 4000], m in {2, 3}, d in {2, 3, 5}, each from the
    small workload's generator with its own seed, float32 Delta, 150 transforms each.
    (a) one autotuned plan (fjofc_plan_autotune: schedule constants chosen by timed
    probes; fjofc_plan_run: one CUDA graph) against (b) the plain path, one fjofc_embed
    call per problem in sequence; also reported: the plan whose tuner may store Delta as
    float16.  value = pair-updates/s of (a) summed over the problems; every plan's final
    configurations are re-scored with float32 Delta against the plain path's stress."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_03391_gb300 as fj
    import synthetic
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(device)
    iters = 150
    shapes = synthetic.batched_problem_shapes(args.problems or 256, seed=3000 + rank)
    probs, X0s, Xs = [], [], []
    ppt_total, bytes_pass = 0, 0
    for sh in shapes:
        prob = synthetic.make_insample(0, n=sh["n"], m=sh["m"], d=sh["d"], seed=sh["seed"], with_deltas=False)
        dev = []
        for Fi in prob.F:
            buf = fj.empty_delta(sh["n"], torch.float32, device)
            buf.copy_(synthetic.torch_distances(Fi, device, torch.float32))
            dev.append(buf)
        X0 = torch.as_tensor(np.asarray(prob.X0, np.float32), device=device).contiguous()
        probs.append((dev, prob.W))
        X0s.append(X0)
        Xs.append(X0.clone())
        ppt_total += pairs_per_transform(sh["m"], sh["n"])
        bytes_pass += sh["m"] * sh["n"] * (sh["n"] - 1) // 2 * 4
    t0 = time.perf_counter()
    plan = fj.Plan([(dv, W, X) for (dv, W), X in zip(probs, Xs)], max_iter=iters, autotune=True, probe_iters=8)
    create_s = time.perf_counter() - t0
    plan16 = fj.Plan([(dv, W, X) for (dv, W), X in zip(probs, Xs)], max_iter=iters, autotune=True, probe_iters=8,
                     allow_f16=True)
    info = plan.info()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def reset():
        for X, X0 in zip(Xs, X0s):
            X.copy_(X0)

    def run_plan():
        plan.run()

    def run_plan16():
        plan16.run()

    plain_stress = [0.0] * len(probs)

    def run_plain():
        for i, ((dv, W), X) in enumerate(zip(probs, Xs)):
            plain_stress[i] = fj.embed(dv, W, X, max_iter=iters, history=False).stress

    res = {}
    with ClockSampler(local_rank) as clk:
        for name, fn in (("plan", run_plan), ("plan_f16_allowed", run_plan16), ("plain", run_plain)):
            for _ in range(args.warmup):
                reset()
                fn()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            torch.cuda.synchronize()
            for k in range(args.steps):
                reset()
                flush.fill_(float(k))
                evs[k][0].record(stream)
                fn()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in evs]
            res[name] = {"ms": sum(ms) / len(ms)}
    clocks = clk.summary()
    # final stress of the plan's results, re-scored with the float32 Delta (the tuner may
    # have chosen float16 storage), against the plain path's
    for name, pl in (("plan", plan), ("plan_f16_allowed", plan16)):
        for X, X0 in zip(Xs, X0s):
            X.copy_(X0)
        pl.run()
        r = pl.results()
        rescored = np.array([fj.stress(dv, W, X) for (dv, W), X in zip(probs, Xs)])
        rel = np.abs(rescored - np.array(plain_stress)) / np.array(plain_stress)
        res[name]["all_status_ok"] = bool(np.all(r.status == 0))
        res[name]["final_stress_rel_to_plain_max"] = float(rel.max())
        res[name]["final_stress_rel_to_plain_mean"] = float(rel.mean())
        res[name]["tuning"] = pl.tuning
    value = ppt_total * iters / (res["plan"]["ms"] / 1e3)
    peaks, src = measured_peaks()
    achieved = bytes_pass * (iters + 1) / (res["plan"]["ms"] / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": "Guttman pair-updates/s (batched)", "value": value, "unit": "pair-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["plan"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-256: n ~ U[100,4000], m in {2,3}, d in {2,3,5}, float32 Delta, "
                                   "150 transforms each, one plan (CUDA graph)", "problems": len(shapes),
                       "l2": "L2 flushed before every timed step; Delta 14 GB in total"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "kernel": "k_embed_batched (3 classes)"},
            "forms": res, "speedup_vs_one_call_each": res["plain"]["ms"] / res["plan"]["ms"],
            "plan": {"graphed": info["graphed"], "launches": info["launches"],
                     "groups_max": int(info["groups"].max()), "multi_sm_problems": int((info["groups"] > 1).sum()),
                     "create_and_tune_s": create_s},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    plan16.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="precision workload: objects (default 20000; a smaller "
                                                       "case for profiling)")
    ap.add_argument("--max-iter", type=int, default=0, help="precision / relaxed / paper-oos workloads: "
                    "iteration cap (default 300 / 3000 / 2000)")
    ap.add_argument("--k", type=int, default=0, help="oos / learned workloads: test objects (default 100000)")
    ap.add_argument("--paper-case", default="", help="paper-oos workload: run only the case 'm,n' (e.g. 30,200)")
    ap.add_argument("--problems", type=int, default=0, help="batched workload: problems (default 256)")
    ap.add_argument("--workload", default="insample",
                    choices=["insample", "precision", "oos", "learned", "batched", "relaxed", "paper",
                             "paper-oos"],
                    help="insample: the headline line (m=2, n=5000, d=3); precision: m=3, n=20000, d=10 "
                         "with float16/bfloat16 Delta vs float32; oos: 100000 out-of-sample objects "
                         "against the m=2, n=10000, d=5 configuration; learned: the same objects from the "
                         "trained network's warm start vs the standard start; batched: 256 problems "
                         "(n ~ U[100,4000], m in {2,3}, d in {2,3,5}) in one plan vs one call each; relaxed: "
                         "the headline workload to a relative stress change of 1e-6 with relaxed updates "
                         "(relax 1.9, 2) vs the plain transform; paper: the paper's Sec. 4.3 run-time "
                         "experiment (m = 2..6, n = 200..1000) beside the dense float64 Algorithm 1; paper-oos: "
                         "its Sec. 4.4 out-of-sample experiment (one held-out object, m = 2..8, n = 200..600)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "precision":
        run_precision(args, rank, world, local_rank)
    elif args.workload == "oos":
        run_oos(args, rank, world, local_rank)
    elif args.workload == "learned":
        run_learned(args, rank, world, local_rank)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "relaxed":
        run_relaxed(args, rank, world, local_rank)
    elif args.workload == "paper":
        run_paper(args, rank, world, local_rank)
    elif args.workload == "paper-oos":
        run_paper_oos(args, rank, world, local_rank)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
