#!/usr/bin/env python
"""Benchmark: beam-splitter MPO updates/s of the U(1) MPO mesh on GB300.

One step = one pass of the whole hot path over one batch of synthetic input: the
state is restored to the lossy squeezed initial MPO (device copy) and the whole
Clements mesh is applied (every gate: bookkeeping, Fock tables, Theta contraction,
Gram, eigensolver, keep-chi selection, re-split with entropy), then the final phase
screen.  The mesh is a plan (gate list resident in HBM, captured in a CUDA graph).
`value` = gates applied per second of device time (CUDA events on the library's
stream), L2 flushed by a 512 MiB write before every timed step (not timed).
`e2e` = the same metric through mpo_sweep_mesh with host buffers (pinned staging,
gate list H2D and per-gate discarded weights D2H inside the timed region).

--impl reference times the FP64 CPU oracle (the reference of this build) on a
bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): replicas only -- every rank runs its own instance(s), no
collective on the data path; value = all ranks' gates / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beam-splitter MPO updates/s at (M,d,chi); mixed vs FP64 at stated observable error"
DEFAULT_WORKLOAD = "M48_d8_chi512"
# nominal figures, used only when the live measurement (mpo_measure_peaks) fails
FP64_PEAK_TFLOPS = 1.25   # 152 SMs x 2.07 GHz x ~4 flop/clk
FP32_PEAK_TFLOPS = 80.5   # 152 SMs x 2.07 GHz x 128 FMA (256 flop) per clock
ORACLE_SAMPLE_GATES = {"exact_M4_d4": 6, "M16_d6_chi64": 120, "M32_d8_chi256": 12,
                       "batched_64x_M16_d6": 60, "M48_d8_chi512": 24}
# tensor-pipe passes per real product of the contraction kernel, by path
MMA_PASSES = {"mixed_tf32": 3, "mixed_bf16": 1}
# DRAM bytes of one launch of the dominant kernel, from an ncu capture of the same
# kernel code on the same workload (dram__bytes_read.sum + dram__bytes_write.sum);
# to be retaken whenever the kernel changes
TRAFFIC = {}


def measured_peaks() -> dict:
    """FP64/FP32 FMA and TF32/BF16 tcgen05 peaks of this GPU, measured now (best of
    three), with MEASURED_PEAKS.json's measured HBM and cuBLAS bf16 beside."""
    import paper_2301_12814_gb300 as lib
    out = {"source": "mpo_measure_peaks (FMA chains; tcgen05.mma on smem operands), best of 3"}
    try:
        runs = [lib.mpo.measure_peaks() for _ in range(3)]
        for k in ("fp64", "fp32", "tf32", "bf16"):
            out[k] = max(r[k] for r in runs)
    except Exception as e:  # never lose the line over the probe
        out.update(fp64=FP64_PEAK_TFLOPS, fp32=FP32_PEAK_TFLOPS, tf32=None, bf16=None,
                   source=f"nominal (probe failed: {str(e)[-120:]})")
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        out["hbm_gbs"] = mp.get("hbm_gbs")
        out["bf16_cublas"] = mp.get("bf16_tflops")
    except (OSError, ValueError):
        pass
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        t0, t1 = (self.marks + [0, 0])[:2] if len(self.marks) >= 2 else (0, time.time())
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [(t, l) for t, l in self.lines if t0 - 0.25 <= t <= t1 + 0.25] or self.lines[-3:]
        for _, l in rows:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(name: str, n_gates: int, repeats: int = 1, threads: int = 1) -> dict:
    """The oracle on the first n_gates gates, in a child process whose BLAS/OpenMP
    thread count is pinned to `threads`."""
    env = dict(os.environ)
    t = str(int(threads))
    env.update(OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-m", "oracle.timing", name, str(n_gates), str(repeats)],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def workload_arrays(wl, rank: int, gates: int = 0):
    """(instances, meshes) for this rank; batched workloads shift their seeds by rank.
    gates > 0 keeps each mesh's first `gates` gates (and drops its phase screen): a
    prefix of the workload, the small case for profiler captures."""
    import gbs_workloads as w
    if wl.batch > 1 and rank > 0:
        wl = w.batched_instances(n=wl.batch, first_seed=100 + rank * wl.batch)
    meshes = [wl.mesh(i) for i in range(wl.batch)]
    if gates > 0:
        meshes = [w.Mesh(m.M, m.k[:gates], m.theta[:gates], m.phi[:gates], np.zeros(m.M))
                  if gates < m.n_gates else m for m in meshes]
    return wl, meshes


def aggregate_value(units: int, ms: float, ws: int, device) -> float:
    """Whole-job updates/s: every rank processed `units` updates; the job took the
    slowest rank's `ms` (max over ranks)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ws * units / (ms / 1e3)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import gbs_workloads as w
    wl = w.workload(args.workload)
    n = ORACLE_SAMPLE_GATES.get(args.workload, 12)
    res = oracle_sample(args.workload, n, repeats=args.warmup + args.steps)
    t = res["seconds"][args.warmup:] or res["seconds"]
    ms = 1e3 * float(np.mean(t))
    val = n / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "M": wl.M, "d": wl.d, "chi": wl.chi, "instances": 1,
                   "sample_gates": n},
        "cpu_baseline": {"value": val, "unit": "updates/s", "cores": res["cores"], "kind": "oracle",
                         "sample": f"first {n} gates of instance 0's mesh from the initial state, per step"},
        "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def observable_errors(a, b) -> dict:
    """Largest error of run a against run b per observable: <n>, <n^2> relative,
    S (bits) and Tr absolute, per-gate discarded weight relative to the largest."""
    tr_a, n1_a, n2_a, S_a, d_a = a
    tr_b, n1_b, n2_b, S_b, d_b = b
    rel = lambda x, y: float(np.max(np.abs(x - y) / np.maximum(np.abs(y), 1e-300)))
    return {"n_rel": rel(n1_a, n1_b), "n2_rel": rel(n2_a, n2_b), "S_abs": float(np.max(np.abs(S_a - S_b))),
            "tr_abs": float(np.max(np.abs(tr_a - tr_b))),
            "eps_rel": float(np.max(np.abs(d_a - d_b)) / max(float(np.max(np.abs(d_b))), 1e-300))}


def compare_precision(args, wl, n_gates, k, th, ph, fp, obs, stream, other, peaks, tuning=None):
    """The same workload on another path: its updates/s (graph replays timed with
    CUDA events, a few steps), its per-stage device times, the observable errors of
    the mixed run against the FP64 run, and the tensor-pipe roofline of its
    contraction kernel (F_Theta flops of Eq. `theta` / its device time)."""
    import torch
    import paper_2301_12814_gb300 as lib
    G = lib.MPO(wl.M, wl.d, wl.r, wl.eta, chi_max=wl.chis, batch=wl.batch, precision=other, stream=stream)
    if tuning:
        G.set_tuning(**tuning)
    choices = G.get_tuning()
    plan = G.plan_mesh(n_gates, k, th, ph, fp)
    G.reset(); plan.run()
    steps = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    live = {s_: 0.0 for s_ in lib.mpo.Plan.STAGES}
    for _ in range(steps):
        G.reset()
        e0.record(stream); plan.run(); e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        for s_, v in plan.stage_times().items():
            live[s_] += v / steps
    disc = plan.discarded()
    tr, n1, n2 = G.observables()
    S, _, _ = G.operator_entropy()
    G.reset()
    prof, jac = plan.profile(with_jacobi=True)
    G.close()
    out = {"precision": other, "tuning": choices, "value": int(sum(n_gates)) * steps / (ms / 1e3),
           "unit": "updates/s", "steps": steps, "stages_ms": {s_: round(v, 4) for s_, v in live.items()}}
    if other != "fp64":
        out["mixed_vs_fp64"] = observable_errors((tr, n1, n2, S, disc), obs)
        fth = jac["theta_F_flops"]
        t_ms = live["theta"]
        tc_form = choices["theta_form"] == 2 or (choices["theta_form"] == 0 and other == "mixed_bf16")
        if tc_form:
            peak = peaks.get("tf32" if other == "mixed_tf32" else "bf16")
            ach = fth / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
            passes = MMA_PASSES.get(other, 1)
            out["contraction_roofline"] = {
                "kernel": "k_theta_tc", "bound": "tensor", "unit": "TFLOP/s",
                "algorithmic_flops_per_step": fth, "achieved": ach, "peak": peak,
                "frac": ach / peak if peak else None,
                "tensor_pipe_frac": passes * ach / peak if peak else None,
                "mma_passes": passes,
                "peak_source": f"{'TF32' if other == 'mixed_tf32' else 'BF16'} tcgen05 peak measured in this run",
                "note": "frac = F_Theta / stage time / peak; tensor_pipe_frac counts the MMA passes of the "
                        "split (3xTF32: 3 products per real product), not the padding of partial tiles"}
        else:
            fl = prof["theta"][2]  # the executed two-stage form's flops
            ach = fl / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
            out["contraction_roofline"] = {
                "kernel": "k_theta", "bound": "alu", "unit": "TFLOP/s", "executed_flops_per_step": fl,
                "F_theta_flops_per_step": fth, "achieved": ach, "peak": peaks["fp32"],
                "frac": ach / peaks["fp32"], "peak_source": "FP32 FMA-chain peak measured in this run"}
        out["jacobi"] = {"cluster_blocks": jac["cluster_blocks"],
                         "cluster_ms_per_block": jac["cluster_cycles"] / max(1, jac["cluster_blocks"]) / 2.07e6,
                         "cluster_ms_split": {k_: jac[f"cluster_{k_}_cycles"] / max(1, jac["cluster_blocks"]) / 2.07e6
                                              for k_ in ("seed", "ns", "polish")}}
    return out


def run_native(args, ws, rank, local):
    import torch
    import gbs_workloads as w
    import paper_2301_12814_gb300 as lib
    from paper_2301_12814_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl0 = w.workload(args.workload)
    wl, meshes = workload_arrays(wl0, rank, args.gates)
    prec = args.precision or wl.precision
    if prec not in lib.mpo.PRECISIONS:
        prec = "fp64"
    n_gates = [m.n_gates for m in meshes]
    k = np.concatenate([m.k for m in meshes]).astype(np.int32)
    th = np.concatenate([m.theta for m in meshes])
    ph = np.concatenate([m.phi for m in meshes])
    fp = np.concatenate([m.final_phase for m in meshes])
    units = int(sum(n_gates))
    stream = torch.cuda.Stream(device=dev)
    peaks = measured_peaks()
    G = lib.MPO(wl.M, wl.d, wl.r, wl.eta, chi_max=wl.chis, batch=wl.batch, precision=prec, stream=stream)
    tuning = {"autotuned": False, "choices": G.get_tuning()}
    if args.autotune:
        from paper_2301_12814_gb300 import autotune as at
        res = at.autotune(G, n_gates, k, th, ph, fp, precision=prec)
        tuning = {"autotuned": True, "choices": res["best"], "best_ms_per_mesh": res["best_ms"],
                  "default_ms_per_mesh": res["default_ms"], "candidates": len(res["table"]),
                  "fastest": [(round(ms_, 3), c_) for ms_, c_ in res["table"][:4]],
                  "method": "grid over the launch choices; stage device times of plan replays, best of 2"}
    plan = G.plan_mesh(n_gates, k, th, ph, fp)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        G.reset(); plan.run()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.6)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    live = {s: 0.0 for s in lib.mpo.Plan.STAGES}
    barrier()
    clocks.mark()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        G.reset()
        plan.run()
        ev[i][1].record(stream)
        # per-stage device times of this replay, from the event nodes inside the graph
        # (reading them synchronises the host after the step's last event)
        for s_, v in plan.stage_times().items():
            live[s_] += v
    barrier()
    wall = time.perf_counter() - wall0
    clocks.mark()
    time.sleep(0.3)
    clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = float(np.sum(step_ms))
    value = aggregate_value(units * args.steps, tot_ms, ws, dev)
    if ws > 1:
        tot_ms = ws * units * args.steps / value * 1e3
    disc = plan.discarded()

    # per-stage breakdown and algorithmic flops: one instrumented replay (not timed above)
    G.reset()
    prof, jac = plan.profile(with_jacobi=True)
    # end to end through the public API with host buffers
    e2e_t = []
    for i in range(max(1, min(args.steps, 2))):
        t0 = time.perf_counter()
        G.reset()
        d_host = G.sweep_mesh(n_gates, k, th, ph, fp)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = aggregate_value(units, 1e3 * float(np.mean(e2e_t)), ws, dev)
    assert np.array_equal(d_host, disc), "sweep and plan disagree"
    tr, n1, n2 = G.observables()
    S, pur, smax = G.operator_entropy()
    G.close()

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    # roofline on the dominant kernel of the timed replays; its arithmetic pipe sets the
    # peak (SIMT FP64 or FP32).  Durations: graph event nodes around each launch over the
    # timed steps; flops: the executed form's counted flops from one instrumented replay
    # (identical work: same mesh, same state, deterministic).
    live_step = {s_: v / args.steps for s_, v in live.items()}
    stage = max(("theta", "gram", "svd", "resplit"), key=lambda s_: live_step[s_])
    _, nl_s, fl_s = prof[stage]
    ms_s = live_step[stage]
    fp64_stage = prec == "fp64" and stage in ("theta", "svd")
    fl32 = 0.0
    if stage == "svd" and prec == "fp64":
        fl_s = jac["refine_flops"]  # the FP64 part; the FP32 seed is reported beside it
        fl32 = jac["seed_flops"]
    peak = peaks["fp64"] if fp64_stage else peaks["fp32"]
    achieved = fl_s / (ms_s / 1e3) / 1e12 if ms_s > 0 else 0.0
    roofline = {"bound": "alu", "kernel": f"k_{stage}", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": ("FP64" if fp64_stage else "FP32") + " FMA-chain peak measured in this run "
                               "(mpo_measure_peaks)" + (
                                   "; the counted flops are the FP64-accurate refinement's (run in double-float "
                                   "arithmetic on the FP32 pipe), so frac compares with doing that work on the "
                                   "FP64 pipe" if fp64_stage and stage == "svd" else ""),
                "traffic": TRAFFIC.get((args.workload, prec, f"k_{stage}"), (None,))[0] if not args.gates else None,
                "traffic_source": TRAFFIC.get((args.workload, prec, f"k_{stage}"), (None, None))[1]
                if not args.gates else None,
                "flops_per_launch": fl_s / max(1, nl_s),
                "avg_launch_ms": ms_s / max(1, nl_s), "launches_per_step": nl_s,
                "timing": "CUDA event record nodes inside the replayed graph, timed steps only"}
    if fl32 > 0:
        # both pipes the kernel uses: the time the FP64 refinement and the FP32 seed
        # would take at their measured peaks, against the kernel's time
        roofline["fp32_seed_flops_per_launch"] = fl32 / max(1, nl_s)
        roofline["two_pipe_frac"] = (fl_s / (peaks["fp64"] * 1e12) + fl32 / (peaks["fp32"] * 1e12)) / (ms_s / 1e3)
    compare = None
    if not args.no_compare:
        # the mixed paths with their default launch choices, and the TF32 path with its
        # contraction on the tensor cores (3xTF32) for the tensor-core roofline
        others = ([("mixed_tf32", None), ("mixed_tf32", {"theta_form": 2}), ("mixed_bf16", None)]
                  if prec == "fp64" else [("fp64", None)])
        compare = [compare_precision(args, wl, n_gates, k, th, ph, fp, (tr, n1, n2, S, disc), stream, o, peaks, t)
                   for o, t in others]
    # CPU oracle on a bounded sample (host cores, single BLAS thread)
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        n = ORACLE_SAMPLE_GATES.get(args.workload, 12)
        try:
            res = oracle_sample(args.workload, n)
            cpu = {"value": res["updates_per_s"][0], "unit": "updates/s", "cores": res["cores"], "kind": "oracle",
                   "sample": f"first {n} gates of instance 0's mesh from the initial state ({res['seconds'][0]:.1f} s)"}
            ncores = os.cpu_count() or 1
            if ncores > 1:
                res_all = oracle_sample(args.workload, n, threads=ncores)
                cpu["all_cores"] = {"value": res_all["updates_per_s"][0], "cores": ncores,
                                    "note": "same sample with BLAS/OpenMP threads = all host cores"}
        except Exception as e:  # the baseline is reported, never a reason to lose the GPU line
            cpu = {"value": None, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {str(e)[-200:]}"}
    h2d = 32 * units + 8 * wl.batch * wl.M
    d2h = 8 * units + 16
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "M": wl.M, "d": wl.d, "chi": wl.chi, "instances": wl.batch,
                   "gates_per_step": units, "precision": prec,
                   "mesh_prefix_gates": args.gates or None,
                   "tuning": tuning,
                   "r": float(wl.r[0, 0]), "eta": float(wl.eta[0, 0]), "seeds": wl.seeds[:4],
                   "l2": "flushed: 512 MiB write before each timed step (untimed)",
                   "svd_cluster": lib.mpo.svd_cluster_shape(),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": plan.launches * args.steps,
        "clocks": clocks.summary(),
        "compare": compare,
        "stages_ms": {s_: round(v, 4) for s_, v in live_step.items()},
        "stages_gflop": {s: round(v[2] / 1e9, 4) for s, v in prof.items() if v[2] > 0},
        "theta_F_gflop": round(jac["theta_F_flops"] / 1e9, 4),
        "peaks_tflops": peaks,
        "jacobi": {"blocks": jac["blocks"], "sweeps_per_block": jac["sweeps"] / max(1, jac["blocks"]),
                   "refine_sweeps_per_block": jac["refine_sweeps"] / max(1, jac["blocks"]),
                   "seed_gflop_fp32": jac["seed_flops"] / 1e9, "refine_gflop": jac["refine_flops"] / 1e9,
                   "cluster_blocks": jac["cluster_blocks"],
                   "cluster_ms_per_block": jac["cluster_cycles"] / max(1, jac["cluster_blocks"]) / 2.07e6,
                   "cta_ms_per_block": jac["cta_cycles"] / max(1, jac["blocks"] - jac["cluster_blocks"]
                                                                - jac["warp_blocks"]) / 2.07e6,
                   "warp_blocks": jac["warp_blocks"],
                   "warp_ms_per_block": jac["warp_cycles"] / max(1, jac["warp_blocks"]) / 2.07e6,
                   "cluster_ms_split": {k: jac[f"cluster_{k}_cycles"] / max(1, jac["cluster_blocks"]) / 2.07e6
                                        for k in ("seed", "ns", "polish")}},
        "wall_s": wall,
        "observables": {"trace": float(tr[0]), "discarded_sum": float(np.sum(disc[:n_gates[0]])),
                        "S_max": float(smax[0])},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


ASYM_WORKLOAD = "asymptotic_fig1"
ASYM_METRIC = "App. C asymptotic operator-EE estimates/s over the Fig. 1 grid (r=0.88, n_max=8)"


def oracle_asymptotic(n_points: int, repeats: int = 1) -> dict:
    env = dict(os.environ)
    env.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-m", "oracle.timing", "asymptotic", str(n_points), str(repeats)],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def asym_flops(n_max: int, sweeps: np.ndarray) -> float:
    """Algorithmic FP64 flops of the block Jacobi.  A block of nb columns has
    nb (nb - 1) / 2 column pairs.  In every sweep each pair costs 6 nb flops for its
    three dot products (3 FMAs per row).  A rotation costs 6 nb more (per row, two
    products and two FMAs); every pair is counted as rotated in every sweep but the
    last, which by definition rotates nothing -- an upper bound on the rotations of
    the earlier sweeps, since pairs that are already orthogonal skip theirs."""
    L = n_max + 1
    E = n_max // 2 + 1
    O = L - E
    nbs = [E * (E + 1) // 2 + O * (O + 1) // 2, E * O, E * (E - 1) // 2 + O * (O - 1) // 2, E * O]
    sw = sweeps.reshape(-1, 4)
    tot = 0.0
    for j, nb in enumerate(nbs):
        pairs = nb * (nb - 1) / 2
        tot += float(np.sum(sw[:, j] * pairs * 6 * nb + np.maximum(sw[:, j] - 1, 0) * pairs * 6 * nb))
    return tot


def run_asymptotic(args, ws, rank, local):
    """The App. C estimator over the Fig. 1 grid: one step = every grid point's
    mode spectrum and entropies (two kernel launches on device-resident inputs)."""
    import gbs_workloads as w
    g = w.asymptotic_grid()
    npts = g.size
    if args.impl == "reference":
        if rank != 0:
            return
        res = oracle_asymptotic(npts, repeats=args.warmup + args.steps)
        t = res["seconds"][args.warmup:] or res["seconds"]
        ms = 1e3 * float(np.mean(t))
        val = npts / (ms / 1e3)
        line = {"impl": "reference", "metric": ASYM_METRIC, "value": val, "unit": "estimates/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": g.name, "points": npts, "r": g.r, "n_max": g.n_max},
                "cpu_baseline": {"value": val, "unit": "estimates/s", "cores": res["cores"], "kind": "oracle",
                                 "sample": f"the whole grid ({npts} points) per step"},
                "e2e": {"value": val, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import torch
    import paper_2301_12814_gb300 as lib
    from paper_2301_12814_gb300 import build as libbuild, experiments as ex
    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mu = ex.transmission(g.N, g.beta, g.gamma)
    K = (g.n_max + 1) ** 2
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        t_r = torch.full((npts,), g.r, dtype=torch.float64, device=dev)
        t_mu = torch.tensor(mu, dtype=torch.float64, device=dev)
        t_th = torch.full((npts,), math.pi / 4, dtype=torch.float64, device=dev)
        S1 = torch.empty(npts, dtype=torch.float64, device=dev)
        spec = torch.empty(npts * K, dtype=torch.float64, device=dev)
        sw = torch.zeros(4 * npts, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    call = lambda: lib.mpo.asymptotic_ee_device(t_r, t_mu, t_th, g.n_max, S1, spec, sweeps=sw, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        call()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.6)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    clocks.mark()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        call()
        ev[i][1].record(stream)
    barrier()
    clocks.mark()
    time.sleep(0.3)
    clocks.stop()
    tot_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    value = aggregate_value(npts * args.steps, tot_ms, ws, dev)
    if ws > 1:
        tot_ms = ws * npts * args.steps / value * 1e3
    S_dev = S1.cpu().numpy() * g.N
    sweeps = sw.cpu().numpy()
    # end to end through the public API: host arrays in, host entropies out
    e2e_t = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        S_host = ex.asymptotic_ee(g.N, g.beta, g.gamma, g.r, g.n_max)["S1"]
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = aggregate_value(npts, 1e3 * float(np.mean(e2e_t)), ws, dev)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    ms_step = tot_ms / args.steps
    fl = asym_flops(g.n_max, sweeps)
    achieved = fl / (ms_step / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_asym_block (+ k_asym_finalize)", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "FP64 SIMT FMA peak derived from 152 SMs x 2.07 GHz x 4 flop/clk/SM; "
                               "MEASURED_PEAKS.json has only HBM and bf16 tensor peaks",
                "traffic": None, "flops_per_launch": fl, "avg_launch_ms": ms_step,
                "timing": "CUDA events around the two launches of each timed step"}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        try:
            res = oracle_asymptotic(npts)
            err = float(np.max(np.abs(np.asarray(res["S"]) - S_dev) / np.maximum(np.abs(S_dev), 1e-300)))
            cpu = {"value": res["points_per_s"][0], "unit": "estimates/s", "cores": res["cores"],
                   "kind": "oracle", "sample": f"the whole grid ({npts} points, {res['seconds'][0]:.1f} s)",
                   "max_rel_diff_vs_gpu": err}
        except Exception as e:
            cpu = {"value": None, "unit": "estimates/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {str(e)[-200:]}"}
    line = {
        "metric": ASYM_METRIC, "value": value, "unit": "estimates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": g.name, "points": npts, "r": g.r, "n_max": g.n_max,
                   "gamma": [0.25, 0.5, 1.0], "beta": [0.25, 0.5, 0.75, 1.0],
                   "N_range": [float(g.N.min()), float(g.N.max())],
                   "l2": "flushed: 512 MiB write before each timed step (untimed)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "estimates/s", "h2d_bytes_per_step": 24 * npts,
                "d2h_bytes_per_step": 8 * npts + 16 * npts},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks.summary(),
        "jacobi": {"sweeps_mean": float(sweeps.mean()), "sweeps_max": int(sweeps.max())},
        "host_equals_device": bool(np.array_equal(S_host, S_dev)),
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="fp64",
                    help="path timed as `value` (fp64, mixed_tf32, mixed_bf16); the others go to `compare`")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the handle's launch choices by timing candidates first (recorded in config)")
    ap.add_argument("--gates", type=int, default=0,
                    help="run only each mesh's first GATES gates (a prefix, for profiler captures)")
    ap.add_argument("--no-compare", action="store_true", help="skip the run on the other precision")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = _dist()
    if args.workload == ASYM_WORKLOAD:
        run_asymptotic(args, ws, rank, local)
    elif args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_native(args, ws, rank, local)


if __name__ == "__main__":
    main()
