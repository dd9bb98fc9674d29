"""Throughput benchmark: JTFS forward + backward signals/sec on the B = 64, N = 2^16, Q = 16
workload (J = 12, J_fr = 4, Q_fr = 2, T = 2^12, F = 16; seeded synthetic AM/FM tones).

One step = one jtfs_forward_backward call: forward of the whole batch (inputs resident in
HBM) and backward with fixed cotangents.  Prints one JSON line.  Under torchrun each rank runs the same per-GPU batch
(weak scaling, no data-path collective); the time is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|tf32|bf16|fp32_simt]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores
  python bench.py --workload varlen ...  # uneven-length batch (1024 signals of 2^13-2^17
                                         # samples) in one graph launch vs per-signal launches
  python bench.py --workload mixed ...   # forward by contraction precision with oracle errors
  python bench.py --workload resynth ... # texture resynthesis, B = 16, N = 2^17, 50 Adam steps
  python bench.py --workload eq5 ...     # the Eq. 5 chirp set: K-NN regression and Isomap
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(N=2 ** 16, J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16)
BATCH = 64
METRIC = "JTFS fwd+bwd signals/sec (B=64, N=2^16, Q=16) at rel err <=1e-4; % HBM roofline"
WORKLOAD_NAME = ("jtfs fwd+bwd, B=64 AM/FM tones, N=2^16 at 22050 Hz, J=12, Q=16, Q2=1, "
                 "J_fr=4, Q_fr=2, T=2^12, F=16, oversampling 0")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
SMS = 152
# DRAM bytes (read + write) per step of the contraction stages (forward and backward kernels
# with their phi_F pooling / adjoint) at B = 64, from an ncu capture of dram__bytes_read.sum +
# dram__bytes_write.sum of the current kernels: 715.7 MB at B = 16, scaled by the signals (the
# kernels' traffic is proportional to them); None where no capture of the current kernels
# exists.
CONTRACTION_TRAFFIC = {"fp32": 4 * 715.7e6}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(ms_local, batch, world, device):
    """(slowest rank's ms per step, whole-job signals/s): every rank's mean step time is
    all-reduced with MAX, and the signals of all ranks are divided by it."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, batch * world / (ms_max / 1e3)


def fft_stage_bytes(plan_shapes, schedule, B, planes):
    """Algorithmic HBM bytes per step of the FFT-side stages of the fused step: every array a
    stage must take in or hand on, counted once (intermediates a stage could keep on chip are
    not counted, however often the kernels re-read them).  The Y producer reads U1-hat and
    writes the Y planes (`planes` BF16 copies of re and im); the scalogram reads x-hat and
    writes U1 and U1-hat; the second-order backward reads gY once and writes g_U1; the
    first-order backward reads g_U1 and x-hat and writes gF; g_x reads gF and writes g_x."""
    s1, s2, lm = schedule
    n1, N = plan_shapes.n1, plan_shapes.N
    y = sum((n1 - int(lm[a])) * (N // int(s2[a])) for a in range(len(s2)) if s2[a])
    u1 = plan_shapes.u1_len
    uh = u1 // 2
    xh = N // 2
    per = {
        "second_order": y * 2 * 2 * planes + uh * 8,
        "scalogram": xh * 8 + u1 * 4 + uh * 8,
        "second_order_bwd": y * 8 + u1 * 4,
        "stage1_bwd": u1 * 4 + xh * 8 + u1 * 8,
        "gx": u1 * 8 + N * 4,
    }
    return {k: v * B for k, v in per.items()}


def contraction_flops(plan_shapes, schedule, B):
    """Algorithmic FLOPs of the log-frequency contractions in one forward + backward step:
    the forward Z = W_c Y_alpha, the backward's recomputation of Z and gY = W_c^H gZ; each is
    C * n1 * K_alpha * L_alpha complex multiply-adds (8 real flops) per signal.  Extra passes
    of the split-precision forms are not counted (they are not algorithmic work)."""
    s1, s2, lm = schedule
    n1, C, N = plan_shapes.n1, plan_shapes.C, plan_shapes.N
    per = 0
    for a in range(len(s2)):
        if s2[a] == 0:
            continue
        per += C * n1 * (n1 - int(lm[a])) * (N // int(s2[a]))
    return 3 * 8 * per * B


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth_signals as SS
    from paper_2204_08269_gb300 import JTFSPlan, build

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    global BATCH
    BATCH = args.batch
    plan = JTFSPlan(**WORKLOAD, precision=args.precision)
    sh = plan.shapes
    x = torch.from_numpy(SS.workload_signals(2, BATCH, WORKLOAD["N"])).cuda()
    # the plan's launch shape of the row FFT stages, tuned once for this batch (untimed setup)
    tuned = None if args.no_autotune else plan.autotune(BATCH)
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    g0 = torch.randn(sh.s0(BATCH), device="cuda", generator=gen)
    g1 = torch.randn(sh.s1(BATCH), device="cuda", generator=gen)
    g2 = torch.randn(sh.s2(BATCH), device="cuda", generator=gen)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        # forward and backward in one library call (the backward half reuses the forward's
        # spectra); the separate jtfs_forward / jtfs_backward calls recompute them from the
        # U1 checkpoint
        return plan.forward_backward(x, g0, g1, g2)[3]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.profile_read()  # reset counters
    plan.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))          # evict L2 between timed steps (outside the events)
            starts[i].record()
            step()
            ends[i].record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    stages, launches = plan.profile_read()
    plan.profile(False)
    ms_max, value = job_throughput(ms, BATCH, world, "cuda")

    # end to end through the host-buffer entry point (H2D, fwd, bwd, D2H in one call)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(SS.workload_signals(2, BATCH, WORKLOAD["N"])).pin_memory()
        gh = [g.cpu().pin_memory() for g in (g0, g1, g2)]
        for _ in range(max(1, min(args.warmup, 2))):
            plan.forward_backward_host(xh, *gh)
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            o = plan.forward_backward_host(xh, *gh)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        h2d = xh.numel() * 4 + sum(g.numel() * 4 for g in gh)
        d2h = sum(t.numel() * 4 for t in o)
        e2e = {"value": BATCH / e2e_s, "unit": "signals/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "how": "jtfs_forward_backward_host on pinned host buffers, wall clock"}

    peaks, peaks_kind = _peaks()
    sched = plan.schedule()
    flops = contraction_flops(sh, sched, BATCH)
    joint_ms = (stages["joint_fwd"] + stages["joint_bwd"]) / args.steps
    clocks = clk.summary()
    if args.precision == "fp32_simt":
        # plain FP32 on CUDA cores: 128 FMA lanes per SM at the maximum SM clock
        peak = SMS * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "joint_fwd+joint_bwd (contraction, CUDA cores)",
                "achieved": flops / (joint_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock",
                "traffic": None}
    else:
        # the timed region is well under a second of back-to-back steps: the burst peak
        peak = peaks.get("bf16_tflops")
        if args.precision == "tf32":
            peak = peak / 2.0
        roof = {"bound": "tensor", "kernel": "joint_fwd+joint_bwd (tcgen05 contraction)",
                "achieved": flops / (joint_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"{peaks_kind} bf16 burst" + (" / 2 (tf32)" if args.precision == "tf32" else ""),
                "traffic": (CONTRACTION_TRAFFIC.get(args.precision) if BATCH == 64 else None),
                "traffic_unit": "bytes per step (both contraction launches)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["launch_ms"] = joint_ms
    roof["flops_per_step"] = flops
    # the FFT-side stages (HBM bound by their algorithmic traffic)
    fft = None
    if args.precision in ("fp32", "bf16"):
        fb = fft_stage_bytes(sh, sched, BATCH, 2 if args.precision == "fp32" else 1)
        fms = sum(stages[k] for k in fb) / args.steps
        gbs = sum(fb.values()) / (fms / 1e3) / 1e9
        fft = {"bound": "hbm", "stages": sorted(fb), "achieved": gbs,
               "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
               "frac": gbs / peaks.get("hbm_gbs"), "bytes_per_step": sum(fb.values()),
               "ms_per_step": fms}
    extras = None
    if world == 1 and not args.no_extras and BATCH == 64:
        extras = run_extras(args, plan, x, (g0, g1, g2))
    out = None
    if rank == 0:
        cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu) else None
        out = {
            "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision in ("fp32", "fp32_simt") else args.precision,
            "data": "synthetic (seeded AM/FM tones + -30 dB noise)",
            "config": {"workload": WORKLOAD_NAME, "global_batch": BATCH * world,
                       "batch_per_gpu": BATCH, "N": WORKLOAD["N"], "precision": args.precision,
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed by a 256 MiB write before every timed step",
                       "row_fft_launch": tuned},
            "roofline": roof,
            "fft_roofline": fft,
            "stage_ms_per_step": {k: v / args.steps for k, v in stages.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "peaks": peaks_kind,
            "comparisons": extras,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out


def _oracle_sample(n_signals):
    """FP64 oracle forward + backward of ``n_signals`` signals of the workload; seconds."""
    import synth_signals as SS
    from oracle import jtfs_oracle as O
    cfg = O.Config(**{k: WORKLOAD[k] for k in ("J", "Q", "J_fr", "Q_fr", "T", "F", "N")})
    p = O.Plan(cfg)
    s = O.Schedule(p, 0)
    x = SS.workload_signals(2, n_signals, cfg.N).astype(np.float64)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    for b in range(n_signals):
        out = O.forward_one(x[b], p, s)
        g = {k: rng.standard_normal(v.shape) for k, v in out.items()}
        O.backward_one(x[b], g["S0"], g["S1"], g["S2"], p, s)
    return time.perf_counter() - t0


def cpu_baseline(args, n_signals=3):
    secs = _oracle_sample(n_signals)
    return {"value": n_signals / secs, "unit": "signals/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{n_signals} of the 64 signals, FP64 NumPy oracle forward + backward "
                      "(SCHEDULED mode), one signal at a time; BLAS threads = all cores"}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return None
    # warm-up: one untimed signal at most (each is seconds of CPU work)
    for _ in range(min(args.warmup, 1)):
        _oracle_sample(1)
    secs = 0.0
    for _ in range(args.steps):
        secs += _oracle_sample(1)
    value = args.steps / secs
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "signals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded AM/FM tones)",
        "config": {"workload": WORKLOAD_NAME, "global_batch": BATCH, "N": WORKLOAD["N"]},
        "cpu_baseline": {"value": value, "unit": "signals/s", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": "1 signal of the 64 per step, FP64 oracle forward + backward"},
        "e2e": {"value": value, "unit": "signals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return out


def run_extras(args, plan, x, g):
    """Short measurements beside the headline, in the same run (one GPU only): the plain FP32
    CUDA-core form of the same step, and summaries of the uneven-length, mixed-precision,
    resynthesis and Eq. 5 workloads (each also available alone with --workload).  None of
    them enters the headline value."""
    import torch
    from paper_2204_08269_gb300 import JTFSPlan
    res = {}
    try:
        simt = JTFSPlan(**WORKLOAD, precision="fp32_simt")
        simt.forward_backward(x[:8], *[t[:8].contiguous() for t in g])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        simt.forward_backward(x, *g)
        e1.record()
        torch.cuda.synchronize()
        res["fp32_cuda_cores"] = {"signals_per_s": BATCH / (e0.elapsed_time(e1) / 1e3),
                                  "ms_per_step": e0.elapsed_time(e1),
                                  "how": "the same B=64 step with the contraction on CUDA cores "
                                         "(plain FP32), one timed step"}
        del simt
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup, sub.batch = 3, 2, BATCH
        v = run_varlen(sub, emit=False)
        res["varlen"] = {k: v[k] for k in ("value", "unit", "ms_per_step", "per_signal_launches")}
        res["varlen"]["tuned_sub_batch"] = v["config"].get("tuned_sub_batch")
        m = run_mixed(sub, emit=False)
        res["mixed_precision_forward"] = m["precisions"]
        sub.steps = 50
        r = run_resynth(sub, emit=False)
        res["resynthesis"] = {k: r[k] for k in ("value", "unit", "ms_per_step", "E_adam",
                                                "E_bold_driver")}
        e = run_eq5(sub, emit=False)
        res["eq5_study"] = {"signals_per_s": e["value"],
                            "knn_error_ratio": e["study"]["knn_error_ratio"],
                            "isomap_alignment": e["study"]["isomap_alignment"]}
    except Exception as exc:   # the headline stands on its own
        res["error"] = repr(exc)
    torch.cuda.empty_cache()
    return res


def run_varlen(args, emit=True):
    """Uneven-length batch: J=12, Q=16, J_fr=4, Q_fr=2, T=2^12, F=16, lengths log-uniform in
    2^13..2^17, half AM/FM tones and half click trains; forward + backward with ones as
    cotangents.  The step is one replay of the captured graph (autotuned launch shapes and
    sub-batch size); the comparison is one library call per signal (B = 1) on a sample of the
    batch."""
    import torch
    from paper_2204_08269_gb300 import jtfs
    import synth_signals as SS
    torch.cuda.set_device(0)
    count = args.batch if args.batch != BATCH else 1024
    cfg = dict(J=12, Q=16, J_fr=4, Q_fr=2, T=2 ** 12, F=16)
    xh, lengths = SS.varlen_batch(count, SS.BASE_SEED + 5)
    v = jtfs.JTFSVarlen(lengths, **cfg, precision=args.precision, chunk=args.chunk)
    x = torch.from_numpy(xh).cuda()
    g = [torch.ones(int(o[-1]), device="cuda") for o in (v.s0_off, v.s1_off, v.s2_off)]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        chosen = None
        if not args.no_autotune:   # profiling runs keep the default shapes and sub-batches
            v.autotune()
            chosen = v.tune_schedule(x, g)
        v.capture(x, g)
        for _ in range(args.warmup):
            v.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        side.synchronize()
        e0.record(side)
        for _ in range(args.steps):
            v.replay()
        e1.record(side)
    side.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # per-signal launches on a sample (every 8th signal), one plan per padded length
    sample = list(range(0, count, 8))
    plans = {}
    for i in sample:
        Np = jtfs.varlen_padded_length(int(lengths[i]), J=cfg["J"])
        if Np not in plans:
            plans[Np] = jtfs.JTFSPlan(N=Np, **cfg, precision=args.precision)
    xs = []
    for i in sample:
        Np = jtfs.varlen_padded_length(int(lengths[i]), J=cfg["J"])
        xi = torch.zeros((1, Np), device="cuda")
        xi[0, :int(lengths[i])] = x[int(v.x_off[i]):int(v.x_off[i]) + int(lengths[i])]
        xs.append((plans[Np], xi))

    def per_signal():
        for p, xi in xs:
            s0, s1, s2, u1 = p.forward(xi)
            p.backward(xi, u1, torch.ones_like(s0), torch.ones_like(s1), torch.ones_like(s2))

    per_signal()
    torch.cuda.synchronize()
    e0.record()
    per_signal()
    e1.record()
    torch.cuda.synchronize()
    ms_ps = e0.elapsed_time(e1)
    out = {"metric": "JTFS fwd+bwd signals/sec, uneven lengths 2^13-2^17 in one graph launch",
           "value": count / (ms / 1e3), "unit": "signals/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "bf16" else "bf16",
           "data": "synthetic (seeded AM/FM tones and click trains)",
           "config": {"workload": f"varlen, {count} signals, len log-uniform 2^13..2^17, J=12, Q=16, "
                                  "J_fr=4, Q_fr=2, T=2^12, F=16", "precision": args.precision,
                      "largest_sub_batch_tried": args.chunk, "tuned_sub_batch": chosen,
                      "padded_lengths": {str(k): int(sum(1 for n in lengths if jtfs.varlen_padded_length(int(n), J=12) == k))
                                         for k in sorted(set(jtfs.varlen_padded_length(int(n), J=12) for n in lengths))}},
           "per_signal_launches": {"value": len(sample) / (ms_ps / 1e3), "unit": "signals/s",
                                   "sample": f"{len(sample)} of the {count} signals, one call per signal"}}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_mixed(args, emit=True):
    """Mixed-precision forward: B = 256, N = 2^15, J = 11, Q = 12, J_fr = 4, Q_fr = 1 (AM/FM
    tones).  Forward signals/s of the FP32-grade, TF32 and BF16 contractions, and their
    per-order relative L2 error against the FP64 oracle on two sampled signals."""
    import torch
    from paper_2204_08269_gb300 import jtfs
    import synth_signals as SS
    from oracle import jtfs_oracle as O
    torch.cuda.set_device(0)
    B = args.batch if args.batch != BATCH else 256
    oc = O.WORKLOADS[4]
    cfg = dict(N=oc.N, J=oc.J, Q=oc.Q, J_fr=oc.J_fr, Q_fr=oc.Q_fr, T=oc.T, F=oc.F)
    xh = SS.workload_signals(4, B, cfg["N"])
    x = torch.from_numpy(xh).cuda()
    plan_o = O.Plan(oc)
    sched_o = O.Schedule(plan_o, 0)
    sample = [0, B // 2]
    refs = [O.forward_one(xh[b].astype(np.float64), plan_o, sched_o) for b in sample]
    res = {}
    for prec in ("fp32", "tf32", "bf16"):
        p = jtfs.JTFSPlan(**cfg, precision=prec)
        for _ in range(args.warmup):
            out = p.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            out = p.forward(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        errs = {}
        for name, k in (("S0", 0), ("S1", 1), ("S2", 2)):
            got = out[k].cpu().numpy().astype(np.float64)
            errs[name] = max(float(np.linalg.norm(got[b] - r[name]) / np.linalg.norm(r[name]))
                             for b, r in zip(sample, refs))
        res[prec] = {"signals_per_s": B / (ms / 1e3), "ms_per_forward": ms, "rel_err": errs}
    out = {"metric": "JTFS forward signals/sec by contraction precision (B=256, N=2^15, J=11, Q=12)",
           "value": res["tf32"]["signals_per_s"], "unit": "signals/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "vs_baseline": None, "dtype": "tf32", "data": "synthetic (seeded AM/FM tones + -30 dB noise)",
           "config": {"workload": "mixed precision forward, B=256 AM/FM tones, N=2^15, J=11, Q=12, "
                                  "J_fr=4, Q_fr=1, T=2^11, F=12"},
           "precisions": res, "oracle_sample": f"signals {sample} of {B}"}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_resynth(args, emit=True):
    """Texture resynthesis (Sec. 5): B = 16 click-train targets of N = 2^17 (J = 13, Q = 16,
    J_fr = 4, Q_fr = 2, T = 2^13, F = 16), ``--steps`` Adam iterations (50 by the workload)
    from seeded white noise, each one forward with the U1 checkpoint and one backward through
    the autograd form.  Value: signal-iterations per second.  The paper's bold driver is run
    beside it for 100 iterations and its normalised error E at 20 and 100 iterations is
    reported as context (the paper quotes about 0.10 and 0.03 on bird calls)."""
    import torch
    from paper_2204_08269_gb300 import build, resynth
    import synth_signals as SS
    from oracle import jtfs_oracle as O
    torch.cuda.set_device(0)
    build.build()
    w = O.WORKLOADS[3]
    cfg = dict(J=w.J, Q=w.Q, J_fr=w.J_fr, Q_fr=w.Q_fr, T=w.T, F=w.F)
    B = args.batch if args.batch != BATCH else 16
    steps = args.steps if args.steps != 10 else 50
    x = torch.from_numpy(SS.workload_signals(3, B, w.N)).cuda()
    warm = resynth.Resynthesis(x, method="adam", seed=1, precision=args.precision, **cfg)
    warm.run(max(3, args.warmup))
    r = resynth.Resynthesis(x, method="adam", seed=0, precision=args.precision, **cfg)
    r.model.plan.profile_read()
    with ClockSampler(0) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        out = r.run(steps, timed=False)
        b.record()
        torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    _, launches = r.model.plan.profile_read()
    bold = resynth.Resynthesis(x, method="bold", seed=0, precision=args.precision, **cfg)
    bh = bold.run(100, timed=False)["E"]
    res = {"metric": "JTFS texture resynthesis signal-iterations/sec (B=16, N=2^17, J=13, Q=16), "
                     "Adam through the autograd form",
           "value": B / (ms / 1e3), "unit": "signal-iterations/s", "n_gpus": 1,
           "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if args.precision in ("fp32", "fp32_simt") else args.precision,
           "data": "synthetic (seeded Poisson click trains through random resonators)",
           "config": {"workload": "resynthesis, B=16 click trains, N=2^17, J=13, Q=16, J_fr=4, "
                                  "Q_fr=2, T=2^13, F=16; Adam lr 0.3 x target RMS",
                      "precision": args.precision},
           "E_adam": {"first": out["E"][0], "last": out["E"][-1],
                      "every_10": out["E"][::10]},
           "E_bold_driver": {"at_20": bh[19], "at_100": bh[99], "every_10": bh[::10]},
           "paper_context": "about 720 ms per iteration for one signal of N=2^16 (J=12, Q=12) "
                            "on an unnamed GPU; E about 0.10 at 20 and 0.03 at 100 iterations",
           "gpu_launches": int(launches), "clocks": clk.summary()}
    if emit:
        print(json.dumps(res), flush=True)
    return res


def run_eq5(args, emit=True):
    """The Eq. 5 similarity study (Sec. 3.2-3.4) on the 16^3 chirp grid: transform throughput
    on the dataset and the K-NN / Isomap results for this library's features."""
    import torch
    from paper_2204_08269_gb300 import build, manifold
    torch.cuda.set_device(0)
    build.build()
    res = manifold.run(precision=args.precision)
    out = {"metric": "JTFS Eq. 4 forward signals/sec on the Eq. 5 chirp set (4096 signals, "
                     "N=2^16, J=14, Q=8) with K-NN / Isomap results",
           "value": res["signals_per_s"], "unit": "signals/s", "n_gpus": 1, "steps": 1,
           "warmup": 0, "higher_is_better": True, "vs_baseline": None,
           "dtype": "f32" if args.precision in ("fp32", "fp32_simt") else args.precision,
           "data": "synthetic (the paper's Eq. 5 AM/FM chirps, 16 values per parameter)",
           "config": {"workload": "Eq. 5 study, 4096 signals, N=2^16 at 22050 Hz, J=14, Q=8, "
                                  "J_fr=4, Q_fr=1, T=2^14, Eq. 4, mu-log eps 0.1, K=40"},
           "study": res,
           "paper_context": "K-NN error ratios of JTFS: f_m within 0.75-1.5, gamma within "
                            "0.75-1.25, f_c close to 1 (Sec. 3.4)"}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16", "fp32_simt"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the short comparison measurements after the headline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default row-FFT launch shape (profiling runs: no tuning launches)")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="signals per GPU (the workload is 64; smaller values for profiling)")
    ap.add_argument("--chunk", type=int, default=512,
                    help="varlen: the largest sub-batch of one padded length the schedule "
                         "tuner tries (the workspace is sized for it)")
    ap.add_argument("--workload", default="fixed", choices=["fixed", "varlen", "mixed", "resynth", "eq5"],
                    help="varlen: the uneven-length batch; mixed: forward by contraction "
                         "precision; resynth: texture resynthesis at N = 2^17 (none of them is "
                         "the headline metric)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "varlen":
        run_varlen(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "resynth":
        run_resynth(args)
    elif args.workload == "eq5":
        run_eq5(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
