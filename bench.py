"""Benchmark of the AS-ICP hot path (one grasp set = one step).

A step is one full AS-ICP optimisation of one object: Fibonacci initial poses,
k_max iterations of transform / matching / cost+gradient / collision / SVGD or
SGD update for every preshape and particle, the final evaluation and the
ranking, then the top-k read-back (asicp_run + asicp_best_grasps).

Default workload: 3 preshapes x 256 particles, gripper contact cloud of 2048
points, 8192-point single-view partial object clouds of seeded procedural
shapes, 64^3 SDF grids, 100 iterations (38 SVGD + 62 SGD).  The metric is
forward matching throughput in particle*point pairs per second
(P * K * N * M pairs per iteration, k_max + 1 evaluations per step) plus the
milliseconds per grasp set.

N > 1 GPUs (torchrun): every rank optimises its own object (weak scaling, no
data-path collective); the step time is the maximum over ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a few particles of one iteration per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
# DRAM bytes (read + write) of one launch of each forward-matching kernel from the committed ncu
# captures: the float32 kernel's from the profile case
# (profiles/fwd_match_kernel_profile-case-P1-K256-N2048-M8192.md; every input is L2-resident, so the
# figure holds for the paper-scale launch too), the tensor-core kernel's from a paper-scale launch
# (profiles/fwd_match_tc_kernel_dram_paper-scale-P3-K256-N2048-M8192.md).  None when the kernel has
# changed since the capture.
FWD_DRAM_BYTES_PER_LAUNCH = 397568        # fwd_match_kernel (float32 shapes)
TC_DRAM_BYTES_PER_LAUNCH = 609280         # fwd_match_tc_kernel (tensor-core shape), paper-scale launch
OPS_PER_PAIR = 4          # algorithmic FP32-lane work per particle*point pair: 3 FMA + 1 compare
FMA_PER_PAIR = 3          # of which FMA-pipe work (the compare runs as half a 3-input min on the ALU pipe)
TC_ALG_FLOP_PER_PAIR = 8  # tensor-core shape, algorithmic: |r|^2 - 2 s'.r as an augmented K = 4 contraction
TC_EXEC_FLOP_PER_PAIR = 32  # executed: one M=128 x N=256 x K=16 f16 MMA per 128 x 256 pairs (split operands)
EPILOGUE_OPS_PER_PAIR = 1   # the tensor-core shape's epilogue: one compare per pair
TC_SHAPE = "tc-f16x3-m128-n256"
TOPK = 16
METRIC = "AS-ICP particle*point pairs/s (forward matching) and ms per grasp set"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="asicp", choices=["asicp", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work for the oracle sample")
    ap.add_argument("--small", action="store_true", help="small workload (debugging only)")
    ap.add_argument("--fwd-shape", type=int, default=-1,
                    help="forward-matching kernel shape (index into asicp.FWD_VARIANTS); -1: autotune")
    ap.add_argument("--k-sweep", action="store_true",
                    help="ms per grasp set of the paper-scale workload for K = 32 .. 1024 particles per preshape")
    ap.add_argument("--large", action="store_true",
                    help="mixed-precision configuration (3 x 1024 particles, N 4096, M 65536, SDF 128^3): both "
                         "matching shapes timed and compared")
    ap.add_argument("--batched", type=int, default=0, metavar="OBJECTS",
                    help="time OBJECTS objects (point counts 1k-32k, 128/256/512 particles per preshape) optimised "
                         "together against each object alone; prints its own JSON line")
    ap.add_argument("--learned", default="", metavar="TRAIN,TEST",
                    help="train the initial-pose proposal on TRAIN objects (targets from the plain method) and "
                         "compare it with the plain method on TEST held-out objects; prints its own JSON line")
    ap.add_argument("--learned-epochs", type=int, default=60)
    ap.add_argument("--compare", type=int, default=0, metavar="OBJECTS",
                    help="the plain FP32 GPU method against the tensor-core / batched / shorter-budget forms at "
                         "equal final cost on OBJECTS paper-scale objects; prints its own JSON line")
    ap.add_argument("--profile-proposal", action="store_true",
                    help="one forward and one loss/gradient pass of the proposal network on 32 clouds of 2048 points "
                         "(for profiler captures); no JSON line")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="time the FP64 oracle on the host cores for configurations 1-4 (1 and 2 in full, 3 on two "
                         "objects in full, 4 on 10 of its 100 iterations, extrapolated and labelled)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one short run of a reduced workload (1 preshape x 256 particles, N=2048, M=8192, "
                         "8 iterations, poses close enough to collide) for profiler captures; no JSON line")
    return ap.parse_args()


def workload(rank: int, small: bool):
    from paper_2412_08346_gb300 import synth
    if small:
        return synth.custom_case(P=3, K=64, N=512, M=2048, grid=32, k_max=20, seed=synth.BASE_SEED + 2)
    w = synth.paper_scale_case(seed=synth.BASE_SEED + 2)
    if rank:
        w.objects = [synth.partial_object(8192, synth.BASE_SEED + 2 + 1000 * (rank + 1))]
    return w


def pairs_per_step(w) -> int:
    P, N, M = len(w.preshapes), w.preshapes[0].S.shape[0], len(w.objects[0].points)
    return P * w.K * N * M * (w.k_max + 1)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, power, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(w, seconds: float, nthreads: int, max_iters: int | None = None):
    """Time the FP64 oracle on a bounded sample: a few particles per preshape for one iteration at
    a time (the first SVGD iteration's work: matching, cost/gradient and collision for every pair)."""
    import oracle
    P, N, M = len(w.preshapes), w.preshapes[0].S.shape[0], len(w.objects[0].points)
    Ks = max(1, min(w.K, nthreads))
    orc = oracle.Oracle(np.stack([p.S for p in w.preshapes]), [(p.sdf, p.origin, p.voxel) for p in w.preshapes],
                        w.objects[0].points, K=Ks)
    th = np.tile(oracle.fibonacci_init(Ks, orc.R.mean(0), 0.15), (P, 1))
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, N=N)
    st = orc.new_state(th[None].reshape(P, Ks, 7))
    pairs = 0
    iters = 0
    t0 = time.perf_counter()
    while True:
        orc.step(st, sched, iters % w.k_max, nthreads)
        pairs += P * Ks * N * M
        iters += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_iters and iters >= max_iters):
            break
    return pairs / el, {"particles_per_preshape": Ks, "iterations": iters, "seconds": el, "pairs": pairs}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload(0, args.small)
    nthreads = os.cpu_count() or 1
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(w, 0.0, nthreads, max_iters=1)
    vals, secs, total_pairs = [], 0.0, 0
    for _ in range(args.steps):
        v, info = oracle_sample(w, per_step, nthreads)
        vals.append(v)
        secs += info["seconds"]
        total_pairs += info["pairs"]
    value = total_pairs / secs
    sample = (f"{info['particles_per_preshape']} particles per preshape x {len(w.preshapes)} preshapes, "
              f"whole iterations (N={w.preshapes[0].S.shape[0]}, M={len(w.objects[0].points)}), "
              f"~{per_step:.0f} s per step")
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": nthreads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_timed_run(pre, obj_points, K, k_max, k_stein, schedule, nthreads, iters, evaluate):
    """One FP64 oracle run from the Fibonacci shell: `iters` iterations (and the final evaluation
    when evaluate is set); returns (seconds, forward pairs)."""
    import oracle
    P, N, M = len(pre), pre[0].S.shape[0], len(obj_points)
    orc = oracle.Oracle(np.stack([p.S for p in pre]), [(p.sdf, p.origin, p.voxel) for p in pre], obj_points, K=K)
    th = np.tile(oracle.fibonacci_init(K, orc.R.mean(0), 0.15), (P, 1)).reshape(P, K, 7)
    sched = orc.schedule(k_max=k_max, k_stein=k_stein, schedule=schedule, N=N)
    st = orc.new_state(th)
    t0 = time.perf_counter()
    for k in range(iters):
        orc.step(st, sched, k, nthreads)
    if evaluate:
        orc.evaluate(st, nthreads)
    return time.perf_counter() - t0, P * K * N * M * (iters + (1 if evaluate else 0))


def run_oracle_configs(args):
    """--oracle-configs: the FP64 oracle's time per configuration on this host's cores."""
    import oracle
    from paper_2412_08346_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    rows = []

    def add(config, what, threads, secs, pairs, scale, full_pairs):
        rows.append({"config": config, "timed": what, "threads": threads, "seconds": secs,
                     "pairs_per_s": pairs / secs, "full_run_pairs": full_pairs,
                     "full_run_seconds": secs * scale, "extrapolated": scale != 1.0})

    # config 1: the small box case in full (50 SVGD iterations + the final evaluation)
    w = synth.small_box_case()
    for thr in (1, cores):
        secs, pairs = oracle_timed_run(w.preshapes, w.objects[0].points, w.K, w.k_max, w.k_stein, w.schedule,
                                       thr, w.k_max, True)
        add(1, f"{w.name}, in full", thr, secs, pairs, 1.0, pairs)
    # config 2: the paper-scale grasp set in full on every core; one thread on 2 iterations
    w = synth.paper_scale_case()
    secs, pairs = oracle_timed_run(w.preshapes, w.objects[0].points, w.K, w.k_max, w.k_stein, w.schedule,
                                   cores, w.k_max, True)
    add(2, f"{w.name}, in full", cores, secs, pairs, 1.0, pairs)
    full = pairs
    secs, pairs = oracle_timed_run(w.preshapes, w.objects[0].points, w.K, w.k_max, w.k_stein, w.schedule,
                                   1, 2, False)
    add(2, f"{w.name}, 2 iterations", 1, secs, pairs, full / pairs, full)
    # config 3: two objects of the batched case in full, every preshape with its own particle count
    wb, Kb = synth.batched_case(64)
    secs, pairs = 0.0, 0
    for o in range(2):
        for p in range(len(wb.preshapes)):
            s_, p_ = oracle_timed_run([wb.preshapes[p]], wb.objects[o].points, int(Kb[o, p]), wb.k_max,
                                      wb.k_stein, wb.schedule, cores, wb.k_max, True)
            secs += s_
            pairs += p_
    add(3, f"2 of the 64 objects of {wb.name}, in full", cores, secs, pairs, 1.0, pairs)
    # config 4: the largest workload, 10 of its 100 iterations
    w = synth.large_case(k_max=100)
    secs, pairs = oracle_timed_run(w.preshapes, w.objects[0].points, w.K, w.k_max, w.k_stein, w.schedule,
                                   cores, 10, False)
    add(4, f"{w.name}, 10 iterations", cores, secs, pairs, 10.1, pairs * 101 // 10)
    line = {"metric": "FP64 oracle time per configuration on the host cores", "unit": "s", "kind": "oracle",
            "cpu": host_cpu_model(), "cores": cores, "dtype": "f64", "data": "synthetic", "configs": rows}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU
def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2412_08346_gb300 import asicp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    w = workload(rank, args.small)
    P, K, N, M = len(w.preshapes), w.K, w.preshapes[0].S.shape[0], len(w.objects[0].points)
    # profile 2: CUDA events around the forward-matching kernel only (the roofline's kernel); every
    # event is a node of the captured loop, and timing all kernels (profile 1) costs ~5 % of a grasp set
    cfg = asicp.asicp_config_default(P=P, K=K, k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule,
                                     profile=2, cuda_stream=stream.cuda_stream, fwd_shape=max(0, args.fwd_shape))
    ctx = asicp.asicp_create(cfg)
    obj = w.objects[0].points
    R_dev = torch.from_numpy(obj).to(dev)
    pre_dev = [(torch.from_numpy(p.S).to(dev), torch.from_numpy(p.sdf).to(dev)) for p in w.preshapes]

    def set_inputs(c):
        asicp.asicp_set_object(c, R_dev)
        for p, (S, g) in enumerate(pre_dev):
            asicp.asicp_set_gripper_sdf(c, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
    set_inputs(ctx)
    # pick the forward-matching kernel shape on this workload (outside the timed region)
    if args.fwd_shape < 0:
        shape, shape_ms = asicp.asicp_autotune(ctx)
    else:
        shape = args.fwd_shape
    best = np.zeros(TOPK * 7, np.float32)
    best_c = np.zeros(TOPK, np.float32)
    best_p = np.zeros(TOPK, np.int32)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    # the per-kernel breakdown: the same workload and shape with every kernel timed, run after the
    # timed region (set up here, outside it)
    cfg_all = asicp.asicp_config_default(P=P, K=K, k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule,
                                         profile=1, cuda_stream=stream.cuda_stream, fwd_shape=shape)
    ctx_all = asicp.asicp_create(cfg_all)
    set_inputs(ctx_all)

    def one_step(c=ctx):
        asicp.asicp_run(c)
        asicp.asicp_best_grasps(c, TOPK, best, best_c, best_p)

    for _ in range(args.warmup):
        one_step()
        one_step(ctx_all)
    torch.cuda.synchronize()
    asicp.asicp_kernel_times(ctx, reset=True)

    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()                     # L2 flush between timed steps, outside the timed interval
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_t, launches_t = asicp.asicp_kernel_times(ctx, reset=True)
    # per-kernel breakdown (every kernel timed), the same number of steps after the timed region
    asicp.asicp_kernel_times(ctx_all, reset=True)
    all_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(ctx_all)
        e1.record(stream)
        e1.synchronize()
        all_ms.append(e0.elapsed_time(e1))
    ms, launches = asicp.asicp_kernel_times(ctx_all, reset=True)
    asicp.asicp_destroy(ctx_all)
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    pairs = pairs_per_step(w)
    value = pairs * args.steps * world / (max_ms / 1e3)

    # dominant kernel: forward matching; algorithmic work per launch = P*K*N*M pairs
    tc = asicp.FWD_VARIANTS[shape] == TC_SHAPE
    match_avg_s = ms_t[0] / max(1, launches_t[0]) / 1e3          # timed region
    exact_avg_s = ms[5] / max(1, launches[5]) / 1e3 if tc else 0.0   # breakdown pass
    pairs_per_launch = P * K * N * M
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = roofline_entry(tc, pairs_per_launch, match_avg_s, exact_avg_s, ms, sms, clk)
    # match, collide, collide_nn, finalize per pass (+ the exact choice with the tensor-core shape),
    # Stein direction and Stein update per SVGD pass, + init, reset, select, gather
    launches_per_step = (5 if tc else 4) * (w.k_max + 1) + 2 * w.k_stein + 4

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, ctx, w, stream, best, best_c, best_p, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        nthreads = os.cpu_count() or 1
        v, info = oracle_sample(w, args.cpu_seconds, nthreads)
        v1, info1 = oracle_sample(w, max(1.0, args.cpu_seconds / 3), 1)
        cpu = {"value": v, "unit": "pairs/s", "cores": nthreads, "kind": "oracle",
               "sample": (f"FP64 oracle, {info['particles_per_preshape']} particles per preshape x {P} preshapes, "
                          f"{info['iterations']} whole iterations (N={N}, M={M}), {info['seconds']:.1f} s"),
               "single_thread_value": v1,
               "single_thread_sample": (f"1 thread, {info1['particles_per_preshape']} particle per preshape x {P} "
                                        f"preshapes, {info1['iterations']} whole iterations, "
                                        f"{info1['seconds']:.1f} s")}
    asicp.asicp_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "P": P, "K": K, "N": N, "M": M,
                       "sdf": int(w.preshapes[0].sdf.shape[0]), "iterations": w.k_max, "k_stein": w.k_stein,
                       "pairs_per_step": pairs, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world} (one object per GPU)",
                       "fwd_shape": asicp.FWD_VARIANTS[shape]},
            "ms_per_grasp_set": max_ms / args.steps,
            "roofline": roofline,
            "kernel_ms_per_step": {k: v / args.steps for k, v in zip(asicp.KERNEL_KINDS, ms)},
            "kernel_breakdown": ("kernel_ms_per_step, exact_kernel_ms and the shares come from a second pass of "
                                 f"{args.steps} steps after the timed region with every kernel timed (CUDA events "
                                 f"in the captured loop: {statistics.median(all_ms):.1f} ms per grasp set there); "
                                 "the timed region times the forward-matching kernel only"),
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        if e2e:
            line["e2e"] = e2e
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)


def roofline_entry(tc, pairs_per_launch, match_avg_s, exact_avg_s, ms, sms, clk):
    """Roofline of the dominant kernel, in particle*point pairs per second.

    The FP32 lanes run SMs x 128 lane operations per clock, at the median SM clock sampled during the
    timed region (the nominal maximum if no sample was taken).  Tensor-core shape: the lower of the
    tensor bound (measured sustained dense bf16 rate over the algorithmic 8 flop per pair of the
    augmented K = 4 contraction; f16 has the same nominal rate) and the bound of its one-compare
    epilogue (one lane operation per pair); the executed split-f16 MMA work (32 flop per pair) is
    reported beside it.  Float32 shapes: 4 lane operations per pair (3 FMA + 1 compare)."""
    share = ms[0] / max(1e-9, sum(ms))
    mhz = clk.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
    clk_basis = ("median SM clock sampled during the timed region" if clk.get("sm_mhz")
                 else "nominal maximum SM clock (no clock sample)")
    lane_ops = sms * FP32_LANES_PER_SM * mhz * 1e6
    achieved = pairs_per_launch / match_avg_s
    if tc:
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        bf16_basis = ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 loop under the power cap)"
                      if bf16 else "fallback 1.7 PFLOP/s sustained")
        bf16 = bf16 or 1700.0
        tensor_bound = bf16 * 1e12 / TC_ALG_FLOP_PER_PAIR
        epi_bound = lane_ops / EPILOGUE_OPS_PER_PAIR
        peak = min(tensor_bound, epi_bound)
        return {"bound": "alu" if epi_bound <= tensor_bound else "tensor",
                "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpairs/s", "frac": achieved / peak,
                "traffic": TC_DRAM_BYTES_PER_LAUNCH,
                "traffic_basis": "dram__bytes_read+write of one paper-scale fwd_match_tc_kernel launch (ncu, one "
                                 "pass); the object tiles and gripper clouds are read once, L2-resident after",
                "kernel": "fwd_match_tc_kernel",
                "peak_basis": (f"min(tensor bound {tensor_bound / 1e9:.0f} Gpairs/s = {bf16:.0f} TFLOP/s ({bf16_basis}) / "
                               f"{TC_ALG_FLOP_PER_PAIR} flop per pair, epilogue bound {epi_bound / 1e9:.0f} Gpairs/s = "
                               f"{sms} SMs x {FP32_LANES_PER_SM} lanes x {mhz:.0f} MHz ({clk_basis}) / "
                               f"{EPILOGUE_OPS_PER_PAIR} compare per pair)"),
                "tensor_bound_gpairs": tensor_bound / 1e9, "epilogue_bound_gpairs": epi_bound / 1e9,
                "frac_of_tensor_bound": achieved / tensor_bound,
                "executed_mma_tflops": achieved * TC_EXEC_FLOP_PER_PAIR / 1e12,
                "executed_mma_frac_of_bf16": achieved * TC_EXEC_FLOP_PER_PAIR / 1e12 / bf16,
                "launch_ms": match_avg_s * 1e3, "pairs_per_launch": pairs_per_launch,
                "exact_kernel_ms": exact_avg_s * 1e3,
                "matching_pairs_per_s": pairs_per_launch / (match_avg_s + exact_avg_s),
                "matching_frac_of_fp32_lane_roofline": pairs_per_launch / (match_avg_s + exact_avg_s) /
                                                       (lane_ops / OPS_PER_PAIR),
                "kernel_share": share, "exact_kernel_share": ms[5] / max(1e-9, sum(ms)), "sms": sms, "sm_mhz": mhz}
    peak = lane_ops / OPS_PER_PAIR
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpairs/s",
            "frac": achieved / peak, "traffic": FWD_DRAM_BYTES_PER_LAUNCH,
            "traffic_basis": "dram__bytes_read+write of one fwd_match_kernel launch (ncu); every input is "
                             "L2-resident, so it does not grow with the launch",
            "kernel": "fwd_match_kernel", "peak_basis":
                f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {mhz:.0f} MHz ({clk_basis}) / "
                f"{OPS_PER_PAIR} lane operations per pair (3 FMA + 1 compare)",
            "frac_fma_pipe": achieved / (lane_ops / FMA_PER_PAIR), "peak_fma_pipe": lane_ops / FMA_PER_PAIR / 1e9,
            "launch_ms": match_avg_s * 1e3, "pairs_per_launch": pairs_per_launch, "kernel_share": share,
            "sms": sms, "sm_mhz": mhz}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def measure_e2e(args, ctx, w, stream, best, best_c, best_p, world, dev):
    """Same metric through the public API with host inputs: every step uploads the object, the
    preshape clouds and SDFs from pinned host memory and reads the top-k back."""
    import torch
    import torch.distributed as dist

    from paper_2412_08346_gb300 import asicp
    R_h = torch.from_numpy(w.objects[0].points).pin_memory()
    pre_h = [(torch.from_numpy(p.S).pin_memory(), torch.from_numpy(p.sdf).pin_memory()) for p in w.preshapes]
    out7 = torch.zeros(TOPK * 7, dtype=torch.float32).pin_memory()
    outc = torch.zeros(TOPK, dtype=torch.float32).pin_memory()
    outp = torch.zeros(TOPK, dtype=torch.int32).pin_memory()
    h2d = R_h.numel() * 4 + sum(S.numel() * 4 + g.numel() * 4 for S, g in pre_h)
    d2h = TOPK * (7 * 4 + 4 + 4)

    def one():
        asicp.asicp_set_object(ctx, R_h)
        for p, (S, g) in enumerate(pre_h):
            asicp.asicp_set_gripper_sdf(ctx, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
        asicp.asicp_run(ctx)
        asicp.asicp_best_grasps(ctx, TOPK, out7, outc, outp)

    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    t = torch.tensor([el], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el = float(t.item())
    return {"value": pairs_per_step(w) * args.steps * world / el, "unit": "pairs/s",
            "ms_per_step": 1e3 * el / args.steps, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def run_profile_case(args):
    """Every kernel of the path at full N, M and K but one preshape, for ncu."""
    import torch
    from paper_2412_08346_gb300 import asicp, synth
    w = synth.custom_case(P=1, K=256, N=2048, M=8192, grid=64, k_max=8, seed=synth.BASE_SEED + 2, k_stein=3)
    stream = torch.cuda.current_stream()
    cfg = asicp.asicp_config_default(P=1, K=256, k_max=w.k_max, k_stein=w.k_stein, init_radius=0.06,
                                     cuda_stream=stream.cuda_stream, fwd_shape=max(0, args.fwd_shape))
    ctx = asicp.asicp_create(cfg)
    try:
        asicp.asicp_set_object(ctx, torch.from_numpy(w.objects[0].points).cuda())
        pre = w.preshapes[0]
        asicp.asicp_set_gripper_sdf(ctx, 0, torch.from_numpy(pre.S).cuda(), torch.from_numpy(pre.sdf).cuda(),
                                    pre.origin, pre.voxel)
        for _ in range(max(1, args.steps)):
            asicp.asicp_run(ctx)
        torch.cuda.synchronize()
        cost = np.zeros(4, np.float32)
        n = asicp.asicp_best_grasps(ctx, 4, np.zeros(28, np.float32), cost, np.zeros(4, np.int32))
        print(f"profile case {w.name}: {max(1, args.steps)} runs, best costs {cost[:n].tolist()}")
    finally:
        asicp.asicp_destroy(ctx)


def run_profile_proposal(args):
    """The proposal network's kernels at the training batch size, for ncu."""
    import torch
    from paper_2412_08346_gb300 import learned_init, proposal, synth
    stream = torch.cuda.current_stream().cuda_stream
    clouds = learned_init.object_clouds(32, 2048, synth.BASE_SEED + 50_000)
    tg = np.zeros((32, 3, 16, 7), np.float32)
    tg[..., :3] = clouds.mean(1)[:, None, None, :]
    tg[..., 3] = 1.0
    net = proposal.Proposal(3, 2048, 32, stream)
    try:
        net.set_params(synth.proposal_params(3, synth.BASE_SEED))
        out, _ = net.forward(clouds, 32)
        loss, _ = net.loss_grad(clouds, tg, 32, 16)
        print(f"proposal: outputs {out.shape}, loss {loss:.4f}")
    finally:
        net.close()


def run_batched(args):
    """Many objects in one context (one launch per kernel for all of them, one captured loop) against the
    plain path (each object in its own context, run one after the other); same per-object results."""
    import torch
    from paper_2412_08346_gb300 import asicp, synth
    w, K = synth.batched_case(args.batched)
    nobj, P = len(w.objects), len(w.preshapes)
    stream = torch.cuda.current_stream()
    pre_dev = [(torch.from_numpy(p.S).cuda(), torch.from_numpy(p.sdf).cuda()) for p in w.preshapes]
    obj_dev = [torch.from_numpy(o.points).cuda() for o in w.objects]

    def make(n, counts, shape):
        cfg = asicp.asicp_config_default(P=P, K=int(K.max()), k_max=w.k_max, k_stein=w.k_stein,
                                         schedule=w.schedule, cuda_stream=stream.cuda_stream, n_objects=n,
                                         fwd_shape=max(0, shape))
        ctx = asicp.asicp_create(cfg)
        asicp.asicp_set_particle_counts(ctx, np.ascontiguousarray(counts.ravel(), np.int32))
        for p, (S, g) in enumerate(pre_dev):
            asicp.asicp_set_gripper_sdf(ctx, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
        return ctx

    def best_cost(ctx, o=None):
        th, c, pr = np.zeros(7, np.float32), np.zeros(1, np.float32), np.zeros(1, np.int32)
        if o is None:
            asicp.asicp_best_grasps(ctx, 1, th, c, pr)
        else:
            asicp.asicp_best_grasps_at(ctx, o, 1, th, c, pr)
        return float(c[0])

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    ctx = make(nobj, K, args.fwd_shape)
    try:
        for o, R in enumerate(obj_dev):
            asicp.asicp_set_object_at(ctx, o, R)
        shape = asicp.asicp_autotune(ctx)[0] if args.fwd_shape < 0 else args.fwd_shape

        def batched_set():
            asicp.asicp_run(ctx)
            return [best_cost(ctx, o) for o in range(nobj)]
        batched_set()                                    # warm-up (captures the loop)
        runs = [timed(batched_set) for _ in range(max(1, args.steps))]
        batched_ms = sum(r[0] for r in runs) / len(runs)
        batched_cost = runs[-1][1]
    finally:
        asicp.asicp_destroy(ctx)

    solo_ms, solo_cost = 0.0, []
    for o in range(nobj):
        c1 = make(1, K[o], shape)
        try:
            asicp.asicp_set_object(c1, obj_dev[o])

            def solo_set():
                asicp.asicp_run(c1)
                return best_cost(c1)
            solo_set()                                   # warm-up (captures the loop)
            t, c = timed(solo_set)
            solo_ms += t
            solo_cost.append(c)
        finally:
            asicp.asicp_destroy(c1)
    rel = max(abs(a - b) / max(abs(b), 1e-30) for a, b in zip(batched_cost, solo_cost))
    pairs = sum(int(K[o].sum()) * w.preshapes[0].S.shape[0] * len(w.objects[o].points) for o in range(nobj))
    print(json.dumps({
        "metric": "ms per grasp set, objects optimised together vs each alone, at equal cost",
        "value": batched_ms / nobj, "unit": "ms/grasp set", "higher_is_better": False,
        "solo_ms_per_grasp_set": solo_ms / nobj, "speedup_vs_solo": solo_ms / batched_ms,
        "batched_pairs_per_s": pairs * (w.k_max + 1) / (batched_ms / 1e3),
        "max_best_cost_rel_diff_vs_solo": rel, "steps": len(runs), "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "objects": nobj, "M_min": min(len(o.points) for o in w.objects),
                   "M_max": max(len(o.points) for o in w.objects), "particles": int(K.sum()),
                   "pairs_per_iteration": pairs, "fwd_shape": asicp.FWD_VARIANTS[shape]}}), flush=True)


def run_compare(args):
    """The plain FP32 GPU method (float32 matching, Fibonacci, 256 particles per preshape, 100
    iterations) against faster forms on the same objects, at equal final cost: a form counts for an
    object when its best final cost (non-colliding first) is within 1 % of the plain method's; the
    time to reach equal cost is that of the fastest form that does.  Forms: the tensor-core matching
    at the same budget and at shorter (particles, iterations) budgets, each object alone, and all
    objects optimised together in one batched context."""
    import torch
    from paper_2412_08346_gb300 import asicp, synth
    n_obj = args.compare
    stream = torch.cuda.current_stream()
    w = synth.paper_scale_case(seed=synth.BASE_SEED + 2)
    P, N = len(w.preshapes), w.preshapes[0].S.shape[0]
    objs = [synth.partial_object(8192, synth.BASE_SEED + 2 + 1000 * (o + 1)) for o in range(n_obj)]
    pre_dev = [(torch.from_numpy(p.S).cuda(), torch.from_numpy(p.sdf).cuda()) for p in w.preshapes]
    obj_dev = [torch.from_numpy(o.points).cuda() for o in objs]
    f32_shape = asicp.FWD_VARIANTS.index("qpt8-chunk64-t128-tile1024")
    tc_shape = asicp.FWD_VARIANTS.index(TC_SHAPE)

    def make(nobj, K, k_max, shape):
        cfg = asicp.asicp_config_default(P=P, K=K, k_max=k_max, k_stein=synth.k_stein_for(k_max), schedule=0,
                                         cuda_stream=stream.cuda_stream, n_objects=nobj, fwd_shape=shape)
        ctx = asicp.asicp_create(cfg)
        for p, (S, g) in enumerate(pre_dev):
            asicp.asicp_set_gripper_sdf(ctx, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
        return ctx

    def best_cost(ctx, o):
        c = np.zeros(1, np.float32)
        asicp.asicp_best_grasps_at(ctx, o, 1, np.zeros(7, np.float32), c, np.zeros(1, np.int32))
        return float(c[0])

    def run_form(K, k_max, shape, batched):
        """(ms per grasp set per object, best cost per object); each timed run after a warm-up run."""
        ms, cost = np.zeros(n_obj), np.zeros(n_obj)
        groups = [list(range(n_obj))] if batched else [[o] for o in range(n_obj)]
        for grp in groups:
            ctx = make(len(grp), K, k_max, shape)
            try:
                for i, o in enumerate(grp):
                    asicp.asicp_set_object_at(ctx, i, obj_dev[o])
                asicp.asicp_run(ctx)                          # warm-up (captures the loop)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                asicp.asicp_run(ctx)
                c = [best_cost(ctx, i) for i in range(len(grp))]
                e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1)
                for i, o in enumerate(grp):
                    ms[o] = t / len(grp)
                    cost[o] = c[i]
            finally:
                asicp.asicp_destroy(ctx)
        return ms, cost

    plain_ms, plain_cost = run_form(256, 100, f32_shape, False)
    target = plain_cost * 1.01
    forms = [("tensor cores, 256 x 100", 256, 100, tc_shape, False),
             ("tensor cores, batched, 256 x 100", 256, 100, tc_shape, True),
             ("tensor cores, batched, 256 x 60", 256, 60, tc_shape, True),
             ("tensor cores, batched, 128 x 100", 128, 100, tc_shape, True),
             ("tensor cores, batched, 128 x 60", 128, 60, tc_shape, True),
             ("tensor cores, batched, 64 x 60", 64, 60, tc_shape, True),
             ("tensor cores, batched, 64 x 40", 64, 40, tc_shape, True)]
    res, best_ms = [], np.full(n_obj, np.inf)
    for name, K, k_max, shape, batched in forms:
        ms, cost = run_form(K, k_max, shape, batched)
        ok = cost <= target
        best_ms = np.where(ok, np.minimum(best_ms, ms), best_ms)
        res.append({"form": name, "particles_per_preshape": K, "iterations": k_max,
                    "ms_per_grasp_set": float(np.mean(ms)), "objects_at_equal_cost": int(ok.sum()),
                    "median_cost_ratio_vs_plain": float(np.median(cost / np.maximum(plain_cost, 1e-30)))})
    reached = np.isfinite(best_ms)
    speed = plain_ms[reached] / best_ms[reached]
    print(json.dumps({
        "metric": "ms per grasp set vs the plain FP32 GPU method, at equal cost (best final cost within 1 %)",
        "value": float(np.median(best_ms[reached])) if reached.any() else None, "unit": "ms/grasp set",
        "higher_is_better": False, "plain_ms_per_grasp_set": float(np.mean(plain_ms)),
        "speedup_at_equal_cost_median": float(np.median(speed)) if reached.any() else None,
        "speedup_at_equal_cost_min": float(np.min(speed)) if reached.any() else None,
        "objects_reaching_equal_cost": int(reached.sum()), "objects": n_obj, "forms": res,
        "plain": {"form": "float32 matching, Fibonacci, 256 x 100, one object at a time",
                  "median_best_cost": float(np.median(plain_cost))},
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"partial-P{P}-K256-N{N}-M8192-sdf64-it100 x {n_obj} objects",
                   "equal_cost": "best final cost <= 1.01 x the plain method's, per object"}}), flush=True)


def run_k_sweep(args):
    """Time per grasp set against the particle count (the paper's time-versus-initialisations axis):
    the paper-scale workload with K = 32 .. 1024 particles per preshape, the kernel shape autotuned
    for each K, L2 flushed before every timed run."""
    import torch
    from paper_2412_08346_gb300 import asicp, synth
    w = synth.paper_scale_case()
    P, N, M = len(w.preshapes), w.preshapes[0].S.shape[0], len(w.objects[0].points)
    stream = torch.cuda.current_stream()
    R_dev = torch.from_numpy(w.objects[0].points).cuda()
    pre_dev = [(torch.from_numpy(p.S).cuda(), torch.from_numpy(p.sdf).cuda()) for p in w.preshapes]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rows = []
    for K in (32, 64, 128, 256, 512, 1024):
        cfg = asicp.asicp_config_default(P=P, K=K, k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule,
                                         cuda_stream=stream.cuda_stream)
        ctx = asicp.asicp_create(cfg)
        try:
            asicp.asicp_set_object(ctx, R_dev)
            for p, (S, g) in enumerate(pre_dev):
                asicp.asicp_set_gripper_sdf(ctx, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
            shape, _ = asicp.asicp_autotune(ctx)
            for _ in range(2):
                asicp.asicp_run(ctx)
            times = []
            for _ in range(max(2, args.steps)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                asicp.asicp_run(ctx)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            rows.append({"K": K, "ms_per_grasp_set": ms, "pairs_per_s": P * K * N * M * (w.k_max + 1) / (ms / 1e3),
                         "fwd_shape": asicp.FWD_VARIANTS[shape]})
        finally:
            asicp.asicp_destroy(ctx)
    print(json.dumps({"metric": "ms per grasp set against particles per preshape", "unit": "ms/grasp set",
                      "higher_is_better": False, "config": {"workload": w.name, "P": P, "N": N, "M": M,
                                                            "iterations": w.k_max},
                      "sweep": rows, "data": "synthetic"}), flush=True)


def run_large(args):
    """The mixed-precision configuration (3 preshapes x 1024 particles, N=4096, M=65536 superquadric
    partial view, SDF 128^3): the float32 matching kernel (the autotuner's best float32 shape) and the
    tensor-core screening + exact choice, each timed over a 4-iteration run (per-launch device time
    from the library's event timers), and the fraction of correspondences on which the two agree in
    one step from the same poses."""
    import torch
    from paper_2412_08346_gb300 import asicp, synth
    import oracle
    w = synth.large_case(k_max=4)
    P, K, N, M = len(w.preshapes), w.K, w.preshapes[0].S.shape[0], len(w.objects[0].points)
    stream = torch.cuda.current_stream()
    R_dev = torch.from_numpy(w.objects[0].points).cuda()
    pre_dev = [(torch.from_numpy(p.S).cuda(), torch.from_numpy(p.sdf).cuda()) for p in w.preshapes]
    com = w.objects[0].points.astype(np.float64).mean(0)
    th0 = np.tile(oracle.fibonacci_init(K, com, 0.15), (P, 1)).astype(np.float32)
    tc_shape = asicp.FWD_VARIANTS.index(TC_SHAPE)
    out, idx = {}, {}
    for name, shape in (("float32", 5), ("tensor_core", tc_shape)):
        cfg = asicp.asicp_config_default(P=P, K=K, k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, profile=1,
                                         debug=1, cuda_stream=stream.cuda_stream, fwd_shape=shape)
        ctx = asicp.asicp_create(cfg)
        try:
            asicp.asicp_set_object(ctx, R_dev)
            for p, (S, g) in enumerate(pre_dev):
                asicp.asicp_set_gripper_sdf(ctx, p, S, g, w.preshapes[p].origin, w.preshapes[p].voxel)
            asicp.asicp_set_state(ctx, th0, 0)
            asicp.asicp_step(ctx, 0)
            nn = np.zeros((P * K, N), np.int32)
            asicp.asicp_get_state(ctx, nn_idx=nn)
            idx[name] = nn
            asicp.asicp_run(ctx, th0)                 # warm-up (captures the loop)
            torch.cuda.synchronize()
            asicp.asicp_kernel_times(ctx, reset=True)
            asicp.asicp_run(ctx, th0)
            ms, n = asicp.asicp_kernel_times(ctx, reset=True)
            per = (ms[0] / n[0]) + (ms[5] / n[5] if n[5] else 0.0)
            out[name] = {"fwd_shape": asicp.FWD_VARIANTS[shape], "matching_ms_per_pass": per,
                         "pairs_per_s": P * K * N * M / (per / 1e3),
                         "kernel_ms_per_pass": {k: v / max(c, 1) for k, v, c in zip(asicp.KERNEL_KINDS, ms, n)}}
        finally:
            asicp.asicp_destroy(ctx)
    same = float(np.mean(idx["float32"] == idx["tensor_core"]))
    print(json.dumps({"metric": "matching ms per pass, float32 vs tensor-core shape (mixed-precision configuration)",
                      "config": {"workload": w.name, "P": P, "K": K, "N": N, "M": M,
                                 "pairs_per_pass": P * K * N * M},
                      "float32": out["float32"], "tensor_core": out["tensor_core"],
                      "speedup": out["float32"]["matching_ms_per_pass"] / out["tensor_core"]["matching_ms_per_pass"],
                      "identical_correspondences": same, "queries": int(idx["float32"].size),
                      "data": "synthetic"}), flush=True)


def run_learned(args):
    """Learned initial poses (64 particles per preshape, 30 iterations) against the plain method
    (256 Fibonacci particles, 100 iterations) and against Fibonacci at the learned budget."""
    import torch
    from paper_2412_08346_gb300 import learned_init, proposal, synth
    n_train, n_test = (int(x) for x in args.learned.split(","))
    stream = torch.cuda.current_stream().cuda_stream
    pre = synth.make_preshapes(3, 2048, 64, synth.BASE_SEED + 5)
    train_clouds = learned_init.object_clouds(n_train, 2048, synth.BASE_SEED + 50_000)
    test_clouds = learned_init.object_clouds(n_test, 2048, synth.BASE_SEED + 90_000)
    t0 = time.perf_counter()
    targets, _ = learned_init.converged_targets(train_clouds, pre, stream=stream)
    t_data = time.perf_counter() - t0
    net = proposal.Proposal(3, 2048, 32, stream)
    net.set_params(synth.proposal_params(3, synth.BASE_SEED))
    t0 = time.perf_counter()
    hist = learned_init.train(net, train_clouds, targets, epochs=args.learned_epochs, batch=32, lr=1e-3, seed=1)
    t_train = time.perf_counter() - t0
    res = learned_init.compare(net, test_clouds, pre, stream)
    eq = res["equal_cost"]
    res.update({"metric": "ms per grasp set at equal cost (best final cost within 1 % of the plain method), "
                          "learned initial poses refined by SGD-ICP",
                "value": eq["learned_sgd"]["median_ms_when_reached"], "unit": "ms/grasp set",
                "higher_is_better": False,
                "train_objects": n_train, "test_objects": n_test, "train_targets_s": t_data, "train_s": t_train,
                "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1], "epochs": len(hist),
                "data": "synthetic", "dtype": "bf16 weights, f32 accumulate"})
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.learned:
        run_learned(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.compare:
        run_compare(args)
        return
    if args.large:
        run_large(args)
        return
    if args.k_sweep:
        run_k_sweep(args)
        return
    if args.oracle_configs:
        run_oracle_configs(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_proposal:
        run_profile_proposal(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
