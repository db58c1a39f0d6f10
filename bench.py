"""Benchmark: noisy-inverse Pauli propagation on B300.

A step is one whole backward propagation of the workload's observable through
every layer (R_X layer, inverse noise, R_ZZ layer per Trotter step, with
truncation) plus the expectation on |0..0>.  Metric: Pauli-term updates per
second, the canonical gate-by-gate count (sum over gates of the live terms
entering the gate).

Workload (default): 7x8 open-boundary TFIM, 56 qubits, 20 Trotter steps,
R_ZZ(0.3), R_X(0.6), observable the mean of Z_a Z_b over the 97 edges, rates
uniform [0, 1e-3), weight cap 10, threshold 1e-6 -- the smallest threshold of
its 1e-4..1e-7 sweep that fits one GPU -- in the FP32-coefficient form.  The
6x6 / 10-step FP64 workload needs about 1e10 live strings (more than a B300
holds) and is not a single-GPU configuration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun) are independent replicas: every rank propagates the
same workload, no data-path collective; value = updates of all ranks / the
slowest rank's time.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2606_20441_b300 import inputs  # noqa: E402

METRIC = "Pauli-term updates/s"
UNIT = "updates/s"
PROFILE = os.path.join(ROOT, "profiles", "k_process_warp_tfim7x8.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2606_20441_b300", "csrc", f)
                  for f in ("pp_device.cuh", "pp_kernels.cuh", "pp_warp.cuh")]


def workload(args):
    if args.workload == "tfim7x8":
        return inputs.workload_7x8(eps=args.eps, w_max=10)
    if args.workload == "tfim6x6":
        return inputs.workload_6x6(eps=args.eps)
    raise SystemExit("unknown workload " + args.workload)


def oracle_sample(args, steps):
    """The same workload family cut to its first `steps` Trotter steps (same
    seed, same per-step rates): a bounded sample for the CPU oracle."""
    if args.workload == "tfim7x8":
        return inputs.workload_7x8(eps=args.eps, w_max=10, steps=steps)
    return inputs.workload_6x6(eps=args.eps, steps=steps)


def config_of(args, inst, precision=None):
    m = inst.meta
    return {"workload": "%s_s%d_eps%g_wmax%d" % (args.workload, m["steps"], args.eps, inst.w_max),
            "lattice": "%dx%d" % (m["rows"], m["cols"]), "qubits": inst.n_qubits,
            "trotter_steps": m["steps"], "eps": args.eps, "w_max": inst.w_max,
            "coefficients": "fp%d" % (precision or args.precision), "noise": "inverse sparse Pauli-Lindblad, "
            "3n + 9|E| generators per step", "l2": "working set (>1 GB of strings) larger than L2",
            "parallelism": "replicas"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers

def kernel_source_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def profiled_traffic(strings_per_launch, precision, plan):
    """DRAM bytes per launch of the main-tier kernel from the committed ncu
    summary, scaled by strings processed, or None when the kernel source or
    the plan (fused gates, bucket headroom: they set how full the buckets'
    regions are) changed since the counters were taken."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(r"dram_bytes_per_string_fp%d:\s*([0-9.eE+]+)" % precision, txt)
    m_plan = re.search(r"plan:\s*max_fused_gates=(\d+)\s+bucket_headroom=([0-9.]+)", txt)
    if not m_sha or not m_tr or not m_plan or m_sha.group(1) != kernel_source_sha():
        return None
    if (int(m_plan.group(1)), float(m_plan.group(2))) != (int(plan[0]), round(float(plan[1]), 6)):
        return None
    return float(m_tr.group(1)) * strings_per_launch


def set_difference_counts(a, b):
    """Strings present in export a and not in b, and the reverse, from (x, z,
    c) exports, counted on the GPU (sorted 64-bit hashes of the keys)."""
    import torch

    def hashes(e):
        x = torch.from_numpy(np.ascontiguousarray(e[0]).view(np.int64)).cuda()
        z = torch.from_numpy(np.ascontiguousarray(e[1]).view(np.int64)).cuda()
        h = torch.zeros(x.shape[0], dtype=torch.int64, device="cuda")
        for w in range(x.shape[1]):
            h = h * 0x100000001B3 + x[:, w] * 0x1F3D5B79 + z[:, w] * 0x2545F491 + (x[:, w] ^ (z[:, w] << 7))
        return h
    ha, hb = hashes(a), hashes(b)
    only_a = int((~torch.isin(ha, hb)).sum().item())
    only_b = int((~torch.isin(hb, ha)).sum().item())
    del ha, hb
    torch.cuda.empty_cache()
    return only_a, only_b


def replica_totals(sec, updates, device):
    """Whole-job numbers of independent replicas (one per rank): the slowest
    rank's time and the sum of all ranks' updates."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([sec], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def run_oracle_sample(args, steps):
    from oracle import oracle
    inst = oracle_sample(args, steps)
    t = time.perf_counter()
    r = oracle.run(inst)
    return r.updates, time.perf_counter() - t


def host_cpu():
    """The host's CPU model and logical core count, for the baseline lines."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def _oracle_updates(inst):
    from oracle import oracle
    return oracle.run(inst).updates


def _oracle_warm(_):
    from oracle import oracle
    oracle.lib()
    return 0


def oracle_pool_baseline(instances, updates_hint, seconds=15.0, rate_guess=1.0e6):
    """The oracle on the host's cores over a bounded sample of independent
    instances: the smallest ones (by the GPU run's update counts) whose total,
    at about `rate_guess` updates per second per core, fills about `seconds` of
    every core; one spawned process per core.  Instances still running after
    3 x `seconds` are abandoned and only the finished ones count."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    order = sorted(range(len(instances)), key=lambda k: updates_hint[k])
    budget = rate_guess * seconds * cores
    pick, tot = [], 0.0
    for k in order:
        u = updates_hint[k]
        if u <= 0 or u > rate_guess * seconds or tot + u > budget:
            continue
        pick.append(k)
        tot += u
    if not pick:
        return None
    procs = min(cores, len(pick))
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(processes=procs)
    try:
        pool.map(_oracle_warm, range(procs), chunksize=1)   # start-up (import, load the oracle), untimed
        t = time.perf_counter()
        deadline = t + 3.0 * seconds
        it = pool.imap_unordered(_oracle_updates, [instances[k] for k in pick], chunksize=1)
        upd, done = 0.0, 0
        while done < len(pick):
            left = deadline - time.perf_counter()
            if left <= 0:
                break
            try:
                upd += it.next(timeout=left)
                done += 1
            except mp.TimeoutError:
                break
        sec = time.perf_counter() - t
    finally:
        pool.terminate()
        pool.join()
    if done == 0:
        return None
    return {"value": upd / sec, "unit": UNIT, "cores": procs, "kind": "oracle", "host": host_cpu(),
            "sample": "%d of the %d instances (the smallest by update count; %d finished in the time "
                      "bound), %.2g updates, one process per core, FP64 hash-map oracle, %.1f s"
                      % (len(pick), len(instances), done, upd, sec)}


# ----------------------------------------------------------------------------- arms

def reference_arm(args, rank, world):
    """The CPU oracle as it stands, on the host cores, rank 0 only."""
    if rank != 0:
        return
    inst = workload(args)
    for _ in range(args.warmup):
        run_oracle_sample(args, 1)
    upd, sec = 0.0, 0.0
    for _ in range(args.steps):
        u, s = run_oracle_sample(args, args.sample_steps)
        upd += u
        sec += s
    v = upd / sec
    sample = ("%s cut to its first %d Trotter steps per timed step (warm-up steps: first 1 step); "
              "single-threaded FP64 hash-map oracle" % (args.workload, args.sample_steps))
    cfg = config_of(args, inst, precision=64)
    cfg["sample"] = "first %d of the %d Trotter steps per timed step" % (args.sample_steps, inst.meta["steps"])
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ours_arm(args, rank, world, local_rank):
    import torch
    from paper_2606_20441_b300 import build, pp

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local_rank)
    build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    inst = workload(args)
    h = pp.Handle(inst.n_qubits, precision=args.precision, timing=True)
    plan = h.pp_get_tuning()
    h.load_instance(inst)
    for _ in range(args.warmup):
        h.run_instance(inst)
        h.pp_expect()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = int(vis.split(",")[local_rank]) if vis and vis.split(",")[local_rank].isdigit() else local_rank
    clocks = ClockSampler(phys)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    updates, launches = 0.0, 0
    tier_ms = [0.0] * pp.N_TIERS
    tier_strings = [0.0] * pp.N_TIERS
    tier_launches = [0] * pp.N_TIERS
    expect = None
    for _ in range(args.steps):
        h.run_instance(inst)
        expect = h.pp_expect()
        s = h.pp_get_stats()
        updates += s.updates
        launches += s.kernel_launches
        for t in range(pp.N_TIERS):
            tier_ms[t] += s.tier_ms[t]
            tier_strings[t] += s.tier_strings[t]
            tier_launches[t] += s.tier_launches[t]
        bps = s.bytes_per_string
        n_terms, peak = s.n_terms, s.peak_terms
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1000.0
    tot_updates = updates
    if dist:
        sec, tot_updates = replica_totals(sec, updates, "cuda")

    # end-to-end through the C ABI with host buffers: load circuit and noise,
    # propagate the host observable, read the expectation back, every step
    h2d = (inst.gate_x.nbytes + inst.gate_z.nbytes + inst.theta.nbytes + inst.layer_of.nbytes +
           sum(m.ex.nbytes + m.ez.nbytes + m.lam.nbytes for m in inst.noise) +
           inst.obs_x.nbytes + inst.obs_z.nbytes + inst.obs_c.nbytes)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_upd = 0.0
    for _ in range(args.steps):
        h.load_instance(inst)
        h.run_instance(inst)
        h.pp_expect()
        e2e_upd += h.pp_get_stats().updates
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_sec], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_sec = float(t.item())
        e2e_upd *= world

    # FP32 form against the FP64 form on the same workload (FP64 final sums in
    # both): the expectation error, the strings kept by one form and not the
    # other, the FP64 form's own speed, and how much the FP64 result moves when
    # its threshold moves by one FP32 rounding (2^-24 relative)
    fp32_vs_fp64 = None
    if args.precision == 32 and rank == 0 and not args.no_fp64_check:
        keys32 = h.pp_export_terms()
        h64 = pp.Handle(inst.n_qubits, precision=64)
        h64.load_instance(inst)
        t = time.perf_counter()
        h64.run_instance(inst)
        e64 = h64.pp_expect()
        sec64 = time.perf_counter() - t
        upd64 = h64.pp_get_stats().updates
        keys64 = h64.pp_export_terms()
        sens = []
        for f in (1.0 + 2.0 ** -24, 1.0 - 2.0 ** -24):
            h64.run_instance(inst, eps=args.eps * f)
            sens.append(h64.pp_expect() - e64)
        h64.close()
        only32, only64 = set_difference_counts(keys32, keys64)
        fp32_vs_fp64 = {"abs_err": abs(expect - e64), "expect_fp64": e64,
                        "strings_only_fp32": only32, "strings_only_fp64": only64,
                        "terms_fp32": int(len(keys32[2])), "terms_fp64": int(len(keys64[2])),
                        "fp64_ms_per_step": 1000.0 * sec64, "fp64_updates_per_s": upd64 / sec64,
                        "fp64_threshold_sensitivity": {"eps*(1+2^-24)": sens[0], "eps*(1-2^-24)": sens[1]}}
        del keys32, keys64
    h.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak_gbs, peak_kind = read_peaks()
    main_ms_avg = tier_ms[0] / max(1, tier_launches[0])
    main_bytes = tier_strings[0] * bps / max(1, tier_launches[0])
    achieved = main_bytes / (main_ms_avg / 1000.0) / 1e9 if main_ms_avg > 0 else 0.0
    roofline = {"bound": "hbm", "limiter": "instruction issue and shared-memory latency of the gate rounds, "
                "not DRAM bandwidth (profiles/k_process_warp_tfim7x8.md)",
                "kernel": "k_process_warp<1, float, 4> (tier 0: one warp per bucket, 248-string tiles in shared "
                          "memory, 4 warps per CTA)",
                "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": main_bytes, "avg_launch_ms": main_ms_avg,
                "traffic": profiled_traffic(tier_strings[0] / max(1, tier_launches[0]), args.precision,
                                            plan),
                "share_of_step_time": (tier_ms[0] / 1000.0) / sec if sec > 0 else None,
                "plan": {"max_fused_gates": plan[0], "bucket_headroom": plan[1]}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        u, s_ = run_oracle_sample(args, args.sample_steps)
        cpu = {"value": u / s_, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": "%s cut to its first %d Trotter steps (%.3g updates in %.1f s), "
                         "single-threaded FP64 hash-map oracle" % (args.workload, args.sample_steps, u, s_)}
    line = {"metric": METRIC, "value": tot_updates / sec, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f%d" % args.precision, "data": "synthetic", "config": config_of(args, inst),
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_upd / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 8},
            "clocks": clk, "gpu_launches": launches,
            "result": {"expect": expect, "terms": int(n_terms), "peak_terms": int(peak),
                       "updates_per_step": updates / args.steps,
                       "fp32_abs_err_vs_fp64": fp32_vs_fp64["abs_err"] if fp32_vs_fp64 else None},
            "fp32_vs_fp64": fp32_vs_fp64,
            "tiers_ms_per_step": [m / args.steps for m in tier_ms]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def pool_arm(args, rank, world, local_rank):
    """Many independent instances on one GPU: the 64-instance batch (all
    requests present at once, largest first) or a Poisson request stream,
    through the serving loop (small-share workers plus large-share workers for
    requests that outgrow a small share; each worker on its own CUDA stream
    with its own handle; the plan autotuner learning per workload class on live
    traffic).  The same instances are then run one after another through the
    plain single-instance path in FP64 (the throughput to compare with, and the
    FP32 form's error against FP64 on every instance) and in FP32."""
    import torch
    from paper_2606_20441_b300 import autotune, build, pp, serving
    torch.cuda.set_device(local_rank)
    build.build()
    # the tightest setting at which every instance fits its worker's share of
    # the GPU within seconds (without a weight cap, some instances of the batch
    # outgrow a worker's share and run for tens of seconds)
    eps, w_max = 1e-4, 8
    if args.workers <= 0:
        args.workers = 8 if args.workload == "batch64" else 12
    if args.workload == "batch64":
        insts = inputs.workload_batch64(eps=eps, w_max=w_max)
        reqs = serving.batch_order([inputs.Request(i, 0.0, inst) for i, inst in enumerate(insts)])
        cfg = {"workload": "batch64_eps%g_wmax%d" % (eps, w_max), "instances": len(insts),
               "lattices": "4x4..8x8", "trotter_steps": "5-25"}
    else:
        reqs = inputs.workload_serving(count=args.requests, rate_hz=args.rate, eps_set=(eps,), w_max=w_max)
        insts = [r.instance for r in reqs]
        cfg = {"workload": "serving_poisson%gHz_eps%g_wmax%d" % (args.rate, eps, w_max), "requests": len(reqs),
               "lattices": "4x4..10x10", "trotter_steps": "5-30"}
    n_large = 2
    cfg.update({"coefficients": "fp%d" % args.precision, "parallelism": "replicas",
                "workers": "%d small + %d large" % (args.workers, n_large), "l2": "working set larger than L2"})
    budget = 0.6 * torch.cuda.mem_get_info()[0]
    tuner = autotune.Tuner()
    ex = serving.GpuExecutor(n_small=args.workers, hbm_budget_bytes=budget, precision=args.precision,
                             n_large=n_large, large_fraction=0.3, tuner=tuner)
    # warm-up: every worker runs a small request (not seen by the tuner)
    ex.tuner = None
    small = inputs.workload_batch64(count=args.workers + n_large, eps=1e-3, w_max=6)
    serving.Server(ex, n_workers=args.workers, n_large=n_large).serve(
        [inputs.Request(i, 0.0, x) for i, x in enumerate(small)])
    ex.tuner = tuner
    torch.cuda.synchronize()
    out = serving.Server(ex, n_workers=args.workers, n_large=n_large, route_key=autotune.class_key,
                         backlog="largest_first", exclusive=True).serve(reqs)
    torch.cuda.synchronize()
    ex.close()
    torch.cuda.empty_cache()   # the workers' memory went back to torch's cache
    summ = serving.summarize(out)
    # the plain single-instance path over the same instances, one at a time:
    # FP64 (the comparison point, and the FP32 form's error on every instance)
    # and FP32 (what running them one by one in the same form would give)
    def sequential(precision):
        upd, secs, res = 0.0, 0.0, {}
        per = 16 + (4 if precision == 32 else 8)
        hs = {1: pp.Handle(64, precision=precision, max_terms=int(budget / 2.6 / per / 2)),
              2: pp.Handle(128, precision=precision, max_terms=int(budget / 2.6 / (per + 16) / 2))}
        for r in reqs:
            h = hs[r.instance.W]
            h.load_instance(r.instance)
            t = time.perf_counter()
            try:
                h.run_instance(r.instance)
                res[r.rid] = h.pp_expect()
                upd += h.pp_get_stats().updates
            except pp.PPError:
                pass
            secs += time.perf_counter() - t
        for h in hs.values():
            h.close()
        return (upd / secs if secs > 0 else None), res

    # the batch's instances once more as one lockstep batch (pp_propagate_batch:
    # every instance advances one fused sub-layer per step and each kernel is
    # launched once per step for all of them), FP32
    lockstep = None
    if args.workload == "batch64":
        hs = [pp.Handle(i.n_qubits, precision=args.precision) for i in insts]
        for h, i in zip(hs, insts):
            h.load_instance(i)
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = pp.pp_propagate_batch(hs, insts, eps=eps, w_max=w_max)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t
        upd = sum(h.pp_get_stats().updates for h, x in zip(hs, st) if x == pp.PP_OK)
        lockstep = {"updates_per_s": upd / sec, "seconds": sec,
                    "completed": sum(1 for x in st if x == pp.PP_OK), "instances": len(insts)}
        for h in hs:
            h.close()
        torch.cuda.empty_cache()

    single64 = single32 = None
    errs = []
    if not args.no_single:
        single64, e64 = sequential(64)
        single32, _ = sequential(32)
        for o in out:
            if o.status == pp.PP_OK and o.rid in e64:
                errs.append(abs(o.expect - e64[o.rid]))
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        by_rid = {o.rid: o for o in out}
        ok = [r for r in reqs if by_rid[r.rid].status == pp.PP_OK]
        cpu = oracle_pool_baseline([r.instance for r in ok], [by_rid[r.rid].updates for r in ok])
    line = {"metric": METRIC, "value": summ["updates_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": summ["span_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f%d" % args.precision, "data": "synthetic",
            "config": cfg, "served": summ["served"], "failed": summ["failed"],
            "escalated": summ["escalated"], "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"],
            "single_instance_fp64_updates_per_s": single64, "single_instance_fp32_updates_per_s": single32,
            "lockstep": lockstep,
            "fp32_vs_fp64_abs_err": ({"max": max(errs), "median": statistics.median(errs)} if errs else None),
            "compared": len(errs), "cpu_baseline": cpu,
            "tuned": {k: list(tuner.best(k)) for k in sorted(tuner.samples)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="tfim7x8")
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--precision", type=int, choices=[32, 64], default=32)
    ap.add_argument("--sample-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--workers", type=int, default=0, help="small-share workers (0: 8 for batch64, 12 for serve)")
    ap.add_argument("--requests", type=int, default=150)
    ap.add_argument("--rate", type=float, default=2.0)
    ap.add_argument("--no-single", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
    elif args.workload in ("batch64", "serve"):
        pool_arm(args, rank, world, local_rank)
    else:
        ours_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
