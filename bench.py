"""Benchmark: HPR-LP on the medium sparse planted LP (m = 200k with 50% equalities,
n = 500k, ~5.2M nonzeros, Zipf(1.5) column counts, values +-10^U(-3,3), 20% free
columns), solved to KKT <= 1e-8 on one B300.

One step = one complete solve (power method + HPR iterations + checks; preprocessing
excluded, as in the paper's timing) with the inputs already on the device.  `value` is
the whole-job HPR iteration throughput (iterations of all ranks / max time over ranks);
the time to KKT <= 1e-8 and <= 1e-4 of the same solves are reported beside it.  `e2e`
is the same throughput through the public C ABI with host buffers: upload +
preprocessing + solve + download of (x, y, z) every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the oracle (plain FP64 CPU implementation) on the host cores
on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time-to-KKT≤1e-8 (s), HPR iters/s, HBM GB/s % of peak; chosen form vs plain FP64")
L2_BYTES = 126e6   # B300 L2
BATCH_METRIC = "HPR iterations/s summed over the LPs of the batch workload (LPs solved to tol per second beside it)"

# DRAM bytes per launch from one ncu capture of the medium planted LP (seed 0, full size,
# FP64; see profiles/), valid only for that workload and the kernel source they were
# taken on.
NCU_TRAFFIC = {
    "source_sha1": "5d2582d12f53f06f041989718808621ee9706288",
    "k_phase_x": 87558656,
    "k_phase_y": 72121600,
}
# FP64 warp instructions per launch (ncu smsp__inst_executed_pipe_fp64.sum) of the phase
# kernels on the same workload and kernel source (profiles/k_sell_traffic_medium_lp.md)
NCU_FP64 = {
    "source_sha1": "5d2582d12f53f06f041989718808621ee9706288",
    "k_phase_x": 290668,
    "k_phase_y": 203226,
}


def kernel_source_sha1():
    p = os.path.join(ROOT, "paper_2408_12179_b300", "csrc", "hpr_device.cuh")
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def algorithmic_bytes(nnz, n, m, precision=0):
    """Each array once per launch, gathered vectors counted once, 32-bit indices.
    FP64: x phase: A^T values+indices 12 nnz, row pointers 4n, gather y 8m, read x, x0,
    c, l, u 40n, write x_hat, x 16n; y phase: 12 nnz, 4m, gather x_hat 8n, read y, y0, b
    24m, write y 8m.  FP32 form: values 4 B, iterates x, x_hat, y 4 B (anchors and data
    stay FP64): x phase 8 nnz + 4n + 4m + (4 + 8 + 24)n + 8n, y phase 8 nnz + 4m + 4n +
    (4 + 8 + 8)m + 4m."""
    if precision == 1:
        return 8 * nnz + 4 * n + 4 * m + 36 * n + 8 * n, 8 * nnz + 4 * m + 4 * n + 20 * m + 4 * m
    bx = 12 * nnz + 4 * n + 8 * m + 40 * n + 16 * n
    by = 12 * nnz + 4 * m + 8 * n + 24 * m + 8 * m
    return bx, by


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem"

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR when it is set, else to a temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"hpr_bench_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, pw, mem, reasons = [], [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for dst, v in ((pw, parts[2]), (mem, parts[8] if len(parts) > 8 else "")):
                try:
                    dst.append(float(v))
                except ValueError:
                    pass
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "mem_mhz": statistics.median(mem) if mem else None,
                "power_w": statistics.median(pw) if pw else None}


def aggregate(torch, dist, secs, iters, device):
    """Whole-job figures over the ranks (replicas): the slowest rank's time and the sum
    of all ranks' iterations.  dist None: a single process."""
    if dist is None:
        return float(secs), float(iters)
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    k = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(k, op=dist.ReduceOp.SUM)
    return float(t.item()), float(k.item())


def memory_ceilings(hpr, phase_bytes, stream):
    """Ceilings measured live by the library's own probe kernels (integer consumers, no FP64
    work): a read-only stream of the phase's size and of 1 GiB launched alone after L2 was
    filled with other data, and the rate of random 8-byte gathers from an L2-resident array
    (each costs an L1 cache-tag lookup).  Context for the roofline: a phase reads ~10x more
    bytes than it writes, and every stored matrix entry gathers one vector entry."""
    r_phase, g_rate = hpr.memory_probe(int(max(phase_bytes, 1 << 20)), 1 << 18, stream)
    r_big, _ = hpr.memory_probe(1 << 30, 1 << 18, stream)
    return {"read_gbs_phase_size": r_phase, "read_gbs_1GiB": r_big, "gather_g_per_s": g_rate}


# the Section 4.2 ablation: DR, + restart & Halpern (HDR, fixed sigma), + sigma update (HDR),
# + relaxation (HPR, the method itself)
VARIANTS = {
    "hpr": dict(halpern=1, reflect=1, restart=1, sigma_update=1),
    "hdr": dict(halpern=1, reflect=0, restart=1, sigma_update=1),
    "hdr_fixed_sigma": dict(halpern=1, reflect=0, restart=1, sigma_update=0),
    "dr": dict(halpern=0, reflect=0, restart=0, sigma_update=0),
}


def fp64_per_launch(hpr, lp, layout, phase):
    """FP64 warp instructions of one normal-iteration launch of a phase in the FP64 form,
    counted from its sliced-ELL layout (hpr_layout_plan, the layout hpr_create builds): one
    DFMA per 32 stored entries (three for a slice of 2 or 3 steps, whose batch issues its
    FMAs predicated), one DADD merging the two FMA chains of a slice of 4 or more steps,
    log2(lanes per row) DADDs of the row's lane butterfly per slice, and the epilogue's five
    FP64 instructions (DADD, DFMA, DFMA, DMUL, DFMA) per work unit (each unit applies its
    32-row buffer once)."""
    import numpy as np

    k = 1 if phase == "x" else 0
    M = lp.A.T.tocsr() if phase == "x" else lp.A.tocsr()
    L = hpr.layout_plan(M, int(layout["sell_steps"][k]), float(layout["unit_cost"][k]))
    steps = np.diff(L["sptr"]) // 32
    units = len(L["wstart"]) - 1
    return int(L["sptr"][-1] // 32 + np.count_nonzero(steps == 2) + np.count_nonzero(steps >= 4)
               + int(L["slg"].astype(np.int64).sum()) + 5 * units)


def bucket_of(lp):
    """Size bucket of the batch workload's per-bucket autotuning: floor(log2 nnz)."""
    return int(math.floor(math.log2(max(lp.nnz, 1))))


def layout_opts(args):
    """Explicit sliced-ELL layout for every context (--sell-steps, --unit-cost), else none."""
    o = {}
    if args.sell_steps:
        o.update(sell_steps_a=args.sell_steps, sell_steps_t=args.sell_steps)
    if args.unit_cost:
        o.update(unit_cost_a=args.unit_cost, unit_cost_t=args.unit_cost)
    return o


def workload(args):
    from paper_2408_12179_b300 import lpgen

    if args.workload == "mcf":
        return lpgen.mcf_lp(args.seed, nodes=max(2, int(round(1_000_000 * args.scale))))
    if args.workload == "qap":
        return lpgen.qap_lp(args.seed, args.qap_n)
    if args.workload == "tiny":
        return lpgen.planted_tiny(args.seed)
    if args.workload == "mid":                     # the reference arm: its 1/200-scale LP
        return lpgen.planted_medium(args.seed, 0.005)
    return lpgen.planted_medium(args.seed, args.scale)


def config_dict(args, lp):
    if args.workload == "tiny":
        name = f"tiny planted LP (m={lp.m}, m1={lp.m1}, n={lp.n}, nnz={lp.nnz}, seed {args.seed})"
    elif args.workload == "qap":
        name = (f"QAP LP, Adams-Johnson linearisation, random flows and grid distances, N={args.qap_n} "
                f"(m={lp.m}, n={lp.n}, nnz={lp.nnz}, seed {args.seed})")
    elif args.workload == "mcf":
        name = (f"min-cost multicommodity flow LP (random geometric 8-NN digraph, 4 commodities; "
                f"m={lp.m}, m1={lp.m1}, n={lp.n}, nnz={lp.nnz}, seed {args.seed})")
    else:
        name = (f"medium sparse planted LP (m={lp.m}, m1={lp.m1}, n={lp.n}, nnz={lp.nnz}, "
                f"Zipf(1.5) column counts, values +-10^U(-3,3), 20% free columns, seed {args.seed})")
    bx, by = algorithmic_bytes(lp.nnz, lp.n, lp.m, args.precision)
    l2 = ("working set per iteration larger than L2 (no flush)" if bx + by > L2_BYTES else
          f"working set per iteration ({(bx + by) / 1e6:.0f} MB) fits in L2 (no flush: every iteration "
          f"of a solve re-reads the same data)")
    return {"workload": name,
            "scale": args.scale, "tol": args.tol,
            "precision": "fp64" if args.precision == 0 else "fp32 form, fp64 below kkt 1e-5",
            "variant": args.variant,
            "l2": l2}


def oracle_one_core(args, iters):
    """The oracle on ONE host core (OMP_NUM_THREADS=1 in a child process, as the CPU plan asks
    beside the all-core figure): HPR iterations/s over `iters` iterations of the workload."""
    code = ("import json, sys; sys.path.insert(0, %r); import oracle; import bench; "
            "lp = bench.workload(bench.parse_args(%r)); "
            "r = oracle.solve(lp, max_iter=%d, lambda_fixed=1.0, checks_cap=16, **bench.VARIANTS[%r]); "
            "print(json.dumps(r['info']['seconds']))") % (ROOT, sys.argv[1:], iters, args.variant)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        secs = float(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": iters / secs, "unit": "iter/s", "cores": 1, "sample": f"{iters} oracle iterations, one thread"}


def run_reference(args):
    """The oracle timed on the host cores on a bounded sample: `sample_iters` HPR
    iterations (with one check) of the full workload per step."""
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lp = workload(args)
    oracle.lib()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    it = args.sample_iters
    times = []
    for step in range(args.warmup + args.steps):
        r = oracle.solve(lp, max_iter=it, lambda_fixed=1.0, checks_cap=16, **VARIANTS[args.variant])
        if step >= args.warmup:
            times.append(r["info"]["seconds"])
    tot = sum(times)
    value = it * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, lp),
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": f"{it} oracle iterations (one check) of the full workload per step, "
                                       f"lambda fixed to 1"},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched workload: `count` uneven planted LPs solved together through hpr_batch_*
    (cluster launches for the LPs whose own solve takes the persistent cluster path, fused
    launches for the others), one context per LP.  Warm-up solves are capped at two check
    periods (graph capture, power method); the timed solve runs every LP to tol or the
    iteration cap.  Also times a sample of the LPs solved one by one and as a batch of
    their own (same instances, same options)."""
    import torch

    from paper_2408_12179_b300 import hpr, lpgen

    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    hpr.load()
    m_hi = max(600, int(round(50_000 * args.scale)))
    lps = lpgen.batch_family(args.seed + rank, args.count, 500, m_hi)
    stream = torch.cuda.Stream()
    opts = dict(tol=args.tol, precision=args.precision, persistent=args.persistent, **VARIANTS[args.variant])
    opts.update(layout_opts(args))
    t_create = time.perf_counter()
    if args.autotune:
        # one autotuned context per size bucket (floor(log2 nnz)); its layout is reused
        tuned = {}
        solvers = []
        for lp in lps:
            bucket = bucket_of(lp)
            if bucket not in tuned:
                s_ = hpr.Solver(lp, max_iter=args.max_iter, autotune=1, **opts)
                lay = s_.layout()
                tuned[bucket] = dict(sell_steps_a=lay["sell_steps"][0], sell_steps_t=lay["sell_steps"][1],
                                     unit_cost_a=lay["unit_cost"][0], unit_cost_t=lay["unit_cost"][1])
            else:
                s_ = hpr.Solver(lp, max_iter=args.max_iter, **tuned[bucket], **opts)
            solvers.append(s_)
    else:
        tuned = None
        solvers = [hpr.Solver(lp, max_iter=args.max_iter, **opts) for lp in lps]
    create_secs = time.perf_counter() - t_create
    batch = hpr.Batch(solvers, stream.cuda_stream)
    for s_ in solvers:
        s_.set_options(max_iter=300)
    for _ in range(args.warmup):
        batch.solve(args.tol)
    for s_ in solvers:
        s_.set_options(max_iter=args.max_iter)
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, res = batch.solve(args.tol)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clocks = sampler.stop()
    st = batch.stats()
    batch.close()
    conv = [r for r in res if r["status"] == hpr.HPR_OK]
    iters = sum(int(r["info"]["iters"]) for r in res)
    for s_ in solvers:
        s_.close()
    # the sample: fresh contexts for the first LPs (the layouts a solo solve gets), solved
    # one by one (after a warm-up solve each), then as a batch of their own
    k = min(args.solo_sample, len(solvers))
    sample = [hpr.Solver(lp, max_iter=args.max_iter, **(tuned[bucket_of(lp)] if tuned else {}), **opts)
              for lp in lps[:k]]
    for s_ in sample:
        s_.set_options(max_iter=300)
        s_.solve(args.tol)
        s_.set_options(max_iter=args.max_iter)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    solo_iters = 0
    for s_ in sample:
        solo_iters += int(s_.solve(args.tol)["info"]["iters"])
    torch.cuda.synchronize()
    solo_secs = time.perf_counter() - t1
    with hpr.Batch(sample, stream.cuda_stream) as b2:
        b2.solve(args.tol)
        t2 = time.perf_counter()
        b2.solve(args.tol)
        torch.cuda.synchronize()
        sample_batch_secs = time.perf_counter() - t2
    for s_ in sample:
        s_.close()
    if rank != 0:
        return
    nnz = sum(lp.nnz for lp in lps)
    bsum = sum(sum(algorithmic_bytes(lp.nnz, lp.n, lp.m, args.precision)) for lp in lps)
    batch_l2 = (f"all LPs' working sets together ({bsum / 1e6:.0f} MB a fused iteration) "
                + ("larger than L2 (no flush)" if bsum > L2_BYTES else "fit in L2 (no flush)"))
    line = {
        "metric": BATCH_METRIC, "value": iters / secs, "unit": "iter/s", "lp_per_s": len(conv) / secs,
        "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch of {len(lps)} uneven planted LPs (m log-uniform in [500, {m_hi}], "
                               f"n = 2.5 m, density log-uniform in [0.1%, 1%], medium-LP value rules; "
                               f"total nnz {nnz}, seed {args.seed})",
                   "tol": args.tol, "max_iter": args.max_iter, "variant": args.variant, "persistent": args.persistent,
                   "autotune": ({str(k): v for k, v in sorted(tuned.items())} if tuned else None),
                   "layout": layout_opts(args) or "library default",
                   "l2": batch_l2,
                   "create_s": create_secs},
        "batch_status": hpr.hpr_status_str(int(status)), "converged": len(conv), "count": len(lps),
        "time_to_all_s": secs, "iters_summed": iters, "iters_per_s_summed": iters / secs,
        "periods": st["periods"], "gpu_launches": int(st["fused_launches"] + sum(int(r["info"]["launches"]) for r in res)),
        "paths": {name: sum(int(r["info"]["path"]) == code for r in res)
                  for name, code in (("fused", 0), ("single_cta", 2), ("cluster", 4))},
        "converged_by_path": {name: sum(int(r["info"]["path"]) == code and r["status"] == hpr.HPR_OK for r in res)
                              for name, code in (("fused", 0), ("single_cta", 2), ("cluster", 4))},
        "sample": {"lps": k, "one_by_one_s": solo_secs, "as_batch_s": sample_batch_secs,
                   "speedup": solo_secs / sample_batch_secs, "iters": solo_iters},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_reference_batch(args):
    """The oracle on a bounded sample of the batch workload: `sample_iters` iterations of
    each of the first `solo_sample` LPs, reported as HPR iterations/s summed over LPs."""
    import oracle
    from paper_2408_12179_b300 import lpgen

    if int(os.environ.get("RANK", "0")) != 0:
        return
    m_hi = max(600, int(round(50_000 * args.scale)))
    lps = lpgen.batch_family(args.seed, args.count, 500, m_hi)[:args.solo_sample]
    oracle.lib()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    secs = 0.0
    its = 0
    for step in range(args.warmup + args.steps):
        for lp in lps:
            r = oracle.solve(lp, max_iter=args.sample_iters, lambda_fixed=1.0, checks_cap=16,
                             **VARIANTS[args.variant])
            if step >= args.warmup:
                secs += r["info"]["seconds"]
                its += args.sample_iters
    value = its / secs
    line = {"impl": "reference", "metric": BATCH_METRIC,
            "value": value, "unit": "iter/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"first {len(lps)} LPs of the batch workload", "tol": args.tol},
            "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.sample_iters} oracle iterations of each of {len(lps)} LPs"},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2408_12179_b300 import hpr

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    hpr.load()
    lp = workload(args)
    stream = torch.cuda.Stream()
    opts = dict(tol=args.tol, max_iter=args.max_iter, cuda_stream=stream.cuda_stream,
                precision=args.precision)
    if args.lambda_fixed > 0:
        opts["lambda_fixed"] = args.lambda_fixed   # profiling aid: skips the power method
    opts.update(VARIANTS[args.variant])
    if args.autotune:
        opts["autotune"] = 1
    opts.update(layout_opts(args))
    solver = hpr.Solver(lp, **opts)
    layout = solver.layout()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        solver.solve(args.tol)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        infos.append(solver.solve(args.tol)["info"])
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    iters = sum(i["iters"] for i in infos)
    secs, all_iters = aggregate(torch, dist if world > 1 else None, ms / 1e3, iters, "cuda")
    value = all_iters / secs

    # live per-kernel timing (CUDA events on the solver's stream) for the roofline: each phase
    # launched alone (an event between the phases), and the in-solve time per iteration (the
    # 150-iteration periods run as CUDA graphs with programmatic launches, checks included,
    # power method left out) split between the phases in the same proportion
    ms_x, ms_y, ms_it = solver.time_iteration(50)
    in_graph_ms = statistics.median((i["solve_time_s"] - i["power_time_s"]) * 1e3 / max(1, i["iters"])
                                    for i in infos)
    bx, by = algorithmic_bytes(lp.nnz, lp.n, lp.m, args.precision)
    peak, peak_kind = measured_peak()
    dom, dom_ms, dom_bytes = ("k_phase_x", ms_x, bx) if ms_x >= ms_y else ("k_phase_y", ms_y, by)
    dom_in_graph_ms = in_graph_ms * dom_ms / (ms_x + ms_y)
    ceil = memory_ceilings(hpr, dom_bytes, stream.cuda_stream)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    # every stored entry of the phase's matrix gathers one entry of the other vector
    gathers = lp.nnz
    gather_rate = gathers / (dom_ms * 1e-3) / 1e9
    traffic = None
    if (NCU_TRAFFIC["source_sha1"] == kernel_source_sha1() and args.workload == "medium" and args.scale == 1.0
            and args.seed == 0 and args.precision == 0 and args.variant == "hpr"):
        traffic = NCU_TRAFFIC.get(dom)          # captured on this workload only
    # the phases' second bound: FP64 issue (one DFMA per stored entry on B300's FP64 pipe)
    fp64 = None
    if args.precision == 0 and not args.autotune:
        f_peak = hpr.fp64_probe(stream.cuda_stream)
        f_model = fp64_per_launch(hpr, lp, layout, "x" if dom == "k_phase_x" else "y")
        f_inst, f_src = f_model, "counted from the layout"
        if traffic is not None and NCU_FP64["source_sha1"] == NCU_TRAFFIC["source_sha1"]:
            f_inst, f_src = NCU_FP64[dom], "ncu smsp__inst_executed_pipe_fp64.sum"
        f_ach = f_inst / (dom_ms * 1e-3) / 1e9
        f_ach_graph = f_inst / (dom_in_graph_ms * 1e-3) / 1e9
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        fp64 = {"bound": "alu", "unit": "G FP64 warp instructions/s", "instructions_per_launch": f_inst,
                "instructions_source": f_src, "instructions_model": f_model,
                "achieved": f_ach, "peak": f_peak, "frac": f_ach / f_peak,
                "in_graph_frac": f_ach_graph / f_peak,
                "peak_source": "hpr_fp64_probe (independent DFMA chains, this run)",
                "peak_nominal": sms * 2.032e9 / 16 / 1e9,
                "peak_nominal_source": "one FP64 warp instruction per 16 cycles per SM at 2032 MHz "
                                       "(ncu: the probe runs at 84% of it)"}
    iter_gbs = (bx + by) / (ms_it * 1e-3) / 1e9
    plain = None
    if args.compare_fp64 and args.precision != 0:
        solver.set_options(precision=0)
        p_ev0, p_ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p_ev0.record(stream)
        pinfo = solver.solve(args.tol)["info"]
        p_ev1.record(stream)
        torch.cuda.synchronize()
        plain = {"time_to_kkt_1e-8_s": p_ev0.elapsed_time(p_ev1) / 1e3, "iters": pinfo["iters"],
                 "status": hpr.hpr_status_str(int(pinfo["status"])), "final_kkt": pinfo["kkt"],
                 "primal_obj": pinfo["primal_obj"], "dual_obj": pinfo["dual_obj"]}
        solver.set_options(precision=args.precision)
    solver.close()

    # end to end through the C ABI with host buffers (upload, preprocessing, solve, download)
    h2d = (lp.A1.indptr.size + lp.A2.indptr.size) * 8 + lp.nnz * 12 + lp.m * 8 + lp.n * 24
    d2h = (2 * lp.n + lp.m) * 8
    barrier()
    e2e = None
    if args.e2e_steps > 0:
        e2e_iters = 0
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            with hpr.Solver(lp, **opts) as s2:
                e2e_iters += s2.solve(args.tol)["info"]["iters"]
        torch.cuda.synchronize()
        e2e_secs = time.perf_counter() - t0
        e2e = {"value": e2e_iters / e2e_secs, "unit": "iter/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "seconds_per_step": e2e_secs / args.e2e_steps}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        it = args.sample_iters
        r = oracle.solve(lp, max_iter=it, lambda_fixed=1.0, checks_cap=16, **VARIANTS[args.variant])
        cpu = {"value": it / r["info"]["seconds"], "unit": "iter/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": f"{it} oracle iterations (one check) of the full workload, lambda fixed to 1 "
                         f"(as the reference arm; lambda does not change the cost of an iteration)"}
        one = oracle_one_core(args, max(10, it // 10))
        if one is not None:
            cpu["one_core"] = one

    t8 = [i["solve_time_s"] for i in infos]
    t4 = [i["time_to_1e4_s"] for i in infos]
    cfg = config_dict(args, lp)
    if args.autotune or layout_opts(args):
        cfg["layout"] = layout
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f32+f64",
        "data": "synthetic", "config": cfg,
        "time_to_kkt_1e-8_s": statistics.mean(t8), "time_to_kkt_1e-4_s": statistics.mean(t4),
        "iters_to_kkt_1e-8": infos[-1]["iters"], "iters_to_kkt_1e-4": infos[-1]["iters_to_1e4"],
        "status": hpr.hpr_status_str(int(infos[-1]["status"])), "final_kkt": infos[-1]["kkt"],
        "primal_obj": infos[-1]["primal_obj"], "dual_obj": infos[-1]["dual_obj"],
        "restarts": infos[-1]["restarts"], "power_iters": infos[-1]["power_iters"],
        "power_rel_change": infos[-1]["power_rel_change"],
        "iters_fp32": infos[-1]["iters_fp32"],
        "effective_hbm_gbs": value * (bx + by) / 1e9,
        "effective_hbm_frac": value * (bx + by) / 1e9 / peak,
        "iteration_kernels_gbs": iter_gbs,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind, "bytes_per_launch": dom_bytes,
                     "ms_per_launch": dom_ms, "ms_phase_x": ms_x, "ms_phase_y": ms_y,
                     "in_graph": {"ms_per_iteration": in_graph_ms, "ms_per_launch": dom_in_graph_ms,
                                  "achieved": dom_bytes / (dom_in_graph_ms * 1e-3) / 1e9,
                                  "frac": dom_bytes / (dom_in_graph_ms * 1e-3) / 1e9 / peak},
                     "ceilings": ceil,
                     "frac_of_read_stream_same_size": achieved / ceil["read_gbs_phase_size"],
                     "gathers_per_launch": gathers, "gather_g_per_s": gather_rate,
                     "frac_of_gather_rate": gather_rate / ceil["gather_g_per_s"],
                     "fp64": fp64},
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "e2e": e2e,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if plain is not None:
        line["plain_fp64"] = plain
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_forms(args):
    """The FP32 form against plain FP64 on the same instances: `count` seeded medium planted LPs
    at `scale`, each solved to tol with precision 0 and with precision 1 in the same context
    (power method included in both).  value = geometric mean of the time ratios (FP32 form /
    FP64) over the instances where both converged; one record per instance beside it."""
    import torch

    from paper_2408_12179_b300 import hpr, lpgen

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    hpr.load()
    rows = []
    for seed in range(args.seed, args.seed + args.count):
        lp = lpgen.planted_medium(seed, args.scale)
        row = {"seed": seed, "m": lp.m, "n": lp.n, "nnz": lp.nnz}
        with hpr.Solver(lp, max_iter=args.max_iter, persistent=0) as s:
            for prec in (0, 1):
                s.set_options(precision=prec)
                I = s.solve(args.tol)["info"]
                row[f"p{prec}"] = dict(iters=int(I["iters"]), seconds=I["solve_time_s"], status=int(I["status"]),
                                       iters_fp32=int(I["iters_fp32"]), kkt=I["kkt"])
        rows.append(row)
    ok = [r for r in rows if r["p0"]["status"] == 0 and r["p1"]["status"] == 0]
    ratios = [r["p1"]["seconds"] / r["p0"]["seconds"] for r in ok]
    gm = math.exp(sum(math.log(x) for x in ratios) / max(len(ratios), 1)) if ratios else None
    line = {"metric": "time to KKT<=tol, FP32 form / plain FP64 (geometric mean over instances)",
            "value": gm, "unit": "ratio", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{args.count} medium planted LPs at scale {args.scale} (seeds {args.seed}..)",
                       "tol": args.tol, "max_iter": args.max_iter},
            "instances": len(rows), "both_converged": len(ok), "fp32_form_faster": sum(x < 1 for x in ratios),
            "total_fp64_s": sum(r["p0"]["seconds"] for r in ok),
            "total_fp32_form_s": sum(r["p1"]["seconds"] for r in ok), "rows": rows}
    print(json.dumps(line), flush=True)


def run_tiny(args):
    """Tiny planted LPs (m = 100, n = 200, nnz ~ 1,000; seeds seed .. seed + count - 1), each
    solved to tol on the default path (the persistent single-CTA kernel) and on the
    multi-CTA graph path: median time to KKT <= tol and <= 1e-4 (power method included) and
    microseconds per iteration; value = iterations / s of the default path over all LPs.
    Also all of them as one batch (one launch, one CTA per LP).  e2e: one-shot solves
    through the C ABI from host arrays (create, upload, scaling, solve, download)."""
    import numpy as np
    import torch

    from paper_2408_12179_b300 import hpr, lpgen

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    hpr.load()
    stream = torch.cuda.Stream()
    lps = [lpgen.planted_tiny(s) for s in range(args.seed, args.seed + args.count)]
    res = {}
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    for path, p in (("single_cta", 1), ("multi_cta", 0)):
        rows = []
        for lp in lps:
            with hpr.Solver(lp, max_iter=args.max_iter, cuda_stream=stream.cuda_stream, persistent=p) as s:
                for _ in range(args.warmup):
                    s.solve(args.tol)
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                infos = [s.solve(args.tol)["info"] for _ in range(args.steps)]
                ev1.record(stream)
                torch.cuda.synchronize()
            secs = ev0.elapsed_time(ev1) / 1e3 / args.steps
            I = infos[-1]
            rows.append(dict(secs=secs, iters=int(I["iters"]), t4=I["time_to_1e4_s"], power=I["power_time_s"],
                             launches=int(I["launches"]), status=int(I["status"])))
        res[path] = rows
    clocks = sampler.stop()

    def summary(rows):
        its = sum(r["iters"] for r in rows)
        return {"time_to_kkt_1e-8_s_median": statistics.median(r["secs"] for r in rows),
                "time_to_kkt_1e-4_s_median": statistics.median(r["t4"] for r in rows),
                "power_method_s_median": statistics.median(r["power"] for r in rows),
                "us_per_iter_with_power_method": 1e6 * sum(r["secs"] for r in rows) / its,
                "us_per_iter": 1e6 * sum(r["secs"] - r["power"] for r in rows) / its,
                "launches_per_solve": statistics.median(r["launches"] for r in rows),
                "all_ok": all(r["status"] == 0 for r in rows)}

    single = res["single_cta"]
    total_iters = sum(r["iters"] for r in single)
    total_secs = sum(r["secs"] for r in single)
    # all of them as one batch: one launch, one CTA per LP
    solvers = [hpr.Solver(lp, max_iter=args.max_iter) for lp in lps]
    with hpr.Batch(solvers, stream.cuda_stream) as b:
        for _ in range(args.warmup):
            b.solve(args.tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, bres = b.solve(args.tol)
        torch.cuda.synchronize()
        batch_secs = time.perf_counter() - t0
        bst = b.stats()
    for s_ in solvers:
        s_.close()
    batched = {"lps": len(lps), "seconds": batch_secs, "lp_per_s": len(lps) / batch_secs,
               "iters_per_s_summed": sum(int(r["info"]["iters"]) for r in bres) / batch_secs,
               "launches": bst["fused_launches"], "all_ok": all(r["status"] == 0 for r in bres)}
    # end to end from host arrays
    h2d = sum((lp.A1.indptr.size + lp.A2.indptr.size) * 8 + lp.nnz * 12 + lp.m * 8 + lp.n * 24 for lp in lps)
    d2h = sum((2 * lp.n + lp.m) * 8 for lp in lps)
    t0 = time.perf_counter()
    e2e_iters = 0
    for lp in lps:
        e2e_iters += hpr.solve(lp, tol=args.tol, max_iter=args.max_iter, cuda_stream=stream.cuda_stream)["info"]["iters"]
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        t0 = time.perf_counter()
        o_iters = 0
        for lp in lps:
            o_iters += oracle.solve(lp, tol=args.tol, max_iter=args.max_iter)["info"]["iters"]
        o_secs = time.perf_counter() - t0
        cpu = {"value": o_iters / o_secs, "unit": "iter/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": f"full solves to tol of the same {len(lps)} LPs (power method included)"}
    line = {
        "metric": METRIC, "value": total_iters / total_secs, "unit": "iter/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_secs,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": (f"tiny planted LPs (m=100, m1=40, n=200, nnz ~1000, entries N(0,1) with "
                                f"p=0.05), seeds {args.seed}..{args.seed + len(lps) - 1}"),
                   "count": len(lps), "tol": args.tol,
                   "l2": "working set far below L2 (latency-bound; no flush)"},
        "single_cta": summary(single), "multi_cta": summary(res["multi_cta"]),
        "batched_single_cta": batched,
        "gpu_launches": int(sum(r["launches"] for r in single)) * args.steps,
        "e2e": {"value": e2e_iters / e2e_secs, "unit": "iter/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_secs},
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


MID_SCALES = (0.001, 0.002, 0.005, 0.01)
MID_QAPS = (6, 8)


def mid_lps(args):
    """The mid-size workload: medium planted LPs at 1/1000 .. 1/100 scale and two QAP LPs."""
    from paper_2408_12179_b300 import lpgen

    return ([(f"medium 1/{round(1 / sc)}", lpgen.planted_medium(args.seed, sc)) for sc in MID_SCALES]
            + [(f"QAP N={q}", lpgen.qap_lp(args.seed + 2, q)) for q in MID_QAPS])


def run_mid(args):
    """Mid-size LPs (too much FP64 work for one SM, too little to fill the GPU): per LP the
    microseconds per iteration (lambda fixed, 3,000 iterations after a warm-up solve) on the
    multi-CTA graph path, the persistent single-CTA path and the persistent cluster path (when
    the LP fits them), and the time to KKT <= tol (power method included) on the graph path
    and on the default path (which takes the cluster path for these LPs).  value = iterations
    / s of the default path over all LPs' solves to tol."""
    import torch

    from paper_2408_12179_b300 import hpr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    hpr.load()
    stream = torch.cuda.Stream()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    rows = []
    launches = 0
    for name, lp in mid_lps(args):
        row = {"lp": name, "n": lp.n, "m": lp.m, "nnz": lp.nnz}
        for label, p in (("graph", 0), ("single_cta", 2), ("cluster", 4)):
            try:
                with hpr.Solver(lp, lambda_fixed=1.0, max_iter=3000, persistent=p, cuda_stream=stream.cuda_stream) as s:
                    s.solve(1e-12)
                    I = s.solve(1e-12)["info"]
                row[f"us_per_iter_{label}"] = 1e6 * I["solve_time_s"] / I["iters"]
            except hpr.HprError:
                row[f"us_per_iter_{label}"] = None          # the LP does not fit that path
        for label, p in (("graph", 0), ("default", 1)):
            with hpr.Solver(lp, max_iter=args.max_iter, persistent=p, cuda_stream=stream.cuda_stream) as s:
                for _ in range(args.warmup):
                    s.solve(args.tol)
                I = s.solve(args.tol)["info"]
            row[f"time_to_kkt_{label}_s"] = I["solve_time_s"]
            row[f"iters_{label}"] = int(I["iters"])
            row[f"status_{label}"] = hpr.hpr_status_str(int(I["status"]))
            if label == "default":
                row["default_path"] = {0: "graph", 2: "single_cta", 3: "grid", 4: "cluster"}[int(I["path"])]
                row["default_ctas"] = int(I["path_ctas"])
                launches += int(I["launches"])
        rows.append(row)
    clocks = sampler.stop()
    its = sum(r["iters_default"] for r in rows)
    secs = sum(r["time_to_kkt_default_s"] for r in rows)
    line = {
        "metric": "time to KKT <= tol on mid-size LPs: persistent cluster path (default) vs multi-CTA graph path",
        "value": its / secs, "unit": "iter/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "medium planted LPs at scales " + ", ".join(str(x) for x in MID_SCALES)
                               + " and QAP LPs N = " + ", ".join(str(q) for q in MID_QAPS) + f" (seed {args.seed})",
                   "tol": args.tol, "l2": "working sets far below L2 (latency-bound; no flush)"},
        "time_to_kkt_graph_s_total": sum(r["time_to_kkt_graph_s"] for r in rows),
        "time_to_kkt_default_s_total": secs,
        "lps": rows, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", dest="max_iter", type=int, default=3_000_000)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=1)
    ap.add_argument("--sample-iters", dest="sample_iters", type=int, default=150)
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1],
                    help="0: FP64; 1: FP32 form, then FP64 below KKT 1e-5")
    ap.add_argument("--compare-fp64", dest="compare_fp64", action="store_true",
                    help="also time one plain FP64 solve and report it beside the chosen form")
    ap.add_argument("--workload", choices=["medium", "mcf", "batch", "qap", "tiny", "forms", "mid"], default="medium",
                    help="medium sparse planted LP (default), the min-cost multicommodity flow LP "
                         "(1M nodes at scale 1), a batch of uneven planted LPs solved in one "
                         "batched run (m log-uniform in [500, 50000 * scale]), the FP32 form "
                         "against FP64 on --count medium planted LPs at --scale, or mid-size LPs "
                         "on the persistent cluster path against the multi-CTA path")
    ap.add_argument("--count", type=int, default=None,
                    help="LPs in the batch workload (default 512) or the tiny workload (default 100)")
    ap.add_argument("--qap-n", dest="qap_n", type=int, default=30,
                    help="QAP workload: N (N^4 + N^2 variables)")
    ap.add_argument("--sell-steps", dest="sell_steps", type=int, default=0,
                    help="lanes-per-row bound of both layouts (default: the library's choice)")
    ap.add_argument("--unit-cost", dest="unit_cost", type=float, default=0.0,
                    help="work-unit size of both layouts (default: the library's choice)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the sliced-ELL layouts by timing candidates at creation (batch workload: "
                         "once per size bucket of nnz, reused for the bucket's other LPs)")
    ap.add_argument("--solo-sample", dest="solo_sample", type=int, default=16,
                    help="batch workload: LPs also solved one by one, and as a batch of their own")
    ap.add_argument("--variant", choices=list(VARIANTS), default="hpr",
                    help="ablation variant of Section 4.2 (default: HPR-LP itself)")
    ap.add_argument("--persistent", type=int, default=1, choices=[0, 1, 2, 3, 4],
                    help="batch workload: hpr_options.persistent of every LP (0: the fused path only)")
    ap.add_argument("--lambda-fixed", dest="lambda_fixed", type=float, default=0.0,
                    help="use this lambda instead of the power method (short profiling runs)")
    args = ap.parse_args(argv)
    if args.count is None:
        args.count = {"tiny": 100, "forms": 8}.get(args.workload, 512)
    return args


def main():
    args = parse_args()
    if args.workload == "tiny" and args.impl == "ours":
        run_tiny(args)
    elif args.workload == "mid" and args.impl == "ours":
        run_mid(args)
    elif args.workload == "forms":
        run_forms(args)
    elif args.impl == "reference" and args.workload == "batch":
        run_reference_batch(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
