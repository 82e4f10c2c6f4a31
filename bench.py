"""Benchmark of the fused Kruskal-Wallis scan (one JSON line on stdout).

A step is one pass of the whole hot path over the paper-scale workload
(N=102 samples, T=20,000 traits, S=500,000 SNPs; seeded synthetic stand-in for
the STAGE data): rank transform, genotype packing, fused tcgen05 scan with
threshold and hit compaction, FP64 finalisation of the hit list.  Inputs are
resident in device memory; L2 is flushed between steps (outside the timed
events).  The plain two-pass form (library GEMM to memory, then a separate
epilogue) is timed beside it; the end-to-end number goes through the C ABI's
host-memory entry point (krux_scan_host, page-locked buffers, the copies inside
the timed region); the FP64 CPU oracle is timed on a bounded sample of the same
workload on the host cores.  The roofline carries both bounds of the scan kernel
(FP16 tensor rate, epilogue issue rate) and its fraction of the slower one.  At
N=1 the line also carries the missing-value, permutation-null and multi-cohort
workloads at full size ("missing", "permute", "cohorts"; --no-extra skips them).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fused|reference]
  python bench.py --scan-only [--traits T] [--snps S] [--data hwe|paper] [--reps R] [--perms P]

With --impl reference only the oracle arm runs (the CPU reference program),
on a bounded sample per step, and prints the same JSON line with
"impl": "reference".  Under torchrun (N > 1) every rank scans its own SNP shard
of the same size (weak scaling, no collective on the data path); rank 0
prints the line.
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

METRIC = "Kruskal-Wallis SNP-trait pairs/sec at N=102 (fused vs plain GPU); % roofline"
WORKLOAD = ("paper-scale fused scan: N=102 samples, T=20000 traits, S=500000 SNPs; HWE genotypes "
            "in LD blocks (MAF U[0.01,0.5]); log-normal expression with 1% x10 outliers; planted "
            "1-SD shifts on ~1% of pairs; hits at p<1e-5")


# Per-launch counters of krux_scan_kernel on the benchmark's workload, each with the
# git blob hash of the kernel source it was taken on: reported only while that
# source is unchanged (else null).  Commands (committed files only):
#   traffic: ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#            -k regex:krux_scan_kernel -s 1 -c 1 python bench.py --scan-only --traits 20000
#            --snps 500000 --data paper --tile 1,4,2,0 --reps 2   (1 pass)
#   issue:   ncu --metrics smsp__inst_executed.sum,sm__inst_executed_pipe_fmaheavy.sum,
#            sm__inst_executed_pipe_fmalite.sum,sm__inst_executed_pipe_alu.sum --clock-control none
#            -k regex:krux_scan_kernel -s 1 -c 1 python bench.py --scan-only --traits 20000
#            --snps 100000 --data paper --tile 1,4,2,0 --reps 2
#            (warp instructions x 32 lanes / pairs = lane issue slots per pair)
# Measured on the kernel below: 241.71 MB read + 74.28 MB written per 500k-SNP launch;
# 676.60 M warp instructions (567.48 M on the FMA-heavy, FMA-lite and ALU pipes) per
# 100k-SNP launch of 2x10^9 pairs.
SCAN_TRAFFIC = {"blob": "bcf763037070c5d9692f0da6d0549752132f2260", "bytes": 315.98e6}
SCAN_ISSUE = {"blob": "bcf763037070c5d9692f0da6d0549752132f2260", "slots_per_pair": 10.83,
              "fp32_int_slots_per_pair": 9.08,
              "workload": "planted 20000 x 100000 x 102 (0.19% of pairs are hits)"}
# Epilogue issue slots per pair by the operation count of the fused test: one add
# for D_2, three multiplies by 1/n_i, one multiply and two fused multiply-adds for
# Q, one select of the threshold by df, one compare/branch, plus the amortised
# TMEM load: about 10 lane slots.  The epilogue bound is SMs x 128 lanes x SM clock
# / 10 pairs per second.
EPILOGUE_SLOTS_PER_PAIR = 10.0


def kernel_blob():
    import hashlib
    with open(os.path.join(ROOT, "paper_1307_3519_gb300", "csrc", "scan_sm103.cu"), "rb") as f:
        data = f.read()
    return hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample_rate(d, target_s=12.0, seed=0):
    """Oracle throughput (pairs/s) on a bounded sample of the workload sized for
    about target_s seconds of CPU work: whole trait rows (all SNPs), a multiple of
    the oracle's thread count so that no thread idles."""
    import oracle
    rng = np.random.default_rng(seed)
    T, S = d["expr"].shape[0], d["geno"].shape[0]
    cores = oracle.num_threads()
    probe_t = rng.choice(T, min(T, cores), replace=False)
    probe_s = np.arange(0, S, max(1, S // 20000))
    t0 = time.perf_counter()
    oracle.scan(d["expr"], d["geno"], d["pthresh"], traits=probe_t, snps=probe_s)
    rate0 = probe_t.size * probe_s.size / (time.perf_counter() - t0)
    nt = int(round(rate0 * target_s / S / cores)) * cores
    nt = int(max(cores, min(T, nt)))
    traits = rng.choice(T, nt, replace=False)
    t0 = time.perf_counter()
    oracle.scan(d["expr"], d["geno"], d["pthresh"], traits=traits)
    dt = time.perf_counter() - t0
    return nt * S / dt, dict(traits=nt, snps=S, seconds=dt, cores=cores)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    d = synth.config(2)
    T, S = d["expr"].shape[0], d["geno"].shape[0]
    # each step: the oracle on a bounded sample, one random trait per oracle thread
    # (the oracle runs one trait per thread) x all SNPs
    cores = oracle.num_threads()
    rng = np.random.default_rng(5)
    nt = cores
    times = []
    for i in range(args.warmup + args.steps):
        traits = rng.choice(T, nt, replace=False)
        t0 = time.perf_counter()
        oracle.scan(d["expr"], d["geno"], d["pthresh"], traits=traits)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    pairs = nt * S
    v = pairs * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "T": T, "S": S, "N": d["N"], "pthresh": d["pthresh"]},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{nt} random traits (one per oracle thread) x all {S} SNPs "
                                       f"per step (FP64 per-pair oracle)"},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sm_count_and_clock(dev_index, clocks):
    """SM count of the device and the SM clock (MHz) for the issue-rate bound: the
    median sampled under load, else the maximum nvidia-smi reports, else 2070."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    return sms, float(mhz)


def roofline_bounds(ms, pairs, N, sms, mhz, pk):
    """Both bounds of the fused scan for `pairs` pairs at N samples in `ms`
    milliseconds: the FP16 tensor bound (4N algorithmic flop per pair against the
    measured dense rate) and the epilogue issue bound (EPILOGUE_SLOTS_PER_PAIR lane
    slots per pair against SMs x 128 lanes x SM clock).  The binding bound is the
    slower one; frac is the achieved rate over it."""
    tensor_peak = float(pk["bf16_tflops"])  # FP16 dense rate = BF16 rate (nominal ratio 1)
    flops = 4.0 * N * pairs
    t_achieved = flops / (ms / 1e3) / 1e12
    tensor_pairs = tensor_peak * 1e12 / (4.0 * N)
    slot_peak = sms * 128 * mhz * 1e6  # lane issue slots per second
    e_achieved = EPILOGUE_SLOTS_PER_PAIR * pairs / (ms / 1e3)
    epi_pairs = slot_peak / EPILOGUE_SLOTS_PER_PAIR
    rate = pairs / (ms / 1e3)
    tensor = {"achieved": t_achieved, "peak": tensor_peak, "unit": "TFLOP/s",
              "frac": t_achieved / tensor_peak, "peak_pairs_per_s": tensor_pairs,
              "flops_per_launch": flops}
    epi = {"achieved": e_achieved / 1e12, "peak": slot_peak / 1e12, "unit": "Tslot/s",
           "frac": e_achieved / slot_peak, "peak_pairs_per_s": epi_pairs,
           "slots_per_pair": EPILOGUE_SLOTS_PER_PAIR, "sms": sms, "sm_mhz": mhz}
    bound = "tensor" if tensor_pairs <= epi_pairs else "alu"
    b = tensor if bound == "tensor" else epi
    return bound, b, {"tensor": tensor, "epilogue": epi}, rate / min(tensor_pairs, epi_pairs)


def run_fused(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1307_3519_gb300 import build as kbuild
    kbuild.build()
    import paper_1307_3519_gb300 as k
    import synth

    d = synth.config(2, seed=1309 + rank)  # this rank's SNP shard (same shape on every rank)
    T, S, N, pth = d["T"], d["S"], d["N"], d["pthresh"]
    cap = 50_000_000
    kx = k.Krux(local)
    dev = torch.device("cuda", local)
    expr = torch.from_numpy(d["expr"]).to(dev)
    geno = torch.from_numpy(d["geno"]).to(dev)
    stream = torch.cuda.current_stream()
    hits = torch.empty((cap, 4), dtype=torch.int32, device=dev)
    H = torch.empty(cap, dtype=torch.float64, device=dev)
    P = torch.empty(cap, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # launch shape: the autotuner's choice for this width, timed on this workload's SNPs
    rs_tune = kx.krux_rank(expr)
    tile_shape = kx.autotune(rs_tune, geno, pth)
    kx.set_profiling(True)

    import ctypes
    lib = kx.lib
    opts = kx._opts(pth, cap)
    nh = ctypes.c_int64()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step(scan_fn):
        h = ctypes.c_void_p()
        st = lib.krux_rank(kx.handle, ctypes.c_void_p(expr.data_ptr()), T, N, N, ctypes.byref(h), sptr)
        kx._check(st, "krux_rank")
        prof_r = kx.profile()
        st = scan_fn(kx.handle, h, ctypes.c_void_p(geno.data_ptr()), S, N, ctypes.byref(opts),
                     ctypes.c_void_p(hits.data_ptr()), ctypes.c_void_p(H.data_ptr()),
                     ctypes.c_void_p(P.data_ptr()), ctypes.byref(nh), sptr)
        kx._check(st, "scan")
        prof_s = kx.profile()
        lib.krux_rankset_free(kx.handle, h)
        return prof_r, prof_s, nh.value

    def timed(scan_fn, steps, warmup):
        for _ in range(warmup):
            step(scan_fn)
        torch.cuda.synchronize()
        barrier(world)
        times, scan_ms, launches, profs = [], [], 0, []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            pr, ps, n = step(scan_fn)
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
            scan_ms.append(ps["ms_scan"])
            launches += pr["launches"] + ps["launches"]
            profs.append((pr, ps))
        torch.cuda.synchronize()
        barrier(world)
        return times, scan_ms, launches, profs, n

    with ClockSampler(local) as clk:
        times, scan_ms, launches, profs, n_hits = timed(lib.krux_scan, args.steps, args.warmup)
    tot_ms = max_over_ranks(sum(times), world)
    pairs = T * S
    value = pairs * world * args.steps / (tot_ms / 1e3)

    # plain two-pass form, measured beside (fewer steps)
    psteps = max(1, min(args.steps, 3))
    ptimes, pscan, _, pprofs, pn = timed(lib.krux_scan_plain, psteps, 1)
    pvalue = pairs * psteps / (sum(ptimes) / 1e3)

    # the same scan as a CUDA-graph replay (packing, scan, compaction, finalisation;
    # the ranks of the step before stay in place)
    graph = kx.graph_scan(rs_tune, geno, pth, cap)
    for _ in range(args.warmup):
        graph.launch(stream)
    graph.wait()
    gtimes = []
    gev0, gev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gsteps = max(1, min(args.steps, 10))
    for _ in range(gsteps):
        flush.zero_()
        gev0.record(stream)
        graph.launch(stream)
        gev1.record(stream)
        gev1.synchronize()
        gtimes.append(gev0.elapsed_time(gev1))
    g_hits = graph.wait()[0]["n_hits"]
    graph.close()
    graph_line = {"value": pairs / (float(np.mean(gtimes)) / 1e3), "unit": "pairs/s",
                  "ms_per_step": float(np.mean(gtimes)), "steps": gsteps, "hits": g_hits,
                  "what": "pack + fused scan + compaction + FP64 finalisation, one graph replay"}

    pk, pk_kind = peaks()
    clocks = clk.summary()
    sms, mhz = sm_count_and_clock(local, clocks)
    ms_scan = float(np.mean(scan_ms))
    bound, b, bounds, frac = roofline_bounds(ms_scan, pairs, N, sms, mhz, pk)
    traffic = (SCAN_TRAFFIC["bytes"] if SCAN_TRAFFIC["blob"] == kernel_blob() else None)
    issue = ({k2: v for k2, v in SCAN_ISSUE.items() if k2 != "blob"}
             if SCAN_ISSUE["blob"] == kernel_blob() and SCAN_ISSUE["slots_per_pair"] else None)
    roof = {"bound": bound, "achieved": b["achieved"], "peak": b["peak"], "unit": b["unit"],
            "frac": frac, "traffic": traffic, "kernel": "krux_scan_kernel",
            "peak_kind": f"{pk_kind} bf16 burst (fp16 = bf16 x 1.0) / SMs x 128 lanes x median SM clock",
            "ms_per_launch": ms_scan, "pairs_per_launch": pairs, "bounds": bounds,
            "measured_issue": issue}

    # end to end through the C ABI on host memory (krux_scan_host: pinned host
    # inputs and outputs, the library's H2D copies, rank, scan and D2H copies inside)
    e_h = torch.from_numpy(d["expr"]).pin_memory()
    g_h = torch.from_numpy(d["geno"]).pin_memory()
    outs_h = (torch.empty((cap, 4), dtype=torch.int32).pin_memory(),
              torch.empty(cap, dtype=torch.float64).pin_memory(),
              torch.empty(cap, dtype=torch.float64).pin_memory())
    esteps = max(1, min(args.steps, 5))
    kx.set_profiling(False)
    for _ in range(max(2, args.warmup)):
        r = kx.krux_scan_host(e_h, g_h, pth, cap, out=outs_h)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(esteps):
        r = kx.krux_scan_host(e_h, g_h, pth, cap, out=outs_h)
        d2h += r["d2h_bytes"] + 8
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)  # whole job: the slowest rank
    e2e = {"value": pairs * world * esteps / e2e_s, "unit": "pairs/s",
           "h2d_bytes_per_step": int(e_h.numel() * 4 + g_h.numel()),
           "d2h_bytes_per_step": int(d2h // esteps), "steps": esteps, "hits": r["n_hits"],
           "call": "krux_scan_host (C ABI, page-locked host buffers)"}
    kx.set_profiling(True)

    extra = {}
    if world == 1 and not args.no_extra:
        extra = extra_workloads(kx, flush, stream, pk, sms, mhz)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline: N = 1 only
        import oracle
        oracle.build()
        rate, info = oracle_sample_rate(d)
        cpu = {"value": rate, "unit": "pairs/s", "cores": info["cores"], "kind": "oracle",
               "sample": f"{info['traits']} random traits x all {info['snps']} SNPs "
                         f"({info['seconds']:.1f} s of FP64 per-pair oracle work)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "T": T, "S": S, "N": N, "pthresh": pth,
                           "hit_capacity": cap, "l2": "flushed (256 MB write) between steps",
                           "tile_shape": dict(zip(("layout", "nc", "nA", "ka"), tile_shape)),
                           "parallelism": f"snp-shards x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "hits": n_hits,
                "graph": graph_line,
                "plain": {"value": pvalue, "unit": "pairs/s", "ms_per_step": float(np.mean(ptimes)),
                          "steps": psteps, "fused_speedup": value / world / pvalue, "hits": pn},
                "breakdown_ms": {k2: float(np.mean([p[1][k2] for p in profs]))
                                 for k2 in ("ms_pack", "ms_scan", "ms_finalize")}
                | {"ms_rank": float(np.mean([p[0]["ms_rank"] for p in profs]))}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def extra_workloads(kx, flush, stream, pk, sms, mhz, steps=5, warmup=3):
    """The other three workloads at full size, each step one whole call on
    resident device inputs (rank transform included), L2 flushed between steps
    outside the timed events, CUDA events on the launching stream:
      missing  -- N=102, T=5,000, S=100,000; 10% of SNPs with one of 200 missing
                  patterns, 1% NaN expression; hits at p<1e-4
      permute  -- N=102, T=20,000, S=200,000, P=16 permutations in one call (min p
                  per permutation and trait, FDR histogram of 40 bins, real hits
                  at p<1e-5); (1 + P) T S pairs per step
      cohorts  -- 8 cohorts, N in {48,...,500}, T=15,000, S=300,000 each, one
                  grouped launch; each cohort also scanned alone for its own
                  roofline (4 N_c flop per pair)."""
    import torch
    import synth
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts, outs = [], []
        for _ in range(steps):
            flush.zero_()
            ev0.record(stream)
            out = fn()
            ev1.record(stream)
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
            outs.append(out)
        return float(np.mean(ts)), outs

    out = {}
    # missing values
    d = synth.config(3)
    e, g = dev(d["expr"]), dev(d["geno"])

    def step_missing():
        rs = kx.krux_rank(e)
        pr = kx.profile()
        r = kx.krux_scan(rs, g, d["pthresh"], capacity=10_000_000)
        ps = kx.profile()
        rs.free()
        return r["n_hits"], pr, ps
    ms, outs = timed(step_missing)
    pairs = d["T"] * d["S"]
    ms_scan = float(np.mean([o[2]["ms_scan"] for o in outs]))
    _, _, _, frac = roofline_bounds(ms_scan, pairs, d["N"], sms, mhz, pk)
    out["missing"] = {"value": pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms, "steps": steps,
                      "warmup": warmup, "hits": outs[-1][0], "T": d["T"], "S": d["S"], "N": d["N"],
                      "pthresh": d["pthresh"],
                      "gpu_launches": int(np.mean([o[1]["launches"] + o[2]["launches"] for o in outs])),
                      "breakdown_ms": {"ms_rank": float(np.mean([o[1]["ms_rank"] for o in outs])),
                                       "ms_pack": float(np.mean([o[2]["ms_pack"] for o in outs])),
                                       "ms_scan": ms_scan,
                                       "ms_finalize": float(np.mean([o[2]["ms_finalize"] for o in outs]))},
                      "scan_kernel_roofline_frac": frac,
                      "what": "krux_rank + krux_scan: missing-pattern groups re-ranked per group"}
    del e, g, d
    # permutation null
    d = synth.config(4)
    e, g, pm = dev(d["expr"]), dev(d["geno"]), dev(d["perms"])
    P = int(d["perms"].shape[0])

    def step_perm():
        rs = kx.krux_rank(e)
        pr = kx.profile()
        r = kx.krux_permute(rs, g, pm, d["pthresh"], capacity=50_000_000, fdr_bins=40, fdr_bin_width=0.1)
        ps = kx.profile()
        rs.free()
        return r["n_hits"], pr, ps
    ms, outs = timed(step_perm)
    pairs = (1 + P) * d["T"] * d["S"]
    ms_scan = float(np.mean([o[2]["ms_scan"] for o in outs]))
    _, _, _, frac = roofline_bounds(ms_scan, pairs, d["N"], sms, mhz, pk)
    out["permute"] = {"value": pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms, "steps": steps,
                      "warmup": warmup, "hits": outs[-1][0], "P": P, "T": d["T"], "S": d["S"],
                      "N": d["N"], "pthresh": d["pthresh"],
                      "gpu_launches": int(np.mean([o[1]["launches"] + o[2]["launches"] for o in outs])),
                      "ms_scan": ms_scan, "scan_kernel_roofline_frac": frac,
                      "what": "krux_rank + krux_permute (P=16, min p per permutation and trait, "
                              "FDR histogram, real hits); pairs = (1+P) T S"}
    del e, g, pm, d
    # cohorts
    d = synth.config(5)
    cin = [(dev(c["expr"]), dev(c["geno"]), int(c["expr"].shape[1])) for c in d["cohorts"]]

    def step_cohorts():
        rss = [kx.krux_rank(ce) for ce, _, _ in cin]
        cohorts = [dict(rs=rs, geno=cg, capacity=5_000_000) for rs, (_, cg, _) in zip(rss, cin)]
        r = kx.krux_scan_grouped(cohorts, d["pthresh"])
        ps = kx.profile()
        for rs in rss:
            rs.free()
        return sum(x["n_hits"] for x in r), ps
    ms, outs = timed(step_cohorts)
    tot_pairs = sum(ce.shape[0] * cg.shape[0] for ce, cg, _ in cin)
    ms_grouped = float(np.mean([o[1]["ms_scan"] for o in outs]))
    per, bound_ms = [], 0.0
    for ce, cg, n in cin:
        rs = kx.krux_rank(ce)
        kx.krux_scan(rs, cg, d["pthresh"], capacity=5_000_000)
        t_ = []
        for _ in range(3):
            flush.zero_()
            kx.krux_scan(rs, cg, d["pthresh"], capacity=5_000_000)
            t_.append(kx.profile()["ms_scan"])
        rs.free()
        cp = ce.shape[0] * cg.shape[0]
        mc = float(np.mean(t_))
        bnd, _, bnds, fr = roofline_bounds(mc, cp, n, sms, mhz, pk)
        bound_ms += cp / min(bnds["tensor"]["peak_pairs_per_s"], bnds["epilogue"]["peak_pairs_per_s"]) * 1e3
        per.append({"N": n, "ms_scan_alone": mc, "pairs_per_s": cp / (mc / 1e3), "bound": bnd,
                    "frac": fr, "tensor_frac": bnds["tensor"]["frac"]})
    out["cohorts"] = {"value": tot_pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_step": ms, "steps": steps,
                      "warmup": warmup, "hits": outs[-1][0], "n_cohorts": len(cin),
                      "T": int(cin[0][0].shape[0]), "S": int(cin[0][1].shape[0]),
                      "N": [n for _, _, n in cin], "pthresh": d["pthresh"],
                      "ms_scan_grouped": ms_grouped, "grouped_roofline_frac": bound_ms / ms_grouped,
                      "per_cohort": per,
                      "what": "8 x krux_rank + one krux_scan_grouped launch; per-cohort rows: the "
                              "cohort scanned alone, frac against its slower bound (4 N_c flop "
                              "per pair on the tensor pipe, 10 issue slots per pair)"}
    del cin, d
    torch.cuda.empty_cache()
    return out


def run_scan_only(args):
    """Profiling driver: the fused scan kernel alone, `reps` calls on one seeded
    input (T traits x S SNPs x 102 samples), one text line per call.  data=hwe:
    HWE genotypes (MAF 0.05-0.5) and log-normal expression, almost no hits;
    data=paper: the paper-scale workload's generator at these sizes; data=multi:
    markers with 2..5 genotype groups (codes 0..4; 4N flop per pair counted as for
    biallelic markers, the contraction itself does 8N).  --perms P: the permutation
    form instead (krux_permute with P seeded permutations, (1 + P) T S pairs)."""
    import torch
    from paper_1307_3519_gb300 import build as kbuild
    kbuild.build()
    import paper_1307_3519_gb300 as k
    import synth
    T, S = args.traits, args.snps
    # the autotuner runs first (as in the benchmark) unless --no-autotune
    multi = args.data == "multi"
    if args.data == "paper":
        d = synth.config(2, T=T, S=S)
        geno, expr, pth = d["geno"], d["expr"], d["pthresh"]
    elif multi:  # markers with 2..5 genotype groups (codes 0..4)
        rng = np.random.default_rng(3)
        geno = synth.multiallelic_genotypes(rng, S, 102)
        expr = synth.expression_lognormal(rng, T, 102)
        pth = 1e-5
    else:
        rng = np.random.default_rng(1)
        geno, _ = synth.hwe_genotypes(rng, S, 102, 0.05, 0.5)
        expr = synth.expression_lognormal(rng, T, 102)
        pth = 1e-5
    kx = k.Krux(0)
    rs = kx.krux_rank(torch.from_numpy(expr).cuda())
    g = torch.from_numpy(geno).cuda()
    if args.tile:  # an explicit launch shape (e.g. the one the benchmark's autotuner chose)
        kx.set_tuning(*[int(v) for v in args.tile.split(",")])
    elif not args.no_autotune:  # the launch shape the benchmark uses
        if not multi:  # the autotuner times the biallelic form
            print(f"scan-only autotuned shape (layout, nc, nA, ka) = {kx.autotune(rs, g, pth)}",
                  flush=True)
    kx.set_profiling(True)
    if args.perms > 0:
        perms = torch.from_numpy(synth.make_perms(1307, args.perms, 102)).cuda()
        for i in range(args.reps):
            r = kx.krux_permute(rs, g, perms, pth, capacity=min(50_000_000, T * S))
            pr = kx.profile()
            print(f"scan-only permute P={args.perms} data={args.data} T={T} S={S} call={i} "
                  f"hits={r['n_hits']} scan={pr['ms_scan']:.3f} ms "
                  f"({(1 + args.perms) * T * S / pr['ms_scan'] / 1e6:.4g} Gpairs/s) "
                  f"launches={pr['launches']}", flush=True)
        return
    for i in range(args.reps):
        r = kx.krux_scan(rs, g, pth, capacity=min(50_000_000, T * S), multiallelic=multi)
        pr = kx.profile()
        fl = 4.0 * 102 * T * S
        print(f"scan-only data={args.data} T={T} S={S} call={i} hits={r['n_hits']} "
              f"scan={pr['ms_scan']:.3f} ms ({fl / pr['ms_scan'] / 1e9:.1f} TFLOP/s algorithmic) "
              f"pack={pr['ms_pack']:.3f} ms finalize={pr['ms_finalize']:.3f} ms grid={pr['scan_grid']}",
              flush=True)


def run_row_timings(args):
    """Timing driver for the other entry points on their workloads (text lines,
    not the benchmark's JSON): whole calls timed with CUDA events on the current
    stream, inputs resident, best of `reps` after one warm-up call."""
    import torch
    from paper_1307_3519_gb300 import build as kbuild
    kbuild.build()
    import paper_1307_3519_gb300 as k
    import synth
    kx = k.Krux(0)
    kx.set_profiling(True)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(name, pairs, fn):
        out = fn()  # warm-up
        best = None
        for _ in range(args.reps):
            ev0.record(st)
            out = fn()
            ev1.record(st)
            ev1.synchronize()
            t = ev0.elapsed_time(ev1)
            best = t if best is None else min(best, t)
        hits = out if isinstance(out, int) else -1
        print(f"row {name}: {pairs:.4g} pairs in {best:.3f} ms = {pairs / best * 1e3:.4g} pairs/s "
              f"(hits {hits}, scan kernel form {kx.profile()['scan_form']})", flush=True)

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    want = set(args.rows.split(","))
    if "missing" in want:  # missing genotype patterns and NaN expression
        d = synth.config(3)
        rs, g = kx.krux_rank(dev(d["expr"])), dev(d["geno"])
        timed("missing-values 5000x100000x102", d["T"] * d["S"],
              lambda: kx.krux_scan(rs, g, d["pthresh"], capacity=10_000_000)["n_hits"])
    if "permute" in want:  # 16 permutations and the FDR histogram
        d = synth.config(4)
        rs, g, pm = kx.krux_rank(dev(d["expr"])), dev(d["geno"]), dev(d["perms"])
        timed("permutations 20000x200000x102, P=16, FDR bins", 17 * d["T"] * d["S"],
              lambda: kx.krux_permute(rs, g, pm, d["pthresh"], capacity=50_000_000, fdr_bins=40,
                                      fdr_bin_width=0.1)["n_hits"])
    if "cis" in want:  # 1 Mbp window on a 22-chromosome map
        d = synth.config(2)
        rs, g = kx.krux_rank(dev(d["expr"])), dev(d["geno"])
        sp, tp = synth.genome_positions(np.random.default_rng(7), d["S"], d["T"])
        sp, tp = dev(sp), dev(tp)
        timed("cis 1 Mbp, 20000x500000x102 (pairs of the full product)", d["T"] * d["S"],
              lambda: kx.krux_scan_cis(rs, g, sp, tp, 1_000_000, d["pthresh"],
                                       capacity=50_000_000)["n_hits"])
    if "multi" in want:  # markers with 2..5 genotype groups
        rng = np.random.default_rng(3)
        T, S = 20000, 100000
        rs = kx.krux_rank(dev(synth.expression_lognormal(rng, T, 102)))
        g = dev(synth.multiallelic_genotypes(rng, S, 102))
        timed("multi-allelic 20000x100000x102", T * S,
              lambda: kx.krux_scan(rs, g, 1e-5, capacity=10_000_000, multiallelic=True)["n_hits"])
    for model in ("anova", "linear"):
        if "param-" + model in want:
            d = synth.config(2, S=100000)
            e, g = dev(d["expr"]), dev(d["geno"])
            timed(f"parametric {model} 20000x100000x102", d["T"] * d["S"],
                  lambda: kx.krux_scan_parametric(e, g, model, 1e-5, capacity=10_000_000)["n_hits"])
    if "cohorts" in want:  # 8 cohorts of uneven N in one grouped launch, direct and graph
        d = synth.config(5)
        cohorts = [dict(rs=kx.krux_rank(dev(c["expr"])), geno=dev(c["geno"]), capacity=5_000_000)
                   for c in d["cohorts"]]
        pairs = sum(c["rs"].T * c["geno"].shape[0] for c in cohorts)
        timed("8 cohorts N=48..500, 15000x300000 each", pairs,
              lambda: sum(r["n_hits"] for r in kx.krux_scan_grouped(cohorts, d["pthresh"])))
        graph = kx.graph_grouped(cohorts, d["pthresh"])

        def replay():
            graph.launch(st)
            return sum(r["n_hits"] for r in graph.wait())
        timed("8 cohorts, CUDA-graph replay", pairs, replay)
        graph.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the missing-value, permutation and cohort workloads")
    ap.add_argument("--scan-only", action="store_true",
                    help="profiling driver: only the fused scan, --reps calls, text output")
    ap.add_argument("--traits", type=int, default=20000)
    ap.add_argument("--snps", type=int, default=100000)
    ap.add_argument("--data", default="hwe", choices=["hwe", "paper", "multi"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--perms", type=int, default=0,
                    help="scan-only: the permutation form with this many permutations")
    ap.add_argument("--rows", default="",
                    help="timing driver: comma list of missing,permute,cis,multi,param-anova,"
                         "param-linear,cohorts")
    ap.add_argument("--tile", default="",
                    help="scan-only: launch shape layout,nc,nA,ka instead of the autotuner's")
    ap.add_argument("--no-autotune", action="store_true",
                    help="scan-only: the automatic launch shape instead of the autotuner's")
    args = ap.parse_args()
    if args.rows:
        run_row_timings(args)
        return
    if args.scan_only:
        run_scan_only(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_fused(args)


if __name__ == "__main__":
    main()
