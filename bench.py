"""Benchmark of the fused Kruskal-Wallis scan (one JSON line on stdout).

A step is one pass of the whole hot path over the paper-scale workload
(N=102 samples, T=20,000 traits, S=500,000 SNPs; seeded synthetic stand-in for
the STAGE data): rank transform, genotype packing, fused tcgen05 scan with
threshold and hit compaction, FP64 finalisation of the hit list.  Inputs are
resident in device memory; L2 is flushed between steps (outside the timed
events).  The plain two-pass form (library GEMM to memory, then a separate
epilogue) is timed beside it, the end-to-end number goes through the public
host API with pinned host buffers, and the FP64 CPU oracle is timed on a
bounded sample of the same workload on the host cores.

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


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one krux_scan_kernel
# launch on the paper-scale workload, from one ncu capture, with the git blob hash of
# the kernel source it was taken on: reported only while that source is unchanged.
# ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on "bench.py --scan-only
# --traits 20000 --snps 500000 --data paper --tile 1,4,2,0" (the benchmark's workload
# and autotuned shape): 241.27 MB read + 78.10 MB written in one launch (1 pass).
SCAN_TRAFFIC = {"blob": "02a01e09e5245b5f6c2551f8441774ba6e351d26", "bytes": 319.37e6}


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
    # each step: the oracle on a bounded sample (4 traits x all SNPs)
    rng = np.random.default_rng(5)
    nt = 4
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
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{nt} random traits x all {S} SNPs per step (FP64 per-pair oracle)"},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    flops = 4.0 * N * pairs  # algorithmic: two indicator columns x N samples x multiply-add
    ms_scan = float(np.mean(scan_ms))
    achieved = flops / (ms_scan / 1e3) / 1e12
    peak = float(pk["bf16_tflops"])  # FP16 dense rate equals the BF16 rate (nominal ratio 1)
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (SCAN_TRAFFIC["bytes"] if SCAN_TRAFFIC and SCAN_TRAFFIC["blob"] == kernel_blob()
                        else None),
            "kernel": "krux_scan_kernel", "peak_kind": f"{pk_kind} bf16 burst (fp16 = bf16 x 1.0)",
            "ms_per_launch": ms_scan, "flops_per_launch": flops}

    # end to end through the public host API (pinned host buffers, H2D + D2H inside)
    e_h = torch.from_numpy(d["expr"]).pin_memory()
    g_h = torch.from_numpy(d["geno"]).pin_memory()
    esteps = max(1, min(args.steps, 5))
    kx.set_profiling(False)
    for _ in range(max(2, args.warmup)):  # warm-up (also fills the pinned-block cache)
        r = kx.scan_pinned(e_h, g_h, pth, cap)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(esteps):
        r = kx.scan_pinned(e_h, g_h, pth, cap)
        d2h += r["d2h_bytes"]
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)  # whole job: the slowest rank
    e2e = {"value": pairs * world * esteps / e2e_s, "unit": "pairs/s",
           "h2d_bytes_per_step": int(e_h.numel() * 4 + g_h.numel()),
           "d2h_bytes_per_step": int(d2h // esteps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline: N = 1 only
        import oracle
        oracle.build()
        rate, info = oracle_sample_rate(d)
        cpu = {"value": rate, "unit": "pairs/s", "cores": info["cores"], "kind": "oracle",
               "sample": f"{info['traits']} random traits x all {info['snps']} SNPs "
                         f"({info['seconds']:.1f} s of FP64 per-pair oracle work)"}

    if rank == 0:
        c = clk.summary()
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "T": T, "S": S, "N": N, "pthresh": pth,
                           "hit_capacity": cap, "l2": "flushed (256 MB write) between steps",
                           "tile_shape": dict(zip(("layout", "nc", "nA", "ka"), tile_shape)),
                           "parallelism": f"snp-shards x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": c, "hits": n_hits,
                "graph": graph_line,
                "plain": {"value": pvalue, "unit": "pairs/s", "ms_per_step": float(np.mean(ptimes)),
                          "steps": psteps, "fused_speedup": value / world / pvalue, "hits": pn},
                "breakdown_ms": {k2: float(np.mean([p[1][k2] for p in profs]))
                                 for k2 in ("ms_pack", "ms_scan", "ms_finalize")}
                | {"ms_rank": float(np.mean([p[0]["ms_rank"] for p in profs]))}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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
              f"(hits {hits})", flush=True)

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
