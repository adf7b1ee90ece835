#!/usr/bin/env python
"""Benchmark: CI tests/sec and PC-stable skeleton time on one GB300.

One step = one whole skeleton (every depth: snapshot, edge list, CI tests,
removal) of the workload, through the C ABI, with the data already resident in
HBM.  The default workload is the batched one: 256 independent PC-stable
problems (20-300 variables, 1k-50k samples) learnt together, one work-pool
launch per depth over every problem's edges.  Throughput counts the tests the
sequential Algorithm 1 runs (redundant tests of the parallel pool are not
counted).  The L2 is flushed (a 256 MB device write) before every timed step,
outside its events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batched|mid|small|large|depth0]
                    [--form pool|plain] [--gs G] [--impl ours|reference]

Under torchrun each rank runs an independent replica of the workload on its
own GPU (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CI tests/sec & PC-stable skeleton time, 1 GB300, batched/INT8 vs plain GPU form"
PROFILES = os.path.join(ROOT, "profiles")


def source_hash():
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2212_04259_gb300", "csrc", "*")))
    files += sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, or None if there is none or the kernel sources changed since."""
    path = os.path.join(PROFILES, f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None, None
    text = open(path).read()
    try:
        block = text.split("```json")[1].split("```")[0]
        rec = json.loads(block)
    except Exception:
        return None, None
    if rec.get("src_hash") != source_hash():
        return None, None
    return rec.get("dram_bytes_per_launch"), rec.get("launch")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--problems", type=int, default=256, help="problems of the batched workload (the first K)")
    ap.add_argument("--form", choices=["pool", "plain"], default="pool")
    ap.add_argument("--gs", type=int, default=0)
    ap.add_argument("--group-threads", type=int, default=0, help="pin the threads per CI test (32-256)")
    ap.add_argument("--loop", choices=["device", "host"], default="device",
                    help="who drives the depth loop (host: the same kernels depth by depth, for kernel-by-kernel "
                         "profilers)")
    ap.add_argument("--depth1", choices=["auto", "pool", "tensor"], default="auto",
                    help="depth-1 counting: tensor-core neighbourhood product or work pool")
    ap.add_argument("--statistic", choices=["g2", "x2"], default="g2", help="CI statistic (G^2 or Pearson X^2)")
    ap.add_argument("--df", choices=["fixed", "adjusted"], default="fixed", help="degrees of freedom of each test")
    ap.add_argument("--tune", choices=["auto", "off"], default="auto",
                    help="autotune the counting per depth before the warm-up (fbn_autotune; untimed), or keep the "
                         "fixed rules")
    ap.add_argument("--count", choices=["auto", "hist", "bits"], default="auto",
                    help="table counting: bit planes for small tables (auto), byte histograms only, bit planes "
                         "wherever they fit")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the bench line: the group-size, granularity, sample-size and network-size "
                         "studies, one JSON line per configuration")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="host processes of the oracle baseline (0: every host core, at most 16)")
    return ap.parse_args()


def load_workload(name, problems=256):
    import bnsynth
    if name == "batched":
        probs = bnsynth.batched_workload(problems)
        return {"kind": "batch", "probs": [(d, a) for d, a, _ in probs], "alpha": 0.05, "max_depth": -1}
    data, ar, alpha, md, _ = bnsynth.workload(name)
    return {"kind": "single", "data": data, "ar": ar, "alpha": alpha, "max_depth": md}


def workload_config(name, w, args):
    cfg = {"workload": name, "form": args.form, "group_size": args.gs or "per depth (1 or 4)",
           "l2": "flushed by a 256 MB device write before each timed step"}
    if args.statistic != "g2" or args.df != "fixed":
        cfg.update(statistic=args.statistic, df=args.df, loop=args.loop)
    if args.loop != "device":
        cfg.update(loop=args.loop)
    cfg.update(count=args.count, tune=args.tune)
    if w["kind"] == "single":
        n, N = w["data"].shape
        cfg.update(n_vars=n, n_samples=N, alpha=w["alpha"], max_depth=w["max_depth"],
                   arities=sorted({int(a) for a in w["ar"]}))
    else:
        cfg.update(problems=len(w["probs"]), n_vars_total=sum(d.shape[0] for d, _ in w["probs"]),
                   samples_total=sum(d.shape[1] for d, _ in w["probs"]), alpha=w["alpha"],
                   max_depth=w["max_depth"])
    return cfg


# ----------------------------------------------------------------------------- ranks
def rank_max(x, dist=None):
    """Max of a float over the ranks (each rank runs an independent replica;
    the job is as slow as its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(tests_per_rank, ms_max, world):
    """Whole-job tests per second: every rank's tests over the slowest rank's time."""
    return world * tests_per_rank / (ms_max / 1e3)


# ----------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        self.idx = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.close()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle baseline
def host_procs(args):
    """Host processes of the oracle legs: every core, at most 16, unless pinned."""
    return args.cpu_procs or max(1, min(16, os.cpu_count() or 1))


def _oracle_skeleton(job):
    """Worker of the host-core pool: one whole sequential oracle skeleton."""
    import oracle
    data, ar, alpha, md = job
    return oracle.pc_stable(data, ar, alpha, md).n_tests


def oracle_batch(w, problems, procs):
    """Whole oracle skeletons of the given problems of a batch, one problem per
    host process at a time (a spawned pool: no process is forked after CUDA
    initialised); returns (oracle tests, wall seconds)."""
    import multiprocessing as mp
    jobs = sorted(problems, key=lambda p: -w["probs"][p][0].size)   # largest first: an even end
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_skeleton, [(w["probs"][0][0][:, :64], w["probs"][0][1], w["alpha"], 0)] * procs)
        t0 = time.perf_counter()
        tests = sum(pool.map(_oracle_skeleton, [(w["probs"][p][0], w["probs"][p][1], w["alpha"], w["max_depth"])
                                                for p in jobs], chunksize=1))
        return tests, time.perf_counter() - t0


def oracle_rate(w, stats, args, budget_s=10.0):
    """Time the CPU oracle on a bounded sample of the workload; returns dict."""
    import numpy as np
    import oracle
    if w["kind"] == "batch":
        # every fourth problem (64 of 256, all sizes), whole skeletons
        sample = list(range(0, len(w["probs"]), 4))
        procs = host_procs(args)
        tests, secs = oracle_batch(w, sample, procs)
        return {"value": tests / secs, "unit": "tests/s", "cores": procs, "kind": "oracle",
                "sample": f"whole sequential skeletons of every fourth problem of the batch ({len(sample)} "
                          f"problems, {tests} oracle tests, {secs:.1f} s wall), one problem per host process"}
    if w["data"].shape[0] <= 64:
        # the whole skeleton, repeated until the budget is used
        t0 = time.perf_counter()
        tests, runs = 0, 0
        while True:
            r = oracle.pc_stable(w["data"], w["ar"], w["alpha"], w["max_depth"])
            tests += r.n_tests
            runs += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        dt = time.perf_counter() - t0
        return {"value": tests / dt, "unit": "tests/s", "cores": 1, "kind": "oracle",
                "sample": f"{runs} full sequential skeletons of the workload ({tests // runs} tests each)"}
    # per-depth sample: random tests of the right size, weighted by the GPU's oracle-equivalent counts
    data, ar = w["data"], w["ar"]
    rng = np.random.default_rng(0)
    per_depth = stats["tests_oracle"]
    total = sum(per_depth)
    sec_per_test = []
    done = 0
    for d, cnt in enumerate(per_depth):
        if cnt == 0:
            sec_per_test.append(0.0)
            continue
        share = budget_s * cnt / total
        t0 = time.perf_counter()
        k = 0
        while True:
            v = rng.permutation(data.shape[0])[: d + 2]
            oracle.ci_test(data, ar, int(v[0]), int(v[1]), [int(t) for t in v[2:]])
            k += 1
            if time.perf_counter() - t0 >= share or k >= 200000:
                break
        sec_per_test.append((time.perf_counter() - t0) / k)
        done += k
    est = sum(c * s for c, s in zip(per_depth, sec_per_test))
    return {"value": total / est, "unit": "tests/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} single CI tests drawn per depth in proportion to the skeleton's "
                      f"test mix (depths 0..{len(per_depth) - 1}), sequential"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, w, name, rank, world):
    """The reference arm: this tier's reference program is the CPU oracle,
    timed as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    procs = host_procs(args) if w["kind"] == "batch" else 1

    def one_step(k):
        if w["kind"] == "batch":
            # a sixteenth of the batch per step (problems p = k mod 16), whole skeletons
            probs = [p for p in range(len(w["probs"])) if p % 16 == k % 16]
            t, s = oracle_batch(w, probs, procs)
            return t, s, "a sixteenth of the batch per step (problems p = step mod 16, 16 problems), whole " \
                         "sequential skeletons, one problem per host process"
        if w["data"].shape[0] <= 64:
            t0 = time.perf_counter()
            r = oracle.pc_stable(w["data"], w["ar"], w["alpha"], w["max_depth"])
            return r.n_tests, time.perf_counter() - t0, "one full sequential skeleton per step"
        import numpy as np
        rng = np.random.default_rng(1 + k)
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < 2.0:
            d = int(rng.integers(0, 3))
            v = rng.permutation(w["data"].shape[0])[: d + 2]
            oracle.ci_test(w["data"], w["ar"], int(v[0]), int(v[1]), [int(t) for t in v[2:]])
            n += 1
        return n, time.perf_counter() - t0, "2 s of sampled single CI tests (depths 0-2) per step"
    for k in range(args.warmup):
        one_step(k)
    tests, secs, what = 0, 0.0, ""
    for k in range(args.steps):
        t, s, what = one_step(args.warmup + k)
        tests += t
        secs += s
    val = tests / secs
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "tests/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(name, w, args),
            "cpu_baseline": {"value": val, "unit": "tests/s", "cores": procs, "kind": "oracle", "sample": what},
            "e2e": {"value": val, "unit": "tests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def run_ablation(args):
    """The studies of the paper's Section V on synthetic networks: group size gs
    (tests executed vs time), granularity (CI-level pool, edge-level plain form,
    threads per test), sample size and network size.  Each configuration: 2
    untimed skeletons, then the median of 5 timed ones (CUDA events, L2 flushed
    before each); the oracle's sequential rate is sampled for the sample-size
    study."""
    import bnsynth
    import torch
    import paper_2212_04259_gb300 as F
    from paper_2212_04259_gb300 import build
    build.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")

    def measure(data, ar, alpha, md, **opt):
        h = F.fbn_create(torch.from_numpy(data).cuda(), ar, **opt)
        F.fbn_set_stream(h, stream)
        for _ in range(2):
            F.fbn_learn_skeleton(h, alpha, md)
        ms = []
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.fbn_learn_skeleton(h, alpha, md)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = F.fbn_get_stats(h)
        F.fbn_destroy(h)
        med = statistics.median(ms)
        return {"ms": med, "tests_executed": sum(st["tests"]), "tests_oracle": sum(st["tests_oracle"]),
                "tests_per_s": sum(st["tests_oracle"]) / (med / 1e3), "depths": st["depths"]}

    def emit(kind, config, res):
        print(json.dumps({"ablation": kind, "config": config, **res}), flush=True)

    data, ar, alpha, md, _ = bnsynth.workload("mid")
    for gs in (1, 2, 4, 8, 16, 0):
        emit("group_size", {"workload": "mid", "gs": gs or "per depth (1 or 4)"},
             measure(data, ar, alpha, md, group_size=gs))
    for label, opt in (("CI-level work pool", {}), ("edge-level plain form", {"form": "plain"}),
                       ("CI-level, 32 threads per test", {"group_threads": 32}),
                       ("CI-level, 256 threads per test", {"group_threads": 256})):
        for wl in ("mid", "large"):
            d2, a2, al2, md2, _ = bnsynth.workload(wl)
            emit("granularity", {"workload": wl, "scheme": label}, measure(d2, a2, al2, md2, **opt))
    import oracle
    for N in (5000, 10000, 15000, 50000):
        d2, a2, al2, md2, _ = bnsynth.workload("mid", n_samples=N)
        res = measure(d2, a2, al2, md2)
        t0 = time.perf_counter()
        ref = oracle.pc_stable(d2, a2, al2, md2)
        cpu_s = time.perf_counter() - t0
        res.update(oracle_tests_per_s=ref.n_tests / cpu_s, oracle_cores=1,
                   speedup_vs_oracle=(ref.n_tests / cpu_s and res["tests_per_s"] / (ref.n_tests / cpu_s)))
        emit("sample_size", {"workload": "mid network", "n_samples": N}, res)
    for wl in ("small", "mid", "large"):
        d2, a2, al2, md2, _ = bnsynth.workload(wl)
        emit("network_size", {"workload": wl, "n_vars": int(d2.shape[0]), "n_samples": int(d2.shape[1])},
             measure(d2, a2, al2, md2))


def main():
    args = parse()
    if args.ablation:
        return run_ablation(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    w = load_workload(name, args.problems)
    if args.impl == "reference":
        return run_reference(args, w, name, rank, world)

    import numpy as np
    import torch
    import paper_2212_04259_gb300 as F
    from paper_2212_04259_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    gs = args.gs
    if w["kind"] == "single":
        data_dev = torch.from_numpy(w["data"]).cuda()
        handles = [F.fbn_create(data_dev, w["ar"], form=args.form, group_size=gs, device=local,
                                group_threads=args.group_threads, depth1=args.depth1, statistic=args.statistic,
                                df=args.df, loop=args.loop, count=args.count)]
        F.fbn_set_stream(handles[0], stream)
        outs = [torch.zeros((w["data"].shape[0],) * 2, dtype=torch.uint8, device="cuda")]
    else:
        handles = [F.fbn_create(torch.from_numpy(d).cuda(), a, form=args.form, group_size=gs, device=local,
                                group_threads=args.group_threads, depth1=args.depth1, statistic=args.statistic,
                                df=args.df, loop=args.loop, count=args.count)
                   for d, a in w["probs"]]
        F.fbn_set_stream(handles[0], stream)
        outs = [torch.zeros((d.shape[0],) * 2, dtype=torch.uint8, device="cuda") for d, _ in w["probs"]]

    def step():
        if w["kind"] == "single":
            F.fbn_learn_skeleton(handles[0], w["alpha"], w["max_depth"], adj_out=outs[0])
        else:
            F.fbn_learn_skeleton_batch(handles, w["alpha"], w["max_depth"], adj_out=outs)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 256 MB > L2
    tuning = None
    if args.tune == "auto" and args.form == "pool":   # choices by measurement, before the warm-up (untimed)
        tuning = F.fbn_autotune(handles, w["alpha"], w["max_depth"])
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier()
    # clocks: the sampler (200 ms period) runs over an untimed soak of the same
    # steps (at least 0.6 s) and the timed steps that follow it
    clocks = Clocks(local)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 0.6:
        flush.zero_()
        step()
        torch.cuda.synchronize()
    evs = []
    stats_acc = None
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
        st = F.fbn_get_stats(handles[0])
        if stats_acc is None:
            stats_acc = {k: (list(v) if isinstance(v, list) else v) for k, v in st.items()}
            stats_acc["test_ms"] = list(st["test_ms"])
        else:
            stats_acc["test_ms"] = [a + b for a, b in zip(stats_acc["test_ms"], st["test_ms"])]
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    st = F.fbn_get_stats(handles[0])
    tests = sum(st["tests_oracle"])
    ms = rank_max(ms, dist)
    value = job_throughput(tests, ms, world)

    # rooflines.  Histogram test kernels (the work pool): algorithmic sample
    # bytes (d + 2) N per oracle-equivalent test -- each test weighted by its
    # own problem's N (the library sums N over each depth's tests) -- over
    # their device time, against the measured HBM copy bandwidth.  Depth 0 on
    # the one-hot Gram: algorithmic FLOPs 2 * M^2 * N / 2 (upper triangle,
    # M = sum of arities) over the Gram kernel's time, against the FP8 dense
    # peak (the measured bf16 peak times the nominal FP8/BF16 ratio of 2).
    gram_used = st["gram_ms"] > 0
    pool_depths = [d for d in range(st["depths"]) if not (gram_used and d == 0)]
    alg_bytes = sum((d + 2) * st["test_samples"][d] for d in pool_depths)
    test_ms = sum(stats_acc["test_ms"][d] for d in pool_depths) / args.steps
    achieved = alg_bytes / (test_ms / 1e3) / 1e9 if test_ms > 0 else 0.0
    try:
        peaks = json.load(open(PEAKS))
        peak, peak_src = float(peaks["hbm_gbs"]), "of measured"
        bf16 = float(peaks["bf16_tflops"])
        fp8_peak, fp8_src = 2.0 * bf16, "of measured (bf16 burst x nominal fp8/bf16 ratio 2)"
    except Exception:
        peak, peak_src = FALLBACK_HBM_GBS, "of fallback"
        fp8_peak, fp8_src = 2.0 * 1900.0, "of fallback (bf16 x 2)"
    roofline_hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": peak_src,
                    "kernel": "k_pool_bits / k_pool_small / k_pool_big (depths %s)" % ",".join(str(d) for d in pool_depths)
                    if args.form == "pool" else "k_plain", "kernel_ms_per_step": test_ms,
                    "algorithmic_bytes_per_step": alg_bytes,
                    "note": "sample bytes (d + 2) N of the oracle-equivalent tests over the pool's test windows; the "
                            "data sets are L2-resident, so this is a traffic view, not the unit that binds"}

    # the unit that binds the counting: measured on this device by the
    # library (fbn_measure_unit_rates).  The dominant pool depth's kernel is
    # reported against it: POPC for tables counted from bit planes (cells x
    # 32-sample words of work), shared-memory reductions for byte histograms
    # (one per sample); the work counters are the executed tests' (redundant
    # tests included), the time the depth's test window.
    rates = F.fbn_measure_unit_rates(local)
    per_ms = [stats_acc["test_ms"][d] / args.steps for d in range(st["depths"])]
    dstar = max(pool_depths, key=lambda d: per_ms[d]) if pool_depths else None
    roofline = None
    if dstar is not None and per_ms[dstar] > 0:
        bits = st["popc_work"][dstar] > 0
        work = st["popc_work"][dstar] if bits else st["smem_updates"][dstar]
        peak_u = (rates["popc_per_s"] if bits else rates["smem_red_per_s"]) / 1e9
        ach = work / (per_ms[dstar] / 1e3) / 1e9
        kname = ("k_pool_bits" if bits else "k_pool_small / k_pool_big") if args.form == "pool" else "k_plain"
        traffic, traffic_launch = profiled_traffic(kname.split(" ")[0], name) if args.form == "pool" else (None, None)
        roofline = {"bound": "alu" if bits else "smem", "unit_op": "POPC" if bits else "red.shared.add",
                    "achieved": ach, "peak": peak_u, "unit": "Gop/s", "frac": ach / peak_u,
                    "traffic": traffic, "traffic_launch": traffic_launch,
                    "peak_source": "of measured (this device, fbn_measure_unit_rates, before the line is printed)",
                    "kernel": f"{kname} (depth {dstar}, {100 * per_ms[dstar] / max(sum(per_ms), 1e-9):.0f}% of the "
                              f"pool's test time)",
                    "kernel_ms_per_step": per_ms[dstar], "work_per_step": work}
    hist_depths = [d for d in pool_depths if st["smem_updates"][d] > 0 and st["popc_work"][d] == 0]
    roofline_smem = None
    if hist_depths:
        hw = sum(st["smem_updates"][d] for d in hist_depths)
        hms = sum(per_ms[d] for d in hist_depths)
        if hms > 0:
            roofline_smem = {"bound": "smem", "unit_op": "red.shared.add", "achieved": hw / (hms / 1e3) / 1e9,
                             "peak": rates["smem_red_per_s"] / 1e9, "unit": "Gop/s",
                             "frac": hw / (hms / 1e3) / rates["smem_red_per_s"],
                             "kernel": "k_pool_small / k_pool_big (depths %s)" % ",".join(map(str, hist_depths)),
                             "kernel_ms_per_step": hms, "work_per_step": hw}
    roofline_gram = None
    if gram_used:
        if w["kind"] == "single":
            M = int(w["ar"].astype("int64").sum())
            flops = float(M) * M * w["data"].shape[1]          # 2 M^2 N / 2
        else:
            flops = float(sum(int(a.astype("int64").sum()) ** 2 * d.shape[1] for d, a in w["probs"]))
        gms = st["gram_ms"]
        tf = flops / (gms / 1e3) / 1e12
        gtraffic, _ = profiled_traffic("k_gram", name)
        roofline_gram = {"bound": "tensor", "achieved": tf, "peak": fp8_peak, "unit": "TFLOP/s",
                         "frac": tf / fp8_peak, "traffic": gtraffic, "peak_source": fp8_src, "kernel": "k_gram",
                         "kernel_ms": gms, "algorithmic_flops": flops}

    # end to end through the public API with host buffers: every step copies
    # the samples from pinned host memory into the handle (fbn_update_data),
    # learns the skeleton into a pinned host adjacency and exports the
    # separating sets to host arrays
    e2e = None
    if w["kind"] == "single":
        host = torch.from_numpy(w["data"]).pin_memory()
        n = w["data"].shape[0]
        adj_host = torch.zeros((n, n), dtype=torch.uint8).pin_memory()
        he = F.fbn_create(host, w["ar"], form=args.form, group_size=gs, device=local, depth1=args.depth1,
                          statistic=args.statistic, df=args.df, loop=args.loop, count=args.count)
        F.fbn_set_stream(he, stream)
        hs_e2e, hosts, adjs_host = [he], [host], [adj_host]
    else:
        hosts = [torch.from_numpy(d).pin_memory() for d, _ in w["probs"]]
        adjs_host = [torch.zeros((d.shape[0],) * 2, dtype=torch.uint8).pin_memory() for d, _ in w["probs"]]
        hs_e2e = [F.fbn_create(hh, a, form=args.form, group_size=gs, device=local, depth1=args.depth1,
                               statistic=args.statistic, df=args.df, loop=args.loop, count=args.count)
                  for hh, (_, a) in zip(hosts, w["probs"])]
        F.fbn_set_stream(hs_e2e[0], stream)
    e2e_ms, d2h = [], 0
    for it in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if w["kind"] == "single":
            F.fbn_update_data(hs_e2e[0], hosts[0])
        else:   # every problem's samples in one call (one synchronisation)
            F.fbn_update_data_batch(hs_e2e, hosts)
        if w["kind"] == "single":
            F.fbn_learn_skeleton(hs_e2e[0], w["alpha"], w["max_depth"], adj_out=adjs_host[0])
        else:
            F.fbn_learn_skeleton_batch(hs_e2e, w["alpha"], w["max_depth"], adj_out=adjs_host)
        removed = members = 0
        for hh in hs_e2e:
            prs, _, mem = F.fbn_export_sepsets(hh, as_dict=False)
            removed += len(prs)
            members += len(mem)
        torch.cuda.synchronize()
        if it > 0:   # the first pass warms the handle
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        # adjacency, the two CSR totals, pairs and offsets of the removed
        # pairs, the members
        d2h = sum(hh.n * hh.n + 16 for hh in hs_e2e) + 16 * removed + 4 * members
    e2e = {"value": world * tests / (statistics.median(e2e_ms) / 1e3), "unit": "tests/s",
           "h2d_bytes_per_step": int(sum(hh.numel() for hh in hosts)), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": statistics.median(e2e_ms)}
    for hh in hs_e2e:
        F.fbn_destroy(hh)

    # the plain edge-level GPU form (one CTA per edge, Section IV-A) on the
    # same workload, same launch pattern (a batch: one launch per depth over
    # every problem's edges), for comparison
    plain = None
    if not args.no_plain and args.form == "pool":
        if w["kind"] == "single":
            hps = [F.fbn_create(data_dev, w["ar"], form="plain", device=local)]
        else:
            hps = [F.fbn_create(torch.from_numpy(d).cuda(), a, form="plain", device=local) for d, a in w["probs"]]
        F.fbn_set_stream(hps[0], stream)

        def plain_step():
            if w["kind"] == "single":
                F.fbn_learn_skeleton(hps[0], w["alpha"], w["max_depth"], adj_out=outs[0])
            else:
                F.fbn_learn_skeleton_batch(hps, w["alpha"], w["max_depth"], adj_out=outs)
        plain_step()
        pm = []
        for _ in range(max(2, min(args.steps, 3 if w["kind"] == "batch" else 5))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plain_step()
            e1.record(stream)
            torch.cuda.synchronize()
            pm.append(e0.elapsed_time(e1))
        sp = F.fbn_get_stats(hps[0])
        pms = sum(pm) / len(pm)
        plain = {"value": world * sum(sp["tests_oracle"]) / (pms / 1e3), "ms_per_step": pms,
                 "tests_executed": sum(sp["tests"]), "steps": len(pm),
                 "chosen_over_plain": (world * tests / (ms / 1e3)) / (world * sum(sp["tests_oracle"]) / (pms / 1e3))}
        for hp in hps:
            F.fbn_destroy(hp)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        cpu = oracle_rate(w, st, args)

    if rank == 0:
        clk["window"] = "0.6 s untimed soak of identical steps followed by the timed steps"
        line = {"metric": METRIC, "value": value, "unit": "tests/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": workload_config(name, w, args), "clocks": clk, "e2e": e2e,
                "gpu_launches": int(st["launches"]) * args.steps, "roofline": roofline,
                "roofline_hbm": roofline_hbm, "roofline_smem": roofline_smem, "roofline_gram": roofline_gram,
                "unit_rates": rates, "tuning": tuning,
                "cpu_baseline": cpu, "plain_form": plain,
                "tests_per_step": {"oracle_equivalent": tests, "executed": sum(st["tests"]),
                                   "per_depth_oracle": st["tests_oracle"]},
                "per_depth": {"edges": st["edges"], "tests_executed": st["tests"],
                              "ms": [round(x, 4) for x in st["ms"]],
                              "test_kernel_ms": [round(x, 4) for x in st["test_ms"]],
                              "test_samples": st["test_samples"], "popc_work": st["popc_work"],
                              "smem_updates": st["smem_updates"]},
                "skeleton_ms": ms, "wall_s": wall}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
