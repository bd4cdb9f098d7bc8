"""Benchmark of the super point detection hot path on GB300.

One step = one discrete window of the core-link workload through the whole
path: zero the sketch, scan 2^26 (src, dst) pairs into SEAV + LDCA, restore
candidates from SEAV and filter them by LDCA (sorted result list on the
device).  Inputs are resident in HBM when the timed region starts and are
larger than L2 (512 MiB of pairs vs 129 MB).

Prints ONE JSON line on rank 0 (see the keys below).  N > 1 runs under
torchrun as independent watch points, one per GPU (weak scaling: each rank
scans its own window; no collective in the data path, only the barrier and
the max-over-ranks timing).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IP pairs/sec (scan + detect, one window per step)"
UNIT = "pairs/s"
WORKLOAD = ("core-link window: 2^26 uint32 (src,dst) pairs, ~4M src with Zipf(1.1) "
            "distinct-dst counts, 500 planted super points (1,500-50,000 peers), "
            "10% duplicate pairs, shuffled; threshold 1024; profile D (SEAV 8 MiB, LDCA 32 MiB)")
SCAN_BYTES_PER_PAIR = 8          # algorithmic HBM bytes of the scan: the pair, read once


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def scan_traffic_from_profile():
    """dram bytes per scan launch from the committed ncu summary, or None when
    the scan source changed since that capture."""
    path = os.path.join(ROOT, "profiles", "k_scan_core_link.md")
    src = os.path.join(ROOT, "paper_1901_07306_gb300", "csrc", "sp_scan.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m_sha = re.search(r"scan_source_sha256_16:\s*([0-9a-f]{16})", text)
        m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
        if m_sha and m_b and m_sha.group(1) == sha:
            return int(m_b.group(1))
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = [ln.strip().split(", ") for ln in open(self.file.name) if ln.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for name, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(pairs, theta, seed, budget_s=12.0, chunk=1 << 20):
    """Times the CPU oracle, as it stands, on a bounded prefix of the window:
    whole chunks are scanned until the budget is spent, then one detect."""
    import oracle as O
    sk = O.Sketch(O.Params(seed=seed, theta=theta))
    n = 0
    t0 = time.perf_counter()
    while n < pairs.shape[0] and time.perf_counter() - t0 < budget_s:
        sk.update(pairs[n:n + chunk])
        n += min(chunk, pairs.shape[0] - n)
    sk.detect(theta)
    dt = time.perf_counter() - t0
    return n, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1901_07306_gb300 import workloads as W
    import oracle
    oracle.build()
    pairs, _ = W.core_link(seed=args.seed)
    budget = max(1.0, args.ref_budget / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_sample(pairs, 1024, args.seed, budget_s=budget)
    rates, ns, dts = [], [], []
    for _ in range(args.steps):
        n, dt = cpu_oracle_sample(pairs, 1024, args.seed, budget_s=budget)
        rates.append(n / dt)
        ns.append(n)
        dts.append(dt)
    value = sum(ns) / sum(dts)
    sample = f"first {min(ns)}-{max(ns)} pairs of the window per step (~{budget:.1f} s budget), then one detect"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_pairs": int(pairs.shape[0])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1901_07306_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    B.build()
    from paper_1901_07306_gb300 import sp, workloads as W

    theta = 1024
    seed = args.seed + rank                      # every rank its own watch point
    pairs, planted = W.core_link(seed=seed, n=1 << args.pairs_log2)
    n = int(pairs.shape[0])
    flat = torch.from_numpy(pairs.reshape(-1).view(np.int32))
    dev_pairs = flat.cuda()
    stream = torch.cuda.current_stream()
    params = sp.make_params(seed=seed, theta=theta, scan_mode=args.scan_mode)
    ctx = sp.SuperPoint(params, stream=stream)
    c = ctx.ctx

    def step():
        sp.sp_reset(c, 0)
        sp.sp_update(c, 0, dev_pairs)
        sp.sp_detect_async(c, 0, theta)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(K):
        e = ev[k]
        sp.sp_reset(c, 0)
        e[0].record(stream)
        sp.sp_update(c, 0, dev_pairs)
        e[1].record(stream)
        e[2].record(stream)
        sp.sp_detect_async(c, 0, theta)
        e[3].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    scan_ms = [e[0].elapsed_time(e[1]) for e in ev]
    det_ms = [e[2].elapsed_time(e[3]) for e in ev]
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    recs, n_found, rc = sp.sp_results(c)
    found = set(recs["ip"].tolist())
    recall = len(found & set(planted.tolist())) / len(planted)

    # end to end through the public API: pinned host pairs -> sp_update_host
    # (double-buffered H2D inside) -> sp_detect (results read back to host)
    e2e = None
    if not args.no_e2e:
        host = flat.pin_memory()
        for _ in range(2):
            sp.sp_reset(c, 0)
            sp.sp_update_host(c, 0, host)
            sp.sp_detect(c, 0, theta)
        ke = max(3, min(K, args.e2e_steps))
        d2h = 0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            sp.sp_reset(c, 0)
            sp.sp_update_host(c, 0, host)
            r, nn, _ = sp.sp_detect(c, 0, theta)
            d2h = 16 + r.nbytes
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": world * n * ke / dt, "unit": UNIT, "h2d_bytes_per_step": n * 8,
               "d2h_bytes_per_step": d2h, "steps": ke, "ms_per_step": 1e3 * dt / ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_cpu, dt_cpu = cpu_oracle_sample(pairs, theta, seed, budget_s=args.cpu_budget)
        cpu = {"value": n_cpu / dt_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_cpu} of the 2^26 window pairs, scanned then one detect, "
                         f"{dt_cpu:.1f} s single-threaded on the host"}

    sp.sp_destroy(c)
    ctx.ctx = None
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    peak, peak_kind = measured_peak_hbm()
    scan_avg_ms = sum(scan_ms) / len(scan_ms)
    achieved = n * SCAN_BYTES_PER_PAIR / (scan_avg_ms * 1e-3) / 1e9
    det_sorted = sorted(det_ms)
    line = {
        "metric": METRIC, "value": world * n * K / (total_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": max(3, args.warmup), "ms_per_step": total_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.pairs_log2 == 26 else f"{WORKLOAD} [scaled to 2^{args.pairs_log2} pairs]",
                   "n_pairs": n, "threshold": theta, "profile": "D", "scan_mode": args.scan_mode,
                   "l2": "inputs larger than L2 (512 MiB of pairs per step vs 129 MB L2)",
                   "parallelism": f"{world} independent watch point(s), one per GPU"},
        "roofline": {"kernel": "k_scan", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": scan_traffic_from_profile(),
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                     "bytes_per_launch": n * SCAN_BYTES_PER_PAIR, "avg_launch_ms": scan_avg_ms},
        "scan_pairs_per_sec": n / (scan_avg_ms * 1e-3),
        "detect_latency_ms": {"p50": det_sorted[len(det_sorted) // 2],
                              "p99": det_sorted[min(len(det_sorted) - 1, int(0.99 * len(det_sorted)))]},
        "super_points": {"found": int(n_found), "planted_recall": recall},
        "clocks": clk,
        "gpu_launches": 4 * K,
        "cpu_baseline": cpu,
        "e2e": e2e,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=60.0)
    ap.add_argument("--pairs-log2", type=int, default=26, help="window size (profiling captures use less)")
    ap.add_argument("--scan-mode", type=int, default=0, help="0 auto, 1 direct (L2 RED), 2 binned")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
