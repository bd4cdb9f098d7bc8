"""Benchmark of the super point detection hot path on GB300.

One step = one discrete window of the core-link workload through the whole
path: zero the sketch, scan 2^26 (src, dst) pairs into SEAV + LDCA, restore
candidates from SEAV and filter them by LDCA (sorted result list on the
device).  Inputs are resident in HBM when the timed region starts and are
larger than L2 (512 MiB of pairs vs 129 MB).

Prints ONE JSON line on rank 0 (see the keys below).  N > 1 runs under
torchrun as watch points, one per GPU (weak scaling: each rank scans its own
window in the headline region, whose only collectives are the barrier and the
max-over-ranks timing); after it, the WP -> GS exchange of Sec. 4.2 (NCCL
all-gather of the device sketches, OR on the GPU, detect) is timed and
checked bit-exact against one GPU's scan of the union stream ("exchange").
At N = 1 the line also carries the accuracy of the window against exact
ground truth (Sec. 6 FPR/FNR) and the distributed, sliding-window and
serving workloads ("workloads"), each timed on its own after the headline.

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


def scan_source_hash():
    h = hashlib.sha256()
    for name in ("sp_scan.cu", "sp_scan_binned.cu"):
        h.update(open(os.path.join(ROOT, "paper_1901_07306_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def scan_traffic_from_profile(n_pairs):
    """DRAM bytes (read + write) of one scan stage (k_bin + k_apply) over
    n_pairs, scaled from the committed one-kernel ncu summaries of a smaller
    case (traffic grows in proportion to the pairs); None when the scan
    sources changed since those captures."""
    total = 0.0
    for kernel in ("k_bin", "k_apply"):
        path = os.path.join(ROOT, "profiles", f"{kernel}_core_link_2e25.md")
        try:
            text = open(path).read()
        except OSError:
            return None
        m_sha = re.search(r"scan_sources_sha256_16:\s*([0-9a-f]{16})", text)
        m_b = re.search(r"kernel_dram_bytes:\s*([0-9]+)", text)
        m_n = re.search(r"kernel_pairs:\s*([0-9]+)", text)
        if not (m_sha and m_b and m_n) or m_sha.group(1) != scan_source_hash():
            return None
        total += int(m_b.group(1)) * n_pairs / int(m_n.group(1))
    return int(total)


def launches_per_step(n_pairs, scan_mode):
    """Kernels one core-link step launches: k_zero (sp_reset); the scan
    (k_scan, or per binning round k_bin + k_apply); the detect (k_fold8 after
    a binned scan, k_detect, k_sort_emit).  Auto mode bins updates of 2^22
    pairs and more, in rounds of up to 2^26 pairs."""
    binned = scan_mode == 2 or (scan_mode == 0 and n_pairs >= (1 << 22))
    if not binned:
        return 1 + 1 + 2
    rounds = max(1, -(-n_pairs // (1 << 26)))
    return 1 + 2 * rounds + 1 + 2


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None
        self.n0 = 0

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
            # nvidia-smi's start-up (NVML initialisation) disturbs the GPU's
            # host transfers for ~0.1 s: the timed region starts only once it
            # has written two samples (at most 5 s)
            self._wait_rows(2, 5.0)
            self.n0 = self._rows()
        except Exception:
            self.proc = None

    def _rows(self) -> int:
        with open(self.file.name) as f:
            return sum(1 for ln in f if ln.strip())

    def _wait_rows(self, n: int, limit_s: float):
        deadline = time.perf_counter() + limit_s
        while time.perf_counter() < deadline and self.proc.poll() is None and self._rows() < n:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._wait_rows(self.n0 + 2, 1.0)              # samples from the timed region and just after it
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = [ln.strip().split(", ") for ln in open(self.file.name) if ln.strip()]
        os.unlink(self.file.name)
        rows = rows[self.n0:] or rows                  # the start-up samples precede the timed region
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


def cpu_oracle_threads(pairs, theta, seed, threads=None, chunk=1 << 20):
    """The oracle, as it stands, on every host core: the window is split into
    one contiguous shard per thread, each thread scans its shard into its own
    sketch (the oracle's C calls release the GIL), the sketches are OR-merged
    (the merged sketch equals the sketch of the whole stream) and one detect
    runs.  Returns (pairs, seconds, threads)."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or os.cpu_count() or 1
    params = O.Params(seed=seed, theta=theta)
    bounds = np.linspace(0, pairs.shape[0], threads + 1).astype(np.int64)

    def shard(t):
        sk = O.Sketch(params)
        for a in range(int(bounds[t]), int(bounds[t + 1]), chunk):
            sk.update(pairs[a:min(a + chunk, int(bounds[t + 1]))])
        return sk

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        sketches = list(ex.map(shard, range(threads)))
    merged = sketches[0]
    for sk in sketches[1:]:
        merged.merge(sk)
    merged.detect(theta)
    return int(pairs.shape[0]), time.perf_counter() - t0, threads


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
        if args.exchange:                         # the exchange leg on a one-rank NCCL group
            import socket
            import torch.distributed as dist
            with socket.socket() as sock:
                sock.bind(("127.0.0.1", 0))
                port = sock.getsockname()[1]
            dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                                    device_id=torch.device("cuda", 0))
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
    # router 1 is the global server of the multi-GPU exchange
    with_exchange = world > 1 or args.exchange
    params = sp.make_params(seed=args.seed, theta=theta, scan_mode=args.scan_mode, n_routers=2 if with_exchange else 1)
    ctx = sp.SuperPoint(params, stream=stream)
    c = ctx.ctx
    # the binned scan's staging shape, tuned on a sample of the window
    shape = None
    if args.scan_mode != 1:
        if args.shape < 0:
            shape = sp.sp_autotune_binned(c, dev_pairs[: 2 << 24])
        else:
            sp.sp_set_binned_shape(c, args.shape)
            shape = sp.sp_get_binned_shape(c)

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
    from paper_1901_07306_gb300 import exchange
    total_ms = exchange.reduce_max(total_ms)
    recs, n_found, rc = sp.sp_results(c)
    found_ips = recs["ip"].copy()
    found = set(found_ips.tolist())
    recall = len(found & set(planted.tolist())) / len(planted)

    # end to end through the public API: pinned host pairs -> sp_update_host
    # (double-buffered H2D inside) -> detect -> results read back to the host.
    # Windows are pipelined the way a watch point streams them: two routers
    # take alternate windows, the results come back with sp_results_async and
    # the host reads window s - 1's results while window s is in flight, so a
    # window's detect and result copy overlap the next window's host copies.
    # The synchronous form (sp_detect per window) is reported beside it.
    e2e = None
    if not args.no_e2e:
        host = flat.pin_memory()
        ctx2 = sp.SuperPoint(sp.make_params(seed=seed, theta=theta, scan_mode=args.scan_mode, n_routers=2),
                             stream=stream)
        c2 = ctx2.ctx
        cap = 4096
        outs = [torch.from_numpy(np.zeros(cap, sp.CANDIDATE).view(np.uint8)).pin_memory() for _ in range(2)]
        stats = [torch.zeros(2, dtype=torch.int32).pin_memory() for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]

        def window(s_):
            r = s_ % 2
            sp.sp_reset(c2, r)
            sp.sp_update_host(c2, r, host)
            sp.sp_detect_async(c2, r, theta)
            sp.sp_results_async(c2, outs[r], cap, stats[r])
            evs[r].record(stream)

        def read(s_):
            r = s_ % 2
            evs[r].synchronize()
            cnt = int(stats[r][0])
            return outs[r].numpy().view(sp.CANDIDATE)[:min(cnt, cap)]

        for s_ in range(4):                               # warm up
            window(s_)
        torch.cuda.synchronize()
        ke = max(3, min(K, args.e2e_steps))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        win_found = []
        t0 = time.perf_counter()
        for s_ in range(ke):
            window(s_)
            if s_ > 0:
                win_found.append(read(s_ - 1))            # the previous window's results, on the host
        win_found.append(read(ke - 1))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = exchange.reduce_max(dt)
        assert all(np.array_equal(f["ip"], recs["ip"]) for f in win_found), "pipelined windows disagree"
        d2h = 8 + cap * sp.CANDIDATE.itemsize
        # the synchronous form: one window at a time, sp_detect waits for it
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(max(3, ke // 5)):
            sp.sp_reset(c, 0)
            sp.sp_update_host(c, 0, host)
            sp.sp_detect(c, 0, theta)
        torch.cuda.synchronize()
        sync_ms = 1e3 * (time.perf_counter() - t1) / max(3, ke // 5)
        ctx2.close()
        # context: the plain host-to-device copy rate of the same pinned buffer
        scratch = torch.empty_like(dev_pairs)
        scratch.copy_(host, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(5):
            scratch.copy_(host, non_blocking=True)
        torch.cuda.synchronize()
        h2d = 5 * n * 8 / (time.perf_counter() - t1) / 1e9
        del scratch
        e2e = {"value": world * n * ke / dt, "unit": UNIT, "h2d_bytes_per_step": n * 8,
               "d2h_bytes_per_step": d2h, "steps": ke, "ms_per_step": 1e3 * dt / ke,
               "pipelining": "two routers, alternate windows, results read one window behind",
               "sync_ms_per_step": sync_ms, "pinned_h2d_copy_gbs": h2d}

    cpu = cpu_threads = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_cpu, dt_cpu = cpu_oracle_sample(pairs, theta, seed, budget_s=args.cpu_budget)
        cpu = {"value": n_cpu / dt_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_cpu} of the 2^26 window pairs, scanned then one detect, "
                         f"{dt_cpu:.1f} s single-threaded on the host"}
        n_mt, dt_mt, thr = cpu_oracle_threads(pairs, theta, seed)
        cpu_threads = {"value": n_mt / dt_mt, "unit": UNIT, "cores": thr,
                       "kind": "oracle, one sketch per thread, OR-merged",
                       "sample": f"the whole 2^26-pair window in {thr} shards, then the merge and one detect, "
                                 f"{dt_mt:.1f} s"}

    # N > 1: the WP -> GS exchange (Sec. 4.2) over NCCL, timed after the
    # headline region: every rank's device sketch all-gathered, ORed into a
    # global router and detected on every rank
    xchg = exchange_leg(torch, sp, W, c, args, rank, world) if with_exchange else None
    sp.sp_destroy(c)
    ctx.ctx = None
    acc = accuracy(found_ips, exact_super_points(pairs, theta)) if not args.no_extra else None
    # the batched and served forms, each timed on its own after the headline region
    legs = None
    if rank == 0 and world == 1 and not args.no_extra:
        legs = {"distributed": distributed_leg(torch, sp, W, 24, 64, steps=5, warmup=3),
                "sliding": sliding_leg(torch, sp, W, 28, passes=1, warmup=1),
                "serving": serving_leg(torch, sp, W, requests=400, runs=5, warmup=1),
                "detect_many_results": detect_many_leg(torch, sp),
                "bounds": bounds_leg(torch)}
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
                   "binned_shape": shape,
                   "l2": "inputs larger than L2 (512 MiB of pairs per step vs 129 MB L2)",
                   "parallelism": f"{world} independent watch point(s), one per GPU"},
        "roofline": {"kernel": ("scan stage k_bin + k_apply (binned)" if args.scan_mode != 1 else "k_scan (direct)"),
                     "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": scan_traffic_from_profile(n),
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                     "bytes_per_launch": n * SCAN_BYTES_PER_PAIR, "avg_launch_ms": scan_avg_ms},
        "scan_pairs_per_sec": n / (scan_avg_ms * 1e-3),
        "detect_latency_ms": {"p50": det_sorted[len(det_sorted) // 2],
                              "p99": det_sorted[min(len(det_sorted) - 1, int(0.99 * len(det_sorted)))]},
        "super_points": {"found": int(n_found), "planted_recall": recall},
        "accuracy": acc,
        "clocks": clk,
        "gpu_launches": launches_per_step(n, args.scan_mode) * K,
        "cpu_baseline": cpu,
        "cpu_baseline_threads": cpu_threads,
        "e2e": e2e,
        "workloads": legs,
        "exchange": xchg,
    }
    print(json.dumps(line), flush=True)
    if with_exchange:
        torch.distributed.destroy_process_group()
    return 0


# ---- the other workloads ----------------------------------------------------
# Each leg returns a dict; ``--workload X`` prints it as its own JSON line and
# the default core-link run embeds a compact form of every leg under
# "workloads" (timed after, and outside, the headline region).
D3 = dict(r=16, isb=(0, 4, 8, 12), ibn=(7, 7, 7, 7), lc_log2=18)   # 16 routers x 2^24 pairs merged
# serving windows of 2^24 pairs: a quarter of profile D's SEAs and LDCs keeps
# its load per SE and per LDC (SEAV 2 MiB + LDCA 8 MiB per router)
PROFILE_S = dict(r=12, isb=(0, 5, 10, 15), ibn=(7, 7, 7, 7), lc_log2=14)


def exchange_leg(torch, sp, W, c, args, rank, world, steps=10):
    """Multi-GPU WP -> GS exchange (Sec. 4.2), NCCL device form: time of
    all-gather of the ranks' device sketches + OR into router 1 + detect (max
    over ranks), and a bit-exactness check of the same path on 2^22-pair
    windows against one GPU's scan of the ranks' concatenated streams (rank 0;
    the OR of the sketches equals the sketch of the union stream)."""
    from paper_1901_07306_gb300 import exchange
    theta = 1024

    def gather_merge_detect(ctx_):
        g = exchange.all_gather_sketches(sp, ctx_, 0)
        sp.sp_reset(ctx_, 1)
        exchange.merge_gathered(sp, ctx_, g, 1)
        sp.sp_detect_async(ctx_, 1, theta)
        return g

    for _ in range(3):
        gather_merge_detect(c)
    torch.cuda.synchronize()
    torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        g = gather_merge_detect(c)
    torch.cuda.synchronize()
    ms = exchange.reduce_max(1e3 * (time.perf_counter() - t0) / steps)
    n_found = sp.sp_results(c)[1]
    # the check on small windows: every rank scans its own, the merged result
    # must equal one scan of all ranks' windows
    small = lambda r: W.core_link(seed=args.seed + r, n=1 << 22)[0]  # noqa: E731
    stream = torch.cuda.current_stream()
    chk = sp.SuperPoint(sp.make_params(seed=args.seed, theta=theta, n_routers=2), stream=stream)
    sp.sp_update(chk.ctx, 0, torch.from_numpy(small(rank).reshape(-1).view(np.int32)).cuda())
    gather_merge_detect(chk.ctx)
    got = sp.sp_results(chk.ctx)[0]
    merged_img = chk.sketch_image(1)
    chk.close()
    exact = None
    if rank == 0:
        one = sp.SuperPoint(sp.make_params(seed=args.seed, theta=theta), stream=stream)
        for r in range(world):
            sp.sp_update(one.ctx, 0, torch.from_numpy(small(r).reshape(-1).view(np.int32)).cuda())
        want = one.detect()[0]
        ref_img = one.sketch_image(0)
        one.close()
        exact = bool(np.array_equal(got, want) and all(np.array_equal(a, b) for a, b in zip(merged_img, ref_img)))
        assert exact, "the exchanged global sketch differs from one scan of the union stream"
    return {"form": "NCCL all-gather of device sketch images + OR on the GPU + detect",
            "bytes_per_rank": int(g.shape[1]), "ms": ms, "global_super_points": int(n_found),
            "bit_exact_vs_one_gpu_union_scan": exact, "check": f"{world} ranks x 2^22-pair windows"}


def exact_super_points(pairs, theta):
    """Ground truth of Def. 1-2 (not the method): the hosts with at least
    theta distinct opposite IPs, by sort-unique of the distinct pairs."""
    keys = np.unique(np.ascontiguousarray(pairs, np.uint32).view(np.uint64).reshape(-1))
    hosts, counts = np.unique((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), return_counts=True)
    return hosts[counts >= theta]


def accuracy(found, truth):
    """Sec. 6: FPR = detected hosts that are not super points / super points,
    FNR = super points not detected / super points, FTR = FPR + FNR."""
    found, truth = set(np.asarray(found).tolist()), set(np.asarray(truth).tolist())
    n = max(1, len(truth))
    fpr, fnr = len(found - truth) / n, len(truth - found) / n
    return {"super_points": len(truth), "detected": len(found), "fpr": fpr, "fnr": fnr, "ftr": fpr + fnr}


def _device_setup():
    import torch
    torch.cuda.set_device(0)
    from paper_1901_07306_gb300 import build as B
    B.build()
    from paper_1901_07306_gb300 import sp, workloads as W
    return torch, sp, W


def _gpu_index():
    v = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return int(v.split(",")[0]) if v.split(",")[0].isdigit() else 0


def _pcts(xs):
    s = sorted(xs)
    return {"p50": s[len(s) // 2], "p99": s[min(len(s) - 1, int(0.99 * len(s)))]}


def _timed(torch, fn, steps, warmup, clocks=None):
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def distributed_leg(torch, sp, W, router_log2=24, batches_per_router=64, steps=10, warmup=3, with_accuracy=False):
    """16 simulated border routers, each 2^router_log2 pairs arriving as
    uneven time-slice batches; one step = reset, scan every batch, OR-merge
    into the global router, detect.  Batched (one sp_update_batched call) vs
    one launch per batch (sp_update per batch)."""
    n_routers, per = 16, 1 << router_log2
    routers, sp_hosts = W.distributed(seed=3, n_per_router=per)
    rng = np.random.default_rng(3)
    flats = [torch.from_numpy(pr.reshape(-1).view(np.int32)).cuda() for pr in routers]
    batches = []
    for r, pr in enumerate(routers):
        w = np.exp(rng.uniform(0, np.log(16.0), batches_per_router))
        cuts = np.floor(np.cumsum(w / w.sum())[:-1] * pr.shape[0]).astype(np.int64)
        bounds = [0, *cuts.tolist(), pr.shape[0]]
        batches += [(r, flats[r][2 * a:2 * b]) for a, b in zip(bounds[:-1], bounds[1:])]
    batches = [batches[i] for i in rng.permutation(len(batches))]
    total = sum(t.numel() // 2 for _, t in batches)
    stream = torch.cuda.current_stream()
    ctx = sp.SuperPoint(sp.make_params(theta=1024, seed=3, n_routers=n_routers + 1, **D3), stream=stream)
    c = ctx.ctx
    shape = sp.sp_autotune_binned(c, flats[0])            # staging shape tuned on one router's stream
    rlist, tlist = [r for r, _ in batches], [t for _, t in batches]

    def step(batched):
        sp.sp_reset_range(c, 0, n_routers + 1)
        if batched:
            sp.sp_update_batched(c, rlist, tlist)
        else:
            for r, t in batches:
                sp.sp_update(c, r, t)
        sp.sp_merge(c, list(range(n_routers)), n_routers)
        sp.sp_detect_async(c, n_routers, 1024)

    clocks = ClockSampler(_gpu_index())
    ms_b = _timed(torch, lambda: step(True), steps, warmup, clocks)
    clk = clocks.stop()
    res_b, n_b, _ = sp.sp_results(c)
    ms_p = _timed(torch, lambda: step(False), max(3, steps // 2), 3)
    res_p, n_p, _ = sp.sp_results(c)
    ctx.close()
    assert np.array_equal(res_b, res_p), "batched and per-batch paths disagree"
    out = {"workload": f"distributed: {n_routers} routers x 2^{router_log2} pairs from an overlapping host population, "
                       f"1,000 global super points split across routers, {batches_per_router} uneven batches per "
                       "router; reset + scan + OR-merge + detect per step; profile D3 (r=16, LC=2^18)",
           "n_pairs": total, "batches": len(batches), "steps": steps, "binned_shape": shape,
           "batched": {"value": total / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b},
           "plain_per_batch": {"value": total / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p},
           "batched_speedup": ms_p / ms_b,
           "super_points": {"found": int(n_b),
                            "global_recall": len(set(res_b["ip"].tolist()) & set(sp_hosts.tolist())) / len(sp_hosts)},
           "clocks": clk}
    if with_accuracy:
        out["accuracy"] = accuracy(res_b["ip"], exact_super_points(np.concatenate(routers), 1024))
    return out


def sliding_leg(torch, sp, W, total_log2=28, passes=2, warmup=1, checkpoints=()):
    """A stream of time slices of lognormal size (2^28 pairs in 128 slices at
    full size), window of 32 slices advanced one slice at a time (Sec. 5):
    per slice = slide + scan the slice + detect the window.  checkpoints:
    slices whose window's detection is scored against exact ground truth."""
    T = total_log2
    scale = 1 << max(0, 28 - T)
    sizes = W.slice_sizes(4, n_slices=128, total=1 << T, lo=(1 << 19) // scale, hi=(1 << 22) // scale)
    slices, sp_hosts, sched = W.sliding_stream(seed=4, sizes=sizes, n_sp=64, sp_degree_per_slice=(64, 512))
    dev_slices = [torch.from_numpy(x.reshape(-1).view(np.int32)).cuda() for x in slices]
    stream = torch.cuda.current_stream()
    k = 32
    ctx = sp.SuperPoint(sp.make_params(theta=1024, seed=4, window_slices=k), stream=stream)
    c = ctx.ctx
    found = {}

    def one_pass(keep=()):
        sp.sp_reset(c, 0)
        evs = []
        for t, x in enumerate(dev_slices):
            if t:
                sp.sp_slide(c, 0)
            sp.sp_update(c, 0, x)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sp.sp_detect_async(c, 0, 1024)
            e1.record(stream)
            evs.append((e0, e1))
            if t in keep:
                found[t] = sp.sp_results(c)[0]["ip"]
        return evs

    for _ in range(max(1, warmup)):                   # warm up: whole passes over the stream
        one_pass()
    torch.cuda.synchronize()
    clocks = ClockSampler(_gpu_index())
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    evs = []
    for _ in range(passes):
        evs += one_pass()
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / passes
    det = [e0.elapsed_time(e1) for e0, e1 in evs]
    n_found = sp.sp_results(c)[1]
    total = int(sizes.sum())
    out = {"workload": f"sliding window: 2^{T} pairs in 128 lognormal slices [{int(sizes.min())}, {int(sizes.max())}] "
                       f"pairs, window {k} slices advanced one slice at a time; per slice slide + scan + detect; "
                       "profile D with slice stamps; one step = one pass over the stream",
           "n_pairs": total, "slices": len(slices), "window_slices": k, "passes": passes,
           "value": total / (ms * 1e-3), "unit": UNIT, "ms_per_pass": ms,
           "detect_latency_ms": _pcts(det), "super_points_last_window": int(n_found), "clocks": clk}
    # the per-slice step as one CUDA graph (slide + scan through a one-entry
    # device batch table + detect), recorded once and replayed per slice with
    # the table entry copied in from a device array of all slices' entries
    entries = np.zeros(len(slices), sp.BATCH)
    for t, x in enumerate(dev_slices):
        entries[t] = (x.data_ptr(), slices[t].shape[0], 0, 0)
    dev_entries = torch.from_numpy(entries.view(np.uint8)).cuda().view(len(slices), -1)
    table = torch.empty_like(dev_entries[0])
    g = torch.cuda.CUDAGraph()

    def graph_pass():
        sp.sp_reset(c, 0)
        table.copy_(dev_entries[0])
        sp.sp_update_batched_device(c, table, 1)
        sp.sp_detect_async(c, 0, 1024)
        for t in range(1, len(slices)):
            table.copy_(dev_entries[t])
            g.replay()

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):                     # warm up the captured calls off the capture
        sp.sp_set_stream(c, side)
        sp.sp_slide(c, 0)
        sp.sp_update_batched_device(c, table, 1)
        sp.sp_detect_async(c, 0, 1024)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        sp.sp_set_stream(c, torch.cuda.current_stream())
        sp.sp_slide(c, 0)
        sp.sp_update_batched_device(c, table, 1)
        sp.sp_detect_async(c, 0, 1024)
    sp.sp_set_stream(c, stream)
    graph_pass()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(passes):
        graph_pass()
    b.record(stream)
    torch.cuda.synchronize()
    ms_g = a.elapsed_time(b) / passes
    out["graph"] = {"value": total / (ms_g * 1e-3), "unit": UNIT, "ms_per_pass": ms_g,
                    "form": "per slice one CUDA graph replay: slide + scan (device batch table, direct form) + detect",
                    "super_points_last_window": int(sp.sp_results(c)[1])}
    if checkpoints:
        one_pass(keep=set(checkpoints))
        out["accuracy"] = {str(t): accuracy(found[t], exact_super_points(
            np.concatenate(slices[max(0, t - k + 1):t + 1]), 1024)) for t in sorted(found)}
    ctx.close()
    return out


def serving_leg(torch, sp, W, requests=400, runs=3, warmup=1, window_slices=1):
    """64 routers sending batches of 2^12-2^22 pairs (log-uniform) with Poisson
    arrivals; continuous batching (each step's pinned batches scanned in place
    by one batched call) under a 2 GiB in-flight budget vs the plain
    one-launch-per-batch path, a detect every 2^24 global pairs.  Throughput
    with the offered load above capacity (median of the runs), then
    batch-to-result latency at half the plain path's capacity (the median
    run of each path by ack p50)."""
    from paper_1901_07306_gb300 import serving as S
    n_routers = 64
    reqs = S.poisson_requests(5, n_routers, requests, rate_pairs_per_s=1e13, lo_log2=12, hi_log2=22)
    total = sum(r.n_pairs for r in reqs)

    # one server per path, made once and reused by every run (a server is
    # long-lived: its context and pinned result buffers outlast the runs)
    servers = {b: S.SketchServer(n_routers, dict(PROFILE_S, theta=1024, seed=5), budget_bytes=2 << 30,
                                 detect_every=1 << 24, window_slices=window_slices, batched=b) for b in (True, False)}

    def serve(batched, rate):
        mean = total / len(reqs)
        rng = np.random.default_rng(55)
        gaps = rng.exponential(mean / rate, len(reqs))
        arr = np.cumsum(gaps) - gaps[0]
        rs = [S.Request(router=r.router, pairs=r.pairs, arrival=float(a)) for r, a in zip(reqs, arr)]
        srv = servers[batched]
        wins = srv.run(rs)
        return rs, wins, srv.elapsed

    try:
        return _serving_runs(S, serve, reqs, total, n_routers, runs, warmup, window_slices)
    finally:
        for srv in servers.values():
            srv.close()


def _serving_runs(S, serve, reqs, total, n_routers, runs, warmup, window_slices):
    for _ in range(max(1, warmup)):                                   # warm up: first DMA of the pinned batches
        serve(True, 1e13)
        serve(False, 1e13)
    clocks = ClockSampler(_gpu_index())
    clocks.start()
    # offered load above capacity; host-driven, so the median of several runs
    bat = sorted((serve(True, 1e13) for _ in range(runs)), key=lambda x: x[2])
    pla = sorted((serve(False, 1e13) for _ in range(runs)), key=lambda x: x[2])
    rb, wb, tb = bat[runs // 2]
    rp, wp, tp = pla[runs // 2]
    assert all(a.n_found == b.n_found and np.array_equal(a.records, b.records) for a, b in zip(wb, wp))
    rate = 0.5 * total / tp                                          # half the plain path's capacity
    lat = {"batched": [], "plain": []}
    for _ in range(runs):                                            # alternating; the median run by ack p50
        lat["batched"].append(S.latency_summary(serve(True, rate)[0]))
        lat["plain"].append(S.latency_summary(serve(False, rate)[0]))
    clk = clocks.stop()
    med = {k: sorted(v, key=lambda x: x["ack_ms"]["p50"])[len(v) // 2] for k, v in lat.items()}
    return {"workload": f"serving: {n_routers} routers, {len(reqs)} batches of 2^12-2^22 pairs (log-uniform), Poisson "
                        "arrivals, batched steps read the pinned batches in place, 2 GiB in-flight budget, detect every "
                        "2^24 global pairs (OR-merge into a global "
                        "router), profile S (r=12, LC=2^14), "
                        + (f"sliding window of {window_slices} detect periods" if window_slices > 1
                           else "discrete windows") + "; value = median of the runs (host wall clock)",
            "n_pairs": total, "windows": len(wb), "runs": runs,
            "runs_ms": {"batched": [round(x[2] * 1e3, 3) for x in bat], "plain": [round(x[2] * 1e3, 3) for x in pla]},
            "batched": {"value": total / tb, "unit": UNIT, "ms": tb * 1e3},
            "plain_per_batch": {"value": total / tp, "unit": UNIT, "ms": tp * 1e3},
            "batched_speedup": tp / tb,
            "latency_at_half_plain_capacity": {
                "offered_pairs_per_s": rate, "runs": runs, "batched": med["batched"], "plain": med["plain"],
                "runs_ack_p50_ms": {k: [round(x["ack_ms"]["p50"], 3) for x in v] for k, v in lat.items()}},
            "clocks": clk}


def detect_many_leg(torch, sp, n_hosts=150000, reps=50):
    """Detection with many results: n_hosts hosts of 64 distinct peers each at
    theta = 32 (about n_hosts super points, so the result sort spans runs of
    8,192 keys merged across the grid); detect p50/p99 over reps detects."""
    rng = np.random.default_rng(51)
    hosts = rng.permutation(np.unique(rng.integers(0, 2**32, n_hosts + n_hosts // 4, dtype=np.uint32))[:n_hosts])
    pairs = np.stack([np.repeat(hosts, 64), rng.integers(0, 2**32, hosts.size * 64, dtype=np.uint32)], 1)
    stream = torch.cuda.current_stream()
    ctx = sp.SuperPoint(sp.make_params(r=16, isb=(0, 8), ibn=(9, 9), theta=32, seed=51), stream=stream)
    sp.sp_update(ctx.ctx, 0, torch.from_numpy(np.ascontiguousarray(pairs).reshape(-1).view(np.int32)).cuda())
    evs = []
    for _ in range(reps + 3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sp.sp_detect_async(ctx.ctx, 0, 0)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    n_found = sp.sp_results(ctx.ctx)[1]
    ctx.close()
    return {"workload": f"{n_hosts} hosts x 64 distinct peers, theta 32, r = 16, SR = 2",
            "super_points": int(n_found), "detect_latency_ms": _pcts([a.elapsed_time(b) for a, b in evs[3:]])}


def bounds_leg(torch, reps=10):
    """The hardware rates that bound the scan (include/sp_bounds.h), measured
    on this GPU: streaming reads of 1 GiB (HBM), random 32-bit atomic ORs
    into a 32 MiB array (L2-resident, as the LDCA of the direct scan) and into
    a 32 KiB shared-memory array per block (as a bit plane of the binned
    scan), with the pair rates they allow at LR = 4 bit sets per pair."""
    import ctypes
    from paper_1901_07306_gb300 import build as B
    lib = ctypes.CDLL(B.BOUNDS_LIB)
    for name in ("sp_probe_stream_read", "sp_probe_l2_red", "sp_probe_smem_atomic"):
        getattr(lib, name).restype = ctypes.c_int
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.sp_probe_stream_read.argtypes = [vp, u64, vp, u32, vp]
    lib.sp_probe_l2_red.argtypes = [vp, u32, u32, u32, u32, vp]
    lib.sp_probe_smem_atomic.argtypes = [vp, u32, u32, u32, u32, vp]
    stream = torch.cuda.current_stream()
    h = ctypes.c_void_p(stream.cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    buf = torch.zeros(1 << 30, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    words = torch.zeros(1 << 23, dtype=torch.int32, device="cuda")

    def timed(call):
        for _ in range(3):
            assert call() == 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            call()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e-3

    t_read = timed(lambda: lib.sp_probe_stream_read(buf.data_ptr(), buf.numel(), sink.data_ptr(), 0, h))
    red_ops = 256
    t_red = timed(lambda: lib.sp_probe_l2_red(words.data_ptr(), 23, red_ops, 0, 7, h))
    smem_ops = 1024
    t_smem = timed(lambda: lib.sp_probe_smem_atomic(sink.data_ptr(), 13, smem_ops, 0, 7, h))
    del buf, words
    read_gbs = (1 << 30) / t_read / 1e9
    red_rate = sms * 8 * 256 * red_ops / t_red
    smem_rate = sms * 4 * 512 * smem_ops / t_smem
    peak, _ = measured_peak_hbm()
    return {"hbm_stream_read_gbs": read_gbs,
            "l2_random_red_or_per_s": red_rate,
            "smem_random_atomic_or_per_s": smem_rate,
            "pairs_per_s_if_bound_by": {"hbm_read_8B_per_pair": read_gbs * 1e9 / 8,
                                        "l2_red_4_per_pair": red_rate / 4,
                                        "smem_atomic_4_per_pair": smem_rate / 4},
            "as_frac_of_hbm_roofline": {"l2_red_4_per_pair": red_rate / 4 * 8 / (peak * 1e9),
                                        "smem_atomic_4_per_pair": smem_rate / 4 * 8 / (peak * 1e9)}}


def _line(leg, args, value, ms):
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": leg.pop("workload"), "n_pairs": leg["n_pairs"]},
            "clocks": leg.pop("clocks"), **leg}


def run_distributed(args):
    torch, sp, W = _device_setup()
    leg = distributed_leg(torch, sp, W, args.router_log2, args.batches_per_router, args.steps, args.warmup,
                          with_accuracy=not args.no_extra)
    print(json.dumps(_line(leg, args, leg["batched"]["value"], leg["batched"]["ms_per_step"])), flush=True)
    return 0


def run_sliding(args):
    torch, sp, W = _device_setup()
    leg = sliding_leg(torch, sp, W, args.slide_total_log2, max(1, min(args.steps, 5)), args.warmup,
                      checkpoints=(31, 64, 127))
    print(json.dumps(_line(leg, args, leg["value"], leg["ms_per_pass"])), flush=True)
    return 0


def run_bounds(args):
    torch, sp, W = _device_setup()
    clocks = ClockSampler(_gpu_index())
    clocks.start()
    leg = bounds_leg(torch)
    print(json.dumps({"metric": "hardware rates bounding the scan", "unit": "see keys", "n_gpus": 1,
                      "clocks": clocks.stop(), **leg}), flush=True)
    return 0


def run_serving(args):
    torch, sp, W = _device_setup()
    leg = serving_leg(torch, sp, W, args.requests, max(3, min(args.steps, 5)), args.warmup,
                      args.serve_window_slices)
    print(json.dumps(_line(leg, args, leg["batched"]["value"], leg["batched"]["ms"])), flush=True)
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
    ap.add_argument("--exchange", action="store_true",
                    help="run the multi-GPU exchange leg even on one GPU (a one-rank NCCL group)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the accuracy report and the distributed, sliding and serving legs")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=60.0)
    ap.add_argument("--pairs-log2", type=int, default=26, help="window size (profiling captures use less)")
    ap.add_argument("--scan-mode", type=int, default=0, help="0 auto, 1 direct (L2 RED), 2 binned")
    ap.add_argument("--shape", type=int, default=-1,
                    help="staging shape of the binned scan (sp_binned_shapes index); -1 = autotune on the window")
    ap.add_argument("--workload", default="core_link",
                    choices=["core_link", "distributed", "sliding", "serving", "bounds"])
    ap.add_argument("--router-log2", type=int, default=24)
    ap.add_argument("--batches-per-router", type=int, default=64)
    ap.add_argument("--slide-total-log2", type=int, default=28)
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--serve-window-slices", type=int, default=1)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "distributed":
        return run_distributed(args)
    if args.workload == "sliding":
        return run_sliding(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "bounds":
        return run_bounds(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
