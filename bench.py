#!/usr/bin/env python
"""Benchmark: range-filtered k-NN queries/sec at recall@10 >= 0.95 on GB300.

Workload (default): N = 1,000,000 points, d = 128 float32 drawn from a
1,024-component Gaussian mixture (sigma 0.1), attribute = a random
permutation of the ranks, 10,000 queries from the same mixture with range
widths 2^-j N for j = 0..10 (equal share), k = 10, graph degree M = 32
(row cap R = 64), leaf size 256, squared Euclidean distance. Synthetic data
of the shape of the paper's 1M-point SIFT/DEEP workloads (Table 3).

One step = one esg_search_batch over the whole 10,000-query batch (all steps
of the hot path: decomposition, beam search with the POST filter on graph
pieces, leaf scans, merge) on device-resident inputs. The beam width is the
smallest of an ef sweep whose recall@10 against the exact GPU brute force
reaches 0.95. An L2 flush (a 512 MB write) separates timed steps, outside the
per-step CUDA events.

`--impl reference` times the CPU oracle instead (exact float64 range-filtered
k-NN, recall 1.0) on a bounded query sample per step, on the host cores.

Prints one JSON line (rank 0).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

METRIC_NAME = "RF-kNN queries/sec at recall@10 \u2265 0.95, 1 GB300: learned+mixed vs plain search"
EF_SWEEP = [16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]
TARGET_RECALL = 0.95


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--ef", type=int, default=0, help="fixed beam width (skip the sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--variants", default="", help="comma-separated subset of variant names")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-budget variant")
    ap.add_argument("--learned-trav", default="bf16", choices=["auto", "f32", "bf16", "fp8"],
                    help="row type of the learned variant; auto: the fastest fixed-ef variant's "
                         "(BF16 and FP8 are within 1 %% there and flip between runs; with the "
                         "learned budget BF16 measured 1.40 ms against 1.46 ms for FP8)")
    ap.add_argument("--bf-workload", default="scale", choices=["scale", "learned"],
                    help="workload of --mode bruteforce: the 128-d scale mixture or the 768-d "
                         "anisotropic inner-product workload (its held-out queries)")
    ap.add_argument("--mode", default="search", choices=["search", "bruteforce", "batching"],
                    help="bruteforce: time only the exact filtered k-NN of the workload's queries; "
                         "batching: the 10M-point, 100k-query workload in one CUDA-graph launch")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    return synthetic.scale(n=args.n, nq=args.nq)


def workload_config(args, extra=None):
    cfg = {"workload": f"ESG range-filtered kNN, N={args.n}, d=128 f32 1024-component mixture, "
                       f"{args.nq} queries, widths 2^-j N (j=0..10), k=10, M=32, leaf 256, L2",
           "n": args.n, "d": 128, "nq": args.nq, "k": 10, "M": 32, "leaf_size": 256,
           "l2_flush": True}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    w = workload(args)
    perm = O.rerank(w.attr)
    X = np.ascontiguousarray(w.base[perm].astype(np.float64))
    per_step = 16
    order = np.arange(len(w.queries))
    times = []
    cursor = 0

    def step():
        nonlocal cursor
        t0 = time.perf_counter()
        for _ in range(per_step):
            i = order[cursor % len(order)]
            cursor += 1
            O.bruteforce(X, w.queries[i].astype(np.float64), int(w.l[i]), int(w.r[i]), 10, w.metric)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    for _ in range(args.steps):
        times.append(step())
    total = sum(times)
    qps = per_step * args.steps / total
    cores = 1
    sample = f"{per_step} queries per step in workload order (exact float64 filtered k-NN, recall 1.0)"
    line = {"impl": "reference", "metric": METRIC_NAME, "value": qps, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, {"parallelism": "replicas"}),
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our arm

def recall_at_10(ids, cnt, gt, gcnt):
    tot = 0.0
    for i in range(len(ids)):
        g = gt[i, :gcnt[i]]
        if len(g) == 0:
            tot += 1.0
            continue
        tot += len(np.intersect1d(ids[i, :cnt[i]], g, assume_unique=True)) / len(g)
    return tot / len(ids)


def cpu_baseline(ix, w, ef, seconds):
    """The oracle's ESG search (Algorithm 4 + Algorithm 1 in plain C, float64)
    on the same graph and ef, one host thread, bounded by `seconds`."""
    import oracle as O
    import paper_2504_04018_gb300 as E
    adj, ent, perm = E.esg_index_export(ix)
    X = np.ascontiguousarray(w.base[perm].astype(np.float64))
    oi = O.OracleIndex(X, perm, adj, ent, ix.leaf_size, ix.R // 2, w.metric)
    done = 0
    t0 = time.perf_counter()
    while done < len(w.queries) and time.perf_counter() - t0 < seconds:
        i = done
        O.search(oi, w.queries[i].astype(np.float64), int(w.l[i]), int(w.r[i]), 10, ef)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(w.queries)} workload queries (all widths), "
                      f"Algorithm 4 + Algorithm 1 in C float64 on the same graph, ef={ef}"}


def bruteforce_timing(E, torch, Xr, Q, L, R, w, args):
    """Exact filtered k-NN of the benchmark queries: the tcgen05 path (whole
    call, and its MMA kernel alone with the MMA FLOPs it issued) against the
    SIMT FP32 kernel (CUDA events, median of 3)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    out = {}
    for name, env in (("tcgen05", "0"), ("simt", "1")):
        os.environ["ESG_BF_SIMT"] = env
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            E.esg_bruteforce_filtered_knn(Xr, Q, L, R, 10, w.metric)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out[name + "_ms"] = round(sorted(ts)[1], 3)
    os.environ.pop("ESG_BF_SIMT", None)
    # the MMA kernel alone
    E.esg_profile_enable(True)
    E.esg_bruteforce_filtered_knn(Xr, Q, L, R, 10, w.metric)
    torch.cuda.synchronize()
    kms, _, _ = E.esg_profile_read(reset=True)
    mma_flops = E.esg_profile_tensor_work(reset=True)
    E.esg_profile_enable(False)
    pairs = float(np.sum(w.r - w.l + 1))
    useful = 2.0 * w.d * pairs                      # one dot product per in-range pair
    peak = float(peaks.get("bf16_tflops", 1900.0))
    t = out["tcgen05_ms"] / 1e3
    out.update({"queries": int(len(w.l)), "pairs": pairs,
                "qps_tcgen05": len(w.l) / t, "qps_simt": len(w.l) / (out["simt_ms"] / 1e3),
                "useful_tflops": useful / t / 1e12,
                "mma_kernel_ms": round(kms, 4),
                "mma_tflops_issued": mma_flops,
                "mma_kernel_tflops": (mma_flops / (kms / 1e3) / 1e12) if kms > 0 else None,
                "mma_frac_of_bf16_peak": (mma_flops / (kms / 1e3) / 1e12 / peak) if kms > 0 else None,
                "bf16_peak_tflops": peak,
                "peak_source": "measured" if "bf16_tflops" in peaks else "fallback"})
    return out


# (name, traversal rows, search width); "plain" is Algorithm 1's order on FP32 rows
VARIANTS = [("plain", "f32", 1)] + [(f"{t}-w{wd}", t, wd) for t in ("f32", "bf16", "fp8")
                                    for wd in (1, 2) if not (t == "f32" and wd == 1)]
ESIZE = {"f32": 4, "bf16": 2, "fp8": 1}
N_TRAIN = 20_000
# largest beam width the learned budget may pick: the candidate list and the
# visited table are sized for it, so a tight cap keeps more warps resident
LEARNED_EF_HI = 64
# labels = smallest ef reaching this per-query recall; median regression; the
# calibrated margin then sets the mean recall (on the scale workload this beat
# full-recall labels with quantile 0.9 by 5-8 % in kernel time at equal recall)
LEARNED_LABEL_RECALL = 0.9
LEARNED_QUANTILE = 0.5


def measured_traffic(variant, params):
    """DRAM bytes per launch of the search kernel from the committed ncu
    summary, when it was taken for this variant, these search parameters
    (ef, budget, row type, width; not the launch shape) and the current
    kernel sources (None otherwise)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "search_kernel_traffic.txt")))[variant]
    except Exception:
        return None
    m = hashlib.sha256()
    for p in rec["kernel_sources"]:
        m.update(open(os.path.join(ROOT, p), "rb").read())
    if m.hexdigest()[:16] != rec["kernel_sources_sha256_16"]:
        return None
    if any(params.get(k) != v for k, v in rec["params"].items()):
        return None
    return rec["traffic_bytes_per_launch"]


def run_bruteforce_only(args, local):
    """Exact filtered k-NN of the workload's queries over the rank-ordered
    points, tcgen05 path against the SIMT kernel (no index is built)."""
    import torch
    import paper_2504_04018_gb300 as E
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E.load_library()
    if args.bf_workload == "learned":
        w = synthetic.learned(n=args.n, nq=args.nq, n_train=0)
    else:
        w = workload(args)
    perm = np.argsort(w.attr, kind="stable")      # rank order: attribute, ties by id
    Xr = torch.as_tensor(w.base[perm], device=dev)
    Q = torch.as_tensor(w.queries, device=dev)
    L = torch.as_tensor(w.l, device=dev)
    Rr = torch.as_tensor(w.r, device=dev)
    info = bruteforce_timing(E, torch, Xr, Q, L, Rr, w, args)
    print(json.dumps({"mode": "bruteforce", "metric": "exact RF-kNN queries/sec (k=10)",
                      "value": info["qps_tcgen05"], "unit": "queries/s", "n_gpus": 1,
                      "higher_is_better": True, "dtype": "bf16x3+f32", "data": "synthetic",
                      "config": (workload_config(args) if args.bf_workload == "scale" else
                                 {"workload": f"N={w.n}, d={w.d} anisotropic unit vectors, inner product, "
                                              f"{len(w.l)} queries, widths log-uniform 0.1%-100%, k=10"}),
                      "bruteforce": info}), flush=True)


def run_batching(args, local):
    """10M unit-norm 96-d points (inner product, BF16 rows + FP32 re-rank),
    100,000 queries with widths 0.01%-100% and k in {1, 10, 100} replayed as
    one CUDA graph per step; launch shape and beam width from the autotuner
    on 2,000 training queries; recall on 3,000 sampled queries against the
    exact GPU brute force; per-query device latency percentiles."""
    import torch
    import paper_2504_04018_gb300 as E
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E.load_library()
    w = synthetic.batching()
    t0 = time.perf_counter()
    ix = E.esg_build(w.base, w.attr, M=32, leaf_size=256, n_entries=16, metric="ip", storage="bf16")
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    _, _, perm = E.esg_index_export(ix)
    Xr = torch.as_tensor(w.base[perm], device=dev)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)

    def gt_of(q, l, r):
        gi, _, gc = E.esg_bruteforce_filtered_knn(Xr, t(q), t(l), t(r), 100, "ip")
        torch.cuda.synchronize()
        gi, gc = gi.cpu().numpy(), gc.cpu().numpy()
        return np.where(gi >= 0, perm[np.maximum(gi, 0)], -1), gc

    tq, tl, tr = synthetic.training_queries(w, 2000, 1024, seed=4004)
    tk = np.array([1, 10, 100], np.int32)[np.random.default_rng(4005).integers(0, 3, 2000)]
    tgt, tgc = gt_of(tq, tl, tr)
    params, trec, _ = E.esg_autotune(ix, t(tq), t(tl), t(tr), t(tgt), t(tgc), k_max=100, k=t(tk),
                                     target_recall=0.955, base=E.search_params(ef=64, traversal="bf16"))
    nq = len(w.l)
    b = E.Batch(ix, max_nq=nq, k_max=100, params=params, use_k=True)
    b.view("queries", (nq, ix.d), torch.float32).copy_(t(w.queries))
    b.view("l", (nq,), torch.int64).copy_(t(w.l))
    b.view("r", (nq,), torch.int64).copy_(t(w.r))
    b.view("k", (nq,), torch.int32).copy_(t(w.k))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.run(nq, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(nq, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    stats = b.view("stats", (nq, 6), torch.int64).cpu().numpy()
    ids = b.view("ids", (nq, 100), torch.int64).cpu().numpy()
    cnt = b.view("count", (nq,), torch.int32).cpu().numpy()
    ev = np.random.default_rng(5).choice(nq, 3000, replace=False)
    gt, gc = gt_of(w.queries[ev], w.l[ev], w.r[ev])
    hits = tot = 0
    for j, i in enumerate(ev):
        c = min(int(w.k[i]), int(gc[j]))
        hits += len(set(ids[i, :min(int(cnt[i]), c)].tolist()) & set(gt[j, :c].tolist()))
        tot += c
    lat = stats[:, 5] / 1e3
    print(json.dumps({"mode": "batching", "metric": "RF-kNN queries/sec, 100k queries per CUDA-graph launch",
                      "value": nq * args.steps / (total / 1e3), "unit": "queries/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
                      "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": "N=10,000,000, d=96 unit-norm 1024-component mixture, inner product, "
                                             "100,000 queries, widths log-uniform 0.01%-100%, k in {1,10,100}, M=32",
                                 "params": params.as_dict(), "l2_flush": True},
                      "recall_sampled_3000": hits / tot, "autotune_train_recall": trec,
                      "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                     "max": float(lat.max())},
                      "build_s": round(build_s, 1), "clocks": clk}), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import paper_2504_04018_gb300 as E
    from paper_2504_04018_gb300 import replicas as R

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    E.load_library()
    w = workload(args)
    t0 = time.perf_counter()
    ix = E.esg_build(w.base, w.attr, M=32, leaf_size=256, n_entries=16, ef_construction=200,
                     metric="l2", storage="bf16")
    E.esg_index_add_storage(ix, "fp8")
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    _, _, perm = E.esg_index_export(ix)
    Q = torch.as_tensor(w.queries, device=dev)
    L = torch.as_tensor(w.l, device=dev)
    Rr = torch.as_tensor(w.r, device=dev)
    nq = Q.shape[0]
    Xr = torch.as_tensor(w.base[perm], device=dev)

    def ground_truth(q, l, r):
        """Exact answers (original ids) from the GPU brute force over the
        rank-ordered rows."""
        gi, _, gc = E.esg_bruteforce_filtered_knn(Xr, q, l, r, 10)
        torch.cuda.synchronize()
        gi, gc = gi.cpu().numpy(), gc.cpu().numpy()
        return np.where(gi >= 0, perm[np.maximum(gi, 0)], -1), gc

    gt, gc = ground_truth(Q, L, Rr)
    bf_info = bruteforce_timing(E, torch, Xr, Q, L, Rr, w, args)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = (torch.empty((nq, 10), dtype=torch.int64, device=dev),
           torch.empty((nq, 10), dtype=torch.float32, device=dev),
           torch.empty(nq, dtype=torch.int32, device=dev),
           torch.empty(nq, dtype=torch.int32, device=dev), None)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    results = {}

    def timed(step_fn, name):
        for _ in range(args.warmup):
            step_fn()
        torch.cuda.synchronize()
        R.barrier()
        torch.cuda.nvtx.range_push(f"timed_{name}")
        evs = [step_fn() for _ in range(args.steps)]
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        total_ms = R.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev)
        R.barrier()
        return total_ms

    def measure(name, params, trav):
        """Recall, per-step time, kernel time and algorithmic bytes of one
        parameter setting with direct esg_search_batch calls."""
        ids, dist, cnt, st, stats = E.esg_search_batch(ix, Q, L, Rr, None, 10, params=params,
                                                       want_stats=True)
        torch.cuda.synchronize()
        rec = recall_at_10(ids.cpu().numpy(), cnt.cpu().numpy(), gt, gc)
        stats = stats.cpu().numpy()
        alg_bytes = float(stats[:, 1].sum() * ix.d * ESIZE[trav] + stats[:, 0].sum() * ix.R * 4
                          + stats[:, 3].sum() * ix.d * 4)

        def one_step():
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            E.esg_search_batch(ix, Q, L, Rr, None, 10, params=params, out=out)
            ev1.record(stream)
            return ev0, ev1

        E.esg_profile_enable(True)
        total_ms = timed(one_step, name)
        kernel_ms, launches, nt = E.esg_profile_read(reset=True)
        E.esg_profile_enable(False)
        launches_per_step = launches // max(1, args.steps + args.warmup)
        return {"trav": trav, "params": params.as_dict(), "recall": round(rec, 5),
                "qps": R.job_rate(nq, world, args.steps, total_ms), "ms_per_step": total_ms / args.steps,
                "kernel_ms": kernel_ms / max(1, nt), "alg_bytes": alg_bytes,
                "launches": launches_per_step * args.steps,
                "evals_per_query": float(stats[:, 1].mean()),
                "expansions_per_query": float(stats[:, 0].mean()),
                # per-query device latency inside the batch (first piece taken
                # by a warp to last piece finished), from the kernel's timer
                "latency_us": {"p50": float(np.percentile(stats[:, 5], 50) / 1e3),
                               "p99": float(np.percentile(stats[:, 5], 99) / 1e3)}}

    sweeps = {}
    chosen_variants = [v for v in VARIANTS if not args.variants or v[0] in args.variants.split(",")]
    if not any(v[0] == "plain" for v in chosen_variants):
        chosen_variants = [VARIANTS[0]] + chosen_variants
    for name, trav, width in chosen_variants:
        sweep, chosen = [], args.ef
        for ef in ([args.ef] if args.ef else EF_SWEEP):
            ids, _, cnt, _, _ = E.esg_search_batch(ix, Q, L, Rr, None, 10, ef=ef, traversal=trav,
                                                   width=width)
            torch.cuda.synchronize()
            rec = recall_at_10(ids.cpu().numpy(), cnt.cpu().numpy(), gt, gc)
            sweep.append({"ef": ef, "recall": round(rec, 5)})
            if not args.ef and rec >= TARGET_RECALL:
                chosen = ef
                break
        sweeps[name] = sweep
        results[name] = measure(name, E.search_params(ef=chosen or EF_SWEEP[-1], traversal=trav,
                                                      width=width), trav)

    # learned budget + low-precision rows + autotuned launch shape + CUDA graph
    learned_info = {}
    if not args.no_learned:
        mixed = {k: v for k, v in results.items() if k != "plain" and v["recall"] >= TARGET_RECALL
                 and v["params"]["width"] == 1}
        trav = results[max(mixed, key=lambda k: mixed[k]["qps"])]["trav"] if mixed else "f32"
        if args.learned_trav != "auto":
            trav = args.learned_trav
        tq, tl, tr = synthetic.training_queries(w, N_TRAIN, 1024, seed=4002)
        TQ, TL, TR = (torch.as_tensor(a, device=dev) for a in (tq, tl, tr))
        tgt, tgc = ground_truth(TQ, TL, TR)
        t1 = time.perf_counter()
        rep = E.esg_train_predictor(ix, TQ, TL, TR, torch.as_tensor(tgt, device=dev),
                                    torch.as_tensor(tgc, device=dev), k_max=10,
                                    target_recall=TARGET_RECALL + 0.005, ef_lo=8, ef_hi=LEARNED_EF_HI,
                                    traversal=trav, epochs=40, per_query_recall=LEARNED_LABEL_RECALL,
                                    quantile=LEARNED_QUANTILE)
        train_s = time.perf_counter() - t1
        base = E.search_params(ef=LEARNED_EF_HI, traversal=trav, use_learned=1)
        # launch shape timed on training batches of the benchmark's batch size
        tuned, trec, tms = E.esg_autotune(ix, TQ[:nq], TL[:nq], TR[:nq], torch.as_tensor(tgt[:nq], device=dev),
                                          torch.as_tensor(tgc[:nq], device=dev), k_max=10,
                                          target_recall=TARGET_RECALL, base=base)
        # both search widths with the tuned launch shape, like the fixed-ef
        # variants; the faster one that meets the recall target is replayed
        # as a graph
        cands = []
        for wd in (1, 2):
            pw = E.search_params(**dict(tuned.as_dict(), width=wd))
            nm = f"learned-{trav}" + ("" if wd == 1 else "-w2")
            results[nm] = measure(nm, pw, trav)
            cands.append((nm, pw))
        ok = [c for c in cands if results[c[0]]["recall"] >= TARGET_RECALL] or cands
        name, tuned = max(ok, key=lambda c: results[c[0]]["qps"])
        # the chosen setting replayed as one CUDA graph per batch
        b = E.Batch(ix, max_nq=nq, k_max=10, params=tuned)
        b.view("queries", (nq, ix.d), torch.float32).copy_(Q)
        b.view("l", (nq,), torch.int64).copy_(L)
        b.view("r", (nq,), torch.int64).copy_(Rr)

        def graph_step():
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            b.run(nq, stream=stream)
            ev1.record(stream)
            return ev0, ev1

        E.esg_profile_enable(True)
        total_ms = timed(graph_step, name + "-graph")
        _, launches, _ = E.esg_profile_read(reset=True)
        E.esg_profile_enable(False)
        ids = b.view("ids", (nq, 10), torch.int64).cpu().numpy()
        cnt = b.view("count", (nq,), torch.int32).cpu().numpy()
        g = dict(results[name])
        g.update({"recall": round(recall_at_10(ids, cnt, gt, gc), 5),
                  "qps": R.job_rate(nq, world, args.steps, total_ms), "ms_per_step": total_ms / args.steps,
                  "launches": launches // max(1, args.steps + args.warmup) * args.steps, "graph": True})
        results[name + "-graph"] = g
        learned_info = {"traversal": trav, "train_queries": N_TRAIN, "ef_hi": LEARNED_EF_HI,
                        "label_recall": LEARNED_LABEL_RECALL, "quantile": LEARNED_QUANTILE, "train_s": round(train_s, 2),
                        "train_loss": float(rep[0]), "heldout_recall": float(rep[1]),
                        "ef_margin_log2": float(rep[2]), "heldout_evals_per_query": float(rep[3]),
                        "autotune": {"params": tuned.as_dict(), "recall": trec, "ms": tms}}
    clk = clocks.stop()
    ok = {k: v for k, v in results.items() if v["recall"] >= TARGET_RECALL}
    opt = {k: v for k, v in ok.items() if k != "plain"}
    head_name = max(opt, key=lambda k: opt[k]["qps"]) if opt else "plain"
    head = results[head_name]

    # end to end through the public call with host buffers (headline setting)
    Qh = torch.as_tensor(w.queries).pin_memory()
    Lh = torch.as_tensor(w.l).pin_memory()
    Rh = torch.as_tensor(w.r).pin_memory()
    ids_h = torch.empty((nq, 10), dtype=torch.int64).pin_memory()
    dist_h = torch.empty((nq, 10), dtype=torch.float32).pin_memory()
    cnt_h = torch.empty(nq, dtype=torch.int32).pin_memory()
    Qd, Ld, Rd = torch.empty_like(Q), torch.empty_like(L), torch.empty_like(Rr)
    head_params = E.search_params(**head["params"])

    def e2e_step():
        flush.fill_(1.0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        Qd.copy_(Qh, non_blocking=True)
        Ld.copy_(Lh, non_blocking=True)
        Rd.copy_(Rh, non_blocking=True)
        E.esg_search_batch(ix, Qd, Ld, Rd, None, 10, params=head_params, out=out)
        ids_h.copy_(out[0], non_blocking=True)
        dist_h.copy_(out[1], non_blocking=True)
        cnt_h.copy_(out[2], non_blocking=True)
        ev1.record(stream)
        return ev0, ev1

    e2e_ms = timed(e2e_step, "e2e")
    h2d = Qh.numel() * 4 + Lh.numel() * 8 + Rh.numel() * 8
    d2h = ids_h.numel() * 8 + dist_h.numel() * 4 + cnt_h.numel() * 4

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = head["alg_bytes"] / (head["kernel_ms"] / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": measured_traffic(head_name, head["params"]),
                "kernel": f"search_kernel ({head_name})",
                "kernel_ms_per_launch": round(head["kernel_ms"], 4),
                "algorithmic_bytes_per_launch": head["alg_bytes"],
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    variants = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()
                    if kk not in ("alg_bytes",)} for k, v in results.items()}
    line = {"metric": METRIC_NAME, "value": head["qps"], "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": head["trav"], "data": "synthetic",
            "config": workload_config(args, {"parallelism": f"replicas{world}",
                                             "variant": head_name, "params": head["params"]}),
            "recall_at_10": head["recall"],
            "plain_fp32": {"qps": results["plain"]["qps"], "ef": results["plain"]["params"]["ef"],
                           "recall_at_10": results["plain"]["recall"]},
            "speedup_vs_plain": head["qps"] / results["plain"]["qps"],
            "variants": variants, "ef_sweeps": sweeps, "learned": learned_info,
            "build_s": round(build_s, 2), "roofline": roofline, "clocks": clk,
            "bruteforce": bf_info,
            "e2e": {"value": R.job_rate(nq, world, args.steps, e2e_ms), "unit": "queries/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": head["launches"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ix, w, results["plain"]["params"]["ef"], args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mode == "bruteforce":
        if rank == 0:
            run_bruteforce_only(args, local)
        return
    if args.mode == "batching":
        if rank == 0:
            run_batching(args, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
