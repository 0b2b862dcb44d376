#!/usr/bin/env python
"""Benchmark of the Panorama exact-refinement search on GB300.

A step is one whole search of a batch of synthetic queries through the
library's C-ABI (query transform, coarse probe, work inversion, level-wise
verification with pruning, exact re-ranking, top-k) with the index and the
queries resident in HBM.  The default workload is the 960-d IVF workload:
N = 1,000,000 FP32 vectors from a 1,024-cluster Gaussian mixture (eigen-decay
exp(-0.01 i)), nlist = 1024, nprobe = 32, 10,000 queries, 16 levels x 60
dims, k = 10.

Printed (rank 0, one JSON line): candidates verified per second (query,
candidate pairs resolved per second over all GPUs), QPS, the same through
host buffers (e2e), the plain FP32 full-distance scan of the same candidate
sets as the comparator, the roofline of the dominant kernel, the CPU oracle
baseline and the SM clocks seen during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 2]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("candidates verified/sec and QPS at oracle-exact top-k: "
          "pruned BF16/FP8 vs plain FP32")
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS, FALLBACK_BF16_TFS = 6800.0, 1900.0
KERNELS_PER_SEARCH = 14  # see the launch list in profiles/
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of a smaller case of the same kernel scaled to the full launch
# (profiles/ holds the capture summary); None once the kernel has changed.
TRAFFIC = {"ivf-1m-d960-fp32": 834.49e6 + 3.38e6}  # phase B, ncu at full size, one pass
PQ_TRAFFIC = {}  # pruned pq_verify_kernel: ncu at full size, one pass (none for this version)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--config", type=int, default=2)
    p.add_argument("--impl", default="panorama", choices=["panorama", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--scan-steps", type=int, default=3)
    p.add_argument("--n", type=int, default=0, help="override N (profiling a smaller case)")
    p.add_argument("--queries", type=int, default=0, help="override the query count")
    p.add_argument("--nlist", type=int, default=0, help="override nlist (and clusters)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-bf16", action="store_true",
                   help="skip the BF16-storage run on FP32 workloads")
    p.add_argument("--no-refine", action="store_true",
                   help="skip the candidate-list refine run on FP32 IVF workloads")
    p.add_argument("--no-fp8", action="store_true",
                   help="skip the FP8-storage run on FP32 and BF16 workloads")
    p.add_argument("--pq-levels", type=int, default=0,
                   help="levels of the IVFPQ line (default: the workload's)")
    p.add_argument("--no-pq-sweep", action="store_true",
                   help="skip the IVFPQ kappa sweep (Section 4.3's shaping trade)")
    p.add_argument("--no-pq", action="store_true",
                   help="skip the IVFPQ line (shaped PCA, M = d/2, levels as the headline)")
    p.add_argument("--no-serve", action="store_true",
                   help="skip the arrival traces of the serving workload")
    p.add_argument("--serve-requests", type=int, default=20000)
    return p.parse_args()


def workload_spec(args):
    import dataclasses
    import synth
    s = synth.spec(args.config)
    upd = {}
    if args.n:
        upd["n"] = args.n
    if args.queries:
        upd["n_queries"] = args.queries
    if args.nlist:
        upd["nlist"] = args.nlist
        if s.n_clusters:
            upd["n_clusters"] = args.nlist
    return dataclasses.replace(s, **upd) if upd else s


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_name(s):
    return (f"{s.name}: N={s.n:,} d={s.d} {s.precision.upper()}, nlist={s.nlist}, "
            f"nprobe={s.nprobe}, {s.n_queries:,} queries, {s.n_levels}x{s.d // s.n_levels}"
            f" levels, k={s.k}")


class Clocks:
    """nvidia-smi sampling of SM clock / throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            j = json.load(f)
        return j, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFS,
                "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(X, Q, C, s, sample_queries, npq, kq, target_s=12.0):
    """The oracle (as it stands) on the host cores: FP64 brute force over each
    sampled query's candidate set after its own FP64 list assignment.  A
    first batch of `sample_queries` sizes the timed sample to ~target_s."""
    import numpy as np
    import oracle
    lists, _ = oracle.assign(X, C)
    ptr, rows = oracle.ivf_lists(lists, C.shape[0])

    def run(qs):
        t0 = time.perf_counter()
        probes, _ = oracle.probe(qs, C, npq[:len(qs)])
        oracle.ivf_topk(X, qs, ptr, rows, probes, kq[:len(qs)])
        return time.perf_counter() - t0, probes

    dt0, _ = run(Q[:sample_queries])
    n = int(min(len(Q), max(sample_queries, sample_queries * target_s / max(dt0, 1e-6))))
    qs = Q[:n]
    dt, probes = run(qs)
    pairs = sum(int(ptr[p + 1].sum() - ptr[p].sum()) for p in probes)
    return {"value": pairs / dt, "unit": "candidates/s", "cores": os.cpu_count(),
            "kind": "oracle", "qps": len(qs) / dt,
            "sample": f"{len(qs)} queries of the workload (probe + FP64 brute force "
                      f"over their candidate sets; list assignment untimed)",
            "seconds": dt}


def run_reference(args):
    """Reference arm: the CPU oracle, on the host cores, on bounded samples."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import numpy as np
    import torch
    import synth
    s = workload_spec(args)
    w = synth.generate(s, device="cpu")
    X, Q = w.X.numpy(), w.Q.numpy()
    npq, kq = w.nprobe.numpy(), w.k.numpy()
    import oracle
    g = np.random.default_rng(3000 + s.cfg)
    C = X[np.sort(g.choice(len(X), s.nlist, replace=False))].astype(np.float32)
    lists, _ = oracle.assign(X, C)
    ptr, rows = oracle.ivf_lists(lists, s.nlist)
    per_step = 24
    def step(i):
        o = (i * per_step) % len(Q)
        qs = Q[o:][:per_step]
        probes, _ = oracle.probe(qs, C, npq[o:][:len(qs)])
        oracle.ivf_topk(X, qs, ptr, rows, probes, kq[o:][:len(qs)])
        return sum(int(ptr[p + 1].sum() - ptr[p].sum()) for p in probes)
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    pairs = 0
    for i in range(args.steps):
        pairs += step(args.warmup + i)
    dt = time.perf_counter() - t0
    v = pairs / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "candidates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(s),
                       "step": f"{per_step} queries (bounded sample of the workload)"},
            "qps": per_step * args.steps / dt,
            "cpu_baseline": {"value": v, "unit": "candidates/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{per_step} queries per step, FP64 brute force"},
            "e2e": {"value": v, "unit": "candidates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def e2e_time(idx, Q, npa, ka, k, args, stream, flush, world, dev):
    """Per-step time of the public API call with HOST buffers: pinned H2D of
    the queries, search, D2H of ids and distances, all inside the events."""
    import torch
    import torch.distributed as dist
    nq = Q.shape[0]
    qh = Q.cpu().pin_memory()
    # per-query nprobe / k are inputs of the step too
    par = [(x.cpu().pin_memory(), torch.empty_like(x)) for x in (npa, ka)
           if isinstance(x, torch.Tensor)]
    if par:
        npa = par[0][1] if isinstance(npa, torch.Tensor) else npa
        ka = par[-1][1] if isinstance(ka, torch.Tensor) else ka
    ids_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    d_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    qd = torch.empty_like(Q)
    for _ in range(2):
        qd.copy_(qh, non_blocking=True)
        for h, dv in par:
            dv.copy_(h, non_blocking=True)
        a, b = idx.search(qd, npa, ka, k_max=k)
        ids_h.copy_(a, non_blocking=True)
        d_h.copy_(b, non_blocking=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        qd.copy_(qh, non_blocking=True)
        for h, dv in par:
            dv.copy_(h, non_blocking=True)
        a, b = idx.search(qd, npa, ka, k_max=k)
        ids_h.copy_(a, non_blocking=True)
        d_h.copy_(b, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    t = torch.tensor([total], device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item() / args.steps, Q.numel() * 4 + sum(h.numel() * 4 for h, _ in par)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2510_00566_gb300 as pano
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_2510_00566_gb300 import _build
    if rank == 0 or not os.path.exists(pano.library_path):
        _build.build()
    if world > 1:
        dist.barrier()
    pano.lib()

    s = workload_spec(args)
    # every rank holds a replica of the index and verifies its own query batch
    w = synth.generate(s, device=dev)
    if rank > 0:
        import dataclasses
        sq = dataclasses.replace(s, cfg=s.cfg + 100 * rank)
        w.Q = synth.generate(sq, device=dev, queries_only=True).Q
    X, Q = w.X, w.Q
    t = pano.panorama_fit_transform(X[:65536], n_levels=s.n_levels)
    prec = {"fp32": pano.PANO_FP32, "bf16": pano.PANO_BF16, "fp8": pano.PANO_FP8}[s.precision]
    # per-query nprobe / k (the batching workload) or scalars
    per_query = not isinstance(s.nprobe, int) or not isinstance(s.k, int)
    npa = w.nprobe.to(dev) if not isinstance(s.nprobe, int) else s.nprobe
    ka = w.k.to(dev) if not isinstance(s.k, int) else s.k
    k = int(w.k.max()) if not isinstance(s.k, int) else s.k  # k_max
    widths, tune = None, None
    if per_query:
        # level widths chosen by the autotuner (median search time of each
        # candidate split on a query sample, k-means run once)
        cands = [[w_] * (s.d // w_) for w_ in (16, 32, 64, 128) if s.d % w_ == 0]
        qs = Q[:min(len(Q), 8192)]
        best, ms = pano.panorama_autotune_levels(t, X, qs, s.nlist, 64, 10, cands,
                                                 precision=prec, repeats=2)
        widths = cands[best]
        tune = {"candidates": [f"{len(c)}x{c[0]}" for c in cands],
                "ms": [float(x) for x in ms], "chosen": f"{len(widths)}x{widths[0]}",
                "sample": f"{len(qs)} queries, nprobe 64, k 10"}
    idx = pano.panorama_build_ivf(t, X, nlist=s.nlist, n_levels=s.n_levels, seed=3000 + s.cfg,
                                  precision=prec, level_widths=widths)
    nq = Q.shape[0]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > L2
    # the batching workload runs as one graph-captured launch per step
    plan = pano.Plan(idx, Q, npa, ka, k_max=k) if per_query else None

    def step(mode=0, timing=False):
        if plan is not None and mode == 0 and not timing:
            return plan.launch(stream)
        return idx.search(Q, npa, ka, k_max=k, mode=mode, collect_timing=timing)

    # counters (one instrumented search, outside the timed region)
    step(0)
    idx.search(Q, npa, ka, k_max=k, collect_stats=True)
    st = pano.last_stats().as_dict()

    def timed(mode, steps, warmup, timing=True):
        for _ in range(warmup):
            step(mode)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        total, verify_ms = 0.0, []
        clk = Clocks(local)
        clk.start()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(mode, timing)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if timing:
                sm = pano.last_stats().stage_ms
                verify_ms.append((sm[3], sm[4], list(sm)))
        torch.cuda.synchronize()
        clocks = clk.stop()
        t_all = torch.tensor([total], device=dev)
        if world > 1:
            dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
        return t_all.item(), verify_ms, clocks

    total_ms, vms, clocks = timed(0, args.steps, args.warmup, timing=plan is None)
    if plan is not None:  # stage times from separate, instrumented searches
        _, vms, _ = timed(0, 3, 1, timing=True)
    ms_per_step = total_ms / args.steps
    pairs = st["pairs"]
    value = pairs * world / (ms_per_step / 1e3)
    qps = nq * world / (ms_per_step / 1e3)

    # comparator: plain FP32 full-distance scan of the same candidate sets
    scan_ms, _, _ = timed(1, args.scan_steps, 1, timing=False)
    scan_per = scan_ms / args.scan_steps

    # e2e: through the public API with host buffers (pinned H2D + D2H)
    e2e_per, h2d = None, 0
    if not args.no_e2e:
        e2e_per, h2d = e2e_time(idx, Q, npa, ka, k, args, stream, flush, world, dev)

    # roofline of the dominant kernel (verify phase B: one launch per step),
    # its duration measured live above with CUDA events on the search stream
    pk, pk_kind = peaks()
    va = float(np.median([v[0] for v in vms]))
    vb = float(np.median([v[1] for v in vms]))
    stage = {n: float(np.median([v[2][i] for v in vms])) for i, n in
             enumerate(("transform", "probe", "inversion", "verify_a", "verify_b", "decode"))}
    dims_b = st["dims_scanned"] - st["dims_scanned_a"]
    flops_b = 2.0 * dims_b  # algorithmic: one FMA per coordinate an alive pair reads
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    if s.precision == "fp32":
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA pipes
        bound, kern = "alu", "verify_fp32_kernel<64,64,256,4> (phase B)"
        src = (f"FP32 FMA: 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
               f"(max clock of MEASURED_PEAKS.json, {pk_kind})")
    else:
        peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1900.0)))
        bound, kern = "tensor", "verify_tc_kernel (phase B)"
        src = f"dense bf16, sustained ({pk_kind})"
    achieved = flops_b / (vb / 1e3) / 1e12
    roof = {"bound": bound, "kernel": kern, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": TRAFFIC.get(s.name),
            "peak_source": src, "flops_per_launch": flops_b, "ms_per_launch": vb,
            "phase_a": {"ms": va, "flops": 2.0 * st["dims_scanned_a"],
                        "achieved": 2.0 * st["dims_scanned_a"] / (va / 1e3) / 1e12},
            "slice_bytes_per_step": st["slice_bytes"],
            "slice_GBps": st["slice_bytes"] / ((va + vb) / 1e3) / 1e9,
            "hbm_peak_GBps": pk.get("hbm_gbs")}

    # pruned BF16 and FP8 storage on the same data and queries (the metric's
    # pruned BF16/FP8 vs plain FP32): d / 64 levels of 64 (valid widths for
    # both), same transform and centroids
    def quantised_run(precision):
        idxq = pano.panorama_build_ivf(t, X, nlist=s.nlist, level_widths=[64] * (s.d // 64),
                                       precision=precision,
                                       centroids=idx.centroids() if s.nlist > 1 else None)
        for _ in range(args.warmup):
            idxq.search(Q, npa, ka, k_max=k)
        torch.cuda.synchronize()
        totq = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            idxq.search(Q, npa, ka, k_max=k)
            e1.record(stream)
            e1.synchronize()
            totq += e0.elapsed_time(e1)
        tq = torch.tensor([totq], device=dev)
        if world > 1:
            dist.all_reduce(tq, op=dist.ReduceOp.MAX)
        msq = tq.item() / args.steps
        idxq.search(Q, npa, ka, k_max=k, collect_stats=True)
        stq = pano.last_stats().as_dict()
        out = {"levels": f"{s.d // 64}x64", "ms_per_step": msq,
               "value": pairs * world / (msq / 1e3), "qps": nq * world / (msq / 1e3),
               "speedup_vs_fp32_scan": scan_per / msq if s.precision == "fp32" else None,
               "dims_scanned_frac": stq["dims_scanned"] / max(1, pairs * s.d),
               "reranked": stq["reranked"], "index_gb": idxq.info().device_bytes / 1e9}
        del idxq
        return out

    # the refine workload (point-centric, B = 1): each query's top-1000 of the
    # pruned IVF search as its candidate-id list, refined to the top-k on a
    # flat index of the same data and levels
    refine = None
    if s.precision == "fp32" and not args.no_refine and s.nlist > 1 and s.d % s.n_levels == 0:
        kprime = 1000
        cand, _ = idx.search(Q, npa, kprime, k_max=kprime)
        flat = pano.panorama_build_flat(t, X, level_widths=[s.d // s.n_levels] * s.n_levels)
        for _ in range(args.warmup):
            flat.refine(Q, cand, k)
        torch.cuda.synchronize()
        totr = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flat.refine(Q, cand, k)
            e1.record(stream)
            e1.synchronize()
            totr += e0.elapsed_time(e1)
        tr = torch.tensor([totr], device=dev)
        if world > 1:
            dist.all_reduce(tr, op=dist.ReduceOp.MAX)
        msr = tr.item() / args.steps
        str_ = pano.last_stats().as_dict()
        refine = {"kprime": kprime, "k": k, "ms_per_step": msr,
                  "value": nq * kprime * world / (msr / 1e3), "unit": "candidates/s",
                  "qps": nq * world / (msr / 1e3),
                  "dims_scanned_frac": str_["dims_scanned"] / max(1, str_["pairs"] * s.d),
                  "reranked": str_["reranked"]}
        del flat, cand

    # the IVFPQ workload (Section 6.3): the same data, lists and queries; the
    # PCA basis shaped for PQ (Section 4.3, kappa = 4, seeded Haar draws),
    # M = d / 2 subquantisers of 8 bits (2-d subvectors), codebooks and codes
    # trained by the library; pruned search vs the plain PQ scan
    ivfpq = None
    Lp = args.pq_levels or s.n_levels
    if (s.precision == "fp32" and not args.no_pq and s.nlist > 1 and s.d % Lp == 0
            and (s.d // 2) % Lp == 0 and isinstance(s.nprobe, int)):
        import time as _time
        gd = np.random.default_rng(7000 + s.cfg).standard_normal((2, s.d, s.d))
        b0 = _time.time()
        tsh, blocks = pano.panorama_shape_transform(t, Lp, 4.0, gd)
        idxp = pano.panorama_build_ivfpq(tsh, X, s.nlist, s.d // 2, Lp,
                                         centroids=idx.centroids(), assign=idx.assignment())
        build_s = _time.time() - b0
        del gd

        def pq_timed(mode, steps):
            for _ in range(args.warmup):
                idxp.search_pq(Q, s.nprobe, k, mode=mode)
            torch.cuda.synchronize()
            tot, vms = 0.0, []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                idxp.search_pq(Q, s.nprobe, k, mode=mode, collect_timing=True)
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
                vms.append(pano.last_stats().stage_ms[4])
            tp = torch.tensor([tot], device=dev)
            if world > 1:
                dist.all_reduce(tp, op=dist.ReduceOp.MAX)
            return tp.item() / steps, float(np.median(vms))

        msp, vmsp = pq_timed(0, args.steps)
        msp_scan, _ = pq_timed(1, args.scan_steps)
        idxp.search_pq(Q, s.nprobe, k, collect_stats=True)
        stp = pano.last_stats().as_dict()
        secs = list(pano.last_stats().section_cycles)[:4]
        secs_share = {nm: v / max(1, sum(secs)) for nm, v in
                      zip(("prologue", "level0_tables", "level0_scan", "deeper_levels"), secs)}
        ivfpq = {"M": s.d // 2, "nbits": 8, "levels": f"{Lp}x{s.d // Lp}",
                 "kappa": 4.0, "robin_hood_blocks": blocks, "ms_per_step": msp,
                 "value": stp["pairs"] * world / (msp / 1e3), "unit": "candidates/s",
                 "qps": nq * world / (msp / 1e3),
                 "plain_pq_scan": {"ms_per_step": msp_scan, "qps": nq * world / (msp_scan / 1e3),
                                   "speedup_of_pruned": msp_scan / msp},
                 "dims_scanned_frac": stp["dims_scanned"] / max(1, stp["pairs"] * s.d),
                 "tables_built": stp["tile_levels"], "pairs": stp["pairs"],
                 "block_time_share": secs_share,
                 # the verify kernel: one shared-memory table lookup per
                 # (live pair, subquantiser); peak = one conflict-free 32-lane
                 # shared-memory wavefront per SM per clock
                 "roofline": {"bound": "lsu", "kernel": "pq_verify_kernel",
                              "achieved": stp["dims_scanned"] / 2 / (vmsp / 1e3),
                              "peak": 152 * 32 * sm_max * 1e6, "unit": "lookups/s",
                              "frac": stp["dims_scanned"] / 2 / (vmsp / 1e3)
                              / (152 * 32 * sm_max * 1e6),
                              "traffic": PQ_TRAFFIC.get(s.name), "ms_per_launch": vmsp,
                              "lookups_per_launch": stp["dims_scanned"] / 2},
                 "index_gb": idxp.info().device_bytes / 1e9, "build_s": build_s}
        # recall@k against the exact top-k over the same lists: the IVFFlat
        # search of the same index lists and queries returns it
        ref_ids, _ = idx.search(Q, s.nprobe, k)
        ref_ids = ref_ids.cpu().numpy()

        def recall_of(ids):
            ids = ids.cpu().numpy()
            return float(np.mean([len(set(ids[i]) & set(ref_ids[i])) / k for i in range(nq)]))

        ivfpq["recall_at_k"] = recall_of(idxp.search_pq(Q, s.nprobe, k)[0])
        del idxp
        # the kappa trade of spectrum shaping (Section 4.3): a larger cap
        # keeps more energy up front (more pruning, less even PQ subspaces)
        if not args.no_pq_sweep:
            sweep = []
            for kap in (1.0, 2.0, 4.0, 16.0):
                gk = np.random.default_rng(7000 + s.cfg).standard_normal((2, s.d, s.d))
                tk, bk = pano.panorama_shape_transform(t, Lp, kap, gk)
                del gk
                ik = pano.panorama_build_ivfpq(tk, X, s.nlist, s.d // 2, Lp,
                                               centroids=idx.centroids(),
                                               assign=idx.assignment())
                for _ in range(2):
                    ik.search_pq(Q, s.nprobe, k)
                torch.cuda.synchronize()
                tot = 0.0
                for _ in range(3):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ids_k, _ = ik.search_pq(Q, s.nprobe, k)
                    e1.record(stream)
                    e1.synchronize()
                    tot += e0.elapsed_time(e1)
                ik.search_pq(Q, s.nprobe, k, collect_stats=True)
                stk = pano.last_stats().as_dict()
                sweep.append({"kappa": kap, "robin_hood_blocks": bk, "ms_per_step": tot / 3,
                              "qps": nq * world / (tot / 3 / 1e3),
                              "recall_at_k": recall_of(ids_k),
                              "dims_scanned_frac": stk["dims_scanned"] / max(1, stk["pairs"] * s.d)})
                del ik, tk
            ivfpq["kappa_sweep"] = sweep
        del tsh

    bf16 = fp8 = None
    if s.precision == "fp32" and not args.no_bf16 and s.d % 64 == 0:
        bf16 = quantised_run(pano.PANO_BF16)
    if s.precision in ("fp32", "bf16") and not args.no_fp8 and s.d % 64 == 0:
        fp8 = quantised_run(pano.PANO_FP8)

    # the serving workload: Poisson arrivals through the continuous-batching
    # server (batches of up to 1024 formed from what has arrived, several in
    # flight, admission by memory); QPS and latency percentiles per rate
    serving = None
    if "serving" in s.name and not args.no_serve:
        import dataclasses
        import numpy as np
        n_req = args.serve_requests
        sq = dataclasses.replace(s, n_queries=n_req, cfg=s.cfg + 50)
        wq = synth.generate(sq, device="cpu", queries_only=True)
        srv = pano.Server(idx, max_batch=1024, max_inflight=4, k_max=10)
        rng = np.random.default_rng(6000 + s.cfg)
        serving = []
        for rate in (20_000, 50_000, 100_000, 200_000):
            arr = np.cumsum(rng.exponential(1e6 / rate, size=n_req))
            b0 = srv.stats()
            _, _, lat = srv.run_trace(wq.Q.numpy(), arr, wq.nprobe.numpy(), wq.k.numpy())
            b1 = srv.stats()
            nb = b1["batches"] - b0["batches"]
            nbq = b1["mean_batch"] * b1["batches"] - b0["mean_batch"] * b0["batches"]
            span_us = float(np.max(arr + lat) - arr[0])
            serving.append({"offered_qps": rate, "qps": n_req / (span_us / 1e6),
                            "p50_us": float(np.percentile(lat, 50)),
                            "p99_us": float(np.percentile(lat, 99)),
                            "max_us": float(lat.max()),
                            "mean_batch": nbq / max(nb, 1), "requests": n_req})
        srv.close()

    cpu = None
    if s.n * s.nlist * s.d > 1e13:  # the oracle's FP64 list assignment alone
        cpu = {"kind": "oracle", "value": None,
               "skipped": "the oracle's FP64 assignment of N vectors to nlist lists would take "
                          "hours on the host cores"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        Xh, Qh = X.cpu().numpy(), Q.cpu().numpy()
        cpu = cpu_baseline(Xh, Qh, idx.centroids(), s, 48, w.nprobe.numpy(), w.k.numpy())
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if s.precision == "fp32" else s.precision, "data": "synthetic",
            "config": {"workload": workload_name(s) + (
                           f" (levels autotuned: {tune['chosen']})" if tune else ""),
                       "l2": "256 MB buffer written between timed steps (L2 flushed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "qps": qps,
            # the comparator: a plain full-distance scan of the same index
            "plain_scan": {"storage": s.precision, "value": pairs * world / (scan_per / 1e3),
                           "qps": nq * world / (scan_per / 1e3), "ms_per_step": scan_per,
                           "speedup_of_pruned": scan_per / ms_per_step},
            "e2e": None if e2e_per is None else {
                "value": pairs * world / (e2e_per / 1e3), "unit": "candidates/s",
                "qps": nq * world / (e2e_per / 1e3), "ms_per_step": e2e_per,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": nq * k * 12},
            "bf16_pruned": bf16,
            "fp8_pruned": fp8,
            "refine": refine,
            "ivfpq": ivfpq,
            "autotune": tune,
            "serving": serving,
            "gpu_launches": (KERNELS_PER_SEARCH if s.nlist > 1 else KERNELS_PER_SEARCH - 2)
                            * args.steps,
            "roofline": roof,
            "stage_ms": stage,
            "search_stats": {kk: st[kk] for kk in ("pairs", "pair_levels", "dims_scanned",
                                                     "dims_scanned_a", "tile_levels",
                                                     "slice_bytes", "reranked", "work_items")},
            "dims_scanned_frac": st["dims_scanned"] / max(1, pairs * s.d),
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
