#!/usr/bin/env python
"""Benchmark of the Panorama exact-refinement search on GB300.

A step is one whole search of a batch of synthetic queries through the
library's C-ABI (query transform, coarse probe, work inversion, level-wise
verification with pruning, exact re-ranking, top-k) with the index and the
queries resident in HBM.  The default workload is the 768-d precision
workload: N = 10,000,000 vectors from one Gaussian (eigen-decay
exp(-0.008 i)), IVF nlist = 4096, nprobe = 64, 10,000 queries, 12 levels x
64 dims, k = 10, level slices stored in BF16 (the headline) and in FP8-E4M3,
compared with the plain scans: the tensor-core scan of the same BF16 index
and the plain FP32 full-distance scan of an FP32 index of the same data.

Printed (rank 0, one JSON line): candidates verified per second (query,
candidate pairs resolved per second over all GPUs) and QPS of the pruned
BF16 search, the same through host buffers (e2e), the FP8 and FP32 lines,
a sampled comparison with the CPU oracle at full size (`parity`), the HBM
roofline of the dominant kernel, the CPU oracle baseline, the SM clocks
seen during the timed region, and a secondary line for the 960-d FP32
workload (with the epsilon sweep of Eq. 4, point-centric refine and IVFPQ).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 3]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
"""
import argparse
import dataclasses
import json
import math
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
# DRAM bytes (read + write) of one launch of the dominant kernel, from one
# ncu capture of that launch at full size (one pass: dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the full workload description (so a
# resized run gets none); the command and figures are in profiles/.  An
# entry is removed whenever its kernel changes, so the line then reports
# null instead of a stale figure.
TRAFFIC = {
    # verify_tc_kernel<BF16>, phase B of the pruned search (whole-tile copies,
    # issue warp, one CTA barrier per level, chunk-wise test schedule, level-0
    # tiles staged first, B-tile loads in flight together): 20.58 GB read +
    # 0.018 GB written
    "ivf-10m-d768-bf16: N=10,000,000 d=768 BF16, nlist=4096, nprobe=64, 10,000 queries, "
    "12x64 levels, k=10": 20.58e9 + 17.67e6,
}
PQ_TRAFFIC = {}
EPSILONS = (1.0, 0.9, 0.8, 0.6, 0.5, 0.4)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--config", type=int, default=3)
    p.add_argument("--impl", default="panorama", choices=["panorama", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-parity", action="store_true",
                   help="skip the sampled comparison with the CPU oracle")
    p.add_argument("--parity-queries", type=int, default=256)
    p.add_argument("--scan-steps", type=int, default=3)
    p.add_argument("--n", type=int, default=0, help="override N (profiling a smaller case)")
    p.add_argument("--queries", type=int, default=0, help="override the query count")
    p.add_argument("--nlist", type=int, default=0, help="override nlist (and clusters)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp8", action="store_true", help="skip the FP8-storage line")
    p.add_argument("--no-fp32", action="store_true",
                   help="skip the FP32-storage line of a quantised workload")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the 960-d FP32 workload's secondary line")
    p.add_argument("--no-eps", action="store_true", help="skip the epsilon sweep")
    p.add_argument("--no-refine", action="store_true",
                   help="skip the candidate-list refine run on FP32 IVF workloads")
    p.add_argument("--no-pq", action="store_true",
                   help="skip the IVFPQ line (shaped PCA, M = d/2, levels as the workload's)")
    p.add_argument("--pq-sweep", action="store_true",
                   help="add the IVFPQ kappa sweep (Section 4.3's shaping trade)")
    p.add_argument("--pq-levels", type=int, default=0,
                   help="levels of the IVFPQ line (default: the workload's)")
    p.add_argument("--no-serve", action="store_true",
                   help="skip the arrival traces of the serving workload")
    p.add_argument("--serve-requests", type=int, default=20000)
    return p.parse_args()


def workload_spec(args, cfg=None):
    import synth
    s = synth.spec(cfg or args.config)
    upd = {}
    if cfg is None or cfg == args.config:
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
    npr = s.nprobe if isinstance(s.nprobe, int) else f"U[{s.nprobe[0]},{s.nprobe[1]}]"
    k = s.k if isinstance(s.k, int) else "{" + ",".join(map(str, s.k)) + "}"
    return (f"{s.name}: N={s.n:,} d={s.d} {s.precision.upper()}, nlist={s.nlist}, "
            f"nprobe={npr}, {s.n_queries:,} queries, {s.n_levels}x{s.d // s.n_levels}"
            f" levels, k={k}")


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


# --------------------------------------------------------------- the oracle
class OracleSide:
    """The CPU oracle's view of a workload: the FP32 host arrays, the
    coarse centroids the library's build chose, and the oracle's own FP64
    assignment of every vector to them (Section 6.1); shared by the parity
    sample and the timed CPU baseline."""

    def __init__(self, X, Q, C):
        import numpy as np
        import oracle
        self.X = np.ascontiguousarray(X, dtype=np.float32)
        self.Q = np.ascontiguousarray(Q, dtype=np.float32)
        self.C = np.asarray(C, dtype=np.float32)
        t0 = time.perf_counter()
        self.lists, self.agap = oracle.assign(self.X, self.C)
        self.assign_s = time.perf_counter() - t0
        self.ptr, self.rows = oracle.ivf_lists(self.lists, self.C.shape[0])

    def answer(self, rows, nprobe, k):
        """Oracle top-k of queries `rows` over their FP64 probe sets."""
        import numpy as np
        import oracle
        qs = self.Q[rows]
        probes, pgap = oracle.probe(qs, self.C, nprobe)
        ids, d = oracle.ivf_topk(self.X, qs, self.ptr, self.rows, probes, k)
        return ids, d, probes, pgap


def parity_report(osd, rows, nprobe, k, got_ids, got_d, gpu_probes, lib_assign):
    """Element-by-element comparison of the GPU's results for queries `rows`
    with the oracle's, by the rules of the parity tests: ids equal except
    where the FP64 distances are within 1e-6 relative (near-ties), each
    returned distance within 1e-5 relative of the FP64 distance of its id.
    Queries whose nprobe-th and next FP64 centroid distances are within
    1e-6 relative are left out (either probe set is correct)."""
    import numpy as np
    nq = len(rows)
    npq = np.broadcast_to(np.asarray(nprobe), (nq,))
    kq = np.broadcast_to(np.asarray(k), (nq,)).astype(np.int32)
    ref_i, ref_d, probes, pgap = osd.answer(rows, npq, kq)
    keep = pgap >= 1e-6
    probe_mismatch = 0
    for j in np.nonzero(keep)[0]:
        if not np.array_equal(np.sort(gpu_probes[j][:npq[j]]), np.sort(probes[j])):
            probe_mismatch += 1
    worst, beyond, swaps, bad_pad = 0.0, 0, 0, 0
    for j in np.nonzero(keep)[0]:
        kj = int(kq[j])
        nv = int(np.sum(ref_i[j, :kj] >= 0))
        g = got_ids[j, :nv]
        if np.any(got_ids[j, nv:kj] != -1) or np.any(g < 0):
            bad_pad += 1
            continue
        if nv == 0:
            continue
        diff = osd.X[g].astype(np.float64) - osd.Q[rows[j]].astype(np.float64)
        true_d = np.einsum("ij,ij->i", diff, diff)
        rel = np.abs(got_d[j, :nv].astype(np.float64) - true_d) / np.maximum(true_d, 1e-30)
        worst = max(worst, float(rel.max()))
        mism = g != ref_i[j, :nv]
        if mism.any():
            r = ref_d[j, :nv][mism]
            gap = np.abs(true_d[mism] - r) / np.maximum(r, 1e-30)
            swaps += int(np.sum(gap <= 1e-6))
            beyond += int(np.sum(gap > 1e-6))
    am = None
    if lib_assign is not None:
        am = int(np.sum((lib_assign != osd.lists) & (osd.agap >= 1e-6)))
    return {"queries": int(keep.sum()), "excluded_probe_near_ties": int((~keep).sum()),
            "probe_mismatch": probe_mismatch, "max_rel_err": worst,
            "id_mismatch_beyond_tie": beyond, "near_tie_swaps": swaps,
            "bad_padding": bad_pad, "assignment_mismatch_beyond_tie": am,
            "tolerances": "dist 1e-5 rel vs FP64; ids exact except FP64 near-ties < 1e-6 rel",
            "oracle": "FP64 brute force over the query's FP64 probe set, vectors assigned "
                      "to the library's centroids in FP64"}


def cpu_baseline(osd, nprobe, k, sample_queries=24, target_s=12.0):
    """The oracle (as it stands) on the host cores: FP64 probe + brute force
    over each sampled query's candidate set (the list assignment is done
    once, untimed).  A first batch of `sample_queries` sizes the timed
    sample to ~target_s."""
    import numpy as np
    import oracle
    nq = len(osd.Q)
    npq = np.broadcast_to(np.asarray(nprobe), (nq,))
    kq = np.broadcast_to(np.asarray(k), (nq,)).astype(np.int32)

    def run(n):
        t0 = time.perf_counter()
        probes, _ = oracle.probe(osd.Q[:n], osd.C, npq[:n])
        oracle.ivf_topk(osd.X, osd.Q[:n], osd.ptr, osd.rows, probes, kq[:n])
        return time.perf_counter() - t0, probes

    dt0, _ = run(sample_queries)
    n = int(min(nq, max(sample_queries, sample_queries * target_s / max(dt0, 1e-6))))
    dt, probes = run(n)
    pairs = sum(int(osd.ptr[p + 1].sum() - osd.ptr[p].sum()) for p in probes)
    return {"value": pairs / dt, "unit": "candidates/s", "cores": os.cpu_count(),
            "kind": "oracle", "qps": n / dt,
            "sample": f"the first {n} queries of the workload (FP64 probe + FP64 brute force "
                      f"over their candidate sets; the FP64 list assignment to the library's "
                      f"centroids, {osd.assign_s:.0f} s, untimed)",
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
    dev = "cuda" if torch.cuda.is_available() else "cpu"  # input draws only
    w = synth.generate(s, device=dev)
    X, Q = w.X.cpu().numpy(), w.Q.cpu().numpy()
    del w.X
    npq, kq = w.nprobe.numpy(), w.k.numpy()
    g = np.random.default_rng(3000 + s.cfg)
    C = X[np.sort(g.choice(len(X), s.nlist, replace=False))].astype(np.float32)
    osd = OracleSide(X, Q, C)
    import oracle
    per_step = 24

    def step(i):
        o = (i * per_step) % len(Q)
        qs = osd.Q[o:][:per_step]
        probes, _ = oracle.probe(qs, osd.C, npq[o:][:len(qs)])
        oracle.ivf_topk(osd.X, qs, osd.ptr, osd.rows, probes, kq[o:][:len(qs)])
        return sum(int(osd.ptr[p + 1].sum() - osd.ptr[p].sum()) for p in probes)

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
                       "step": f"{per_step} queries (bounded sample of the workload); coarse "
                               f"centroids = {s.nlist} seeded data rows, FP64 assignment "
                               f"({osd.assign_s:.0f} s, untimed)"},
            "qps": per_step * args.steps / dt,
            "cpu_baseline": {"value": v, "unit": "candidates/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{per_step} queries per step, FP64 brute force"},
            "e2e": {"value": v, "unit": "candidates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU side
class Timer:
    """Timed steps on the search stream: W untimed warm-up steps, then K
    steps each bracketed by CUDA events, a 256 MB buffer written before each
    (L2 flushed), the max over ranks of the total."""

    def __init__(self, dev, world, stream):
        import torch
        self.dev, self.world, self.stream = dev, world, stream
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run(self, fn, steps, warmup, clocks=False, after=None):
        import torch
        import torch.distributed as dist
        for _ in range(warmup):
            fn()
        if self.world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = Clocks(self.dev.index or 0) if clocks else None
        if clk:
            clk.start()
        total, extra = 0.0, []
        for _ in range(steps):
            self.flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if after:
                extra.append(after())
        torch.cuda.synchronize()
        c = clk.stop() if clk else None
        t = torch.tensor([total], device=self.dev)
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item() / steps, extra, c


def e2e_time(idx, Q, npa, ka, k, steps, timer, test_every=0):
    """Per-step time of the public API call with HOST buffers: pinned H2D of
    the queries (and per-query nprobe / k), search, D2H of ids and
    distances, all inside the events."""
    import torch
    nq = Q.shape[0]
    qh = Q.cpu().pin_memory()
    par = [(x.cpu().pin_memory(), torch.empty_like(x)) for x in (npa, ka)
           if isinstance(x, torch.Tensor)]
    if par:
        npa = par[0][1] if isinstance(npa, torch.Tensor) else npa
        ka = par[-1][1] if isinstance(ka, torch.Tensor) else ka
    ids_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    d_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    qd = torch.empty_like(Q)

    def step():
        qd.copy_(qh, non_blocking=True)
        for h, dv in par:
            dv.copy_(h, non_blocking=True)
        a, b = idx.search(qd, npa, ka, k_max=k, test_every=test_every)
        ids_h.copy_(a, non_blocking=True)
        d_h.copy_(b, non_blocking=True)

    ms, _, _ = timer.run(step, steps, 2)
    return ms, Q.numel() * 4 + sum(h.numel() * 4 for h, _ in par), nq * k * 12


def search_launches(pano, st, nlist):
    """Kernels one search launches: prep, transform GEMM, query norms, probe
    GEMM + select (IVF), four inversion kernels (emit twice), the threshold
    seeds, verify phase A (two-phase searches only), verify phase B, decode."""
    one_pass = st["pairs_a"] == 0
    return 14 - (2 if nlist <= 1 else 0) - (1 if one_pass else 0)


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
    stream = torch.cuda.current_stream()
    timer = Timer(dev, world, stream)
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    check_oracle = rank == 0 and world == 1

    s = workload_spec(args)
    # every rank holds a replica of the index and verifies its own query batch
    w = synth.generate(s, device=dev)
    if rank > 0:
        sq = dataclasses.replace(s, cfg=s.cfg + 100 * rank)
        w.Q = synth.generate(sq, device=dev, queries_only=True).Q
    X, Q = w.X, w.Q
    nq = Q.shape[0]
    t = pano.panorama_fit_transform(X[:65536], n_levels=s.n_levels)
    prec = {"fp32": pano.PANO_FP32, "bf16": pano.PANO_BF16, "fp8": pano.PANO_FP8}[s.precision]
    per_query = not isinstance(s.nprobe, int) or not isinstance(s.k, int)
    npa = w.nprobe.to(dev) if not isinstance(s.nprobe, int) else s.nprobe
    ka = w.k.to(dev) if not isinstance(s.k, int) else s.k
    k = int(w.k.max()) if not isinstance(s.k, int) else s.k  # k_max
    npmax = int(w.nprobe.max())
    widths, tune = None, None
    # the bound-test schedule: the library's default for the storage format
    # (FP32 every level as Algorithm 1; BF16 / FP8 every 4th level and nearly
    # dead chunks at every level) unless tuned
    test_every = 0
    if per_query:
        # storage precision and level split chosen by the autotuner: median
        # search time of each (precision, split) pair on a query sample,
        # splits generated per format (uniform and front-loaded), k-means once
        qs = Q[:min(len(Q), 8192)]
        names = {pano.PANO_FP32: "fp32", pano.PANO_BF16: "bf16", pano.PANO_FP8: "fp8"}
        t0 = time.time()
        best, trials = pano.panorama_autotune(
            t, X, qs, s.nlist, 64, 10,
            precisions=(pano.PANO_FP32, pano.PANO_BF16, pano.PANO_FP8), repeats=2)
        widths, prec = trials[best]["widths"], trials[best]["precision"]
        test_every = max(1, trials[best]["test_every"])
        s = dataclasses.replace(s, precision=names[prec], n_levels=len(widths))
        tune = {"trials": [{"precision": names[tr["precision"]], "widths": tr["widths"],
                            "ms": tr["ms"] if math.isfinite(tr["ms"]) else None,
                            "test_every": tr["test_every"]}
                           for tr in trials],
                "chosen": {"precision": names[prec], "widths": widths,
                           "test_every": test_every},
                "sample": f"{len(qs)} queries, nprobe 64, k 10", "seconds": time.time() - t0}
    b0 = time.time()
    idx = pano.panorama_build_ivf(t, X, nlist=s.nlist, n_levels=s.n_levels, seed=3000 + s.cfg,
                                  precision=prec, level_widths=widths)
    torch.cuda.synchronize()
    build_s = time.time() - b0
    C = idx.centroids()
    sizes = np.bincount(idx.assignment(), minlength=s.nlist)
    list_cv = float(sizes.std() / sizes.mean())  # balance of the k-means lists
    plan = pano.Plan(idx, Q, npa, ka, k_max=k, test_every=test_every) if per_query else None

    # counters (one instrumented search, outside the timed region)
    out = idx.search(Q, npa, ka, k_max=k, test_every=test_every)
    idx.search(Q, npa, ka, k_max=k, collect_stats=True, test_every=test_every)
    st = pano.last_stats().as_dict()
    pairs = st["pairs"]

    # the headline: pruned search of the whole batch, timed with the
    # library's stage events on the search stream
    def headline():
        if plan is not None:
            return plan.launch(stream)
        return idx.search(Q, npa, ka, k_max=k, collect_timing=True, test_every=test_every)

    stage_of = (lambda: list(pano.last_stats().stage_ms)) if plan is None else None
    ms_per_step, stages, clocks = timer.run(headline, args.steps, args.warmup, clocks=True,
                                           after=stage_of)
    if plan is not None:  # stage times from separate, instrumented searches
        _, stages, _ = timer.run(lambda: idx.search(Q, npa, ka, k_max=k, collect_timing=True,
                                                    test_every=test_every),
                                 3, 1, after=lambda: list(pano.last_stats().stage_ms))
    stage = {n: float(np.median([v[i] for v in stages])) for i, n in
             enumerate(("transform", "probe", "inversion", "verify_a", "verify_b", "decode"))}
    value = pairs * world / (ms_per_step / 1e3)
    qps = nq * world / (ms_per_step / 1e3)

    # comparator on the same index: the plain scan (no pruning test before
    # the last level; for BF16/FP8 storage the plain tensor-core scan)
    scan_ms, _, _ = timer.run(lambda: idx.search(Q, npa, ka, k_max=k, mode=1),
                              args.scan_steps, 1)
    # the bound-test schedule (which levels test Eq. 3): every level as in
    # Algorithm 1, every other, every fourth, the first and last levels only
    # (the tensor-core formats also test nearly dead chunks at every level)
    schedule_sweep = None
    if not per_query and not args.no_eps:
        schedule_sweep = []
        for te in sorted({1, 2, 4, s.n_levels}):
            mst, _, _ = timer.run(lambda: idx.search(Q, npa, ka, k_max=k, test_every=te),
                                  max(3, args.scan_steps), 1)
            idx.search(Q, npa, ka, k_max=k, test_every=te, collect_stats=True)
            sts = pano.last_stats().as_dict()
            schedule_sweep.append({"test_every": te, "ms_per_step": mst,
                                   "qps": nq * world / (mst / 1e3),
                                   "tile_levels": sts["tile_levels"],
                                   "dims_scanned_frac": sts["dims_scanned"] / max(1, pairs * s.d),
                                   "reranked": sts["reranked"]})
    e2e = None
    if not args.no_e2e:
        e2e_ms, h2d, d2h = e2e_time(idx, Q, npa, ka, k, args.steps, timer, test_every)
        e2e = {"value": pairs * world / (e2e_ms / 1e3), "unit": "candidates/s",
               "qps": nq * world / (e2e_ms / 1e3), "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # the oracle side (rank 0 of a 1-GPU run): FP64 assignment to the
    # library's centroids, then a sampled full-size parity check of every
    # storage format and the timed CPU baseline
    osd = None
    if check_oracle and (not args.no_parity or not args.no_cpu_baseline) and s.nlist > 1:
        osd = OracleSide(X.cpu().numpy(), Q.cpu().numpy(), C)
    prow = None
    if osd is not None and not args.no_parity:
        g = np.random.default_rng(9000 + s.cfg)
        prow = np.sort(g.choice(nq, min(nq, args.parity_queries), replace=False))
    lib_assign = idx.assignment() if osd is not None else None
    npq_host = w.nprobe.numpy()
    kq_host = w.k.numpy()

    def parity_of(ix, ids, dists):
        if prow is None:
            return None
        gp = pano.panorama_probe(ix, Q[torch.from_numpy(prow).to(dev)], npmax).cpu().numpy()
        return parity_report(osd, prow, npq_host[prow], kq_host[prow], ids.cpu().numpy()[prow],
                             dists.cpu().numpy()[prow], gp, lib_assign)

    parity = parity_of(idx, *out)
    del out
    eps_sweep = None
    if not args.no_eps and plan is None:
        ref_ids = osd.answer(prow, npq_host[prow], kq_host[prow])[0] if prow is not None else None
        eps_sweep = epsilon_sweep(idx, Q, npa, ka, k, s.d, timer, max(3, args.scan_steps),
                                  ref_ids, prow)

    # roofline of the dominant kernel: verify phase B (one launch per
    # search), its device time from the stage events of the timed steps
    vb = stage["verify_b"]
    va = stage["verify_a"]
    dims_b = st["dims_scanned"] - st["dims_scanned_a"]
    if s.precision == "fp32":
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA pipes
        flops_b = 2.0 * dims_b  # algorithmic: one FMA per coordinate an alive pair reads
        roof = {"bound": "alu", "kernel": "verify_fp32_kernel (phase B)",
                "achieved": flops_b / (vb / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops_b / (vb / 1e3) / 1e12 / peak,
                "traffic": TRAFFIC.get(workload_name(s)),
                "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                               f"(max clock of MEASURED_PEAKS.json, {pk_kind})",
                "flops_per_launch": flops_b, "ms_per_launch": vb,
                "phase_a": {"ms": va, "flops": 2.0 * st["dims_scanned_a"]}}
    else:
        hbm = float(pk.get("hbm_gbs", FALLBACK_HBM_GBS))
        live_b = st["live_row_bytes"]  # algorithmic: live rows x (w b + 4) per chunk-level
        ach = live_b / (vb / 1e3) / 1e9
        eb = 2 if s.precision == "bf16" else 1
        flops_tc = 2.0 * dims_b * (2 if eb == 2 else 3)  # live pairs, hi+lo (BF16) / 3 terms (FP8)
        tpk = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", FALLBACK_BF16_TFS)))
        roof = {"bound": "hbm", "kernel": f"verify_tc_kernel<{'FP8' if eb == 1 else 'BF16'}> "
                                          f"(phase B)",
                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": TRAFFIC.get(workload_name(s)),
                "peak_source": f"STREAM-style copy of MEASURED_PEAKS.json ({pk_kind})",
                "bytes_per_launch": live_b,
                "bytes_definition": "per (query group, chunk, level): candidates live for at "
                                    "least one query of the group x (level width x bytes per "
                                    "element + 4-byte tail norm)",
                "ms_per_launch": vb,
                "staged_bytes_per_launch": st["slice_bytes"],
                "staged_GBps": st["slice_bytes"] / (vb / 1e3) / 1e9,
                "tensor": {"achieved_tflops": flops_tc / (vb / 1e3) / 1e12,
                           "peak_tflops": tpk, "frac": flops_tc / (vb / 1e3) / 1e12 / tpk,
                           "note": "MMA flops on live (pair, level) coordinates; dense bf16 "
                                   "sustained peak"}}

    def search_line(ix, precision_name, with_scan=True, eps_runs=False):
        """Timed pruned search (and plain scan) of another index of the same
        data and queries, its counters and its parity sample."""
        o = ix.search(Q, npa, ka, k_max=k)
        msx, _, _ = timer.run(lambda: ix.search(Q, npa, ka, k_max=k), args.steps, args.warmup)
        ix.search(Q, npa, ka, k_max=k, collect_stats=True)
        stx = pano.last_stats().as_dict()
        line = {"storage": precision_name, "ms_per_step": msx,
                "value": stx["pairs"] * world / (msx / 1e3), "qps": nq * world / (msx / 1e3),
                "dims_scanned_frac": stx["dims_scanned"] / max(1, stx["pairs"] * s.d),
                "reranked": stx["reranked"], "index_gb": ix.info().device_bytes / 1e9}
        if with_scan:
            scx, _, _ = timer.run(lambda: ix.search(Q, npa, ka, k_max=k, mode=1),
                                  args.scan_steps, 1)
            line["plain_scan"] = {"ms_per_step": scx, "qps": nq * world / (scx / 1e3),
                                  "value": stx["pairs"] * world / (scx / 1e3),
                                  "speedup_of_pruned": scx / msx}
        line["parity"] = parity_of(ix, *o)
        return line

    def other_storage(precision, name):
        """The same data, centroids, levels and queries in another storage
        format (a split the format cannot take is reported, not fatal)."""
        try:
            ixo = pano.panorama_build_ivf(t, X, nlist=s.nlist, level_widths=widths or
                                          [s.d // s.n_levels] * s.n_levels,
                                          precision=precision, centroids=C)
        except pano.LibraryError as ex:
            return {"storage": name, "unavailable": str(ex)}
        line_ = search_line(ixo, name)
        del ixo
        return line_

    fp8 = fp32 = None
    if s.precision == "bf16" and not args.no_fp8 and s.d % 64 == 0:
        fp8 = other_storage(pano.PANO_FP8, "fp8")
    if s.precision != "fp32" and not args.no_fp32:
        fp32 = other_storage(pano.PANO_FP32, "fp32")

    # the serving workload: Poisson arrivals through the continuous-batching
    # server (batches of up to 1024 formed from what has arrived, several in
    # flight, admission by memory); QPS and latency percentiles per rate
    serving = None
    if "serving" in s.name and not args.no_serve:
        n_req = args.serve_requests
        sq = dataclasses.replace(s, n_queries=n_req, cfg=s.cfg + 50)
        wq = synth.generate(sq, device="cpu", queries_only=True)
        srv = pano.Server(idx, max_batch=1024, max_inflight=4, k_max=10)
        rng = np.random.default_rng(6000 + s.cfg)
        serving = []
        for rate in (20_000, 50_000, 100_000, 200_000):
            arr = np.cumsum(rng.exponential(1e6 / rate, size=n_req))
            b0_ = srv.stats()
            _, _, lat = srv.run_trace(wq.Q.numpy(), arr, wq.nprobe.numpy(), wq.k.numpy())
            b1 = srv.stats()
            nb = b1["batches"] - b0_["batches"]
            nbq = b1["mean_batch"] * b1["batches"] - b0_["mean_batch"] * b0_["batches"]
            span_us = float(np.max(arr + lat) - arr[0])
            serving.append({"offered_qps": rate, "qps": n_req / (span_us / 1e6),
                            "p50_us": float(np.percentile(lat, 50)),
                            "p99_us": float(np.percentile(lat, 99)),
                            "max_us": float(lat.max()),
                            "mean_batch": nbq / max(nb, 1), "requests": n_req})
        srv.close()

    cpu = None
    if osd is not None and not args.no_cpu_baseline:
        cpu = cpu_baseline(osd, npq_host, kq_host)
    launches = search_launches(pano, st, s.nlist) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if s.precision == "fp32" else s.precision, "data": "synthetic",
        "config": {"workload": workload_name(s) + (
                       f" (precision and levels autotuned: {tune['chosen']})" if tune else ""),
                   "l2": "index larger than L2, and a 256 MB buffer written between timed "
                         "steps (L2 flushed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "qps": qps,
        "plain_scan": {"storage": s.precision, "what": "plain tensor-core scan of the same "
                       "index" if s.precision != "fp32" else "plain FP32 full-distance scan",
                       "value": pairs * world / (scan_ms / 1e3),
                       "qps": nq * world / (scan_ms / 1e3), "ms_per_step": scan_ms,
                       "speedup_of_pruned": scan_ms / ms_per_step},
        "e2e": e2e,
        "parity": parity,
        "epsilon_sweep": eps_sweep,
        "test_schedule_sweep": schedule_sweep,
        "test_every": test_every if test_every > 0 else (1 if s.precision == "fp32" else 4),
        "fp8_pruned": fp8,
        "fp32": fp32,
        "speedup_vs_plain_fp32_scan": (fp32["plain_scan"]["ms_per_step"] / ms_per_step
                                       if fp32 and "plain_scan" in fp32 else None),
        "autotune": tune,
        "serving": serving,
        "gpu_launches": launches,
        "roofline": roof,
        "stage_ms": stage,
        "search_stats": {kk: st[kk] for kk in ("pairs", "pair_levels", "dims_scanned",
                                                 "dims_scanned_a", "tile_levels",
                                                 "slice_bytes", "live_row_bytes", "reranked",
                                                 "work_items")},
        "dims_scanned_frac": st["dims_scanned"] / max(1, pairs * s.d),
        "candidates_per_query": pairs / nq,
        "list_size_cv": list_cv,
        "build_s": build_s,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    del plan, idx, osd
    del X, Q, w
    torch.cuda.empty_cache()

    if s.cfg != 2 and not args.no_secondary:
        line["secondary"] = secondary(args, timer, dev, world, check_oracle, pk, pk_kind)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def epsilon_sweep(idx, Q, nprobe, k, k_max, d, timer, steps, ref_ids=None, prow=None):
    """Eq. 4 / Proposition 5.3: epsilon-relaxed pruning.  Per epsilon: time,
    coordinates read against the model E[cost_eps] / E[cost_1] = 1 + ln(eps)
    (valid for eps > 1/e), and recall@k against the oracle's exact top-k on
    the parity sample."""
    import numpy as np
    import paper_2510_00566_gb300 as pano
    nq = Q.shape[0]
    sweep, d1 = [], None
    for eps in EPSILONS:
        mse, _, _ = timer.run(lambda: idx.search(Q, nprobe, k, k_max=k_max, epsilon=eps),
                              steps, 1)
        ids_e, _ = idx.search(Q, nprobe, k, k_max=k_max, epsilon=eps, collect_stats=True)
        ste = pano.last_stats().as_dict()
        d1 = d1 or ste["dims_scanned"]
        row = {"epsilon": eps, "ms_per_step": mse, "qps": nq / (mse / 1e3),
               "dims_scanned_frac": ste["dims_scanned"] / max(1, ste["pairs"] * d),
               "dims_ratio_vs_exact": ste["dims_scanned"] / d1,
               "model_ratio_1_plus_ln_eps": 1.0 + math.log(eps)}
        if ref_ids is not None:
            got = ids_e.cpu().numpy()[prow]
            kq = np.broadcast_to(np.asarray(k if isinstance(k, int) else k.cpu().numpy()),
                                 (nq,))[prow]
            row["recall_at_k"] = float(np.mean(
                [len(set(got[i][:kq[i]]) & set(ref_ids[i][:kq[i]])) / max(1, kq[i])
                 for i in range(len(prow))]))
        sweep.append(row)
    return sweep


def secondary(args, timer, dev, world, check_oracle, pk, pk_kind):
    """The 960-d FP32 workload (N = 1M from a 1,024-cluster mixture, nlist
    1024, nprobe 32, 10k queries, 16 x 60 levels, k = 10): pruned FP32
    search, the plain FP32 scan, the FP32 verify roofline, a parity sample,
    the same data in BF16 storage against its plain tensor-core scan, the
    epsilon sweep of Eq. 4, point-centric refine and IVFPQ."""
    import numpy as np
    import torch
    import paper_2510_00566_gb300 as pano
    import synth
    s = synth.spec(2)
    rank = int(os.environ.get("RANK", "0"))
    w = synth.generate(s, device=dev)
    if rank > 0:
        w.Q = synth.generate(dataclasses.replace(s, cfg=s.cfg + 100 * rank), device=dev,
                             queries_only=True).Q
    X, Q = w.X, w.Q
    nq, k = Q.shape[0], s.k
    stream = timer.stream
    t = pano.panorama_fit_transform(X[:65536], n_levels=s.n_levels)
    idx = pano.panorama_build_ivf(t, X, nlist=s.nlist, n_levels=s.n_levels, seed=3002)
    C = idx.centroids()
    out = idx.search(Q, s.nprobe, k)
    idx.search(Q, s.nprobe, k, collect_stats=True)
    st = pano.last_stats().as_dict()
    pairs = st["pairs"]
    ms, stages, _ = timer.run(lambda: idx.search(Q, s.nprobe, k, collect_timing=True),
                              args.steps, args.warmup,
                              after=lambda: list(pano.last_stats().stage_ms))
    vb = float(np.median([v[4] for v in stages]))
    va = float(np.median([v[3] for v in stages]))
    scan_ms, _, _ = timer.run(lambda: idx.search(Q, s.nprobe, k, mode=1), args.scan_steps, 1)
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    flops_b = 2.0 * (st["dims_scanned"] - st["dims_scanned_a"])
    sizes = np.bincount(idx.assignment(), minlength=s.nlist)
    res = {"workload": workload_name(s), "ms_per_step": ms,
           "value": pairs * world / (ms / 1e3), "unit": "candidates/s",
           "qps": nq * world / (ms / 1e3),
           "candidates_per_query": pairs / nq,
           "list_size_cv": float(sizes.std() / sizes.mean()),
           "plain_scan": {"storage": "fp32", "ms_per_step": scan_ms,
                          "qps": nq * world / (scan_ms / 1e3), "speedup_of_pruned": scan_ms / ms},
           "roofline": {"bound": "alu", "kernel": "verify_fp32_kernel (phase B)",
                        "achieved": flops_b / (vb / 1e3) / 1e12, "peak": peak,
                        "unit": "TFLOP/s", "frac": flops_b / (vb / 1e3) / 1e12 / peak,
                        "traffic": TRAFFIC.get(workload_name(s)),
                        "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                                       f"({pk_kind} max clock)",
                        "ms_per_launch": vb, "phase_a_ms": va},
           "dims_scanned_frac": st["dims_scanned"] / max(1, pairs * s.d),
           "gpu_launches": search_launches(pano, st, s.nlist) * args.steps}
    osd = prow = None
    if check_oracle and not args.no_parity:
        osd = OracleSide(X.cpu().numpy(), Q.cpu().numpy(), C)
        g = np.random.default_rng(9002)
        prow = np.sort(g.choice(nq, min(nq, args.parity_queries), replace=False))
        gp = pano.panorama_probe(idx, Q[torch.from_numpy(prow).to(dev)], s.nprobe).cpu().numpy()
        res["parity"] = parity_report(osd, prow, s.nprobe, k, out[0].cpu().numpy()[prow],
                                      out[1].cpu().numpy()[prow], gp, idx.assignment())
    # the same data in BF16 storage (15 levels of 64, same transform basis and
    # centroids): pruned search and the plain tensor-core scan
    if not args.no_fp8:
        ixb = pano.panorama_build_ivf(t, X, nlist=s.nlist, level_widths=[64] * (s.d // 64),
                                      precision=pano.PANO_BF16, centroids=C)
        ob = ixb.search(Q, s.nprobe, k)
        msb, _, _ = timer.run(lambda: ixb.search(Q, s.nprobe, k), args.steps, args.warmup)
        scb, _, _ = timer.run(lambda: ixb.search(Q, s.nprobe, k, mode=1), args.scan_steps, 1)
        ixb.search(Q, s.nprobe, k, collect_stats=True)
        stb = pano.last_stats().as_dict()
        res["bf16_pruned"] = {
            "storage": "bf16", "levels": f"{s.d // 64}x64", "ms_per_step": msb,
            "qps": nq * world / (msb / 1e3), "value": stb["pairs"] * world / (msb / 1e3),
            "dims_scanned_frac": stb["dims_scanned"] / max(1, stb["pairs"] * s.d),
            "plain_tc_scan": {"ms_per_step": scb, "speedup_of_pruned": scb / msb},
            "speedup_vs_plain_fp32_scan": scan_ms / msb}
        if osd is not None:
            gp = pano.panorama_probe(ixb, Q[torch.from_numpy(prow).to(dev)], s.nprobe).cpu().numpy()
            res["bf16_pruned"]["parity"] = parity_report(
                osd, prow, s.nprobe, k, ob[0].cpu().numpy()[prow], ob[1].cpu().numpy()[prow], gp,
                ixb.assignment())
        del ixb, ob
    # Eq. 4 / Proposition 5.3: epsilon-relaxed pruning; recall@k against the
    # oracle's exact top-k on the parity sample, dims read against the model
    # E[cost_eps] / E[cost_1] = 1 + ln(eps) (valid for eps > 1/e)
    if not args.no_eps:
        ref_ids = osd.answer(prow, s.nprobe, k)[0] if osd is not None else None
        res["epsilon_sweep"] = epsilon_sweep(idx, Q, s.nprobe, k, k, s.d, timer,
                                             max(3, args.scan_steps), ref_ids, prow)
    # the refine workload (point-centric, B = 1): each query's top-1000 of the
    # pruned IVF search as its candidate-id list, refined to the top-k on a
    # flat index of the same data and levels
    if not args.no_refine:
        kprime = 1000
        cand, _ = idx.search(Q, s.nprobe, kprime, k_max=kprime)
        flat = pano.panorama_build_flat(t, X, level_widths=[s.d // s.n_levels] * s.n_levels)
        msr, _, _ = timer.run(lambda: flat.refine(Q, cand, k), args.steps, args.warmup)
        str_ = pano.last_stats().as_dict()
        res["refine"] = {"kprime": kprime, "k": k, "ms_per_step": msr,
                         "value": nq * kprime * world / (msr / 1e3), "unit": "candidates/s",
                         "qps": nq * world / (msr / 1e3),
                         "dims_scanned_frac": str_["dims_scanned"] / max(1, str_["pairs"] * s.d),
                         "reranked": str_["reranked"]}
        if osd is not None:
            rc = cand.cpu().numpy()[prow]
            import oracle
            ref_i, ref_d = oracle.candidate_topk(osd.X, osd.Q[prow], rc, k)
            ids_r, d_r = flat.refine(Q[torch.from_numpy(prow).to(dev)],
                                     cand[torch.from_numpy(prow).to(dev)], k)
            ids_r, d_r = ids_r.cpu().numpy(), d_r.cpu().numpy().astype(np.float64)
            ok = (ids_r == ref_i) | (np.abs(d_r - ref_d) <= 1e-6 * np.maximum(ref_d, 1e-30))
            fin = np.isfinite(ref_d)
            res["refine"]["parity"] = {
                "queries": len(prow), "id_mismatch_beyond_tie": int((~ok).sum()),
                "max_rel_err": float(np.max(np.abs(d_r[fin] - ref_d[fin]) / ref_d[fin]))}
        del flat, cand
    # IVFPQ (Section 6.3): the same data, lists and queries; the PCA basis
    # shaped for PQ (Section 4.3, kappa = 4, seeded Haar draws), M = d / 2
    # subquantisers of 8 bits, codebooks and codes trained by the library
    Lp = args.pq_levels or s.n_levels
    if not args.no_pq and s.d % Lp == 0 and (s.d // 2) % Lp == 0:
        gd = np.random.default_rng(7000 + s.cfg).standard_normal((2, s.d, s.d))
        b0 = time.time()
        tsh, blocks = pano.panorama_shape_transform(t, Lp, 4.0, gd)
        idxp = pano.panorama_build_ivfpq(tsh, X, s.nlist, s.d // 2, Lp,
                                         centroids=C, assign=idx.assignment())
        build_s = time.time() - b0
        msp, vm, _ = timer.run(lambda: idxp.search_pq(Q, s.nprobe, k, collect_timing=True),
                               args.steps, args.warmup,
                               after=lambda: pano.last_stats().stage_ms[4])
        vmsp = float(np.median(vm))
        msp_scan, _, _ = timer.run(lambda: idxp.search_pq(Q, s.nprobe, k, mode=1),
                                   args.scan_steps, 1)
        idxp.search_pq(Q, s.nprobe, k, collect_stats=True)
        stp = pano.last_stats().as_dict()
        look = stp["dims_scanned"] / 2
        lpk = 152 * 32 * sm_max * 1e6
        ref_ids, _ = idx.search(Q, s.nprobe, k)
        ref_ids = ref_ids.cpu().numpy()
        pq_ids = idxp.search_pq(Q, s.nprobe, k)[0].cpu().numpy()
        res["ivfpq"] = {
            "M": s.d // 2, "nbits": 8, "levels": f"{Lp}x{s.d // Lp}", "kappa": 4.0,
            "robin_hood_blocks": blocks, "ms_per_step": msp,
            "value": stp["pairs"] * world / (msp / 1e3), "unit": "candidates/s",
            "qps": nq * world / (msp / 1e3),
            "plain_pq_scan": {"ms_per_step": msp_scan, "qps": nq * world / (msp_scan / 1e3),
                              "speedup_of_pruned": msp_scan / msp},
            "dims_scanned_frac": stp["dims_scanned"] / max(1, stp["pairs"] * s.d),
            "recall_at_k_vs_exact_same_lists": float(np.mean(
                [len(set(pq_ids[i]) & set(ref_ids[i])) / k for i in range(nq)])),
            "roofline": {"bound": "lsu", "kernel": "pq_verify_kernel",
                         "achieved": look / (vmsp / 1e3), "peak": lpk, "unit": "lookups/s",
                         "frac": look / (vmsp / 1e3) / lpk, "traffic": PQ_TRAFFIC.get(s.name),
                         "ms_per_launch": vmsp},
            "index_gb": idxp.info().device_bytes / 1e9, "build_s": build_s}
        del idxp, tsh, gd
    del idx, osd
    return res


if __name__ == "__main__":
    main()
