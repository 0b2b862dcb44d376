"""Serving: continuous batching over a device-resident BF16 index (the
recipe of the 50M-vector serving workload, d = 128, 8 x 16 levels, at 60k
vectors, with coarse centroids from the seeded generator).  Every served
result is checked against the CPU oracle (the FP64 top-k over the query's
FP64 probe set; ids equal except at near-ties, distances within 1e-5
relative), and each request's result must also be the same alone and in the
mix; Poisson arrivals are batched; a tiny memory budget serialises batches
but still completes every request."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_00566_gb300 as pano
import synth
from parity import check_topk, gamma_of

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def serving_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()
    s = synth.scaled(5, n=60_000, n_queries=600, nlist=64)
    w = synth.generate(s)
    C = synth.initial_centroids(w.X, 64, seed=3005).numpy()
    t = pano.panorama_fit_transform(w.X.numpy(), n_levels=8)
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=64, level_widths=[16] * 8,
                                  precision=pano.PANO_BF16, centroids=C)
    npq = np.clip(w.nprobe.numpy(), 1, 64)
    lists, _ = oracle.assign(w.X.numpy(), C)
    return s, w, idx, npq, C, lists


def _check_oracle(w, C, lists, npq, rows, ids, dists, k=10):
    """The served results of queries `rows` against the oracle's FP64 top-k
    over each query's FP64 probe set (queries whose nprobe-th and next
    centroid distances are within 1e-6 are left out, as in every IVF
    parity test)."""
    X, Q = w.X.numpy(), w.Q.numpy()[rows]
    ref = oracle.ivf_search(X, Q, C, npq[rows], k, lists_of_vector=lists)
    keep = ref["probe_gap"] >= 1e-6
    assert keep.mean() > 0.9
    G = gamma_of(lists, [ref["probes"][i] for i in np.nonzero(keep)[0]])
    check_topk(X, Q[keep], np.asarray(ids)[keep], np.asarray(dists)[keep], ref["ids"][keep],
               ref["dists"][keep], k, gamma_rows=G)


def _alone(idx, q, nprobe, k=10):
    ids, d = idx.search(torch.from_numpy(q[None]).to(DEV), int(nprobe), k)
    return ids.cpu().numpy()[0], d.cpu().numpy()[0]


def _same(ia, da, ib, db):
    fin = np.isfinite(da)
    assert np.array_equal(fin, np.isfinite(db))
    assert np.all(np.abs(da[fin] - db[fin]) <= 1e-5 * np.abs(da[fin]))
    diff = ia != ib
    assert np.all(np.abs(da[diff] - db[diff]) <= 1e-6 * np.abs(da[diff]))


def test_results_match_oracle_and_alone_in_mix(serving_index):
    s, w, idx, npq, C, lists = serving_index
    Q = w.Q.numpy()
    srv = pano.Server(idx, max_batch=64, max_inflight=3, k_max=10)
    tickets = [srv.submit(Q[i], int(npq[i]), 10) for i in range(400)]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 400 and st["batches"] >= 400 / 64
    rows = np.arange(400)
    _check_oracle(w, C, lists, npq, rows, np.stack([g[0] for g in got]),
                  np.stack([g[1] for g in got]))
    for i in range(0, 400, 7):
        ia, da = _alone(idx, Q[i], npq[i])
        _same(ia, da, got[i][0], got[i][1])


def test_poisson_trace_batches_requests(serving_index):
    s, w, idx, npq, C, lists = serving_index
    Q = w.Q.numpy()
    n = 600
    rng = np.random.default_rng(5005)
    arrivals = np.cumsum(rng.exponential(1e6 / 50_000.0, size=n))  # 50k QPS
    srv = pano.Server(idx, max_batch=256, max_inflight=2, k_max=10)
    ids, d, lat = srv.run_trace(Q[:n], arrivals, npq[:n], 10)
    st = srv.stats()
    srv.close()
    assert st["completed"] == n
    assert st["mean_batch"] > 1.0  # arrivals during a batch were grouped
    assert np.all(lat > 0) and st["p99_us"] >= st["p50_us"] > 0
    _check_oracle(w, C, lists, npq, np.arange(n), ids, d)
    for i in range(0, n, 37):
        ia, da = _alone(idx, Q[i], npq[i])
        _same(ia, da, ids[i], d[i])


def test_memory_budget_admits_one_batch_at_a_time(serving_index):
    s, w, idx, npq, C, lists = serving_index
    Q = w.Q.numpy()
    srv = pano.Server(idx, max_batch=32, max_inflight=4, k_max=10, memory_budget=1)
    tickets = [srv.submit(Q[i], int(npq[i]), 10) for i in range(100)]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 100
    _check_oracle(w, C, lists, npq, np.arange(100), np.stack([g[0] for g in got]),
                  np.stack([g[1] for g in got]))
    ia, da = _alone(idx, Q[3], npq[3])
    _same(ia, da, got[3][0], got[3][1])
