"""Batching pieces: a search captured into a CUDA graph (plan) replays the
same results as the direct call, also after the bound query buffer is
refilled; the level-width autotuner times valid candidates and skips invalid
ones.  Workload: the recipe of the 5M-vector Zipf workload (d = 384, Zipf(1.1)
cluster sizes, per-query nprobe in [1, 128] and k in {1, 10, 100}) at 30k
vectors."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2510_00566_gb300 as pano
import synth
from parity import check_topk

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def zipf_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()
    s = synth.scaled(4, n=30_000, n_queries=256, nlist=64, n_clusters=64)
    w = synth.generate(s)
    t = pano.panorama_fit_transform(w.X.numpy(), n_levels=6)
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=64, level_widths=[64] * 6,
                                  precision=pano.PANO_BF16, kmeans_iters=8)
    return s, w, t, idx


def test_plan_replays_direct_search(zipf_index):
    s, w, t, idx = zipf_index
    npq = torch.clamp(w.nprobe, max=64).to(DEV)
    kq = w.k.to(DEV)
    q = w.Q.to(DEV).clone()
    plan = pano.Plan(idx, q, npq, kq, k_max=100)
    for round_ in range(2):
        ids, d = plan.launch()
        ref_ids, ref_d = idx.search(q, npq, kq, k_max=100)
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids) and torch.equal(d, ref_d)
        # the oracle agrees with the replayed result as well
        X, Qh = w.X.numpy(), q.cpu().numpy()
        C = idx.centroids()
        lists = idx.assignment().astype(np.int64)
        probes, pgap = oracle.probe(Qh, C, npq.cpu().numpy())
        ri, rd = oracle.ivf_topk(X, Qh, *oracle.ivf_lists(lists, 64), probes,
                                 kq.cpu().numpy())
        keep = [i for i in range(len(Qh)) if pgap[i] >= 1e-6][:64]
        for i in keep:
            check_topk(X, Qh[i:i + 1], ids.cpu().numpy()[i:i + 1], d.cpu().numpy()[i:i + 1],
                       ri[i:i + 1], rd[i:i + 1], int(kq[i]))
        # refill the bound buffer with other queries for the second replay
        q.copy_(torch.flip(w.Q, dims=[0]).to(DEV) * 1.01)


def test_autotune_levels_picks_a_valid_split(zipf_index):
    s, w, t, idx = zipf_index
    cands = [[64] * 6, [128] * 3, [32] * 12, [48] * 8]
    best, ms = pano.panorama_autotune_levels(t, w.X[:20_000].to(DEV), w.Q[:128].to(DEV),
                                             nlist=32, nprobe=8, k=10, candidates=cands,
                                             precision=pano.PANO_BF16, repeats=2)
    assert best in (0, 1, 2)
    assert all(math.isfinite(x) and x > 0 for x in ms[:3])
    assert math.isinf(ms[3])  # 48-wide bf16 levels are not a supported tile width
    assert ms[best] == min(ms)


def test_autotune_precision_and_generated_splits(zipf_index):
    """The precision x split tuner (generated candidates): every trial is a
    valid split of d for its storage format, the best is the fastest, and
    the configuration it picks returns the oracle's exact top-k."""
    s, w, t, idx = zipf_index
    X = w.X[:20_000]
    Qs = w.Q[:128].to(DEV)
    best, trials = pano.panorama_autotune(
        t, X.to(DEV), Qs, nlist=32, nprobe=8, k=10,
        precisions=(pano.PANO_FP32, pano.PANO_BF16, pano.PANO_FP8), repeats=2)
    assert len(trials) >= 6
    precs = {tr["precision"] for tr in trials}
    assert precs == {pano.PANO_FP32, pano.PANO_BF16, pano.PANO_FP8}
    ok_w = {pano.PANO_BF16: {16, 32, 64, 128}, pano.PANO_FP8: {32, 64, 128, 256}}
    for tr in trials:
        assert sum(tr["widths"]) == s.d
        if tr["precision"] in ok_w:
            assert set(tr["widths"]) <= ok_w[tr["precision"]]
    # uniform and front-loaded (non-uniform) splits were both tried
    assert any(len(set(tr["widths"])) > 1 for tr in trials)
    finite = [tr["ms"] for tr in trials if math.isfinite(tr["ms"])]
    assert trials[best]["ms"] == min(finite)
    # the chosen configuration, built on the same data, answers exactly
    bt = trials[best]
    C = synth.initial_centroids(X, 32, seed=3004).numpy()
    ix = pano.panorama_build_ivf(t, X.to(DEV), nlist=32, level_widths=bt["widths"],
                                 precision=bt["precision"], centroids=C)
    ids, d = ix.search(Qs, 8, 10)
    Xh, Qh = X.numpy(), Qs.cpu().numpy()
    lists, _ = oracle.assign(Xh, C)
    ref = oracle.ivf_search(Xh, Qh, C, 8, 10, lists_of_vector=lists)
    keep = ref["probe_gap"] >= 1e-6
    check_topk(Xh, Qh[keep], ids.cpu().numpy()[keep], d.cpu().numpy()[keep], ref["ids"][keep],
               ref["dists"][keep], 10)
