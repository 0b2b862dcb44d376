"""GPU parity of the BF16 tensor-core path: level slices stored in bf16,
partial products on tcgen05 with bf16 hi/lo query splits, margined bounds,
exact FP32 re-rank.  The answer must equal the oracle's exact top-k (same
tolerances as the FP32 path) -- quantisation only loosens the bounds."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_00566_gb300 as pano
import synth
from parity import check_topk, gamma_of, oracle_dims_fraction

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()


def _ivf(s, C, widths, nprobe, k, mode=0, Qn=None):
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    t = pano.panorama_fit_transform(X, n_levels=len(widths))
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=C.shape[0], level_widths=widths,
                                  precision=pano.PANO_BF16, centroids=C)
    assert idx.info().precision == pano.PANO_BF16 and idx.info().chunk == 128
    ids, d = idx.search(torch.from_numpy(Q).to(DEV), nprobe, k, mode=mode,
                        collect_stats=True)
    st = pano.last_stats()
    lists, _ = oracle.assign(X, C)
    ref = oracle.ivf_search(X, Q, C, nprobe, k, lists_of_vector=lists)
    keep = ref["probe_gap"] >= 1e-6
    G = gamma_of(lists, ref["probes"])
    check_topk(X, Q[keep], ids.cpu().numpy()[keep], d.cpu().numpy()[keep], ref["ids"][keep],
               ref["dists"][keep], k, gamma_rows=[G[i] for i in np.nonzero(keep)[0]])
    return st, idx, X, Q


@pytest.mark.parametrize("mode", [0, 1])
def test_bf16_768d_single_gaussian(mode):
    """The 10M-vector workload's recipe (d = 768, decay 0.008, 12 x 64
    levels) at 30k vectors, 32 fixed lists, nprobe 4."""
    s = synth.scaled(3, n=30_000, n_queries=120, nlist=32)
    w = synth.generate(s)
    C = synth.initial_centroids(w.X, 32, seed=3003).numpy()
    st, idx, X, Q = _ivf(s, C, [64] * 12, nprobe=4, k=10, mode=mode)
    assert st.device_error == 0
    if mode == 1:
        assert st.dims_scanned == st.pairs * 768
        return
    # pruning at least about as effective as the oracle's Algorithm 1 (the
    # bound tested at every level, as there)
    idx.search(torch.from_numpy(Q[:20]).to(DEV), 4, 10, collect_stats=True, test_every=1)
    st = pano.last_stats()
    frac = st.dims_scanned / (st.pairs * 768)
    lists, _ = oracle.assign(X, C)
    ref = oracle_dims_fraction(X, Q[:20], C, lists, 4, [64] * 12, 10)
    assert frac <= 1.2 * ref + 0.02, (frac, ref)


def test_bf16_128d_narrow_levels_large_groups():
    """d = 128 with 16- and 32-wide levels (32- and 64-byte swizzled rows)
    and 3 lists probed by all 200 queries (groups of 64 and a ragged 8)."""
    s = synth.scaled(5, n=12_000, n_queries=200, nlist=3)
    w = synth.generate(s)
    C = synth.initial_centroids(w.X, 3, seed=3005).numpy()
    _ivf(s, C, [16, 16, 32, 64], nprobe=2, k=10)
    _ivf(s, C, [16] * 8, nprobe=3, k=25)


def test_bf16_384d_per_query_nprobe_k():
    s = synth.scaled(4, n=25_000, n_queries=150, nlist=40, n_clusters=40)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 40, seed=3004).numpy()
    t = pano.panorama_fit_transform(X, n_levels=6)
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=40, level_widths=[64] * 6,
                                  precision=pano.PANO_BF16, centroids=C)
    g = np.random.default_rng(4)
    npq = g.integers(1, 17, size=len(Q)).astype(np.int32)
    kq = g.choice([1, 10, 100], size=len(Q)).astype(np.int32)
    ids, d = idx.search(torch.from_numpy(Q).to(DEV), torch.from_numpy(npq).to(DEV),
                        torch.from_numpy(kq).to(DEV), k_max=100)
    lists, _ = oracle.assign(X, C)
    probes, pgap = oracle.probe(Q, C, npq)
    ref_i, ref_d = oracle.ivf_topk(X, Q, *oracle.ivf_lists(lists, 40), probes, kq)
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    for i in range(len(Q)):
        if pgap[i] >= 1e-6:
            check_topk(X, Q[i:i + 1], ids[i:i + 1], d[i:i + 1], ref_i[i:i + 1],
                       ref_d[i:i + 1], int(kq[i]))


def test_bf16_rejects_unsupported_widths():
    s = synth.scaled(5, n=2_000, n_queries=4, nlist=1)
    w = synth.generate(s)
    t = pano.panorama_fit_transform(w.X.numpy(), n_levels=2)
    with pytest.raises(pano.LibraryError):
        pano.panorama_build_ivf(t, w.X.to(DEV), nlist=1, level_widths=[48, 80],
                                precision=pano.PANO_BF16)


@pytest.mark.parametrize("precision", [pano.PANO_BF16, pano.PANO_FP32])
def test_test_schedule_keeps_the_exact_answer(precision):
    """The bound-test schedule (test_every: which levels test Eq. 3, the last
    always; 0 = the format's default) changes the work, never the answer:
    every schedule returns the oracle's exact top-k, the same ids and
    distances bit for bit, and none reads more coordinates than the plain
    scan (the test at the last level only)."""
    s = synth.scaled(3, n=20_000, n_queries=80, nlist=16)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 16, seed=3013).numpy()
    t = pano.panorama_fit_transform(X, n_levels=12)
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=16, level_widths=[64] * 12,
                                  precision=precision, centroids=C)
    q = torch.from_numpy(Q).to(DEV)
    lists, _ = oracle.assign(X, C)
    ref = oracle.ivf_search(X, Q, C, 4, 10, lists_of_vector=lists)
    keep = ref["probe_gap"] >= 1e-6
    G = gamma_of(lists, ref["probes"])
    first = None
    dims = []
    for te in (1, 2, 5, 12, 100, 0):
        ids, d = idx.search(q, 4, 10, test_every=te, collect_stats=True)
        dims.append(pano.last_stats().dims_scanned)
        ids, d = ids.cpu().numpy(), d.cpu().numpy()
        check_topk(X, Q[keep], ids[keep], d[keep], ref["ids"][keep], ref["dists"][keep], 10,
                   gamma_rows=[G[i] for i in np.nonzero(keep)[0]])
        if first is None:
            first = (ids, d)
        else:
            assert np.array_equal(first[0], ids) and np.array_equal(first[1], d), te
    # the plain scan reads every coordinate of every pair; no schedule reads
    # more, and testing every level reads less (how much less depends on the
    # thresholds of the moment, which the order of the work items decides)
    idx.search(q, 4, 10, mode=1, collect_stats=True)
    st = pano.last_stats()
    assert st.dims_scanned == st.pairs * 768
    assert all(x <= st.dims_scanned for x in dims), (dims, st.dims_scanned)
    assert dims[0] < st.dims_scanned
