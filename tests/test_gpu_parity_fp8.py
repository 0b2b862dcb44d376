"""GPU parity of the FP8 tensor-core path: level slices stored in E4M3 with a
power-of-two scale per vector, partial products on tcgen05 (kind::f8f6f4)
with the query split into three E4M3 terms at one scale per group, margined
bounds, exact FP32 re-rank.  The answer must equal the oracle's exact top-k
(same tolerances as the FP32 path): quantisation only loosens the bounds."""
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


def _check(idx, X, Q, C, nprobe, k, mode=0):
    ids, d = idx.search(torch.from_numpy(Q).to(DEV), nprobe, k, mode=mode, collect_stats=True)
    st = pano.last_stats()
    assert st.device_error == 0
    lists, _ = oracle.assign(X, C)
    ref = oracle.ivf_search(X, Q, C, nprobe, k, lists_of_vector=lists)
    keep = ref["probe_gap"] >= 1e-6
    G = gamma_of(lists, ref["probes"])
    check_topk(X, Q[keep], ids.cpu().numpy()[keep], d.cpu().numpy()[keep], ref["ids"][keep],
               ref["dists"][keep], k, gamma_rows=[G[i] for i in np.nonzero(keep)[0]])
    return st


def _build(X, C, widths):
    t = pano.panorama_fit_transform(X, n_levels=len(widths))
    idx = pano.panorama_build_ivf(t, torch.from_numpy(X).to(DEV), nlist=C.shape[0],
                                  level_widths=widths, precision=pano.PANO_FP8, centroids=C)
    info = idx.info()
    assert info.precision == pano.PANO_FP8 and info.chunk == 128
    return idx


@pytest.mark.parametrize("mode", [0, 1])
def test_fp8_768d_single_gaussian(mode):
    """The 10M-vector workload's recipe (d = 768, decay 0.008, 12 x 64
    levels) at 30k vectors, 32 fixed lists, nprobe 4."""
    s = synth.scaled(3, n=30_000, n_queries=120, nlist=32)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 32, seed=3003).numpy()
    idx = _build(X, C, [64] * 12)
    st = _check(idx, X, Q, C, 4, 10, mode=mode)
    if mode == 1:
        assert st.dims_scanned == st.pairs * 768
        return
    # the bounds still prune (E4M3 loosens them by its quantisation error):
    # with the bound tested at every level, as the oracle's Algorithm 1
    idx.search(torch.from_numpy(Q).to(DEV), 4, 10, collect_stats=True, test_every=1)
    st = pano.last_stats()
    frac = st.dims_scanned / (st.pairs * 768)
    lists, _ = oracle.assign(X, C)
    ref = oracle_dims_fraction(X, Q[:20], C, lists, 4, [64] * 12, 10)
    assert frac <= 1.6 * ref + 0.05, (frac, ref)


def test_fp8_128d_narrow_levels_large_groups():
    """d = 128 with 32- and 64-wide levels (32- and 64-byte swizzled rows of
    E4M3) and 3 lists probed by all 200 queries (groups of 64 and a ragged 8)."""
    s = synth.scaled(5, n=12_000, n_queries=200, nlist=3)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 3, seed=3005).numpy()
    _check(_build(X, C, [32, 32, 64]), X, Q, C, 2, 10)
    _check(_build(X, C, [32] * 4), X, Q, C, 3, 25)


def test_fp8_960d_multi_panel_levels():
    """256-wide levels (two 128-byte panels per row) next to 128 and 64."""
    s = synth.scaled(2, n=20_000, n_queries=80, nlist=16, n_clusters=16)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 16, seed=3002).numpy()
    _check(_build(X, C, [256, 256, 256, 128, 64]), X, Q, C, 4, 10)


def test_fp8_384d_per_query_nprobe_k():
    s = synth.scaled(4, n=25_000, n_queries=150, nlist=40, n_clusters=40)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 40, seed=3004).numpy()
    idx = _build(X, C, [128] * 3)
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


def test_fp8_vector_and_query_scales_far_apart():
    """Vectors and queries whose magnitudes span 2^-20 .. 2^20 (per-vector
    and per-group power-of-two scales; small query elements fall below
    E4M3's normal range)."""
    s = synth.scaled(5, n=8_000, n_queries=100, nlist=4)
    w = synth.generate(s)
    g = np.random.default_rng(11)
    X = (w.X.numpy() * np.exp2(g.integers(-20, 21, size=(w.X.shape[0], 1)))).astype(np.float32)
    Q = (w.Q.numpy() * np.exp2(g.integers(-20, 21, size=(w.Q.shape[0], 1)))).astype(np.float32)
    C = synth.initial_centroids(torch.from_numpy(X), 4, seed=3006).numpy()
    _check(_build(X, C, [32] * 4), X, Q, C, 2, 10)


def test_fp8_save_load_roundtrip(tmp_path):
    s = synth.scaled(5, n=6_000, n_queries=30, nlist=4)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, 4, seed=3007).numpy()
    idx = _build(X, C, [64, 64])
    q = torch.from_numpy(Q).to(DEV)
    a_ids, a_d = idx.search(q, 2, 10)
    path = str(tmp_path / "fp8.pano")
    pano.panorama_save(idx, path)
    idx2 = pano.panorama_load(path)
    assert idx2.info().precision == pano.PANO_FP8
    b_ids, b_d = idx2.search(q, 2, 10)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)


def test_fp8_rejects_unsupported_widths():
    s = synth.scaled(5, n=2_000, n_queries=4, nlist=1)
    w = synth.generate(s)
    for widths in ([16] * 8, [96, 32], [48, 80]):
        t = pano.panorama_fit_transform(w.X.numpy(), n_levels=len(widths))
        with pytest.raises(pano.LibraryError):
            pano.panorama_build_ivf(t, w.X.to(DEV), nlist=1, level_widths=widths,
                                    precision=pano.PANO_FP8)
