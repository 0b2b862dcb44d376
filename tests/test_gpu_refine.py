"""GPU parity of point-centric refinement (the paper's no-batch variant,
IndexRefinePanorama over an IndexFlatPanorama): each query's own candidate-id
list is refined level by level and re-ranked exactly.  The answer must equal
the FP64 top-k over the candidate set (ties by id, -1 ignored, repeats kept
once); the coordinates read follow the oracle's Algorithm 1 with the same
batching (the first k candidates seed the threshold, then batches of 256)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_00566_gb300 as pano
import synth
from parity import check_topk

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()


def _candidates(X, Q, kp, n_true, seed):
    """n_true exact nearest ids plus random ids, shuffled (a coarse index's
    top-k' stand-in)."""
    g = np.random.default_rng(seed)
    out = np.empty((len(Q), kp), np.int64)
    for i, q in enumerate(Q):
        d = ((X.astype(np.float64) - q) ** 2).sum(1)
        near = np.argsort(d, kind="stable")[:n_true]
        rest = g.choice(np.setdiff1d(np.arange(len(X)), near), kp - n_true, replace=False)
        row = np.concatenate([near, rest])
        g.shuffle(row)
        out[i] = row
    return out


def _check(X, Q, cand, k, got_i, got_d):
    ref_i, ref_d = oracle.candidate_topk(X, Q, cand, k)
    gam = [np.unique(c[c >= 0]) for c in cand]
    check_topk(X, Q, got_i.cpu().numpy(), got_d.cpu().numpy(), ref_i, ref_d, k,
               gamma_rows=gam)


def test_refine_960d_matches_fp64_and_prunes_like_algorithm1():
    s = synth.scaled(2, n=20_000, n_queries=64, nlist=16, n_clusters=16)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    widths = [60] * 16
    t = pano.panorama_fit_transform(X, n_levels=16)
    idx = pano.panorama_build_flat(t, w.X.to(DEV), level_widths=widths)
    cand = _candidates(X, Q, 400, 40, seed=1)
    ids, d = idx.refine(torch.from_numpy(Q).to(DEV), torch.from_numpy(cand).to(DEV), 10)
    st = pano.last_stats()
    _check(X, Q, cand, 10, ids, d)
    assert st.pairs == cand.size and st.reranked >= 10 * len(Q)
    # coordinates read vs the oracle's Algorithm 1 (FP64 bounds, same batches)
    mu, T, _ = oracle.pca_fit(X[:65536])
    m = oracle.level_thresholds(960, widths)
    tX = oracle.transform(T, mu, X)
    tQ = oracle.transform(T, mu, Q)
    rho = 0
    for i in range(len(Q)):
        _, _, r = oracle.refine(tQ[i], tX[cand[i]], cand[i], m, 10, B=256)
        rho += r.sum()
    assert st.dims_scanned <= 1.2 * rho + 0.02 * cand.size * 960, (st.dims_scanned, rho)
    # seeded by the best first-level candidates, most others stop early
    assert st.dims_scanned < 0.5 * cand.size * 960, st.dims_scanned / (cand.size * 960)


def test_refine_padding_repeats_and_short_lists():
    s = synth.scaled(5, n=5_000, n_queries=40, nlist=1)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    t = pano.panorama_fit_transform(X, n_levels=4)
    idx = pano.panorama_build_flat(t, w.X.to(DEV), level_widths=[32] * 4)
    g = np.random.default_rng(5)
    cand = g.integers(0, len(X), size=(len(Q), 300))
    cand[:, 150:200] = cand[:, :50]           # repeats
    cand[g.random(cand.shape) < 0.2] = -1     # padding
    cand[3, :] = -1                           # no candidate at all
    cand[4, 5:] = -1                          # fewer than k
    for k in (1, 10, 100):
        ids, d = idx.refine(torch.from_numpy(Q).to(DEV), torch.from_numpy(cand).to(DEV), k)
        _check(X, Q, cand, k, ids, d)
    ids, d = idx.refine(torch.from_numpy(Q).to(DEV),
                        torch.empty((len(Q), 0), dtype=torch.int64, device=DEV), 5)
    assert torch.all(ids == -1) and torch.all(torch.isinf(d))


def test_refine_unaligned_dimension():
    """d = 130 (no float4 rows) with uneven levels."""
    g = np.random.default_rng(9)
    X = (g.standard_normal((3_000, 130)) * np.exp(-0.03 * np.arange(130))).astype(np.float32)
    Q = (g.standard_normal((30, 130)) * np.exp(-0.03 * np.arange(130))).astype(np.float32)
    t = pano.panorama_fit_transform(X, n_levels=3)
    idx = pano.panorama_build_flat(t, torch.from_numpy(X).to(DEV), level_widths=[10, 40, 80])
    cand = _candidates(X, Q, 120, 15, seed=2)
    ids, d = idx.refine(torch.from_numpy(Q).to(DEV), torch.from_numpy(cand).to(DEV), 7)
    _check(X, Q, cand, 7, ids, d)


def test_refine_epsilon_relaxed_keeps_exact_distances():
    s = synth.scaled(2, n=8_000, n_queries=32, nlist=8, n_clusters=8)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    t = pano.panorama_fit_transform(X, n_levels=16)
    idx = pano.panorama_build_flat(t, w.X.to(DEV), level_widths=[60] * 16)
    cand = _candidates(X, Q, 300, 30, seed=3)
    qd, cd = torch.from_numpy(Q).to(DEV), torch.from_numpy(cand).to(DEV)
    idx.refine(qd, cd, 10)
    dims1 = pano.last_stats().dims_scanned
    ids, d = idx.refine(qd, cd, 10, epsilon=0.5)
    dims_e = pano.last_stats().dims_scanned
    assert dims_e <= dims1
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    ref_i, _ = oracle.candidate_topk(X, Q, cand, 10)
    recall = np.mean([len(set(ids[i]) & set(ref_i[i])) / 10 for i in range(len(Q))])
    assert recall >= 0.5
    for i in range(len(Q)):  # whatever is returned carries its exact distance
        v = ids[i] >= 0
        ex = ((X[ids[i][v]].astype(np.float64) - Q[i]) ** 2).sum(1)
        assert np.allclose(d[i][v], ex, rtol=1e-5)


def test_refine_save_load_and_argument_errors(tmp_path):
    s = synth.scaled(5, n=3_000, n_queries=8, nlist=1)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    t = pano.panorama_fit_transform(X, n_levels=2)
    idx = pano.panorama_build_flat(t, w.X.to(DEV), level_widths=[64, 64])
    qd = torch.from_numpy(Q).to(DEV)
    cand = torch.from_numpy(_candidates(X, Q, 50, 5, seed=4)).to(DEV)
    a = idx.refine(qd, cand, 5)
    path = str(tmp_path / "flat.pano")
    pano.panorama_save(idx, path)
    idx2 = pano.panorama_load(path)
    b = idx2.refine(qd, cand, 5)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    bad = cand.clone()
    bad[0, 0] = len(X)
    with pytest.raises(pano.LibraryError):
        idx.refine(qd, bad, 5)
    with pytest.raises(pano.LibraryError):  # the IVF search does not take a flat index
        idx.search(qd, 1, 5)
    ivf = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=1, level_widths=[64, 64])
    with pytest.raises(pano.LibraryError):  # refine needs the flat layout
        ivf.refine(qd, cand, 5)
