"""GPU parity of IVFPQ Panorama (Section 6.3) with spectrum shaping (Section
4.3).  The oracle supplies the shaped transform, centroids, lists, codebooks
and codes (or checks the library's own), and computes the FP64 answer; the
library's pruned search must equal its plain scan bit for bit, and both must
match the oracle: ids equal except where FP64 distances tie within 2e-5
(two FP32 sums of M terms, each within 1e-5, may swap), distances within
1e-5 relative."""
import numpy as np
import pytest
import torch

import oracle
from oracle import pq
import paper_2510_00566_gb300 as pano
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RTOL_D = 1e-5
RTOL_TIE = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()


def _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes):
    """Per query: candidate ids and FP64 asymmetric distances over its probes."""
    tq = oracle.transform(Ts, mu, Q)
    tc = oracle.transform(Ts, mu, C)
    xh = pq.pq_reconstruct(codes, cb)
    out = []
    for i in range(len(Q)):
        mem = np.concatenate([np.nonzero(lists == c)[0] for c in probes[i]])
        own = lists[mem]
        D = ((tq[i][None] - tc[own] - xh[mem]) ** 2).sum(1)
        out.append((mem, D))
    return out


def _check(got_i, got_d, cand, k, keep):
    got_i, got_d = got_i.cpu().numpy(), got_d.cpu().numpy().astype(np.float64)
    worst = 0.0
    for i in np.nonzero(keep)[0]:
        mem, D = cand[i]
        order = np.lexsort((mem, D))[:k]
        nv = order.size
        assert np.all(got_i[i, nv:] == -1) and np.all(np.isinf(got_d[i, nv:])), i
        if nv == 0:
            continue
        g = got_i[i, :nv]
        assert len(set(g.tolist())) == nv and np.all(np.isin(g, mem)), (i, g)
        pos = {int(v): j for j, v in enumerate(mem)}
        true = D[[pos[int(v)] for v in g]]
        rel = np.abs(got_d[i, :nv] - true) / np.maximum(true, 1e-30)
        worst = max(worst, float(rel.max()))
        assert np.all(rel <= RTOL_D), (i, rel.max())
        mism = g != mem[order]
        if mism.any():
            gap = np.abs(true[mism] - D[order][mism]) / np.maximum(D[order][mism], 1e-30)
            assert np.all(gap <= RTOL_TIE), (i, g[mism], mem[order][mism], gap)
        assert np.all(np.diff(got_d[i, :nv]) >= 0)
    return worst


def _shaped(X, L, kappa, seed):
    mu, T, lam = oracle.pca_fit(X[:65536])
    G = np.random.default_rng(seed).standard_normal((2, X.shape[1], X.shape[1]))
    Ts, vs, _ = pq.shape_transform(T, lam, L, kappa, G[0], G[1])
    return Ts, mu, vs


def _search_both(idx, Q, nprobe, k):
    q = torch.from_numpy(Q).to(DEV)
    a = idx.search_pq(q, nprobe, k, mode=0, collect_stats=True)
    st0 = pano.last_stats()
    b = idx.search_pq(q, nprobe, k, mode=1, collect_stats=True)
    st1 = pano.last_stats()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), "pruned != plain scan"
    return a, st0, st1


def test_pq_960d_shaped_parity_and_pruning():
    """The 1M x 960 workload's recipe at 12k vectors: 16 lists, M = 480
    (2-d subvectors), 16 levels of 60 coordinates, kappa = 4."""
    s = synth.scaled(2, n=12_000, n_queries=40, nlist=16, n_clusters=16)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    d, L, M, nl = 960, 16, 480, 16
    Ts, mu, vs = _shaped(X, L, 4.0, 11)
    C = synth.initial_centroids(w.X, nl, seed=3002).numpy()
    lists, _ = oracle.assign(X, C)
    R = oracle.transform(Ts, mu, X) - oracle.transform(Ts, mu, C)[lists]
    g = np.random.default_rng(12)
    cb = pq.pq_train(R[g.choice(len(R), 2000, replace=False)], M, iters=1, seed=13)
    codes = pq.pq_encode32(R.astype(np.float32), cb)
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, w.X.to(DEV), nl, M, L, centroids=C, assign=lists,
                                    codebooks=cb, codes=codes)
    info = idx.info()
    assert info.precision == pano.PANO_PQ and info.chunk == 256
    k, nprobe = 10, 4
    (ids, dd), st0, st1 = _search_both(idx, Q, nprobe, k)
    probes, gap = oracle.probe(Q, C, nprobe)
    cand = _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes)
    worst = _check(ids, dd, cand, k, gap >= 1e-6)
    assert worst < RTOL_D
    pairs = sum(len(c[0]) for c in cand)
    assert st1.pairs == pairs and st1.dims_scanned == pairs * d
    assert st0.pairs == pairs and st0.dims_scanned < 0.9 * st1.dims_scanned
    # Algorithm 1 over the same codes (lists in probe order, batches of 1024)
    tq = oracle.transform(Ts, mu, Q)
    tc = oracle.transform(Ts, mu, C)
    xh = pq.pq_reconstruct(codes, cb)
    m = oracle.level_thresholds(d, [d // L] * L)
    dims = 0
    for i in range(len(Q)):
        mems = [np.nonzero(lists == c)[0] for c in probes[i]]
        _, _, di = pq.ivfpq_panorama([tq[i] - tc[c] for c in probes[i]],
                                     [xh[mm] for mm in mems], mems, m, k)
        dims += di
    assert st0.dims_scanned <= 1.5 * dims + 0.02 * pairs * d, (st0.dims_scanned, dims)


def test_pq_ragged_lists_slabs_and_padding():
    """Lists of 4500 (three slabs), 1, 0 and the rest of 7000 vectors; random
    codes; k from 1 to 100; a query whose only probed list has one member."""
    g = np.random.default_rng(20)
    d, L, M = 64, 4, 32
    n = 7000
    X = (g.standard_normal((n, d)) * np.exp(-0.04 * np.arange(d))).astype(np.float32)
    lists = np.full(n, 3, np.int32)
    lists[:4500] = 0
    lists[4500] = 1
    C = np.stack([X[lists == 0].mean(0), X[4500], 5 + X[:10].mean(0), X[lists == 3].mean(0)])
    C = C.astype(np.float32)
    C[0] += 0.3
    Ts, mu, vs = _shaped(X, L, 2.0, 21)
    cb = (g.standard_normal((M, 256, d // M)) * 0.3).astype(np.float32)
    codes = g.integers(0, 256, (n, M)).astype(np.uint8)
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, X, 4, M, L, centroids=C, assign=lists, codebooks=cb,
                                    codes=codes)
    Q = np.concatenate([g.standard_normal((30, d)).astype(np.float32) * 0.5,
                        X[4500:4501] + 1e-3]).astype(np.float32)
    for nprobe, k in ((1, 1), (1, 10), (2, 10), (4, 100), (3, 37)):
        (ids, dd), _, _ = _search_both(idx, Q, nprobe, k)
        probes, gap = oracle.probe(Q, C, nprobe)
        cand = _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes)
        _check(ids, dd, cand, k, gap >= 1e-6)
    ids, dd = idx.search_pq(torch.from_numpy(Q[-1:]).to(DEV), 1, 10)
    assert ids[0, 0].item() == 4500 and torch.all(ids[0, 1:] == -1)


@pytest.mark.parametrize("dsub", [1, 2, 3, 8])
def test_pq_encoder_bit_exact(dsub):
    g = np.random.default_rng(30 + dsub)
    M, n = 12, 3000
    d = M * dsub
    cb = g.standard_normal((M, 256, dsub)).astype(np.float32)
    cb[:, 200] = cb[:, 17]  # duplicated codewords: the lower index wins
    R = g.standard_normal((n, d)).astype(np.float32)
    R[:50] = cb[:, 17].reshape(-1)[None, :]
    got = pano.panorama_debug_pq_encode(torch.from_numpy(R).to(DEV),
                                        torch.from_numpy(cb).to(DEV)).cpu().numpy()
    want = pq.pq_encode32(R, cb)
    assert np.array_equal(got, want)
    assert np.all(got[:50] == 17)


def test_pq_library_trained_index():
    """The quantiser trained by the library (lists from given centroids, PQ
    k-means, the device encoder), checked without feeding any library output
    to the oracle: the lists agree with the oracle's nearest centroids; each
    code is the nearest codeword of the oracle's own FP64 residual up to FP32
    rounding; the pruned search equals the plain scan; and the recall of the
    oracle's exact neighbours (over its own probes and lists) is that of a
    working PQ."""
    s = synth.scaled(4, n=20_000, n_queries=60, nlist=20, n_clusters=20)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    d, L, M, nl, k, nprobe = X.shape[1], 8, 96, 20, 10, 5
    Ts, mu, vs = _shaped(X, L, 2.0, 40)
    C = synth.initial_centroids(w.X, nl, seed=41).numpy()
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, w.X.to(DEV), nl, M, L, centroids=C, pq_iters=8)
    lists, _ = oracle.assign(X, C)
    agree = idx.assignment() == lists
    assert agree.mean() > 0.999, agree.mean()
    cb, codes = pano.panorama_pq_export(idx)  # outputs under test
    R = oracle.transform(Ts, mu, X) - oracle.transform(Ts, mu, C)[lists]
    dsub = d // M
    for m in range(0, M, 7):
        sub = R[agree, m * dsub:(m + 1) * dsub]
        dd = ((sub[:, None, :] - cb[m][None].astype(np.float64)) ** 2).sum(-1)
        got = dd[np.arange(len(sub)), codes[agree, m]]
        assert np.all(got <= dd.min(1) + 1e-4 * (1 + dd.min(1))), m
    (ids, dd), _, _ = _search_both(idx, Q, nprobe, k)
    probes, gap = oracle.probe(Q, C, nprobe)
    ids = ids.cpu().numpy()
    rec = []
    for i in np.nonzero(gap >= 1e-6)[0]:
        mem = np.concatenate([np.nonzero(lists == c)[0] for c in probes[i]])
        assert np.all(np.isin(ids[i][ids[i] >= 0], mem)), i
        ex = ((X[mem].astype(np.float64) - Q[i]) ** 2).sum(1)
        true = mem[np.lexsort((mem, ex))[:k]]
        rec.append(len(set(true) & set(ids[i])) / k)
    assert np.mean(rec) >= 0.4, np.mean(rec)


def test_pq_epsilon_relaxed_pruning():
    """Eq. 4 on the IVFPQ path: epsilon = 0.5 reads no more subvector terms
    than the exact test, keeps most of the exact top-k, and every returned
    candidate carries its computed distance (as the plain scan computes it)."""
    s = synth.scaled(5, n=15_000, n_queries=60, nlist=8)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    d, L, M = X.shape[1], 8, X.shape[1] // 2
    Ts, mu, vs = _shaped(X, L, 2.0, 71)
    C = synth.initial_centroids(w.X, 8, seed=72).numpy()
    lists, _ = oracle.assign(X, C)
    R = oracle.transform(Ts, mu, X) - oracle.transform(Ts, mu, C)[lists]
    cb = pq.pq_train(R[:2000], M, iters=2, seed=73)
    codes = pq.pq_encode32(R.astype(np.float32), cb)
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, X, 8, M, L, centroids=C, assign=lists, codebooks=cb,
                                    codes=codes)
    q = torch.from_numpy(Q).to(DEV)
    ids1, d1 = idx.search_pq(q, 3, 10, collect_stats=True)
    dims1 = pano.last_stats().dims_scanned
    ids_e, d_e = idx.search_pq(q, 3, 10, collect_stats=True, epsilon=0.5)
    assert pano.last_stats().dims_scanned <= dims1
    probes, _ = oracle.probe(Q, C, 3)
    cand = _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes)
    ids_e, d_e = ids_e.cpu().numpy(), d_e.cpu().numpy().astype(np.float64)
    ids1 = ids1.cpu().numpy()
    rec = np.mean([len(set(ids_e[i]) & set(ids1[i])) / 10 for i in range(len(Q))])
    assert rec >= 0.5, rec
    for i in range(len(Q)):
        mem, D = cand[i]
        pos = {int(v): j for j, v in enumerate(mem)}
        v = ids_e[i] >= 0
        true = D[[pos[int(x)] for x in ids_e[i][v]]]
        assert np.allclose(d_e[i][v], true, rtol=RTOL_D)


def test_pq_per_query_nprobe_and_k():
    """Each query its own nprobe (1..6 of 6 lists) and k (0, 1, 10 or 37) in
    rows of k_max = 40: every row matches the oracle for its own probes and
    k, and is padded past it; the pruned search equals the plain scan."""
    g = np.random.default_rng(80)
    d, L, M, n, nl, nq = 64, 4, 32, 8000, 6, 50
    X = (g.standard_normal((n, d)) * np.exp(-0.04 * np.arange(d))).astype(np.float32)
    C = X[g.choice(n, nl, replace=False)]
    lists, _ = oracle.assign(X, C)
    Ts, mu, vs = _shaped(X, L, 2.0, 81)
    R = oracle.transform(Ts, mu, X) - oracle.transform(Ts, mu, C)[lists]
    cb = pq.pq_train(R[:2000], M, iters=2, seed=82)
    codes = pq.pq_encode32(R.astype(np.float32), cb)
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, X, nl, M, L, centroids=C, assign=lists, codebooks=cb,
                                    codes=codes)
    Q = (X[:nq] + 0.05 * g.standard_normal((nq, d))).astype(np.float32)
    npq = g.integers(1, nl + 1, nq).astype(np.int32)
    kq = g.choice([0, 1, 10, 37], nq).astype(np.int32)
    q = torch.from_numpy(Q).to(DEV)
    a = idx.search_pq(q, torch.from_numpy(npq).to(DEV), torch.from_numpy(kq).to(DEV), k_max=40)
    b = idx.search_pq(q, torch.from_numpy(npq).to(DEV), torch.from_numpy(kq).to(DEV), k_max=40,
                      mode=1)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[0].shape == (nq, 40)
    probes, gap = oracle.probe(Q, C, npq)
    cand = _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes)
    for i in range(nq):
        if gap[i] >= 1e-6:
            _check(a[0][i:i + 1], a[1][i:i + 1], [cand[i]], int(kq[i]), np.array([True]))


@pytest.mark.parametrize("M,L", [(48, 4), (16, 1), (6, 3), (16, 8), (12, 2)])
def test_pq_subvector_widths_and_level_counts(M, L):
    """d = 48 with 1-, 3-, 4- and 8-coordinate subvectors (vector and scalar
    table builders), a single level (no bound test at all) and up to 8
    levels; lists large enough for tables at level 0."""
    g = np.random.default_rng(60 + M + L)
    d, n = 48, 3000
    X = (g.standard_normal((n, d)) * np.exp(-0.05 * np.arange(d))).astype(np.float32)
    C = X[g.choice(n, 3, replace=False)]
    lists, _ = oracle.assign(X, C)
    Ts, mu, vs = _shaped(X, L, 2.0, 61)
    cb = (g.standard_normal((M, 256, d // M)) * 0.2).astype(np.float32)
    R = oracle.transform(Ts, mu, X) - oracle.transform(Ts, mu, C)[lists]
    codes = pq.pq_encode32(R.astype(np.float32), cb)
    t = pano.panorama_transform_import(Ts, mu, vs)
    idx = pano.panorama_build_ivfpq(t, X, 3, M, L, centroids=C, assign=lists, codebooks=cb,
                                    codes=codes)
    Q = (X[:40] + 0.05 * g.standard_normal((40, d))).astype(np.float32)
    for nprobe, k in ((1, 10), (2, 25)):
        (ids, dd), st0, st1 = _search_both(idx, Q, nprobe, k)
        probes, gap = oracle.probe(Q, C, nprobe)
        cand = _oracle_dists(Q, Ts, mu, C, lists, cb, codes, probes)
        _check(ids, dd, cand, k, gap >= 1e-6)
        assert st1.dims_scanned == st1.pairs * d
        assert st0.dims_scanned <= st1.dims_scanned


def test_pq_argument_errors_and_save_load(tmp_path):
    g = np.random.default_rng(50)
    X = g.standard_normal((600, 32)).astype(np.float32)
    t = pano.panorama_fit_transform(X, n_levels=4)
    for M, L in ((5, 4), (8, 3), (12, 4)):
        with pytest.raises(pano.LibraryError):
            pano.panorama_build_ivfpq(t, X, 2, M, L)
    idx = pano.panorama_build_ivfpq(t, X, 2, 16, 4, pq_iters=2)
    q = torch.from_numpy(X[:4]).to(DEV)
    with pytest.raises(pano.LibraryError):
        idx.search(q, 1, 5)
    with pytest.raises(pano.LibraryError):
        idx.search_pq(q, 3, 5)  # nprobe > nlist
    path = str(tmp_path / "pq.pano")
    pano.panorama_save(idx, path)  # the quantiser survives a round trip bit for bit
    idx2 = pano.panorama_load(path)
    assert idx2.info().precision == pano.PANO_PQ
    a, b = idx.search_pq(q, 2, 5), idx2.search_pq(q, 2, 5)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    cb1, c1 = pano.panorama_pq_export(idx)
    cb2, c2 = pano.panorama_pq_export(idx2)
    assert np.array_equal(cb1, cb2) and np.array_equal(c1, c2)
    with pytest.raises(pano.LibraryError):
        idx2.search(q, 1, 5)
    flat = pano.panorama_build_ivf(t, X, 2, n_levels=4)
    with pytest.raises(pano.LibraryError):
        flat.search_pq(q, 1, 5)
    ids, dd = idx.search_pq(q, 2, 5)
    assert torch.all(ids[:, 0] >= 0)
