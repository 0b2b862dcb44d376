"""Comparison of library results with oracle results (used by GPU tests)."""
import numpy as np


def fp64_dists(q, X, ids):
    ids = np.asarray(ids)
    diff = X[ids].astype(np.float64) - q.astype(np.float64)
    return np.einsum("ij,ij->i", diff, diff)


def check_topk(X, Q, got_ids, got_d, ref_ids, ref_d, k, gamma_rows=None,
               rtol_tie=1e-6, rtol_d=1e-5):
    """Checks one batch of results against the oracle.

    * every row holds exactly min(k, |Gamma|) distinct valid ids followed by
      (-1, +inf) padding, like the oracle's row;
    * the id at each position equals the oracle's, or its FP64 distance is
      within rtol_tie (relative) of the oracle's distance at that position
      (a near-tie, which FP32 arithmetic may order either way);
    * each reported distance is within rtol_d of the FP64 distance of the
      reported id (and so of the oracle's distance at that position);
    * ids belong to the query's candidate set when gamma_rows is given.
    Returns (max relative distance error, number of near-tie swaps).
    """
    got_ids = np.asarray(got_ids)
    got_d = np.asarray(got_d, dtype=np.float64)
    k_arr = np.broadcast_to(np.asarray(k), (Q.shape[0],))
    worst, swaps = 0.0, 0
    for i in range(Q.shape[0]):
        ki = int(k_arr[i])
        nvalid = int(np.sum(ref_ids[i, :ki] >= 0))
        assert np.all(got_ids[i, nvalid:] == -1), (i, got_ids[i])
        assert np.all(np.isinf(got_d[i, nvalid:])), (i, got_d[i])
        g = got_ids[i, :nvalid]
        assert np.all(g >= 0), (i, g)
        assert len(set(g.tolist())) == nvalid, (i, g)
        if gamma_rows is not None:
            assert np.all(np.isin(g, gamma_rows[i])), (i, "id outside Gamma")
        if nvalid == 0:
            continue
        true_d = fp64_dists(Q[i], X, g)
        rel = np.abs(got_d[i, :nvalid] - true_d) / np.maximum(true_d, 1e-30)
        worst = max(worst, float(rel.max()))
        assert np.all(rel <= rtol_d), (i, rel.max())
        mism = g != ref_ids[i, :nvalid]
        if mism.any():
            r = ref_d[i, :nvalid][mism]
            gap = np.abs(true_d[mism] - r) / np.maximum(r, 1e-30)
            assert np.all(gap <= rtol_tie), (i, g[mism], ref_ids[i, :nvalid][mism], gap)
            swaps += int(mism.sum())
    return worst, swaps


def gamma_of(lists_of_vector, probes):
    return [np.nonzero(np.isin(lists_of_vector, p))[0] for p in probes]


def oracle_dims_fraction(X, Q, C, lists, nprobe, widths, k, B=1024):
    """Fraction of coordinates Algorithm 1 (the oracle) reads, averaged over
    the queries Q, with each query's nearest list first (as the GPU's phase
    A) and the PCA transform fitted on (up to) 65,536 rows of X."""
    import oracle
    d = X.shape[1]
    probes, _ = oracle.probe(Q, C, nprobe)
    mu, T, _ = oracle.pca_fit(X[:65536])
    tX = oracle.transform(T, mu, X)
    m = oracle.level_thresholds(d, widths)
    fr = []
    for i in range(len(Q)):
        order = np.concatenate([np.nonzero(lists == p)[0] for p in probes[i]])
        tq = oracle.transform(T, mu, Q[i:i + 1])[0]
        _, _, rho = oracle.refine(tq, tX[order], order, m, k, B=B)
        fr.append(rho.mean() / d)
    return float(np.mean(fr))
