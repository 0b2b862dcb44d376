"""Plain FP64 restatement of Panorama's mathematics (test infrastructure only).

Every function cites the passage of the paper it follows.  Nothing is blocked,
fused or reordered beyond what the passage states; numpy routines (matmul,
eigh, sort) serve as single steps.

Pins (tests/test_oracle_pins.py):
  pca_fit           exact-spectrum construction, orthogonality < 1e-10,
                    distance preservation, Ky Fan optimality, spectrum recovery
  level_stats/bounds level-0 closed form (reverse triangle inequality),
                    level-L exactness vs scipy, gap identity (Appendix A),
                    hand-derived integer example, monotone tightening
  topk / assign / probe  hand lattice example with ties, scipy cdist
  candidate_topk    hand-derived golden with repeated and padded ids
  refine (Alg. 1)   equals brute force on random inputs (any B, k > |Gamma|)
  energy_fraction / fit_alpha  closed form on an exact exponential spectrum,
                    the least-squares optimum of a two-level spectrum solved
                    by hand (cubic), MAE < 0.04 on the 128-d workload
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

__all__ = [
    "pca_fit", "transform", "level_thresholds", "level_stats", "bounds",
    "exact_sqdist", "topk", "assign", "probe", "refine", "energy_fraction",
    "fit_alpha", "ivf_lists", "ivf_search", "candidate_topk", "KEY_INF",
]

KEY_INF = np.inf


# ---------------------------------------------------------------- Section 4.1
def pca_fit(X: np.ndarray):
    """PCA basis of a data set (Section 4.1 "PCA as the closed-form transform").

    Returns (mu, T, lam): the sample mean, the orthogonal matrix whose ROWS are
    the eigenvectors of the empirical covariance (1/n normalisation), ordered
    by eigenvalue descending (ties by eigen-solver index), and the eigenvalues.
    Centring by the mean is a translation, which preserves distances, so the
    transformed vector of x is T (x - mu).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    mu = X.mean(axis=0)
    Xc = X - mu
    cov = (Xc.T @ Xc) / n
    lam, V = np.linalg.eigh(cov)              # ascending, columns
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    T = V[:, order].T.copy()                  # rows = eigenvectors
    return mu, T, lam


def transform(T: np.ndarray, mu: np.ndarray, V: np.ndarray) -> np.ndarray:
    """T(v) = T (v - mu) for each row v of V (Eq. 1 uses T; centring per C1)."""
    V = np.asarray(V, dtype=np.float64)
    return (V - mu) @ np.asarray(T, dtype=np.float64).T


def level_thresholds(d: int, widths: Sequence[int]) -> np.ndarray:
    """0 = m_0 < m_1 < ... < m_L = d from level widths (Section 3)."""
    m = np.concatenate([[0], np.cumsum(np.asarray(widths, dtype=np.int64))])
    if m[-1] != d or np.any(np.diff(m) <= 0):
        raise ValueError("level widths must be positive and sum to d")
    return m


# ------------------------------------------------------------- Section 3
def level_stats(tq: np.ndarray, tX: np.ndarray, m: np.ndarray):
    """Partial inner products and tail energies of Eq. 2.

    tq: (d,) transformed query; tX: (n, d) transformed candidates.
    Returns, for l = 0..L:
      p[l]  = p^{(0,l)}(q, x)   = sum_{j <= m_l} T(q)_j T(x)_j      (n, L+1)
      Rq[l] = R_{T(q)}^{(l,L)}  = sum_{j >  m_l} T(q)_j^2           (L+1,)
      Rx[l] = R_{T(x)}^{(l,L)}  = sum_{j >  m_l} T(x)_j^2           (n, L+1)
    (indices are 0-based here: coordinates m_l .. d-1 form the tail.)
    """
    tq = np.asarray(tq, dtype=np.float64)
    tX = np.atleast_2d(np.asarray(tX, dtype=np.float64))
    L = len(m) - 1
    n = tX.shape[0]
    p = np.zeros((n, L + 1))
    Rx = np.zeros((n, L + 1))
    Rq = np.zeros(L + 1)
    for l in range(L + 1):
        head = slice(0, m[l])
        tail = slice(m[l], m[-1])
        p[:, l] = tX[:, head] @ tq[head]
        Rx[:, l] = np.sum(tX[:, tail] ** 2, axis=1)
        Rq[l] = np.sum(tq[tail] ** 2)
    return p, Rq, Rx


def bounds(tq: np.ndarray, tX: np.ndarray, m: np.ndarray, eps: float = 1.0):
    """Cauchy-Schwarz bounds per level (Eq. 3, Eq. 4 and the matching UB).

    With A^l = R_q^{(0,d)} + R_x^{(0,d)} - 2 p^{(0,l)} and
    C^l = sqrt(R_q^{(l,d)} R_x^{(l,d)}) (Section 3, "pruning aggressiveness"):
      LB^l     = A^l - 2 C^l        (Eq. 3; eps = 1)
      LB_eps^l = A^l - 2 eps C^l    (Eq. 4)
      UB^l     = A^l + 2 C^l        (the other side of the same Cauchy-Schwarz
                                     step, |tail inner product| <= C^l; the
                                     gap identity of Appendix A with rho >= -1)
    Returns (LB_eps, UB, A, C), each (n, L+1).
    """
    p, Rq, Rx = level_stats(tq, tX, m)
    A = Rq[0] + Rx[:, [0]] - 2.0 * p
    C = np.sqrt(Rq[None, :] * Rx)
    return A - 2.0 * eps * C, A + 2.0 * C, A, C


# ------------------------------------------------------------- Problem 1
def exact_sqdist(q: np.ndarray, X: np.ndarray) -> np.ndarray:
    """||q - x||^2 = sum_j (q_j - x_j)^2 in FP64 (Problem 1)."""
    diff = np.atleast_2d(np.asarray(X, dtype=np.float64)) - \
        np.asarray(q, dtype=np.float64)
    return np.einsum("ij,ij->i", diff, diff)


def topk(dists: np.ndarray, ids: np.ndarray, k: int):
    """The k smallest (dist, id) pairs, ascending, ties by id (Problem 1).

    Fewer than k candidates: the result is padded with (id -1, dist +inf).
    """
    dists = np.asarray(dists, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    order = np.lexsort((ids, dists))[:k]
    out_i = np.full(k, -1, dtype=np.int64)
    out_d = np.full(k, np.inf)
    out_i[:len(order)] = ids[order]
    out_d[:len(order)] = dists[order]
    return out_i, out_d


# ------------------------------------------------------------- Section 6.1
def _sq_to_centroids(V: np.ndarray, C: np.ndarray) -> np.ndarray:
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    out = np.empty((V.shape[0], C.shape[0]))
    for j in range(C.shape[0]):
        diff = V - C[j]
        out[:, j] = np.einsum("ij,ij->i", diff, diff)
    return out


def _sq_to_centroids_fast(V: np.ndarray, C: np.ndarray,
                          block: int = 65536) -> np.ndarray:
    # FP64 expansion; error ~1e-16 * (|v|+|c|)^2, far below the 1e-6 relative
    # near-tie band the tests allow.
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    cn = np.sum(C * C, axis=1)
    out = np.empty((V.shape[0], C.shape[0]))
    for s in range(0, V.shape[0], block):
        v = V[s:s + block]
        vn = np.sum(v * v, axis=1)
        out[s:s + block] = vn[:, None] + cn[None, :] - 2.0 * (v @ C.T)
    return out


def assign(X: np.ndarray, C: np.ndarray, block: int = 65536, threads: int = 0):
    """Nearest centroid of every vector (IVF, Section 6.1), ties -> lowest id.

    Returns (list_of_vector, relative gap between the best and second-best
    centroid distance); gaps below 1e-6 mark assignments that FP32 arithmetic
    may legitimately resolve the other way.  Distances are the FP64
    expansion |v|^2 + |c|^2 - 2 v.c (one matmul per block of rows); the
    argmin (first = lowest id among equal values) and the second-smallest
    value of each row are taken in parallel over slices of rows.
    """
    import concurrent.futures as cf
    import os
    n = X.shape[0]
    C = np.asarray(C, dtype=np.float64)
    cn = np.sum(C * C, axis=1)
    lists = np.empty(n, dtype=np.int64)
    gap = np.full(n, np.inf)
    nt = threads if threads > 0 else (os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(nt) as ex:
        for s in range(0, n, block):
            v = np.asarray(X[s:s + block], dtype=np.float64)
            vn = np.sum(v * v, axis=1)
            G = v @ C.T

            def rows(a, b):
                D = vn[a:b, None] + cn[None, :]
                D -= 2.0 * G[a:b]
                best = np.argmin(D, axis=1)
                r = np.arange(b - a)
                lists[s + a:s + b] = best
                if D.shape[1] > 1:
                    d0 = D[r, best].copy()
                    D[r, best] = np.inf
                    d1 = np.min(D, axis=1)
                    gap[s + a:s + b] = (d1 - d0) / np.maximum(d1, 1e-300)

            step = max(256, -(-v.shape[0] // nt))
            list(ex.map(lambda a: rows(a, min(a + step, v.shape[0])),
                        range(0, v.shape[0], step)))
    return lists, gap


def probe(Qv: np.ndarray, C: np.ndarray, nprobe):
    """The nprobe nearest lists of every query, by (FP64 distance, list id).

    Returns (probes as a list of int arrays, relative gap between the
    nprobe-th and (nprobe+1)-th centroid distances; inf if nprobe = nlist).
    """
    D = _sq_to_centroids_fast(Qv, C)
    nq, nlist = D.shape
    nprobe = np.broadcast_to(np.asarray(nprobe), (nq,))
    out, gaps = [], np.full(nq, np.inf)
    for i in range(nq):
        order = np.lexsort((np.arange(nlist), D[i]))
        p = int(nprobe[i])
        out.append(order[:p].copy())
        if p < nlist:
            a, b = D[i, order[p - 1]], D[i, order[p]]
            gaps[i] = (b - a) / max(b, 1e-300)
    return out, gaps


def ivf_lists(lists_of_vector: np.ndarray, nlist: int):
    """CSR of list membership: rows of list c are rows[ptr[c]:ptr[c+1]]."""
    order = np.argsort(lists_of_vector, kind="stable")
    counts = np.bincount(lists_of_vector, minlength=nlist)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return ptr, order.astype(np.int64)


def ivf_search(X, Qv, C, nprobe, k, lists_of_vector=None, threads=0):
    """The answer of Problem 1 over IVF candidate sets (Problem 2 + Section 6.1).

    Gamma(q) is the union of the q's nprobe nearest lists; the result is the
    brute-force FP64 top-k over Gamma(q), ties by id, padded with (-1, inf).
    Returns dict(ids, dists, probes, probe_gap, lists, assign_gap).
    """
    from .native import ivf_topk
    X = np.ascontiguousarray(X, dtype=np.float32)
    Qv = np.ascontiguousarray(Qv, dtype=np.float32)
    nlist = C.shape[0]
    agap = None
    if lists_of_vector is None:
        lists_of_vector, agap = assign(X, C)
    ptr, rows = ivf_lists(lists_of_vector, nlist)
    probes, pgap = probe(Qv, C, nprobe)
    nq = Qv.shape[0]
    k_arr = np.broadcast_to(np.asarray(k), (nq,)).astype(np.int32)
    ids, dists = ivf_topk(X, Qv, ptr, rows, probes, k_arr, threads=threads)
    return dict(ids=ids, dists=dists, probes=probes, probe_gap=pgap,
                lists=lists_of_vector, assign_gap=agap)


def candidate_topk(X, Qv, cand, k):
    """The answer of Problem 1 over an explicit candidate-id list per query.

    This is the refine workload of Section 6.4 ("IndexRefinePanorama"):
    another index hands each query its top-k' ids, and the refinement
    returns the exact top-k among them.  Reading: Gamma(q) is the set of
    DISTINCT ids in the query's row that are >= 0 (-1 pads a short list; an
    id listed twice is one candidate).  Distances are sum_j (q_j - x_j)^2 in
    FP64 from the FP32 inputs; the k smallest (dist, id) pairs ascending,
    ties by id, padded with (-1, +inf) when |Gamma(q)| < k.
    Returns (ids int64 [nq, k], dists float64 [nq, k]).
    """
    X = np.asarray(X)
    Qv = np.asarray(Qv)
    cand = np.asarray(cand, dtype=np.int64)
    out_i = np.full((Qv.shape[0], k), -1, dtype=np.int64)
    out_d = np.full((Qv.shape[0], k), np.inf)
    for i in range(Qv.shape[0]):
        gamma = np.unique(cand[i][cand[i] >= 0])
        out_i[i], out_d[i] = topk(exact_sqdist(Qv[i], X[gamma]), gamma, k)
    return out_i, out_d


# ------------------------------------------------------------- Algorithm 1
def refine(tq: np.ndarray, tX: np.ndarray, ids: np.ndarray, m: np.ndarray,
           k: int, B: int = 1024, eps: float = 1.0):
    """Algorithm 1 (iterative distance refinement), FP64, in the paper's order.

    * precompute T(q), ||T(q)||^2 and the query tail energies;
    * seed the exact-distance heap H with the first k candidates and set d_k
      to the k-th smallest of them (+inf while H holds fewer than k);
    * for every following batch of B candidates, for l = 1..L, mark as pruned
      every still-active candidate with LB_eps^l > d_k (strict, d_k fixed for
      the whole batch);
    * push each unpruned candidate's LB^L (= its exact distance) into H and,
      when it is below d_k, refresh d_k as the k-th smallest entry of H.
    Returns (top-k ids, top-k dists, rho) where rho[i] is the number of
    coordinates read for candidate i (the dimension at which it was pruned,
    or d) -- the cost measure of Section 3.
    Readings: the batches cover the candidates after the first k; "d" in the
    heap-update test is the pushed distance LB^L.
    """
    tX = np.atleast_2d(np.asarray(tX, dtype=np.float64))
    ids = np.asarray(ids, dtype=np.int64)
    n = tX.shape[0]
    L = len(m) - 1
    d = int(m[-1])
    LB, _, _, _ = bounds(tq, tX, m, eps=eps)
    exact = bounds(tq, tX, m, eps=1.0)[0][:, L]     # LB^L = exact distance
    rho = np.full(n, d, dtype=np.int64)

    heap_d = list(exact[:k])
    heap_i = list(ids[:k])

    def kth():
        if len(heap_d) < k:
            return np.inf
        order = np.lexsort((np.asarray(heap_i), np.asarray(heap_d)))
        return float(np.asarray(heap_d)[order[k - 1]])

    def crop():
        order = np.lexsort((np.asarray(heap_i), np.asarray(heap_d)))[:k]
        hd = [heap_d[o] for o in order]
        hi = [heap_i[o] for o in order]
        heap_d[:] = hd
        heap_i[:] = hi

    dk = kth()
    for s in range(min(k, n), n, B):
        e = min(n, s + B)
        active = np.ones(e - s, dtype=bool)
        for l in range(1, L + 1):
            prune = active & (LB[s:e, l] > dk)
            rho[s:e][prune] = m[l]
            active &= ~prune
        for j in np.nonzero(active)[0]:
            dist = exact[s + j]
            heap_d.append(dist)
            heap_i.append(ids[s + j])
            if dist < dk or len(heap_d) <= k:
                crop()
                dk = kth()
        crop()
        dk = kth()
    crop()
    out_i = np.full(k, -1, dtype=np.int64)
    out_d = np.full(k, np.inf)
    out_i[:len(heap_i)] = heap_i
    out_d[:len(heap_d)] = heap_d
    return out_i, out_d, rho


# ------------------------------------------- Section 4.1 energy compaction
def energy_fraction(lam: np.ndarray) -> np.ndarray:
    """E(m) = sum_{j>m} lambda_j / sum_j lambda_j for m = 0..d (Section 4.1)."""
    lam = np.asarray(lam, dtype=np.float64)
    tail = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
    return tail / tail[0]


def fit_alpha(lam: np.ndarray):
    """Least-squares alpha in E(m) ~ exp(-alpha m / d) (Section 4.1).

    Returns (alpha, mean absolute error of the fit over m = 0..d).
    """
    from scipy.optimize import minimize_scalar
    E = energy_fraction(lam)
    d = len(lam)
    x = np.arange(d + 1) / d

    def loss(a):
        return float(np.sum((E - np.exp(-a * x)) ** 2))

    # the loss is flat for large alpha (exp(-alpha x) ~ 0 beyond m = 0), so a
    # bounded search over the whole range can stop on that plateau: bracket
    # the minimum on a log-spaced grid first, then refine inside the bracket
    grid = np.geomspace(1e-6, 1e4, 4001)
    i = int(np.argmin([loss(a) for a in grid]))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    res = minimize_scalar(loss, bounds=(lo, hi), method="bounded",
                          options=dict(xatol=1e-12))
    a = float(res.x)
    mae = float(np.mean(np.abs(E - np.exp(-a * x))))
    return a, mae
