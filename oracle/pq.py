"""IVFPQ Panorama in plain FP64 (test infrastructure only).

Follows Section 4.3 (spectrum shaping for PQ compatibility: Procedure 1,
Robin Hood inter-level shaping; Procedure 2, intra-level isotropisation; the
combined transform U R T) and Section 6.3 (IndexIVFPQPanorama: product
quantisation of IVF residuals, per-level look-up-table distances, the same
bound / prune loop as IVFFlat).  Product quantisation itself is the textbook
method the paper recalls in Section 4.3 ("What PQ expects"): M contiguous
subvectors, one 2^nbits-entry codebook each, asymmetric distance
sum_m ||r_m - C_m[code_m]||^2.

Readings (the paper leaves these open):
  * Levels for shaping and for pruning are the same L contiguous blocks of
    b = d / L coordinates; a level holds M / L whole subvectors.
  * "Expected energy" is the expectation over the Haar draw: a Haar rotation
    of n coordinates with variances v gives each output coordinate expected
    variance sum(v) / n.  Procedure 1 tracks these expected variances.
  * The "minimal suffix" of Procedure 1 is the smallest s >= 1 with
    b * (sum of the level's and the next s variances) / (b + s) <= cap; a
    relative tolerance of 1e-12 keeps exact ties (sum equal to the cap)
    inside the cap.
  * A Haar-random orthogonal matrix is drawn from a Gaussian matrix G as the
    Q factor of G = QR with R's diagonal made positive (Mezzadri, "How to
    generate random matrices from the classical compact groups", 2007).
    The Gaussian draws are inputs: the block [a, a+n) of Procedure 1 uses
    G1[a:a+n, a:a+n] and level l of Procedure 2 uses G2 on the level's
    diagonal block.
  * IVF residuals: a vector of list c is encoded as r = T(x - mu) - T(c - mu)
    (the coarse centroid removed in the transformed basis).
  * The distance the index ranks by is the asymmetric distance in FP32 as a
    plain scan computes it: per subvector the entry sum_j fl(fl(r_j - C_j)^2)
    added left to right, then the M entries added in subquantiser order; the
    oracle's answer is the same quantity in FP64, and ties are broken by id.
  * Bounds of Eq. 3 in partial-distance form: with D_head the distance over
    the subvectors of levels <= l and R_q, R_x the tail energies of the query
    residual and of the reconstruction, LB = D_head + (sqrt R_q - sqrt R_x)^2
    and UB = D_head + (sqrt R_q + sqrt R_x)^2, which equal A - 2C and A + 2C
    of Eq. 3 (A = ||r||^2 + ||x^||^2 - 2 p).

Pins (tests/test_pq_oracle.py): hand-derived Robin Hood examples
(tests/golden/robin_hood.txt), orthogonality, energy conservation and the
cap, minimality of each suffix, Haar moments by Monte Carlo, the encoder's
codes against an FP64 argmin, ADC equal to the exact distance when the
codebooks hold the data, LB <= ADC <= UB with equality at the last level, the
Eq. 3 identity, Algorithm 1 over ADC equal to the plain ADC top-k, the
invariance of every level bound under Procedure 2, and the trade Procedure 1
makes (more coordinates read by Algorithm 1, lower PQ reconstruction error
than the PCA basis at the same bit budget), and pq_train's Lloyd steps (the
blob means as the fixed point on separated blobs, a non-increasing
quantisation error).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .reference import probe

__all__ = [
    "haar_from_gaussian", "robin_hood", "isotropize", "shape_transform",
    "pq_entries32", "pq_encode32", "pq_train", "pq_reconstruct",
    "adc_dists", "pq_level_bounds", "ivfpq_search", "ivfpq_panorama",
    "level_energies",
]

_TIE = 1e-12


def haar_from_gaussian(G: np.ndarray) -> np.ndarray:
    """Haar-distributed orthogonal matrix from an n x n standard Gaussian
    matrix: the Q of G = QR with diag(R) > 0 (Mezzadri 2007, Section 5)."""
    G = np.asarray(G, dtype=np.float64)
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def level_energies(v: np.ndarray, L: int) -> np.ndarray:
    """E_l = sum of the coordinate variances of level l (Section 4.3,
    Procedure 1), levels of b = d / L coordinates."""
    v = np.asarray(v, dtype=np.float64)
    return v.reshape(L, -1).sum(axis=1)


def robin_hood(lam: np.ndarray, L: int, kappa: float, G1: np.ndarray):
    """Procedure 1 (Section 4.3): cap tau = kappa * mean level energy; sweep
    the levels front to back; a level above the cap is rotated, together
    with the smallest suffix of following coordinates that brings its
    expected energy down to the cap, by a Haar rotation.

    Returns (R d x d, v expected coordinate variances after R, blocks as a
    list of (first coordinate, size))."""
    lam = np.asarray(lam, dtype=np.float64)
    d = lam.size
    assert d % L == 0, "levels of equal width"
    b = d // L
    v = lam.copy()
    cap = kappa * v.sum() / L
    R = np.eye(d)
    blocks = []
    for l in range(L):
        a = l * b
        if v[a:a + b].sum() <= cap * (1 + _TIE):
            continue
        s = 1
        while a + b + s < d and b * v[a:a + b + s].sum() > cap * (b + s) * (1 + _TIE):
            s += 1
        n = b + s
        R[a:a + n, a:a + n] = haar_from_gaussian(G1[a:a + n, a:a + n])
        v[a:a + n] = v[a:a + n].sum() / n
        blocks.append((a, n))
    return R, v, blocks


def isotropize(d: int, L: int, G2: np.ndarray) -> np.ndarray:
    """Procedure 2 (Section 4.3): block-diagonal U with an independent Haar
    rotation U_l of each level's b coordinates."""
    b = d // L
    U = np.zeros((d, d))
    for l in range(L):
        a = l * b
        U[a:a + b, a:a + b] = haar_from_gaussian(G2[a:a + b, a:a + b])
    return U


def shape_transform(T: np.ndarray, lam: np.ndarray, L: int, kappa: float,
                    G1: np.ndarray, G2: np.ndarray):
    """The combined transform U R T (Section 4.3) and the expected coordinate
    variances after it (each level's energy spread evenly by U)."""
    R, v, blocks = robin_hood(lam, L, kappa, G1)
    U = isotropize(T.shape[0], L, G2)
    Ts = U @ (R @ np.asarray(T, dtype=np.float64))
    vs = np.repeat(level_energies(v, L) / (T.shape[0] // L), T.shape[0] // L)
    return Ts, vs, blocks


def pq_entries32(R32: np.ndarray, C32: np.ndarray) -> np.ndarray:
    """FP32 entries sum_j fl(fl(r_j - c_j)^2), added left to right (no fused
    multiply-add), of each row of R32 (n x dsub) against each codeword of
    C32 (ksub x dsub): an n x ksub float32 array."""
    R32 = np.asarray(R32, dtype=np.float32)
    C32 = np.asarray(C32, dtype=np.float32)
    s = np.zeros((R32.shape[0], C32.shape[0]), dtype=np.float32)
    for j in range(R32.shape[1]):
        t = R32[:, j:j + 1] - C32[None, :, j]
        s = s + t * t
    return s


def pq_encode32(R32: np.ndarray, codebooks32: np.ndarray) -> np.ndarray:
    """Product-quantisation codes (Section 4.3): for each subvector the
    codeword with the smallest FP32 entry, ties to the lowest index.
    R32 n x d, codebooks32 M x ksub x dsub -> n x M uint8."""
    R32 = np.asarray(R32, dtype=np.float32)
    M, ksub, dsub = codebooks32.shape
    codes = np.empty((R32.shape[0], M), dtype=np.uint8)
    for m in range(M):
        e = pq_entries32(R32[:, m * dsub:(m + 1) * dsub], codebooks32[m])
        codes[:, m] = np.argmin(e, axis=1)  # first minimum
    return codes


def pq_train(R: np.ndarray, M: int, ksub: int = 256, iters: int = 10,
             seed: int = 0) -> np.ndarray:
    """Per-subspace Lloyd k-means in FP64 (the PQ codebooks of Section 4.3),
    initialised with distinct training rows; empty cells keep their
    codeword.  Returns M x ksub x dsub float32."""
    R = np.asarray(R, dtype=np.float64)
    n, d = R.shape
    dsub = d // M
    g = np.random.default_rng(seed)
    init = g.choice(n, size=ksub, replace=False)
    out = np.empty((M, ksub, dsub), dtype=np.float32)
    for m in range(M):
        X = R[:, m * dsub:(m + 1) * dsub]
        C = X[init].copy()
        for _ in range(iters):
            dd = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
            a = np.argmin(dd, axis=1)
            for j in range(ksub):
                sel = a == j
                if sel.any():
                    C[j] = X[sel].mean(axis=0)
        out[m] = C.astype(np.float32)
    return out


def pq_reconstruct(codes: np.ndarray, codebooks: np.ndarray) -> np.ndarray:
    """x^ = concat_m C_m[code_m] in FP64 (n x d)."""
    M, ksub, dsub = codebooks.shape
    cb = np.asarray(codebooks, dtype=np.float64)
    return np.concatenate([cb[m][codes[:, m]] for m in range(M)], axis=1)


def adc_dists(rq: np.ndarray, codes: np.ndarray, codebooks: np.ndarray) -> np.ndarray:
    """Asymmetric distance sum_m ||rq_m - C_m[code_m]||^2 in FP64."""
    xh = pq_reconstruct(codes, codebooks)
    return ((np.asarray(rq, dtype=np.float64)[None, :] - xh) ** 2).sum(axis=1)


def pq_level_bounds(rq: np.ndarray, xh: np.ndarray, m: Sequence[int]):
    """LB / UB of Eq. 3 in partial-distance form for each level l = 1..L
    (coordinates < m_l known): LB_l = D_head + (sqrt R_q - sqrt R_x)^2,
    UB_l = D_head + (sqrt R_q + sqrt R_x)^2.  Returns (L x n, L x n)."""
    rq = np.asarray(rq, dtype=np.float64)
    xh = np.asarray(xh, dtype=np.float64)
    L = len(m) - 1
    lb = np.empty((L, xh.shape[0]))
    ub = np.empty((L, xh.shape[0]))
    for l in range(1, L + 1):
        h = m[l]
        head = ((rq[None, :h] - xh[:, :h]) ** 2).sum(axis=1)
        sq = np.sqrt((rq[h:] ** 2).sum())
        sx = np.sqrt((xh[:, h:] ** 2).sum(axis=1))
        lb[l - 1] = head + (sq - sx) ** 2
        ub[l - 1] = head + (sq + sx) ** 2
    return lb, ub


def ivfpq_search(Q, T, mu, C, lists_of_vector, codebooks, codes, nprobe: int, k: int):
    """The IVFPQ answer (Section 6.3 without pruning): probe the nprobe
    nearest lists (FP64, ties by list id), score every member x of those
    lists by the asymmetric distance of the query residual T(q - c) to its
    code, return the k smallest (distance, id), padded with (-1, inf).

    Returns dict(ids, dists, probes, probe_gap)."""
    T = np.asarray(T, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    tq = (np.asarray(Q, dtype=np.float64) - mu) @ T.T
    tc = (np.asarray(C, dtype=np.float64) - mu) @ T.T
    probes, gap = probe(np.asarray(Q, np.float32), np.asarray(C, np.float32), nprobe)
    xh = pq_reconstruct(codes, codebooks)
    nq = tq.shape[0]
    ids = np.full((nq, k), -1, np.int64)
    dists = np.full((nq, k), np.inf)
    members = [np.nonzero(lists_of_vector == c)[0] for c in range(C.shape[0])]
    for i in range(nq):
        cand, dd = [], []
        for c in probes[i]:
            mem = members[c]
            r = tq[i] - tc[c]
            cand.append(mem)
            dd.append(((r[None, :] - xh[mem]) ** 2).sum(axis=1))
        cand = np.concatenate(cand)
        dd = np.concatenate(dd)
        order = np.lexsort((cand, dd))[:k]
        ids[i, :order.size] = cand[order]
        dists[i, :order.size] = dd[order]
    return {"ids": ids, "dists": dists, "probes": probes, "probe_gap": gap}


def ivfpq_panorama(rq_lists, xh_lists, id_lists, m: Sequence[int], k: int, B: int = 1024):
    """Algorithm 1 over asymmetric distances (Section 6.3 keeps the IVFFlat
    loop): the lists of one query in probe order, each in batches of B
    candidates; the threshold is the k-th smallest distance found so far
    (seeded with the first k candidates met); level by level every live
    candidate's lower bound is compared with it (strict >).  Returns
    (ids, dists, dims) with dims the coordinates whose subvector distances
    were added."""
    L = len(m) - 1
    best_d: list = []
    best_i: list = []
    dims = 0

    def kth():
        return best_d[k - 1] if len(best_d) >= k else np.inf

    def push(dist, i):
        best_d.append(dist)
        best_i.append(i)
        order = np.lexsort((np.array(best_i), np.array(best_d)))[:k]
        bd = [best_d[j] for j in order]
        bi = [best_i[j] for j in order]
        best_d[:] = bd
        best_i[:] = bi

    for rq, xh, ids in zip(rq_lists, xh_lists, id_lists):
        rq = np.asarray(rq, np.float64)
        xh = np.asarray(xh, np.float64)
        for s in range(0, xh.shape[0], B):
            X = xh[s:s + B]
            I = ids[s:s + B]
            live = np.arange(X.shape[0])
            lb, _ = pq_level_bounds(rq, X, m)
            for l in range(1, L + 1):
                dims += live.size * (m[l] - m[l - 1])
                if l < L:
                    live = live[~(lb[l - 1][live] > kth())]
                else:
                    for j in live:
                        dist = float(((rq - X[j]) ** 2).sum())
                        if len(best_d) < k or dist <= kth():
                            push(dist, int(I[j]))
    ids = np.full(k, -1, np.int64)
    dd = np.full(k, np.inf)
    ids[:len(best_i)] = best_i
    dd[:len(best_d)] = best_d
    return ids, dd, dims
