"""A CPU model of the IVFPQ search's FP32 arithmetic, checking the rounding
allowance of its pruning test (Eq. 3 in partial-distance form, margined).

The model follows the operation order the library documents for an IVFPQ
search (include/panorama_pq.h): each subvector term sum_j fl(fl(r_j - c_j)^2)
left to right, terms of a level added in subquantiser order, level sums added
in level order; tail norms sqrt of FP64 sums rounded to FP32; the test
(1 - gamma) * (D_head + max(0, |s_q - s_x| - 8u (s_q + s_x))^2) > tau.  A
candidate may only be dropped when its computed distance exceeds tau, so the
margined lower bound must never exceed the computed distance.  The hardest
case is a reconstruction whose tail is a positive multiple of the residual's
tail: there the Cauchy-Schwarz bound is exact and only rounding separates it
from the distance.  (The GPU tests check the kernels themselves: a pruned
search returns the plain scan's result bit for bit.)"""
import numpy as np
import pytest

U = 2.0 ** -24
f32 = np.float32


def gamma(n):
    return n * U / (1 - n * U)


def model(r, X, L, ML, dsub, fused):
    """Computed level prefix sums P (n, L), tails s_x (n, L), s_q (L), and the
    lower bound of each level before its tail test (n, L - 1)."""
    n, d = X.shape
    M = d // dsub
    t = (r[None, :] - X).astype(f32)           # fl(r_j - c_j)
    sq_t = (t * t).astype(f32)                 # fl(t^2)
    e = np.zeros((n, M), f32)
    for m in range(M):                         # left to right within a term
        acc = sq_t[:, m * dsub]
        for j in range(1, dsub):
            acc = (acc + sq_t[:, m * dsub + j]).astype(f32)
        e[:, m] = acc
    P = np.zeros((n, L), f32)
    run = np.zeros(n, f32)
    for l in range(L):
        S = e[:, l * ML]
        for mm in range(1, ML):
            S = (S + e[:, l * ML + mm]).astype(f32)
        run = (run + S).astype(f32)
        P[:, l] = run
    b = d // L
    r64, X64 = r.astype(np.float64), X.astype(np.float64)
    sq = np.array([np.sqrt((r64[(l + 1) * b:] ** 2).sum()) for l in range(L)]).astype(f32)
    sx = np.stack([np.sqrt((X64[:, (l + 1) * b:] ** 2).sum(1)) for l in range(L)], 1).astype(f32)
    erel = f32(8 * U)
    lo64 = 1 - gamma(L + ML + dsub + 6)
    lo = f32(lo64)
    if float(lo) > lo64:
        lo = np.nextafter(lo, f32(0))
    lbs = np.zeros((n, L - 1), f32)
    for l in range(L - 1):
        diff = np.abs((sq[l] - sx[:, l]).astype(f32))
        ssum = (sq[l] + sx[:, l]).astype(f32)
        if fused:   # fl(|d| - erel * s) with one rounding
            gap = (diff.astype(np.float64) - float(erel) * ssum.astype(np.float64)).astype(f32)
        else:
            gap = (diff - (erel * ssum).astype(f32)).astype(f32)
        gap = np.maximum(gap, f32(0))
        # fma(gap, gap, P): the FP64 value of gap^2 + P is exact or within
        # FP64 rounding, then one rounding to FP32
        lb = (gap.astype(np.float64) ** 2 + P[:, l].astype(np.float64)).astype(f32)
        lbs[:, l] = (lb * lo).astype(f32)
    return P, lbs


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("dsub,ML,L", [(2, 30, 16), (1, 12, 4), (4, 6, 8), (8, 2, 3)])
def test_margined_bound_never_exceeds_the_computed_distance(dsub, ML, L, fused):
    g = np.random.default_rng(dsub * 100 + ML + L)
    d = dsub * ML * L
    b = d // L
    worst = 0.0
    for trial in range(6):
        scale = 10.0 ** g.uniform(-3, 3)
        r = (g.standard_normal(d) * scale).astype(f32)
        # random reconstructions, and ones whose tail after every level is a
        # positive multiple of the residual's (Cauchy-Schwarz tight) plus a
        # near-equal copy (|s_q - s_x| ~ 0)
        Xr = (g.standard_normal((200, d)) * scale).astype(f32)
        Xt = np.empty((3 * L, d), f32)
        for l in range(L):
            for j, lam in enumerate((0.5, 1.0 + 1e-7, 3.0)):
                x = (g.standard_normal(d) * scale).astype(f32)
                x[(l + 1) * b:] = (lam * r[(l + 1) * b:]).astype(f32)
                Xt[3 * l + j] = x
        X = np.concatenate([Xr, Xt])
        P, lbs = model(r, X, L, ML, dsub, fused)
        D = P[:, -1]
        assert np.all(lbs <= D[:, None]), (trial, np.max(lbs - D[:, None]))
        worst = max(worst, float(np.max(lbs / np.maximum(D[:, None], 1e-30))))
    # the bound is tight: for Cauchy-Schwarz-tight candidates it comes within
    # a few parts in 10^5 of the distance
    assert worst > 0.999


def test_without_the_allowance_the_bound_can_exceed_the_distance():
    """Dropping the margins (lo = 1, no 8u allowance) lets rounding push the
    bound above the computed distance on tight candidates: the allowance is
    needed, not decorative."""
    g = np.random.default_rng(7)
    dsub, ML, L = 2, 30, 16
    d = dsub * ML * L
    b = d // L
    over = 0
    for trial in range(40):
        r = (g.standard_normal(d) * 10.0 ** g.uniform(-2, 2)).astype(f32)
        X = np.empty((L, d), f32)
        for l in range(L):
            x = (g.standard_normal(d)).astype(f32) * r.std()
            x[(l + 1) * b:] = (1.7 * r[(l + 1) * b:]).astype(f32)
            X[l] = x
        t = (r[None, :] - X).astype(f32)
        e = (t * t).astype(f32).reshape(L, -1, dsub).sum(-1, dtype=f32)
        D = np.zeros(L, f32)
        for m in range(e.shape[1]):
            D = (D + e[:, m]).astype(f32)
        for l in range(L - 1):
            head = np.zeros(L, f32)
            for m in range((l + 1) * ML):
                head = (head + e[:, m]).astype(f32)
            sq = f32(np.sqrt((r[(l + 1) * b:].astype(np.float64) ** 2).sum()))
            sx = np.sqrt((X[:, (l + 1) * b:].astype(np.float64) ** 2).sum(1)).astype(f32)
            lb = (head + ((sq - sx).astype(f32)) ** 2).astype(f32)
            over += int(np.sum(lb > D))
    assert over > 0
