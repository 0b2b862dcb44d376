"""Pins of the IVFPQ oracle (oracle/pq.py) against hand-derived values, closed
forms, textbook special cases and brute force: spectrum shaping (Section 4.3,
Procedures 1 and 2), the PQ encoder, asymmetric distances, the Eq. 3 bounds
in partial-distance form and Algorithm 1 over asymmetric distances."""
import os

import numpy as np
import pytest

from oracle import pq
from oracle import reference as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "robin_hood.txt")


def _golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, lam, blocks, energies = [p.strip() for p in line.split("|")]
        d, L, kappa = head.split()
        bl = [] if blocks == "-" else [tuple(int(v) for v in b.split(":")) for b in blocks.split()]
        cases.append((int(d), int(L), float(kappa), np.array(lam.split(), float), bl,
                      np.array(energies.split(), float)))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: f"d{c[0]}L{c[1]}k{c[2]}")
def test_robin_hood_golden(case):
    d, L, kappa, lam, blocks, energies = case
    G = np.random.default_rng(0).standard_normal((d, d))
    R, v, got = pq.robin_hood(lam, L, kappa, G)
    assert got == blocks
    np.testing.assert_allclose(pq.level_energies(v, L), energies, rtol=1e-12, atol=1e-12)
    assert np.abs(R.T @ R - np.eye(d)).max() < 1e-12


def test_haar_sampler_moments():
    """Q of a Gaussian matrix with diag(R) > 0 is Haar: each column is uniform
    on the sphere, so E[Q_ij] = 0, E[Q_ij^2] = 1/n, E[Q_ij^4] = 3/(n(n+2)).
    Without the sign correction E[Q_11] is far from 0 (LAPACK's Householder
    QR returns R_11 < 0 for every input, making Q_11 = -|.|)."""
    n, trials = 4, 4000
    g = np.random.default_rng(1)
    Q = np.stack([pq.haar_from_gaussian(g.standard_normal((n, n))) for _ in range(trials)])
    assert np.abs(np.einsum("tij,tik->tjk", Q, Q) - np.eye(n)).max() < 1e-12
    m1, m2, m4 = Q.mean(0), (Q ** 2).mean(0), (Q ** 4).mean(0)
    se2 = np.sqrt(3 / (n * (n + 2)) / trials)
    assert np.abs(m1).max() < 5 * np.sqrt(1 / n / trials)
    assert np.abs(m2 - 1 / n).max() < 5 * se2
    assert np.abs(m4 - 3 / (n * (n + 2))).max() < 0.02
    # the same draws without the correction are visibly biased
    raw = np.stack([np.linalg.qr(g.standard_normal((n, n)))[0] for _ in range(trials)])
    assert abs(raw[:, 0, 0].mean()) > 10 * np.sqrt(1 / n / trials)


@pytest.mark.parametrize("kappa", [1.0, 2.0, 4.0])
def test_shaping_cap_conservation_and_minimal_suffix(kappa):
    d, L = 64, 8
    b = d // L
    lam = np.exp(-0.08 * np.arange(d))
    g = np.random.default_rng(2)
    G1, G2 = g.standard_normal((d, d)), g.standard_normal((d, d))
    T = pq.haar_from_gaussian(g.standard_normal((d, d)))
    R, v, blocks = pq.robin_hood(lam, L, kappa, G1)
    cap = kappa * lam.sum() / L
    E = pq.level_energies(v, L)
    assert E.max() <= cap * (1 + 1e-9)
    assert abs(v.sum() - lam.sum()) < 1e-12 * lam.sum()
    for a, n in blocks:  # the suffix is the smallest that meets the cap
        s = n - b
        assert b * lam[a:a + n].sum() / n <= cap * (1 + 1e-9)
        if s > 1:
            assert b * lam[a:a + n - 1].sum() / (n - 1) > cap
    # disjoint blocks; outside them R is the identity
    mask = np.ones(d, bool)
    for a, n in blocks:
        mask[a:a + n] = False
    assert np.array_equal(R[np.ix_(mask, mask)], np.eye(mask.sum()))
    Ts, vs, _ = pq.shape_transform(T, lam, L, kappa, G1, G2)
    assert np.abs(Ts @ Ts.T - np.eye(d)).max() < 1e-12
    np.testing.assert_allclose(pq.level_energies(vs, L), E, rtol=1e-12)


def test_no_rotation_when_the_cap_holds():
    d, L = 32, 4
    lam = np.exp(-0.1 * np.arange(d))
    E = pq.level_energies(lam, L)
    kappa = E.max() / E.mean() * 1.0001
    R, v, blocks = pq.robin_hood(lam, L, kappa, np.random.default_rng(3).standard_normal((d, d)))
    assert blocks == [] and np.array_equal(R, np.eye(d)) and np.array_equal(v, lam)


def test_expected_energies_match_monte_carlo():
    """The level energies Procedure 1 tracks are expectations over the Haar
    draw: averaging the realised diag(R Lambda R^T) over many draws gives
    them; Procedure 2 leaves each level's realised energy unchanged."""
    d, L, trials = 16, 4, 3000
    lam = np.exp(-0.3 * np.arange(d))
    g = np.random.default_rng(4)
    acc = np.zeros(L)
    for _ in range(trials):
        G1 = g.standard_normal((d, d))
        R, v, _ = pq.robin_hood(lam, L, 1.0, G1)
        cov = R @ np.diag(lam) @ R.T
        realised = pq.level_energies(np.diag(cov), L)
        acc += realised
        U = pq.isotropize(d, L, g.standard_normal((d, d)))
        cov2 = U @ cov @ U.T
        np.testing.assert_allclose(pq.level_energies(np.diag(cov2), L), realised, rtol=1e-10)
    np.testing.assert_allclose(acc / trials, pq.level_energies(v, L), rtol=0.03)


def test_encoder_matches_fp64_argmin_and_breaks_ties_low():
    g = np.random.default_rng(5)
    M, ksub, dsub, n = 6, 256, 3, 500
    cb = g.standard_normal((M, ksub, dsub)).astype(np.float32)
    X = g.standard_normal((n, M * dsub)).astype(np.float32)
    codes = pq.pq_encode32(X, cb)
    for m in range(M):
        d64 = ((X[:, None, m * dsub:(m + 1) * dsub].astype(np.float64)
                - cb[m][None].astype(np.float64)) ** 2).sum(-1)
        best = d64.min(1)
        got = d64[np.arange(n), codes[:, m]]
        assert np.all(got <= best * (1 + 1e-5) + 1e-30)
        srt = np.sort(d64, axis=1)
        clear = srt[:, 1] - srt[:, 0] > 1e-5 * srt[:, 1]
        assert np.array_equal(codes[clear, m], d64.argmin(1)[clear])
    cb2 = cb.copy()
    cb2[0, 7] = cb2[0, 3]  # a duplicated codeword: the lower index wins
    X2 = np.tile(cb2[0, 3], (1, M)).astype(np.float32)
    assert pq.pq_encode32(X2, cb2)[0, 0] == 3


def test_adc_is_the_exact_distance_when_codebooks_hold_the_data():
    g = np.random.default_rng(6)
    n, M, dsub = 200, 8, 4
    X = g.standard_normal((n, M * dsub))
    cb = np.empty((M, 256, dsub), np.float32)
    cb[:, :n] = X.astype(np.float32).reshape(n, M, dsub).transpose(1, 0, 2)
    cb[:, n:] = 1e3 + g.standard_normal((M, 256 - n, dsub))
    codes = pq.pq_encode32(X.astype(np.float32), cb)
    assert np.array_equal(codes, np.tile(np.arange(n)[:, None], (1, M)))
    q = g.standard_normal(M * dsub)
    np.testing.assert_allclose(pq.adc_dists(q, codes, cb),
                               ref.exact_sqdist(q, X.astype(np.float32).astype(np.float64)),
                               rtol=1e-12)


def test_pq_bounds_enclose_adc_and_equal_eq3():
    g = np.random.default_rng(7)
    d, L = 48, 6
    m = ref.level_thresholds(d, [d // L] * L)
    lam = np.exp(-0.1 * np.arange(d))
    rq = g.standard_normal(d) * np.sqrt(lam)
    xh = g.standard_normal((300, d)) * np.sqrt(lam)
    exact = ((rq[None] - xh) ** 2).sum(1)
    lb, ub = pq.pq_level_bounds(rq, xh, m)
    assert np.all(lb <= exact[None] * (1 + 1e-12) + 1e-12)
    assert np.all(ub >= exact[None] * (1 - 1e-12) - 1e-12)
    np.testing.assert_allclose(lb[-1], exact, rtol=1e-12)
    np.testing.assert_allclose(ub[-1], exact, rtol=1e-12)
    LB3, UB3, _, _ = ref.bounds(rq, xh, m)  # Eq. 3: A - 2C, A + 2C
    np.testing.assert_allclose(lb, LB3[:, 1:].T, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ub, UB3[:, 1:].T, rtol=1e-9, atol=1e-9)
    assert np.all(np.diff(lb, axis=0) >= -1e-9)  # tightening with depth
    assert np.all(np.diff(ub, axis=0) <= 1e-9)


@pytest.mark.parametrize("k,B", [(1, 7), (10, 64), (50, 1024)])
def test_algorithm1_over_adc_equals_plain_topk(k, B):
    g = np.random.default_rng(8 + k)
    d, L, M = 32, 4, 16
    m = ref.level_thresholds(d, [d // L] * L)
    lam = np.exp(-0.15 * np.arange(d))
    cb = (g.standard_normal((M, 256, d // M)) * np.sqrt(lam).reshape(M, d // M)[:, None, :]
          ).astype(np.float32)
    rq_l, xh_l, id_l, all_d, all_i = [], [], [], [], []
    start = 0
    for n in (40, 300, 3):
        codes = g.integers(0, 256, (n, M)).astype(np.uint8)
        rq = g.standard_normal(d) * np.sqrt(lam)
        xh = pq.pq_reconstruct(codes, cb)
        ids = np.arange(start, start + n)
        start += n
        rq_l.append(rq)
        xh_l.append(xh)
        id_l.append(ids)
        all_d.append(pq.adc_dists(rq, codes, cb))
        all_i.append(ids)
    ids, dd, dims = pq.ivfpq_panorama(rq_l, xh_l, id_l, m, k, B)
    D, I = np.concatenate(all_d), np.concatenate(all_i)
    order = np.lexsort((I, D))[:k]
    assert np.array_equal(ids[:order.size], I[order])
    np.testing.assert_allclose(dd[:order.size], D[order], rtol=1e-12)
    assert dims <= D.size * d


def test_ivfpq_search_reduces_to_ivf_flat_when_codes_are_exact():
    """With T = I, mu = 0 and codebooks that hold every residual exactly, the
    asymmetric distance is the exact distance, so the IVFPQ answer is the
    IVFFlat answer (a residual sign or centroid error would break this)."""
    g = np.random.default_rng(9)
    d, M, nlist = 16, 4, 3
    dsub = d // M
    X = (g.standard_normal((240, d)) + 3 * g.integers(0, 3, (240, 1))).astype(np.float32)
    C = np.stack([X[i::3].mean(0) for i in range(nlist)]).astype(np.float32)
    lists, _ = ref.assign(X, C)
    R = X.astype(np.float64) - C[lists].astype(np.float64)
    cb = np.full((M, 256, dsub), 1e4, np.float32)
    cb[:, :240] = R.astype(np.float32).reshape(240, M, dsub).transpose(1, 0, 2)
    codes = np.tile(np.arange(240)[:, None], (1, M)).astype(np.uint8)
    Q = g.standard_normal((20, d)).astype(np.float32) * 3
    got = pq.ivfpq_search(Q, np.eye(d), np.zeros(d), C, lists, cb, codes, 2, 7)
    # X - C in FP32 may differ from the FP64 residual by one rounding: compare
    # with the FP64 distance of the reconstructed points c + r32
    Xr = C[lists].astype(np.float64) + pq.pq_reconstruct(codes, cb)
    want = ref.ivf_search(Xr.astype(np.float64), Q, C, 2, 7, lists_of_vector=lists)
    assert np.array_equal(got["ids"], want["ids"])
    np.testing.assert_allclose(got["dists"], want["dists"], rtol=1e-9)


def test_procedure2_leaves_every_level_bound_unchanged():
    """A rotation inside each level keeps every level's head distance and
    tail energy, so the bounds of Eq. 3 are the same before and after
    Procedure 2 (only the coordinates within a level mix)."""
    g = np.random.default_rng(10)
    d, L = 40, 5
    m = ref.level_thresholds(d, [d // L] * L)
    lam = np.exp(-0.1 * np.arange(d))
    q = g.standard_normal(d) * np.sqrt(lam)
    X = g.standard_normal((200, d)) * np.sqrt(lam)
    U = pq.isotropize(d, L, g.standard_normal((d, d)))
    lb0, ub0 = pq.pq_level_bounds(q, X, m)
    lb1, ub1 = pq.pq_level_bounds(U @ q, X @ U.T, m)
    np.testing.assert_allclose(lb1, lb0, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ub1, ub0, rtol=1e-9, atol=1e-9)


def test_robin_hood_trades_pruning_for_pq_balance():
    """Section 4.3's trade: on a fast-decaying spectrum, kappa = 1 moves energy
    out of the leading level, so Algorithm 1 reads more coordinates than in
    the PCA basis, while product quantisation with the same bit budget
    reconstructs the vectors better (equal-bit codebooks fit a flat profile)."""
    g = np.random.default_rng(11)
    d, L, M, n = 32, 4, 8, 3000
    lam = np.exp(-0.2 * np.arange(d))
    X = g.standard_normal((n, d)) * np.sqrt(lam)  # already in its PCA basis
    q = g.standard_normal((20, d)) * np.sqrt(lam)
    m = ref.level_thresholds(d, [d // L] * L)
    G = g.standard_normal((2, d, d))
    Ts, vs, blocks = pq.shape_transform(np.eye(d), lam, L, 1.0, G[0], G[1])
    assert blocks and pq.level_energies(vs, L).max() <= lam.sum() / L * (1 + 1e-9)

    def dims(T):
        tot = 0
        for i in range(len(q)):
            tq, tX = T @ q[i], X @ T.T
            _, _, r = ref.refine(tq, tX, np.arange(n), m, 10, B=256)
            tot += r.sum()
        return tot

    assert dims(Ts) > dims(np.eye(d))

    def pq_mse(T):
        R = X @ T.T
        cb = pq.pq_train(R[:2000], M, iters=6, seed=3)
        codes = pq.pq_encode32(R.astype(np.float32), cb)
        return float(((pq.pq_reconstruct(codes, cb) - R) ** 2).sum(1).mean())

    assert pq_mse(Ts) < pq_mse(np.eye(d))


def test_pq_train_lloyd_properties():
    """pq_train is Lloyd's algorithm per subspace: on two well-separated blobs
    with two codewords its fixed point is the pair of blob means (closed
    form), and more iterations never raise the quantisation error (each
    step cannot increase the objective)."""
    g = np.random.default_rng(12)
    A = g.standard_normal((500, 2)) * 0.1 + 10.0
    B = g.standard_normal((700, 2)) * 0.1 - 10.0
    X = np.concatenate([A, B])
    cb = pq.pq_train(X, 1, ksub=2, iters=10, seed=1)[0].astype(np.float64)
    cb = cb[np.argsort(cb[:, 0])]
    np.testing.assert_allclose(cb, np.stack([B.mean(0), A.mean(0)]), atol=1e-6)
    Y = g.standard_normal((4000, 8)) * np.exp(-0.2 * np.arange(8))
    errs = []
    for it in (0, 1, 3, 8):
        cb = pq.pq_train(Y, 2, iters=it, seed=2)
        codes = pq.pq_encode32(Y.astype(np.float32), cb)
        errs.append(((pq.pq_reconstruct(codes, cb) - Y) ** 2).sum(1).mean())
    assert all(b <= a * (1 + 1e-6) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0]
