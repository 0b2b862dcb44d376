"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an invariant, a construction with a known answer, a different
library routine, or a different algorithm (Algorithm 1 vs brute force).
"""
import numpy as np
import pytest
import scipy.spatial.distance as ssd

import oracle
import synth


def rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- PCA, 4.1
def _exact_spectrum_data(d, lam, seed):
    """2d points mu +- sqrt(d lam_i) o_i: sample mean mu, covariance
    sum_i lam_i o_i o_i^T exactly (1/n normalisation)."""
    g = rng(seed)
    O, _ = np.linalg.qr(g.standard_normal((d, d)))
    mu = g.standard_normal(d)
    pts = []
    for i in range(d):
        a = np.sqrt(d * lam[i])
        pts.append(mu + a * O[:, i])
        pts.append(mu - a * O[:, i])
    return np.array(pts), O, mu


def test_pca_recovers_constructed_spectrum():
    d = 12
    lam = np.array([9.0, 7.5, 6.0, 4.0, 3.0, 2.5, 2.0, 1.0, 0.5, 0.25, 0.1,
                    0.01])
    X, O, mu = _exact_spectrum_data(d, lam, 7)
    mu_o, T, lam_o = oracle.pca_fit(X)
    np.testing.assert_allclose(mu_o, mu, atol=1e-12)
    np.testing.assert_allclose(lam_o, lam, rtol=1e-10, atol=1e-12)
    # rows of T are the generating axes up to sign, in eigenvalue order
    overlap = np.abs(T @ O)
    np.testing.assert_allclose(overlap, np.eye(d), atol=1e-8)


def test_pca_orthogonal_and_distance_preserving():
    g = rng(3)
    X = g.standard_normal((500, 40)) @ g.standard_normal((40, 40))
    mu, T, lam = oracle.pca_fit(X)
    assert np.linalg.norm(T.T @ T - np.eye(40)) < 1e-10
    assert np.all(np.diff(lam) <= 0)
    a, b = X[:50], X[50:100]
    ta, tb = oracle.transform(T, mu, a), oracle.transform(T, mu, b)
    lhs = np.sum((ta - tb) ** 2, axis=1)
    rhs = np.sum((a - b) ** 2, axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_ky_fan_tail_optimality():
    """Appendix A: the PCA basis minimises the mean tail energy at every m;
    the minimum is sum_{j>m} lambda_j."""
    g = rng(11)
    d = 24
    X = g.standard_normal((3000, d)) * np.exp(-0.1 * np.arange(d))
    X = X @ np.linalg.qr(g.standard_normal((d, d)))[0].T
    mu, T, lam = oracle.pca_fit(X)
    Xc = X - mu
    tails_pca = np.mean(np.cumsum((Xc @ T.T)[:, ::-1] ** 2, axis=1)[:, ::-1],
                        axis=0)
    expect = np.cumsum(lam[::-1])[::-1]
    np.testing.assert_allclose(tails_pca, expect, rtol=1e-9)
    for basis in (np.eye(d), np.linalg.qr(g.standard_normal((d, d)))[0].T):
        tails = np.mean(np.cumsum((Xc @ basis.T)[:, ::-1] ** 2,
                                  axis=1)[:, ::-1], axis=0)
        assert np.all(tails[1:] >= expect[1:] - 1e-9)


def test_spectrum_recovery_and_alpha_on_128d_workload():
    """lambda_i = exp(-0.05 i): a 20k-sample PCA recovers the spectrum within
    sampling error, and E(m) ~ exp(-alpha m / d) fits with MAE < 0.04
    (Section 5 fit quality); alpha ~ 0.05 * 128 = 6.4."""
    s = synth.scaled(1, n=20_000, n_queries=1)
    w = synth.generate(s)
    mu, T, lam = oracle.pca_fit(w.X.numpy())
    true = w.eigvals.numpy()
    tol = 6 * np.sqrt(2.0 / 20_000) * true + 1e-4
    assert np.all(np.abs(lam - true) <= tol)
    alpha, mae = oracle.fit_alpha(lam)
    assert mae < 0.04
    assert 5.5 < alpha < 7.5


def test_fit_alpha_recovers_an_exact_exponential():
    """lambda_i = exp(-beta i) with beta d = 50: E(m) equals exp(-50 m / d)
    up to exp(-50) ~ 2e-22, so the fit must return alpha = 50 to 1e-6 and a
    vanishing error."""
    d, beta = 1000, 0.05
    alpha, mae = oracle.fit_alpha(np.exp(-beta * np.arange(d)))
    assert abs(alpha - beta * d) < 1e-6 * beta * d, alpha
    assert mae < 1e-9


def test_fit_alpha_least_squares_optimum_by_hand():
    """Two levels (d = 2): E = (1, r, 0).  The squared error of exp(-a m / 2)
    over m = 0..2 is (r - u)^2 + u^4 with u = exp(-a / 2); it is least where
    2 u^3 + u - r = 0.  Taking u = 0.35 gives r = 0.43575, i.e. the spectrum
    (0.56425, 0.43575), alpha = -2 ln 0.35, and the mean absolute error over
    the three points (0 + 2u^3 + u^2) / 3 = 0.0694166...  A fit of log E, or
    an error averaged over m = 1..d only, gives other numbers."""
    u = 0.35
    r = 2 * u ** 3 + u
    alpha, mae = oracle.fit_alpha(np.array([1.0 - r, r]))
    assert abs(alpha - (-2.0 * np.log(u))) < 1e-6, alpha
    assert abs(mae - (2 * u ** 3 + u ** 2) / 3) < 1e-9, mae


def test_candidate_topk_golden():
    """tests/golden/refine_candidates.txt: hand-derived answers of Problem 1
    over explicit candidate lists with repeats, -1 padding, ties and an empty
    set (the refine workload's reading of a candidate list)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "refine_candidates.txt")
    X, cases = {}, []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("X "):
            f = line.split()
            X[int(f[1])] = (float(f[2]), float(f[3]))
        else:
            q, cand, k, ids, dists = [p.split() for p in line[2:].split("|")]
            cases.append((np.array(q, float), np.array(cand, np.int64), int(k[0]),
                          np.array(ids, np.int64), np.array([float(v) for v in dists])))
    Xa = np.array([X[i] for i in range(len(X))], dtype=np.float32)
    assert len(cases) == 4
    for q, cand, k, ids, dists in cases:
        gi, gd = oracle.candidate_topk(Xa, q[None].astype(np.float32), cand[None], k)
        np.testing.assert_array_equal(gi[0], ids)
        np.testing.assert_array_equal(gd[0], dists)


def test_energy_fraction_closed_form():
    # geometric spectrum: E(m) = r^m (1 - r^(d-m)) / (1 - r^d)
    d, r = 50, 0.9
    lam = r ** np.arange(d)
    E = oracle.energy_fraction(lam)
    m = np.arange(d + 1)
    np.testing.assert_allclose(E, (r ** m - r ** d) / (1 - r ** d),
                               rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------- bounds, Eq. 1-4
def test_bounds_hand_example():
    """d = 4, levels (2, 2): T(q) = (3, 0, 4, 0), T(x) = (0, 0, 0, 5).
    ||q||^2 = ||x||^2 = 25, exact distance 9 + 16 + 25 = 50.
    l=0: p=0, C = sqrt(25*25) = 25 -> LB = 0, UB = 100.
    l=1: p=0, tails 16 and 25, C = 20 -> LB = 10, UB = 90.
    l=2: LB = UB = 50."""
    tq = np.array([3.0, 0.0, 4.0, 0.0])
    tx = np.array([[0.0, 0.0, 0.0, 5.0]])
    m = oracle.level_thresholds(4, [2, 2])
    LB, UB, A, C = oracle.bounds(tq, tx, m)
    np.testing.assert_array_equal(LB[0], [0.0, 10.0, 50.0])
    np.testing.assert_array_equal(UB[0], [100.0, 90.0, 50.0])
    LBe, _, _, _ = oracle.bounds(tq, tx, m, eps=0.5)
    np.testing.assert_array_equal(LBe[0], [25.0, 30.0, 50.0])


def test_bounds_level0_is_reverse_triangle_and_levelL_exact():
    g = rng(5)
    d = 64
    tq = g.standard_normal(d) * 2
    tX = g.standard_normal((200, d))
    m = oracle.level_thresholds(d, [8] * 8)
    LB, UB, _, _ = oracle.bounds(tq, tX, m)
    nq = np.linalg.norm(tq)
    nx = np.linalg.norm(tX, axis=1)
    np.testing.assert_allclose(LB[:, 0], (nq - nx) ** 2, rtol=1e-10,
                               atol=1e-9)
    np.testing.assert_allclose(UB[:, 0], (nq + nx) ** 2, rtol=1e-12)
    exact = ssd.cdist(tq[None, :], tX, "sqeuclidean")[0]
    np.testing.assert_allclose(LB[:, -1], exact, rtol=1e-11, atol=1e-10)
    np.testing.assert_allclose(UB[:, -1], exact, rtol=1e-11, atol=1e-10)


def test_gap_identity_and_monotone_tightening():
    """Appendix A gap identity: exact - LB_eps^m = 2 C^m (eps - rho_m) with
    rho_m = pi_m / C^m, pi_m the tail inner product; so LB <= exact <= UB."""
    g = rng(9)
    d = 96
    tq = g.standard_normal(d) * np.exp(-0.02 * np.arange(d))
    tX = g.standard_normal((300, d)) * np.exp(-0.02 * np.arange(d))
    m = oracle.level_thresholds(d, [12] * 8)
    exact = ssd.cdist(tq[None, :], tX, "sqeuclidean")[0]
    for eps in (1.0, 0.7):
        LB, UB, A, C = oracle.bounds(tq, tX, m, eps=eps)
        for l in range(len(m)):
            pi = tX[:, m[l]:] @ tq[m[l]:]
            gap = exact - LB[:, l]
            np.testing.assert_allclose(gap, 2 * (eps * C[:, l] - pi),
                                       atol=1e-9)
            rho = np.where(C[:, l] > 0, pi / np.maximum(C[:, l], 1e-300), 0)
            assert np.all(np.abs(rho) <= 1 + 1e-12)
    LB, UB, _, _ = oracle.bounds(tq, tX, m)
    assert np.all(LB <= exact[:, None] + 1e-9)
    assert np.all(UB >= exact[:, None] - 1e-9)
    assert np.all(np.diff(LB, axis=1) >= -1e-9)
    assert np.all(np.diff(UB, axis=1) <= 1e-9)


# ------------------------------------------------------------ top-k, assign
def test_topk_lattice_with_ties():
    X = np.array([[1, 0], [0, 1], [1, 1], [2, 0], [-1, 0]], dtype=np.float32)
    q = np.zeros(2, dtype=np.float32)
    d = oracle.exact_sqdist(q, X)
    ids, dd = oracle.topk(d, np.arange(5), 4)
    assert ids.tolist() == [0, 1, 4, 2]
    assert dd.tolist() == [1.0, 1.0, 1.0, 2.0]
    ids, dd = oracle.topk(d, np.arange(5), 7)
    assert ids.tolist() == [0, 1, 4, 2, 3, -1, -1]
    assert dd[-1] == np.inf
    # the C brute force on the same lattice, one list holding every row
    ci, cd = oracle.ivf_topk(X, q[None, :], np.array([0, 5]),
                             np.arange(5), [np.array([0])], np.array([7]))
    assert ci[0].tolist() == [0, 1, 4, 2, 3, -1, -1]
    assert cd[0, :5].tolist() == [1.0, 1.0, 1.0, 2.0, 4.0]


def test_ivf_search_matches_scipy():
    g = rng(21)
    X = g.standard_normal((3000, 16)).astype(np.float32)
    Q = g.standard_normal((40, 16)).astype(np.float32)
    C = X[g.choice(3000, 20, replace=False)].astype(np.float64)
    res = oracle.ivf_search(X, Q, C, nprobe=4, k=7, threads=3)
    D = ssd.cdist(X.astype(np.float64), C, "sqeuclidean")
    lists = np.argmin(D, axis=1)
    np.testing.assert_array_equal(res["lists"], lists)
    DQ = ssd.cdist(Q.astype(np.float64), C, "sqeuclidean")
    DX = ssd.cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for i in range(40):
        pr = np.lexsort((np.arange(20), DQ[i]))[:4]
        assert res["probes"][i].tolist() == pr.tolist()
        cand = np.nonzero(np.isin(lists, pr))[0]
        order = cand[np.lexsort((cand, DX[i, cand]))][:7]
        assert res["ids"][i].tolist() == order.tolist()
        np.testing.assert_allclose(res["dists"][i], DX[i, order], rtol=1e-12)


def test_assign_ties_go_to_lowest_centroid():
    C = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 3.0]])
    X = np.array([[0.0, 0.0], [0.0, 2.0], [0.5, 0.0]])
    lists, gap = oracle.assign(X, C)
    assert lists.tolist() == [0, 2, 0]
    assert gap[0] == 0.0


# ---------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("B", [1, 7, 64, 10_000])
@pytest.mark.parametrize("k", [1, 10, 600])
def test_refine_equals_brute_force(B, k):
    g = rng(100 + B + k)
    d = 48
    lam = np.exp(-0.08 * np.arange(d))
    X = g.standard_normal((500, d)) * np.sqrt(lam)
    q = g.standard_normal(d) * np.sqrt(lam)
    mu, T, _ = oracle.pca_fit(X)
    tX, tq = oracle.transform(T, mu, X), oracle.transform(T, mu, q[None])[0]
    m = oracle.level_thresholds(d, [6] * 8)
    ids = np.arange(500)
    ri, rd, rho = oracle.refine(tq, tX, ids, m, k, B=B)
    bi, bd = oracle.topk(oracle.exact_sqdist(q, X), ids, k)
    assert ri.tolist() == bi.tolist()
    np.testing.assert_allclose(rd, bd, rtol=1e-9)
    assert np.all(rho >= m[1]) and np.all(rho <= d)


def test_refine_single_level_and_identity_transform():
    """L = 1 reduces Algorithm 1 to brute-force kNN; T = I (raw axes, Section
    7.4) returns the same answer with more coordinates read."""
    g = rng(77)
    d = 32
    X = g.standard_normal((400, d)) * np.exp(-0.1 * np.arange(d))
    X = X @ np.linalg.qr(g.standard_normal((d, d)))[0].T
    q = X[:1] + 0.01
    ids = np.arange(400)
    bi, _ = oracle.topk(oracle.exact_sqdist(q[0], X), ids, 5)
    m1 = oracle.level_thresholds(d, [d])
    ri, _, rho1 = oracle.refine(q[0], X, ids, m1, 5, B=64)
    assert ri.tolist() == bi.tolist() and np.all(rho1 == d)
    m = oracle.level_thresholds(d, [4] * 8)
    ri, _, rho_raw = oracle.refine(q[0], X, ids, m, 5, B=64)
    assert ri.tolist() == bi.tolist()
    mu, T, _ = oracle.pca_fit(X)
    ri, _, rho_pca = oracle.refine(oracle.transform(T, mu, q)[0],
                                   oracle.transform(T, mu, X), ids, m, 5, B=64)
    assert ri.tolist() == bi.tolist()
    assert rho_pca.mean() < rho_raw.mean()


def test_dims_scanned_plausible_on_128d_workload():
    """Table 2 / Proposition 5.1: exhaustive-search fraction of dimensions
    scanned tracks 1/alpha; here a plausibility band of a factor 3."""
    s = synth.scaled(1, n=20_000, n_queries=20)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    mu, T, lam = oracle.pca_fit(X)
    alpha, _ = oracle.fit_alpha(lam)
    tX = oracle.transform(T, mu, X)
    m = oracle.level_thresholds(128, [16] * 8)
    fr = []
    for i in range(20):
        tq = oracle.transform(T, mu, Q[i:i + 1])[0]
        _, _, rho = oracle.refine(tq, tX, np.arange(len(X)), m, 10, B=1024)
        fr.append(rho.mean() / 128)
    phi = float(np.mean(fr))
    assert 1 / (3 * alpha) < phi < 3 / alpha, (phi, 1 / alpha)


def test_alg1_golden_trace():
    """tests/golden/alg1_trace.txt (written by make_golden.py from the oracle;
    each row hand-checkable from Eq. 3) still matches, and its hand facts hold:
    candidate 2 is pruned at level 1, candidate 3 at level 2, and the tie at
    distance 1 between candidates 1 and 4 goes to the lower id."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "alg1_trace.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "mk", os.path.join(os.path.dirname(path), "make_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    m = oracle.level_thresholds(4, mk.M)
    ids, dists, rho = oracle.refine(mk.TQ, mk.TX, np.arange(5), m, k=1, B=2)
    LB, UB, _, _ = oracle.bounds(mk.TQ, mk.TX, m)
    for i in range(5):
        vals = list(map(float, rows[i][1:7]))
        np.testing.assert_allclose(vals[:3], LB[i], atol=1e-6)
        np.testing.assert_allclose(vals[3:], UB[i], atol=1e-6)
        assert int(rows[i][7]) == rho[i]
    assert rows[5][0] == "topk" and int(rows[5][1]) == ids[0] == 1
    assert rho[2] == 2 and LB[2, 1] == 160.0 and LB[3, 2] == 64.0
