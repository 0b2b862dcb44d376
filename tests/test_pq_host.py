"""Host-side parts of the IVFPQ path in the C-ABI library, checked on the CPU
against the oracle: transform import and spectrum shaping (Section 4.3,
Procedures 1 and 2) from the same Gaussian draws.  These entry points do no
GPU work."""
import numpy as np
import pytest

from oracle import pq
from oracle import reference as ref
import paper_2510_00566_gb300 as pano
from paper_2510_00566_gb300 import _build

from test_pq_oracle import _golden_cases


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    pano.lib()


def test_import_roundtrip_and_rejects_bad_input():
    g = np.random.default_rng(0)
    d = 24
    T = pq.haar_from_gaussian(g.standard_normal((d, d)))
    mu = g.standard_normal(d)
    lam = np.sort(g.random(d))[::-1]
    t = pano.panorama_transform_import(T, mu, lam)
    T2, mu2, lam2 = t.export()
    assert np.array_equal(T2, T) and np.array_equal(mu2, mu) and np.array_equal(lam2, lam)
    bad = lam.copy()
    bad[3] = -1.0
    with pytest.raises(pano.LibraryError):
        pano.panorama_transform_import(T, mu, bad)
    T3 = T.copy()
    T3[0, 0] = np.nan
    with pytest.raises(pano.LibraryError):
        pano.panorama_transform_import(T3, mu, lam)


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: f"d{c[0]}L{c[1]}k{c[2]}")
def test_library_shaping_golden(case):
    """The hand-derived Robin Hood cases through the library (T = I)."""
    d, L, kappa, lam, blocks, energies = case
    t = pano.panorama_transform_import(np.eye(d), np.zeros(d), lam)
    G = np.random.default_rng(1).standard_normal((2, d, d))
    ts, got = pano.panorama_shape_transform(t, L, kappa, G)
    assert got == blocks
    _, _, v = ts.export()
    np.testing.assert_allclose(pq.level_energies(v, L), energies, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kappa", [1.0, 1.7, 4.0, 100.0])
def test_library_shaping_matches_oracle(kappa):
    """Same PCA basis and draws on both sides: the shaped transform agrees to
    rounding, blocks and expected variances exactly."""
    g = np.random.default_rng(2)
    d, L = 96, 8
    lam = np.exp(-0.05 * np.arange(d))
    O = pq.haar_from_gaussian(g.standard_normal((d, d)))
    X = (g.standard_normal((6000, d)) * np.sqrt(lam)) @ O.T + 0.5
    mu, T, lam_f = ref.pca_fit(X)
    G = g.standard_normal((2, d, d))
    Ts, vs, blocks = pq.shape_transform(T, lam_f, L, kappa, G[0], G[1])
    t = pano.panorama_transform_import(T, mu, lam_f)
    ts, got = pano.panorama_shape_transform(t, L, kappa, G)
    T2, mu2, v2 = ts.export()
    assert got == blocks
    assert np.abs(T2 - Ts).max() < 1e-10
    np.testing.assert_allclose(v2, vs, rtol=1e-12, atol=1e-15)
    assert np.array_equal(mu2, mu)
    assert np.abs(T2 @ T2.T - np.eye(d)).max() < 1e-12


def test_shaping_argument_errors():
    d = 16
    t = pano.panorama_transform_import(np.eye(d), np.zeros(d), np.ones(d))
    G = np.zeros((2, d, d))
    for L, kappa in ((3, 2.0), (4, 0.5), (4, float("nan"))):
        with pytest.raises(pano.LibraryError):
            pano.panorama_shape_transform(t, L, kappa, G)


def test_ivfpq_argument_checks_before_any_device_work():
    """Sizes the IVFPQ build and search reject on the host (no GPU needed):
    the C entry points are called directly with a null stream."""
    import ctypes
    L_ = pano.lib()

    def build(d, M, L, n=600, nlist=2, assign=None):
        t = pano.panorama_transform_import(np.eye(d), np.zeros(d), np.ones(d))
        X = np.zeros((n, d), np.float32)
        o = pano.PQBuildOpts(M=M, n_levels=L)
        if assign is not None:
            o.assign = assign.ctypes.data
        out = ctypes.c_void_p()
        return L_.panorama_build_ivfpq(t.handle, X.ctypes.data, n, nlist, ctypes.byref(o),
                                       None, ctypes.byref(out))

    for M, L in ((5, 4), (8, 3), (12, 4), (32, 64), (1, 2)):
        assert build(32, M, L) == -1, (M, L)
    assert build(130, 130, 2) == -1      # 65 subquantisers per level
    assert build(32, 16, 4, nlist=0) == -1
    assert build(32, 16, 4, n=100) == -1  # codebooks to train on fewer than 256 rows
    a = np.zeros(600, np.int32)
    assert build(32, 16, 4, assign=a) == -1  # an assignment without its centroids
    assert L_.panorama_search_pq(None, None, 0, 1, 1, None, None, 0, 0, 1.0, None) == -1
    assert L_.panorama_pq_export(None, None, None, None) == -1
    assert L_.panorama_debug_pq_encode(None, 0, 32, 5, None, None, None) == -1
