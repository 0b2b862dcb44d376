"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/*.h declares, reports errors, and its host-only PCA fit agrees
with the oracle (no GPU compute is called here)."""
import ctypes
import re

import numpy as np
import pytest

import oracle
import paper_2510_00566_gb300 as pano
from paper_2510_00566_gb300 import _build

HEADER = _build.os.path.join(_build.ROOT, "include", "panorama.h")


@pytest.fixture(scope="module")
def L():
    _build.build()
    return pano.lib()


def declared_functions():
    import glob
    text = "".join(open(h).read() for h in
                   sorted(glob.glob(_build.os.path.join(_build.ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(panorama_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
        assert n in pano.SIGNATURES, f"binding lacks {n}"


def test_version_and_error_reporting(L):
    assert b"sm_103a" in L.panorama_version()
    out = ctypes.c_void_p()
    rc = L.panorama_fit_transform(None, 0, 0, None, ctypes.byref(out))
    assert rc == -1
    assert L.panorama_last_error() != b""
    assert L.panorama_search(None, None, 0, None, 1, None, 1, 1, None, None,
                             None) == -1


def test_host_pca_fit_matches_oracle(L):
    g = np.random.default_rng(4)
    d = 48
    lam = np.exp(-0.08 * np.arange(d))
    O = np.linalg.qr(g.standard_normal((d, d)))[0]
    X = (g.standard_normal((4000, d)) * np.sqrt(lam)) @ O.T + 0.3
    X = X.astype(np.float32)
    t = pano.panorama_fit_transform(X, fit_sample=4000)
    T, mu, ev = t.export()
    mu_o, T_o, lam_o = oracle.pca_fit(X.astype(np.float64))
    np.testing.assert_allclose(mu, mu_o, atol=1e-12)
    np.testing.assert_allclose(ev, lam_o, rtol=1e-9, atol=1e-13)
    assert np.linalg.norm(T @ T.T - np.eye(d)) < 1e-10
    # same axes up to sign (eigenvalues are distinct here)
    np.testing.assert_allclose(np.abs(np.sum(T * T_o, axis=1)), 1.0, atol=1e-7)


def test_host_pca_fit_on_constructed_spectrum(L):
    g = np.random.default_rng(8)
    d = 16
    lam = np.linspace(5.0, 0.2, d)
    O = np.linalg.qr(g.standard_normal((d, d)))[0]
    pts = []
    for i in range(d):
        a = np.sqrt(d * lam[i])
        pts += [a * O[:, i], -a * O[:, i]]
    X = np.array(pts, dtype=np.float32)
    t = pano.panorama_fit_transform(X)
    T, mu, ev = t.export()
    # the FP32 rounding of the constructed points perturbs the spectrum ~1e-7
    np.testing.assert_allclose(ev, lam, rtol=1e-5)
    np.testing.assert_allclose(np.abs(T @ O), np.eye(d), atol=1e-4)
    assert all(T[r, np.argmax(np.abs(T[r]))] > 0 for r in range(d))


def test_device_error_word_maps_to_status(L):
    """The serving loop retires each batch with the status of its device
    error word: a bounded wait that gave up -> PANO_ETIMEOUT, an input the
    search had to clamp or cannot represent -> PANO_EINVAL, a capacity note
    alone -> success."""
    f = L.panorama_status_of_device_error
    assert f(0) == 0
    assert f(1) == -4 and f(1 | 2) == -4 and f(1 | 4) == -4
    assert f(4) == -1 and f(4 | 2) == -1
    assert f(2) == 0
