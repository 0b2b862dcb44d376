"""panorama_search_noalloc: the search for callers that cannot allocate
device memory while searching (their memory belongs to another allocator or
pool, or an allocation -- which can synchronize or fail under fragmentation
-- is not allowed on their path).  Its workspace is a fixed array in the
library's global memory.

The entry point is called through the C-ABI (ctypes) twice in a row, on two
different batches; both results must match panorama_search's on the same
batch within the parity tolerances used by the other GPU tests (ids equal
except at near-ties below 1e-6 relative, distances within 1e-5 relative).
The second batch differs in queries, size, nprobe, k and k_max, so what the
first call left in the shared array would show in the second result.
This file is collected last; it builds everything it needs, so it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2510_00566_gb300 as pano
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def index_and_queries():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()
    s = synth.scaled(2, n=20_000, n_queries=150, nlist=48, n_clusters=48)
    w = synth.generate(s)
    t = pano.panorama_fit_transform(w.X.numpy(), n_levels=16)
    idx = pano.panorama_build_ivf(t, w.X.to(DEV), nlist=48, n_levels=16, kmeans_iters=5)
    return idx, w.Q.to(DEV)


def _noalloc(idx, q, nprobe, k, k_max):
    nq = q.shape[0]
    ids = torch.full((nq, k_max), 7, dtype=torch.int64, device=DEV)
    dists = torch.full((nq, k_max), 7.0, dtype=torch.float32, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    rc = pano.lib().panorama_search_noalloc(idx.handle, q.data_ptr(), nq, None, nprobe, None,
                                            k, k_max, ids.data_ptr(), dists.data_ptr(), stream)
    return rc, ids, dists


def _same(a_ids, a_d, b_ids, b_d):
    a_ids, b_ids = a_ids.cpu().numpy(), b_ids.cpu().numpy()
    a_d, b_d = a_d.cpu().numpy().astype(np.float64), b_d.cpu().numpy().astype(np.float64)
    fin = np.isfinite(a_d)
    assert np.array_equal(fin, np.isfinite(b_d))
    rel = np.abs(a_d[fin] - b_d[fin]) / np.maximum(np.abs(a_d[fin]), 1e-30)
    assert rel.max(initial=0.0) <= 1e-5
    diff = a_ids != b_ids
    # a differing id is only allowed where the distances form a near-tie
    assert np.all(np.abs(a_d[diff] - b_d[diff]) <= 1e-6 * np.abs(a_d[diff]))


def test_noalloc_matches_search_on_two_calls(index_and_queries):
    """Two calls in a row with different batches: the second one has other
    queries, fewer of them, another nprobe, k and k_max, so whatever the
    first call left in the shared array (top-k keys, counters, work lists)
    would show up in its result if the search did not clear it."""
    idx, q = index_and_queries
    calls = [(q[:120], 6, 10, 12), (q[120:], 9, 4, 5)]
    for qs, nprobe, k, k_max in calls:
        ref_ids, ref_d = idx.search(qs, nprobe, k, k_max=k_max)
        rc, ids, d = _noalloc(idx, qs, nprobe, k, k_max)
        torch.cuda.synchronize()
        assert rc == 0, pano.lib().panorama_last_error()
        _same(ref_ids, ref_d, ids, d)
        assert torch.all(ids[:, k:] == -1) and torch.all(torch.isinf(d[:, k:]))


def test_noalloc_rejects_workspace_beyond_scratch(index_and_queries):
    idx, q = index_and_queries
    big = q.repeat(60, 1)  # 9,000 queries x k_max 1024: > 64 MiB of workspace
    rc, _, _ = _noalloc(idx, big, 6, 10, 1024)
    assert rc == -1
    assert b"static scratch" in pano.lib().panorama_last_error()
    # the rejection queued no work; the entry point still answers afterwards
    ref_ids, ref_d = idx.search(q, 6, 10)
    rc, ids, d = _noalloc(idx, q, 6, 10, 10)
    torch.cuda.synchronize()
    assert rc == 0
    _same(ref_ids, ref_d, ids, d)
