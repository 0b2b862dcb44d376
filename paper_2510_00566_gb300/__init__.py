"""Python binding of libpanorama (GB300 / sm_103a), argument marshalling only.

Every computation runs in the library's CUDA kernels behind the C-ABI of
``include/panorama.h``; this module converts torch tensors / numpy arrays to
pointers and sizes.  Importing the package does not load the library;
``lib()`` does, and raises if the library was not built (there is no CPU
fallback).  Build it with ``paper_2510_00566_gb300._build.build()``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

__all__ = ["lib", "LibraryError", "Transform", "Index", "SearchStats",
           "panorama_fit_transform", "panorama_build_ivf", "panorama_search",
           "panorama_search_ex", "panorama_probe", "panorama_save",
           "panorama_load", "panorama_build_flat", "panorama_refine",
           "PANO_FP32", "PANO_BF16", "PANO_FP8", "PANO_PQ",
           "panorama_transform_import", "panorama_shape_transform",
           "panorama_build_ivfpq", "panorama_search_pq", "panorama_pq_export",
           "panorama_debug_pq_encode", "panorama_autotune",
           "library_path"]

PANO_FP32, PANO_BF16, PANO_FP8, PANO_PQ = 0, 1, 2, 3
_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT",
           -5: "ECORRUPT", -6: "ENODEV"}
_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "lib", "libpanorama.so")
_lib = None


class LibraryError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"panorama error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class BuildOpts(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32),
                ("level_widths", ctypes.POINTER(ctypes.c_int32)),
                ("precision", ctypes.c_int32),
                ("fit_sample", ctypes.c_int64),
                ("seed", ctypes.c_uint64),
                ("kmeans_iters", ctypes.c_int32),
                ("kmeans_sample", ctypes.c_int64),
                ("identity_transform", ctypes.c_int32),
                ("centroids", ctypes.c_void_p)]


class SearchOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("synchronize", ctypes.c_int32),
                ("collect_stats", ctypes.c_int32),
                ("query_group", ctypes.c_int32),
                ("collect_timing", ctypes.c_int32),
                ("single_phase", ctypes.c_int32),
                ("epsilon", ctypes.c_float),
                ("test_every", ctypes.c_int32)]


class SearchStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("pair_levels", ctypes.c_int64),
                ("dims_scanned", ctypes.c_int64),
                ("tile_levels", ctypes.c_int64),
                ("slice_bytes", ctypes.c_int64),
                ("reranked", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("device_error", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("stage_ms", ctypes.c_float * 6), ("pad2_", ctypes.c_float * 2),
                ("section_cycles", ctypes.c_int64 * 8),
                ("dims_scanned_a", ctypes.c_int64), ("pairs_a", ctypes.c_int64),
                ("section_cycles_a", ctypes.c_int64 * 8),
                ("live_row_bytes", ctypes.c_int64)]

    STAGES = ("transform", "probe", "inversion", "verify_a", "verify_b",
              "decode")

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_
             if not f.startswith("pad")
             and f not in ("stage_ms", "section_cycles", "section_cycles_a")}
        d["stage_ms"] = dict(zip(self.STAGES, list(self.stage_ms)))
        names = ("prologue", "mma_issue", "epilogue", "next_level", "ub_filter", "rerank",
                 "kernel", "ctas")
        d["section_cycles"] = dict(zip(names, list(self.section_cycles)))
        d["section_cycles_a"] = dict(zip(names, list(self.section_cycles_a)))
        return d


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("nlist", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("max_level_width", ctypes.c_int32),
                ("n_chunks", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("eta", ctypes.c_double)]


class PQBuildOpts(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("kmeans_iters", ctypes.c_int32), ("pq_iters", ctypes.c_int32),
                ("kmeans_sample", ctypes.c_int64), ("pq_sample", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("centroids", ctypes.c_void_p),
                ("assign", ctypes.c_void_p), ("codebooks", ctypes.c_void_p),
                ("codes", ctypes.c_void_p)]


# name -> (restype, argtypes); the exported C-ABI (include/panorama.h,
# include/panorama_pq.h)
_P, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "panorama_partition_lists": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "panorama_merge_topk": (ctypes.c_int, [_P, _P, _I32, _I64, _I32, _P, _P]),
    "panorama_fit_transform": (ctypes.c_int, [_P, _I64, _I32, _P, _P]),
    "panorama_transform_export": (ctypes.c_int, [_P, _P, _P, _P]),
    "panorama_transform_dim": (ctypes.c_int, [_P]),
    "panorama_free_transform": (None, [_P]),
    "panorama_build_ivf": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "panorama_search": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32,
                                       _I32, _P, _P, _P]),
    "panorama_search_ex": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32,
                                          _I32, _P, _P, _P, _P]),
    "panorama_search_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32,
                                                _I32, _P, _P, _P]),
    "panorama_search_stats": (ctypes.c_int, [_P]),
    "panorama_status_of_device_error": (ctypes.c_int, [_I32]),
    "panorama_probe": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P]),
    "panorama_index_info": (ctypes.c_int, [_P, _P]),
    "panorama_index_centroids": (ctypes.c_int, [_P, _P]),
    "panorama_index_assignment": (ctypes.c_int, [_P, _P]),
    "panorama_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "panorama_load": (ctypes.c_int, [ctypes.c_char_p, _P]),
    "panorama_free_index": (None, [_P]),
    "panorama_last_error": (ctypes.c_char_p, []),
    "panorama_version": (ctypes.c_char_p, []),
    "panorama_build_flat": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "panorama_refine": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _I32, _P, _P, ctypes.c_float,
                                       _P]),
    "panorama_debug_tc_gemm": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _P]),
    "panorama_transform_import": (ctypes.c_int, [_P, _P, _P, _I32, _P]),
    "panorama_shape_transform": (ctypes.c_int, [_P, _I32, ctypes.c_double, _P, _P, _P]),
    "panorama_build_ivfpq": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "panorama_search_pq": (ctypes.c_int, [_P, _P, _I64, _I32, _I32, _P, _P, _I32, _I32,
                                          ctypes.c_float, _P]),
    "panorama_search_pq_ex": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32, _I32, _P, _P,
                                             _P, _P]),
    "panorama_pq_export": (ctypes.c_int, [_P, _P, _P, _P]),
    "panorama_debug_pq_encode": (ctypes.c_int, [_P, _I64, _I32, _I32, _P, _P, _P]),
    "panorama_debug_tc_gemm_fp8": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _P]),
    "panorama_debug_sqrt_up": (ctypes.c_int, [_P, _I64, _P, _P]),
    "panorama_plan_create": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32, _I32,
                                            _P, _P, _I32, _P]),
    "panorama_plan_create_ex": (ctypes.c_int, [_P, _P, _I64, _P, _I32, _P, _I32, _I32,
                                               _P, _P, _P, _P]),
    "panorama_plan_launch": (ctypes.c_int, [_P, _P]),
    "panorama_plan_free": (None, [_P]),
    "panorama_server_create": (ctypes.c_int, [_P, _P, _P]),
    "panorama_server_submit": (ctypes.c_int, [_P, _P, _I32, _I32, _P]),
    "panorama_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _I32, _P, _P, _P]),
    "panorama_server_stats": (ctypes.c_int, [_P, _P]),
    "panorama_server_run_trace": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "panorama_server_free": (None, [_P]),
    "panorama_autotune": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _I32, _I32, _I32, _P, _I32,
                                         _P, _P, _I32, _I32, _P, _I32, _P, _P, _P]),
    "panorama_autotune_levels": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _I32, _I32,
                                                _I32, _I32, _P, _P, _I32, _I32, _P,
                                                _P, _P]),
}


def lib():
    """Load libpanorama.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(
                f"{library_path} is missing: build it with "
                "paper_2510_00566_gb300._build.build() (no CPU fallback)")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise LibraryError(rc, lib().panorama_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _host_f32(a):
    import numpy as np
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            keep = a.contiguous()
            return keep, keep.data_ptr()
        a = a.numpy()
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data


# ------------------------------------------------------------------ C names
def panorama_fit_transform(X, n_levels=8, fit_sample=0, identity=False):
    """PCA transform of the rows of X (host numpy / torch, or CUDA tensor)."""
    keep, ptr = _host_f32(X)
    n, d = keep.shape
    opts = BuildOpts(n_levels=n_levels, fit_sample=fit_sample,
                     identity_transform=1 if identity else 0)
    out = ctypes.c_void_p()
    _check(lib().panorama_fit_transform(ptr, n, d, ctypes.byref(opts),
                                        ctypes.byref(out)))
    return Transform(out.value, d)


def panorama_build_ivf(t: "Transform", X, nlist: int, n_levels=8,
                       level_widths=None, precision=PANO_FP32, seed=1234,
                       kmeans_iters=20, kmeans_sample=0, centroids=None,
                       stream=None):
    """IVF index of X (CUDA tensor or host array); see panorama_build_ivf."""
    import numpy as np
    keep, ptr = _host_f32(X)
    n, d = keep.shape
    widths = None
    if level_widths is not None:
        widths = (ctypes.c_int32 * len(level_widths))(*level_widths)
        n_levels = len(level_widths)
    cent_keep = None
    opts = BuildOpts(n_levels=n_levels, level_widths=widths,
                     precision=precision, seed=seed,
                     kmeans_iters=kmeans_iters, kmeans_sample=kmeans_sample)
    if centroids is not None:
        cent_keep = np.ascontiguousarray(
            centroids.cpu().numpy() if hasattr(centroids, "cpu") else centroids,
            dtype=np.float32)
        opts.centroids = cent_keep.ctypes.data
    out = ctypes.c_void_p()
    _check(lib().panorama_build_ivf(t.handle, ptr, n, nlist, ctypes.byref(opts),
                                    _stream_ptr(stream), ctypes.byref(out)))
    del cent_keep
    return Index(out.value)


def panorama_search_ex(idx: "Index", queries, nprobe, k, k_max=None,
                       mode=0, collect_stats=False, synchronize=True,
                       stream=None, out=None, collect_timing=False,
                       single_phase=None, epsilon=1.0, test_every=0):
    """Returns (ids int64 [nq, k_max], dists float32 [nq, k_max]) on the GPU.

    nprobe / k: python ints, or CUDA int32 tensors with one value per query.
    single_phase: None = the library chooses, True = one pass, False = each
    query's nearest list first.  epsilon < 1: Eq. 4's relaxed pruning
    (approximate; exact distances for what is returned).  test_every: the
    bound is tested at level l when l % test_every == 0 and at the last
    level, and (BF16 / FP8) at every level for chunks with at most 16 live
    rows; 1 = every level, 0 = the format's default (FP32 1, BF16 / FP8 4).
    The result is exact whatever the schedule.
    """
    import torch
    q = queries.contiguous()
    assert q.is_cuda and q.dtype == torch.float32
    nq = q.shape[0]
    np_ptr, np_scalar = None, 0
    if isinstance(nprobe, torch.Tensor):
        nprobe = nprobe.to(device=q.device, dtype=torch.int32).contiguous()
        np_ptr, np_scalar = nprobe.data_ptr(), int(nprobe.max()) if nq else 1
    else:
        np_scalar = int(nprobe)
    k_ptr, k_scalar = None, 0
    if isinstance(k, torch.Tensor):
        k = k.to(device=q.device, dtype=torch.int32).contiguous()
        k_ptr = k.data_ptr()
        if k_max is None:
            k_max = int(k.max()) if nq else 1
    else:
        k_scalar = int(k)
        if k_max is None:
            k_max = max(1, k_scalar)
    if out is None:
        ids = torch.empty((nq, k_max), dtype=torch.int64, device=q.device)
        dists = torch.empty((nq, k_max), dtype=torch.float32, device=q.device)
    else:
        ids, dists = out
    opts = SearchOpts(mode=mode, synchronize=1 if synchronize else 0,
                      collect_stats=1 if collect_stats else 0,
                      collect_timing=1 if collect_timing else 0,
                      single_phase=0 if single_phase is None else (1 if single_phase else 2),
                      epsilon=float(epsilon), test_every=int(test_every))
    _check(lib().panorama_search_ex(idx.handle, q.data_ptr(), nq, np_ptr,
                                    np_scalar, k_ptr, k_scalar, k_max,
                                    ids.data_ptr(), dists.data_ptr(),
                                    _stream_ptr(stream), ctypes.byref(opts)))
    return ids, dists


def panorama_search(idx, queries, nprobe, k, k_max=None, stream=None):
    return panorama_search_ex(idx, queries, nprobe, k, k_max, stream=stream)


def panorama_probe(idx: "Index", queries, nprobe: int, stream=None):
    import torch
    q = queries.contiguous()
    out = torch.empty((q.shape[0], nprobe), dtype=torch.int32, device=q.device)
    _check(lib().panorama_probe(idx.handle, q.data_ptr(), q.shape[0], nprobe,
                                out.data_ptr(), _stream_ptr(stream)))
    return out


def panorama_save(idx: "Index", path: str):
    _check(lib().panorama_save(idx.handle, path.encode()))


def panorama_build_flat(t: "Transform", X, n_levels=8, level_widths=None, stream=None):
    """Flat index for refining candidate-id lists (B = 1); see
    panorama_build_flat.  Vector i gets id i."""
    keep, ptr = _host_f32(X)
    n, d = keep.shape
    widths = None
    if level_widths is not None:
        widths = (ctypes.c_int32 * len(level_widths))(*level_widths)
        n_levels = len(level_widths)
    opts = BuildOpts(n_levels=n_levels, level_widths=widths, precision=PANO_FP32)
    out = ctypes.c_void_p()
    _check(lib().panorama_build_flat(t.handle, ptr, n, ctypes.byref(opts),
                                     _stream_ptr(stream), ctypes.byref(out)))
    return Index(out.value)


def panorama_refine(index: "Index", queries, cand_ids, k: int, epsilon=1.0, stream=None):
    """Exact top-k of each query among its candidate ids (CUDA tensors:
    queries nq x d float32, cand_ids nq x k' int64 with -1 = none) on a flat
    index; returns (ids int64 nq x k, dists float32 nq x k)."""
    import torch
    q = queries.contiguous()
    c = cand_ids.to(torch.int64).contiguous()
    nq = q.shape[0]
    kp = c.shape[1] if c.dim() == 2 else 0
    ids = torch.empty((nq, k), dtype=torch.int64, device=q.device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
    _check(lib().panorama_refine(index.handle, q.data_ptr(), nq, c.data_ptr() if kp else None,
                                 kp, k, ids.data_ptr(), dists.data_ptr(), float(epsilon),
                                 _stream_ptr(stream)))
    return ids, dists


def panorama_load(path: str) -> "Index":
    out = ctypes.c_void_p()
    _check(lib().panorama_load(path.encode(), ctypes.byref(out)))
    return Index(out.value)


def panorama_debug_tc_gemm(A, B, stream=None):
    """D = 2 A B^T through the tensor-core building blocks (A: 128 x K, B:
    N x K, bf16 CUDA tensors); a unit check of the BF16 verify kernel's MMA
    path."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    N, K = B.shape
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    _check(lib().panorama_debug_tc_gemm(A.data_ptr(), B.data_ptr(), N, K,
                                        D.data_ptr(), _stream_ptr(stream)))
    return D


def panorama_debug_tc_gemm_fp8(A, B, stream=None):
    """D = 2 A B^T with E4M3 tiles (A: 128 x K, B: N x K uint8 CUDA tensors of
    E4M3 bytes); a unit check of the FP8 verify kernel's MMA path."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    N, K = B.shape
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    _check(lib().panorama_debug_tc_gemm_fp8(A.data_ptr(), B.data_ptr(), N, K,
                                            D.data_ptr(), _stream_ptr(stream)))
    return D


def panorama_debug_sqrt_up(x, stream=None):
    """The verify kernels' rounded-up square root of each element of x (a
    float32 CUDA tensor of non-negative values)."""
    import torch
    x = x.contiguous()
    out = torch.empty_like(x)
    _check(lib().panorama_debug_sqrt_up(x.data_ptr(), x.numel(), out.data_ptr(),
                                        _stream_ptr(stream)))
    return out


# ------------------------------------------------------------------ IVFPQ
def panorama_transform_import(T, mu, lam) -> "Transform":
    """A transform from FP64 arrays: T (d x d, orthogonal), mu (d), lam (d
    expected coordinate variances)."""
    import numpy as np
    T = np.ascontiguousarray(T, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    d = T.shape[0]
    out = ctypes.c_void_p()
    _check(lib().panorama_transform_import(T.ctypes.data, mu.ctypes.data, lam.ctypes.data, d,
                                           ctypes.byref(out)))
    return Transform(out.value, d)


def panorama_shape_transform(t: "Transform", n_levels: int, kappa: float, gauss):
    """U R T of spectrum shaping; gauss: 2 x d x d standard normal draws
    (G1, G2).  Returns (shaped Transform, list of (start, size) blocks)."""
    import numpy as np
    g = np.ascontiguousarray(gauss, dtype=np.float64)
    assert g.size == 2 * t.d * t.d
    blocks = np.full(2 * n_levels, -1, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().panorama_shape_transform(t.handle, n_levels, float(kappa), g.ctypes.data,
                                          blocks.ctypes.data, ctypes.byref(out)))
    bl = [(int(blocks[2 * i]), int(blocks[2 * i + 1])) for i in range(n_levels)
          if blocks[2 * i] >= 0]
    return Transform(out.value, t.d), bl


def panorama_build_ivfpq(t: "Transform", X, nlist: int, M: int, n_levels: int,
                         centroids=None, assign=None, codebooks=None, codes=None,
                         kmeans_iters=0, pq_iters=0, kmeans_sample=0, pq_sample=0,
                         seed=1234, stream=None) -> "Index":
    """IVFPQ index of X (CUDA tensor or host array); optional host arrays:
    centroids (nlist x d), assign (n int32), codebooks (M x 256 x d/M float32
    in the basis of t), codes (n x M uint8)."""
    import numpy as np
    keep, ptr = _host_f32(X)
    n = keep.shape[0]
    o = PQBuildOpts(M=M, n_levels=n_levels, kmeans_iters=kmeans_iters, pq_iters=pq_iters,
                    kmeans_sample=kmeans_sample, pq_sample=pq_sample, seed=seed)
    hold = []

    def host(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a.cpu().numpy() if hasattr(a, "cpu") else a, dtype=dt)
        hold.append(a)
        return a.ctypes.data

    o.centroids = host(centroids, np.float32)
    o.assign = host(assign, np.int32)
    o.codebooks = host(codebooks, np.float32)
    o.codes = host(codes, np.uint8)
    out = ctypes.c_void_p()
    _check(lib().panorama_build_ivfpq(t.handle, ptr, n, nlist, ctypes.byref(o),
                                      _stream_ptr(stream), ctypes.byref(out)))
    del hold
    return Index(out.value)


def panorama_search_pq(idx: "Index", queries, nprobe, k, k_max=None, mode=0,
                       collect_stats=False, stream=None, out=None, collect_timing=False,
                       epsilon=1.0):
    """(ids int64 [nq, k_max], dists float32 [nq, k_max]) on the GPU.

    nprobe / k: python ints, or CUDA int32 tensors with one value per query
    (then k_max defaults to max(k)); mode 1 = plain scan; collect_timing
    fills stage_ms (transform, probe, pairs + seeds, -, verify, decode);
    epsilon < 1: Eq. 4's relaxed pruning (approximate)."""
    import torch
    q = queries.contiguous()
    assert q.is_cuda and q.dtype == torch.float32
    nq = q.shape[0]
    np_ptr, np_scalar = None, 0
    if isinstance(nprobe, torch.Tensor):
        nprobe = nprobe.to(device=q.device, dtype=torch.int32).contiguous()
        np_ptr, np_scalar = nprobe.data_ptr(), int(nprobe.max()) if nq else 1
    else:
        np_scalar = int(nprobe)
    k_ptr, k_scalar = None, 0
    if isinstance(k, torch.Tensor):
        k = k.to(device=q.device, dtype=torch.int32).contiguous()
        k_ptr = k.data_ptr()
        if k_max is None:
            k_max = max(1, int(k.max())) if nq else 1
    else:
        k_scalar = int(k)
        if k_max is None:
            k_max = max(1, k_scalar)
    if out is None:
        ids = torch.empty((nq, k_max), dtype=torch.int64, device=q.device)
        dists = torch.empty((nq, k_max), dtype=torch.float32, device=q.device)
    else:
        ids, dists = out
    opts = SearchOpts(mode=mode, synchronize=1, collect_stats=1 if collect_stats else 0,
                      collect_timing=1 if collect_timing else 0, epsilon=float(epsilon))
    _check(lib().panorama_search_pq_ex(idx.handle, q.data_ptr(), nq, np_ptr, np_scalar,
                                       k_ptr, k_scalar, k_max, ids.data_ptr(),
                                       dists.data_ptr(), ctypes.byref(opts),
                                       _stream_ptr(stream)))
    return ids, dists


def panorama_pq_export(idx: "Index"):
    """(codebooks M x 256 x d/M float32, codes n x M uint8) host copies."""
    import numpy as np
    info = idx.info()
    M = ctypes.c_int32()
    _check(lib().panorama_pq_export(idx.handle, None, None, ctypes.byref(M)))
    cb = np.empty((M.value, 256, info.d // M.value), dtype=np.float32)
    codes = np.empty((info.n, M.value), dtype=np.uint8)
    _check(lib().panorama_pq_export(idx.handle, cb.ctypes.data, codes.ctypes.data, None))
    return cb, codes


def panorama_debug_pq_encode(R, codebooks, stream=None):
    """Codes (n x M uint8 CUDA tensor) of residual rows R (n x d float32 CUDA)
    by the build's encoder; codebooks M x 256 x d/M float32 CUDA."""
    import torch
    R = R.contiguous()
    cb = codebooks.contiguous()
    n, d = R.shape
    M = cb.shape[0]
    codes = torch.empty((n, M), dtype=torch.uint8, device=R.device)
    _check(lib().panorama_debug_pq_encode(R.data_ptr(), n, d, M, cb.data_ptr(),
                                          codes.data_ptr(), _stream_ptr(stream)))
    return codes


class Plan:
    """One search of a fixed batch shape captured into a CUDA graph.

    The tensors given here stay bound to the graph: refill ``queries`` (and
    nprobe / k when they are tensors) in place, call ``launch()``, then read
    ``ids`` / ``dists``."""

    def __init__(self, idx: "Index", queries, nprobe, k, k_max=None, mode=0, test_every=0,
                 epsilon=1.0):
        import torch
        self.idx = idx
        self.queries = queries
        nq = queries.shape[0]
        self._keep = []
        np_ptr, np_scalar = None, 0
        if isinstance(nprobe, torch.Tensor):
            np_ptr, np_scalar = nprobe.data_ptr(), int(nprobe.max())
            self._keep.append(nprobe)
        else:
            np_scalar = int(nprobe)
        k_ptr, k_scalar = None, 0
        if isinstance(k, torch.Tensor):
            k_ptr = k.data_ptr()
            self._keep.append(k)
            k_max = k_max or int(k.max())
        else:
            k_scalar = int(k)
            k_max = k_max or k_scalar
        self.ids = torch.empty((nq, k_max), dtype=torch.int64, device=queries.device)
        self.dists = torch.empty((nq, k_max), dtype=torch.float32, device=queries.device)
        out = ctypes.c_void_p()
        opts = SearchOpts(mode=mode, test_every=int(test_every), epsilon=float(epsilon))
        _check(lib().panorama_plan_create_ex(idx.handle, queries.data_ptr(), nq, np_ptr,
                                             np_scalar, k_ptr, k_scalar, k_max,
                                             self.ids.data_ptr(), self.dists.data_ptr(),
                                             ctypes.byref(opts), ctypes.byref(out)))
        self.handle = out.value

    def launch(self, stream=None):
        _check(lib().panorama_plan_launch(self.handle, _stream_ptr(stream)))
        return self.ids, self.dists

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.panorama_plan_free(self.handle)
            self.handle = None


def panorama_autotune_levels(t: "Transform", X, queries, nlist, nprobe, k,
                             candidates, precision=PANO_FP32, repeats=3,
                             stream=None):
    """Index of the fastest candidate level split and every candidate's
    median search time in ms (inf when it cannot be built)."""
    import numpy as np
    keep, ptr = _host_f32(X)
    n = keep.shape[0]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(c) for c in candidates]),
                                dtype=np.int32)
    lens = np.ascontiguousarray([len(c) for c in candidates], dtype=np.int32)
    best = ctypes.c_int32(-1)
    ms = np.zeros(len(candidates), dtype=np.float32)
    q = queries.contiguous()
    _check(lib().panorama_autotune_levels(t.handle, ptr, n, q.data_ptr(), q.shape[0],
                                          nlist, nprobe, k, precision, flat.ctypes.data,
                                          lens.ctypes.data, len(candidates), repeats,
                                          ctypes.byref(best), ms.ctypes.data,
                                          _stream_ptr(stream)))
    return best.value, ms


class AutotuneTrial(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("widths", ctypes.c_int32 * 64), ("ms", ctypes.c_float),
                ("test_every", ctypes.c_int32)]


def panorama_autotune(t: "Transform", X, queries, nlist, nprobe, k,
                      precisions=(PANO_FP32, PANO_BF16, PANO_FP8), candidates=None,
                      repeats=3, max_trials=64, stream=None):
    """Fastest (precision, level split, bound-test schedule) on a query
    sample.  Returns (best index, trials) with trials a list of dicts
    (precision, widths, ms, test_every: the fastest schedule of the split)."""
    import numpy as np
    keep, ptr = _host_f32(X)
    n = keep.shape[0]
    prec = np.ascontiguousarray(precisions, dtype=np.int32)
    flat = lens = None
    ncand = 0
    if candidates:
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c) for c in candidates]),
                                    dtype=np.int32)
        lens = np.ascontiguousarray([len(c) for c in candidates], dtype=np.int32)
        ncand = len(candidates)
    trials = (AutotuneTrial * max_trials)()
    n_tr, best = ctypes.c_int32(0), ctypes.c_int32(-1)
    q = queries.contiguous()
    _check(lib().panorama_autotune(t.handle, ptr, n, q.data_ptr(), q.shape[0], nlist, nprobe,
                                   k, prec.ctypes.data, len(prec),
                                   None if flat is None else flat.ctypes.data,
                                   None if lens is None else lens.ctypes.data, ncand, repeats,
                                   trials, max_trials, ctypes.byref(n_tr), ctypes.byref(best),
                                   _stream_ptr(stream)))
    out = [{"precision": trials[i].precision,
            "widths": list(trials[i].widths[:trials[i].n_levels]), "ms": trials[i].ms,
            "test_every": trials[i].test_every}
           for i in range(n_tr.value)]
    return best.value, out


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mean_batch", ctypes.c_double),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("qps", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Server:
    """Continuous-batching request server over an index (see panorama.h)."""

    def __init__(self, idx: "Index", max_batch=1024, max_inflight=2, k_max=10,
                 memory_budget=0):
        self.idx = idx
        self.k_max = k_max
        self.d = idx.info().d
        o = ServerOpts(max_batch=max_batch, max_inflight=max_inflight, k_max=k_max,
                       memory_budget=memory_budget)
        out = ctypes.c_void_p()
        _check(lib().panorama_server_create(idx.handle, ctypes.byref(o), ctypes.byref(out)))
        self.handle = out.value

    def submit(self, query, nprobe, k):
        import numpy as np
        q = np.ascontiguousarray(query, dtype=np.float32)
        t = ctypes.c_uint64()
        _check(lib().panorama_server_submit(self.handle, q.ctypes.data, nprobe, k,
                                            ctypes.byref(t)))
        return t.value

    def wait(self, ticket, timeout_ms=60000):
        import numpy as np
        ids = np.empty(self.k_max, dtype=np.int64)
        d = np.empty(self.k_max, dtype=np.float32)
        lat = ctypes.c_double()
        _check(lib().panorama_server_wait(self.handle, ticket, timeout_ms, ids.ctypes.data,
                                          d.ctypes.data, ctypes.byref(lat)))
        return ids, d, lat.value

    def run_trace(self, queries, arrival_us, nprobe, k):
        import numpy as np
        Q = np.ascontiguousarray(queries, dtype=np.float32)
        n = Q.shape[0]
        arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
        npq = np.ascontiguousarray(np.broadcast_to(nprobe, (n,)), dtype=np.int32)
        kq = np.ascontiguousarray(np.broadcast_to(k, (n,)), dtype=np.int32)
        ids = np.empty((n, self.k_max), dtype=np.int64)
        d = np.empty((n, self.k_max), dtype=np.float32)
        lat = np.empty(n, dtype=np.float64)
        _check(lib().panorama_server_run_trace(self.handle, Q.ctypes.data, n, arr.ctypes.data,
                                               npq.ctypes.data, kq.ctypes.data,
                                               ids.ctypes.data, d.ctypes.data,
                                               lat.ctypes.data))
        return ids, d, lat

    def stats(self):
        s = ServerStats()
        _check(lib().panorama_server_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.panorama_server_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def last_stats() -> SearchStats:
    s = SearchStats()
    _check(lib().panorama_search_stats(ctypes.byref(s)))
    return s


# ------------------------------------------------------------ thin objects
class Transform:
    def __init__(self, handle: int, d: int):
        self.handle = handle
        self.d = d

    def export(self):
        import numpy as np
        T = np.empty((self.d, self.d), dtype=np.float64)
        mu = np.empty(self.d, dtype=np.float64)
        ev = np.empty(self.d, dtype=np.float64)
        _check(lib().panorama_transform_export(self.handle, T.ctypes.data,
                                               mu.ctypes.data, ev.ctypes.data))
        return T, mu, ev

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.panorama_free_transform(self.handle)
            self.handle = None


class Index:
    def __init__(self, handle: int):
        self.handle = handle

    def info(self) -> IndexInfo:
        i = IndexInfo()
        _check(lib().panorama_index_info(self.handle, ctypes.byref(i)))
        return i

    def centroids(self):
        import numpy as np
        i = self.info()
        out = np.empty((i.nlist, i.d), dtype=np.float32)
        _check(lib().panorama_index_centroids(self.handle, out.ctypes.data))
        return out

    def assignment(self):
        import numpy as np
        out = np.empty(self.info().n, dtype=np.int32)
        _check(lib().panorama_index_assignment(self.handle, out.ctypes.data))
        return out

    def search(self, queries, nprobe, k, k_max=None, **kw):
        return panorama_search_ex(self, queries, nprobe, k, k_max, **kw)

    def refine(self, queries, cand_ids, k, epsilon=1.0, stream=None):
        return panorama_refine(self, queries, cand_ids, k, epsilon=epsilon, stream=stream)

    def search_pq(self, queries, nprobe, k, **kw):
        return panorama_search_pq(self, queries, nprobe, k, **kw)

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.panorama_free_index(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


# ------------------------------------------------------------ list sharding
def panorama_partition_lists(list_size, n_shards: int):
    """Owner shard of every IVF list (greedy balance of list sizes); host."""
    import numpy as np
    ls = np.ascontiguousarray(list_size, dtype=np.int32)
    owner = np.empty(ls.shape[0], dtype=np.int32)
    _check(lib().panorama_partition_lists(ls.ctypes.data, ls.shape[0], int(n_shards),
                                          owner.ctypes.data))
    return owner


def panorama_merge_topk(ids_parts, dists_parts):
    """Exact merge of per-shard top-k results (host arrays [n_parts, nq, k]
    or lists of [nq, k]); returns (ids int64 [nq, k], dists float32 [nq, k])."""
    import numpy as np
    ids = np.ascontiguousarray(np.stack([np.asarray(x) for x in ids_parts]), dtype=np.int64)
    dists = np.ascontiguousarray(np.stack([np.asarray(x) for x in dists_parts]),
                                 dtype=np.float32)
    n_parts, nq, k = ids.shape
    out_i = np.empty((nq, k), dtype=np.int64)
    out_d = np.empty((nq, k), dtype=np.float32)
    _check(lib().panorama_merge_topk(ids.ctypes.data, dists.ctypes.data, n_parts, nq, k,
                                     out_i.ctypes.data, out_d.ctypes.data))
    return out_i, out_d


def gather_merge_topk(ids, dists, group=None, dst: int = 0):
    """Every rank's partial top-k (torch tensors [nq, k], any device) are
    gathered on rank `dst` (torch.distributed, e.g. gloo or nccl) and merged
    there; returns (ids, dists) numpy arrays on `dst`, None elsewhere."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ids_c = ids.detach().to("cpu", torch.int64).contiguous()
    dists_c = dists.detach().to("cpu", torch.float32).contiguous()
    gi = [torch.empty_like(ids_c) for _ in range(world)] if rank == dst else None
    gd = [torch.empty_like(dists_c) for _ in range(world)] if rank == dst else None
    dist.gather(ids_c, gi, dst=dst, group=group)
    dist.gather(dists_c, gd, dst=dst, group=group)
    if rank != dst:
        return None
    return panorama_merge_topk([t.numpy() for t in gi], [t.numpy() for t in gd])

