"""Seeded synthetic workloads for Panorama-style exact kNN refinement.

This module is the only code shared by the CUDA library's tests/benchmark and
the CPU oracle.  It draws inputs and nothing else: it holds none of the
method's arithmetic (no PCA, no bounds, no distances, no clustering).

Recipe (the same for every workload):

* a Haar-random orthogonal basis O (d x d): QR of an FP64 Gaussian matrix with
  the signs of R's diagonal folded into Q, drawn on the CPU from seed
  ``1000 + cfg``;
* per-axis standard deviations sqrt(lambda_i), lambda_i = exp(-decay * i),
  i = 0..d-1 (the covariance spectrum the paper's cost model is written in,
  Section 4.1 "Energy compaction and the parameter alpha");
* cluster centres c ~ N(0, centre_std^2 I) (mixtures only), drawn from the same
  CPU generator;
* each vector x = c_{a} + O diag(sqrt(lambda)) z with z ~ N(0, I), cast to FP32
  once; database vectors use seed ``1000 + cfg`` on the target device, queries
  an independent stream with seed ``2000 + cfg`` (queries pick their cluster
  with the same weights as the data);
* per-query nprobe / k draws (the batching and serving workloads) come from a
  CPU generator with seed ``4000 + cfg``.

The five named workloads mirror the shapes of the paper's benchmark datasets
(Section 7, Table "Datasets used"): 128-d (SIFT-like), 960-d (GIST-like),
768-d (arXiv-embedding-like) and 384-d.  None of those datasets is used; the
vectors are synthetic draws from the recipe above.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import torch

__all__ = ["Spec", "SPECS", "spec", "scaled", "Workload", "generate",
           "haar_orthogonal", "zipf_sizes"]


@dataclasses.dataclass(frozen=True)
class Spec:
    """Shape of one synthetic workload."""
    cfg: int                      # seed base (1..5 for the named workloads)
    name: str
    n: int                        # database vectors
    d: int                        # dimension
    n_queries: int
    decay: float                  # lambda_i = exp(-decay * i)
    n_clusters: int = 0           # 0 -> one Gaussian centred at the origin
    centre_std: float = 1.0
    sizes: str = "equal"          # "equal" (iid labels) or "zipf"
    zipf_s: float = 1.1
    nlist: int = 1                # IVF lists (1 -> flat / exhaustive)
    nprobe: int | tuple = 1       # int, or (lo, hi) inclusive uniform range
    k: int | tuple = 10           # int, or tuple of values drawn uniformly
    n_levels: int = 8
    precision: str = "fp32"       # "fp32", "bf16" or "fp8"
    query_decay: Optional[float] = None  # queries' own eigen-decay (out of
                                         # distribution, same total energy);
                                         # None = decay

    @property
    def level_width(self) -> int:
        return self.d // self.n_levels


SPECS = {
    1: Spec(1, "plain-20k-d128-flat", n=20_000, d=128, n_queries=100,
            decay=0.05, nlist=1, nprobe=1, k=10, n_levels=8),
    2: Spec(2, "ivf-1m-d960-fp32", n=1_000_000, d=960, n_queries=10_000,
            decay=0.01, n_clusters=1024, centre_std=1.0, nlist=1024,
            nprobe=32, k=10, n_levels=16),
    3: Spec(3, "ivf-10m-d768-bf16", n=10_000_000, d=768, n_queries=10_000,
            decay=0.008, nlist=4096, nprobe=64, k=10, n_levels=12,
            precision="bf16"),
    4: Spec(4, "ivf-5m-d384-zipf-batch", n=5_000_000, d=384,
            n_queries=65_536, decay=0.02, n_clusters=2048, centre_std=0.5,
            sizes="zipf", zipf_s=1.1, nlist=2048, nprobe=(1, 128),
            k=(1, 10, 100), n_levels=12, precision="bf16"),
    5: Spec(5, "ivf-50m-d128-serving", n=50_000_000, d=128, n_queries=1024,
            decay=0.05, nlist=16384, nprobe=(8, 64), k=10, n_levels=8,
            precision="bf16"),
}


def spec(cfg: int) -> Spec:
    return SPECS[cfg]


def scaled(cfg: int, n: int, n_queries: int, nlist: Optional[int] = None,
           n_clusters: Optional[int] = None, **kw) -> Spec:
    """A smaller workload with the same recipe and seeds as ``cfg``."""
    s = SPECS[cfg]
    upd = dict(n=n, n_queries=n_queries)
    if nlist is not None:
        upd["nlist"] = nlist
    if n_clusters is not None:
        upd["n_clusters"] = n_clusters
    upd.update(kw)
    return dataclasses.replace(s, **upd)


def haar_orthogonal(d: int, gen: torch.Generator) -> torch.Tensor:
    """Haar-distributed orthogonal d x d matrix (FP64, CPU)."""
    g = torch.randn(d, d, generator=gen, dtype=torch.float64)
    q, r = torch.linalg.qr(g)
    sgn = torch.sign(torch.diagonal(r))
    sgn[sgn == 0] = 1.0
    return q * sgn.unsqueeze(0)


def zipf_sizes(n: int, m: int, s: float) -> torch.Tensor:
    """Cluster sizes proportional to r^-s (r = 1..m) summing to n.

    Largest-remainder rounding; every cluster gets at least one vector.
    """
    w = torch.arange(1, m + 1, dtype=torch.float64).pow(-s)
    w = w / w.sum()
    raw = w * (n - m)
    base = torch.floor(raw)
    rem = int(n - m - base.sum().item())
    order = torch.argsort(raw - base, descending=True, stable=True)
    base[order[:rem]] += 1
    return (base + 1).to(torch.int64)


@dataclasses.dataclass
class Workload:
    spec: Spec
    X: torch.Tensor               # n x d float32 (on `device`)
    Q: torch.Tensor               # n_queries x d float32 (on `device`)
    nprobe: torch.Tensor          # n_queries int32 (CPU)
    k: torch.Tensor               # n_queries int32 (CPU)
    basis: torch.Tensor           # d x d float64 (CPU): the generating basis O
    eigvals: torch.Tensor         # d float64 (CPU): lambda_i
    centres: Optional[torch.Tensor]  # n_clusters x d float64 (CPU) or None


def _draw(count: int, labels: Optional[torch.Tensor], O32: torch.Tensor,
          sd32: torch.Tensor, C32: Optional[torch.Tensor],
          gen: torch.Generator, device, block: int) -> torch.Tensor:
    d = O32.shape[0]
    out = torch.empty(count, d, dtype=torch.float32, device=device)
    for s in range(0, count, block):
        e = min(count, s + block)
        z = torch.randn(e - s, d, generator=gen, dtype=torch.float32,
                        device=device)
        y = (z * sd32) @ O32.t()
        if C32 is not None:
            y += C32[labels[s:e]]
        out[s:e] = y
    return out


def generate(s: Spec, device="cpu", block: int = 1 << 18,
             queries_only: bool = False) -> Workload:
    """Draw the database and query set of workload ``s`` on ``device``."""
    device = torch.device(device)
    cpu = torch.Generator().manual_seed(1000 + s.cfg)
    O = haar_orthogonal(s.d, cpu)
    lam = torch.exp(-s.decay * torch.arange(s.d, dtype=torch.float64))
    C = None
    weights = None
    if s.n_clusters > 0:
        C = torch.randn(s.n_clusters, s.d, generator=cpu,
                        dtype=torch.float64) * s.centre_std
        if s.sizes == "zipf":
            sizes = zipf_sizes(s.n, s.n_clusters, s.zipf_s)
            weights = sizes.to(torch.float64) / s.n
        else:
            sizes = None
            weights = torch.full((s.n_clusters,), 1.0 / s.n_clusters,
                                 dtype=torch.float64)
    O32 = O.to(torch.float32).to(device)
    sd32 = lam.sqrt().to(torch.float32).to(device)
    C32 = C.to(torch.float32).to(device) if C is not None else None

    def gdev(seed):
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        return g

    X = None
    if not queries_only:
        gx = gdev(1000 + s.cfg)
        labels = None
        if C is not None:
            if s.sizes == "zipf":
                labels = torch.repeat_interleave(
                    torch.arange(s.n_clusters, device=device),
                    sizes.to(device))
                perm = torch.randperm(s.n, generator=gx, device=device)
                labels = labels[perm]
            else:
                labels = torch.randint(0, s.n_clusters, (s.n,), generator=gx,
                                       device=device)
        X = _draw(s.n, labels, O32, sd32, C32, gx, device, block)

    gq = gdev(2000 + s.cfg)
    qlabels = None
    if C is not None:
        qlabels = torch.multinomial(weights.to(torch.float32).to(device),
                                    s.n_queries, replacement=True,
                                    generator=gq)
    sdq32 = sd32
    if s.query_decay is not None:  # same basis and total energy, another decay
        lam_q = torch.exp(-s.query_decay * torch.arange(s.d, dtype=torch.float64))
        lam_q *= lam.sum() / lam_q.sum()
        sdq32 = lam_q.sqrt().to(torch.float32).to(device)
    Qm = _draw(s.n_queries, qlabels, O32, sdq32, C32, gq, device, block)

    gp = torch.Generator().manual_seed(4000 + s.cfg)
    if isinstance(s.nprobe, tuple):
        lo, hi = s.nprobe
        nprobe = torch.randint(lo, hi + 1, (s.n_queries,), generator=gp)
    else:
        nprobe = torch.full((s.n_queries,), s.nprobe)
    if isinstance(s.k, tuple):
        vals = torch.tensor(s.k)
        k = vals[torch.randint(0, len(s.k), (s.n_queries,), generator=gp)]
    else:
        k = torch.full((s.n_queries,), s.k)
    nprobe = torch.clamp(nprobe, max=s.nlist).to(torch.int32)
    return Workload(s, X, Qm, nprobe, k.to(torch.int32), O, lam, C)


def initial_centroids(X: torch.Tensor, nlist: int, seed: int) -> torch.Tensor:
    """``nlist`` distinct database rows picked with a seeded permutation.

    Used by tests that hand fixed coarse centroids to both sides (so that the
    oracle's list assignment does not depend on the library's k-means).
    """
    g = torch.Generator().manual_seed(seed)
    idx = torch.randperm(X.shape[0], generator=g)[:nlist]
    return X[idx.to(X.device)].clone()
