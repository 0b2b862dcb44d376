"""The synthetic inputs follow their stated recipe (host only).

Every workload draws x = c_a + O diag(sqrt(lambda)) z with a Haar-random
orthogonal O, lambda_i = exp(-decay i), z ~ N(0, I), optional Gaussian
cluster centres (equal or Zipf-sized clusters) and per-query nprobe / k
draws.  These checks pin the draws against that recipe, so that a mistake
in the generator (a transposed basis, a variance used as a standard
deviation, Zipf sizes that do not follow r^-s) cannot slip into every
workload unnoticed.  They also pin the five workloads' shapes."""
import math

import numpy as np
import pytest
import torch

import synth


def test_haar_basis_is_orthogonal():
    g = torch.Generator().manual_seed(5)
    O = synth.haar_orthogonal(64, g)
    assert torch.allclose(O.t() @ O, torch.eye(64, dtype=torch.float64), atol=1e-12)
    # Haar: the diagonal of R was made positive, so the draw is not biased
    # towards one orientation; the first column's entries look N(0, 1/d)
    g2 = torch.Generator().manual_seed(6)
    cols = torch.stack([synth.haar_orthogonal(64, g2)[:, 0] for _ in range(200)])
    assert abs(float(cols.mean())) < 0.01
    assert abs(float((cols ** 2).mean()) - 1 / 64) < 0.002


def test_covariance_spectrum_in_the_generating_basis():
    """Projected onto the generating basis, the per-axis variances of a
    single-Gaussian workload are exp(-decay i), not their square roots, and
    the axes are uncorrelated."""
    s = synth.scaled(3, n=40_000, n_queries=8_000, d=96, decay=0.03)
    w = synth.generate(s)
    Y = w.X.double() @ w.basis  # coordinates along O's columns
    var = Y.var(dim=0)
    lam = torch.exp(-0.03 * torch.arange(96, dtype=torch.float64))
    rel = (var / lam - 1).abs()
    assert float(rel.max()) < 0.05, float(rel.max())
    C = torch.corrcoef(Y[:, :8].t())
    off = C - torch.diag(torch.diagonal(C))
    assert float(off.abs().max()) < 0.03
    # queries: an independent draw from the same distribution
    Yq = w.Q.double() @ w.basis
    assert float(((Yq.var(dim=0) / lam) - 1).abs().max()) < 0.1
    assert not torch.equal(w.X[: len(w.Q)], w.Q)


def test_cluster_centres_and_equal_sizes():
    s = synth.scaled(2, n=60_000, n_queries=100, d=32, n_clusters=6, nlist=6)
    w = synth.generate(s)
    C = w.centres
    assert C.shape == (6, 32)
    # every vector sits near one centre; the clusters are about equal
    d2 = torch.cdist(w.X.double(), C)
    lab = d2.argmin(dim=1)
    counts = torch.bincount(lab, minlength=6).double()
    assert float((counts / counts.mean() - 1).abs().max()) < 0.1
    # within a cluster the spread is the recipe's, around that centre
    lam = torch.exp(-s.decay * torch.arange(32, dtype=torch.float64))
    Y = (w.X.double()[lab == 0] - C[0]) @ w.basis
    assert float(((Y.var(dim=0) / lam) - 1).abs().max()) < 0.25


def test_zipf_sizes_follow_the_power_law():
    sizes = synth.zipf_sizes(1_000_000, 100, 1.1)
    assert int(sizes.sum()) == 1_000_000 and int(sizes.min()) >= 1
    assert torch.all(sizes[:-1] >= sizes[1:])
    r = torch.arange(1, 101, dtype=torch.float64)
    expect = r.pow(-1.1) / r.pow(-1.1).sum() * 1_000_000
    assert float(((sizes.double() - expect).abs() / expect).max()) < 0.01
    tiny = synth.zipf_sizes(10, 10, 1.1)
    assert torch.equal(tiny, torch.ones(10, dtype=torch.int64))


def test_per_query_nprobe_and_k_draws():
    s = synth.scaled(4, n=5_000, n_queries=20_000, d=16, n_clusters=8, nlist=256)
    w = synth.generate(s)
    npq, kq = w.nprobe.numpy(), w.k.numpy()
    assert npq.min() == 1 and npq.max() == 128
    assert set(np.unique(kq)) == {1, 10, 100}
    # uniform: every value about equally often
    counts = np.bincount(npq, minlength=129)[1:]
    assert counts.min() > 0.6 * counts.mean() and counts.max() < 1.4 * counts.mean()
    # nprobe is clamped to the list count
    s2 = synth.scaled(4, n=5_000, n_queries=1_000, d=16, n_clusters=8, nlist=40)
    assert int(synth.generate(s2).nprobe.max()) == 40


def test_out_of_distribution_queries_keep_the_total_energy():
    s = synth.scaled(1, n=2_000, n_queries=20_000, query_decay=0.2)
    w = synth.generate(s)
    lam = torch.exp(-s.decay * torch.arange(s.d, dtype=torch.float64))
    lam_q = torch.exp(-0.2 * torch.arange(s.d, dtype=torch.float64))
    lam_q *= lam.sum() / lam_q.sum()
    Yq = w.Q.double() @ w.basis
    assert float(((Yq.var(dim=0)[:16] / lam_q[:16]) - 1).abs().max()) < 0.1
    e_x = float((w.X.double() ** 2).sum(1).mean())
    e_q = float((w.Q.double() ** 2).sum(1).mean())
    assert abs(e_q / e_x - 1) < 0.1


def test_workload_shapes():
    """The five workloads (sizes, levels, lists, probes, k, storage)."""
    exp = {
        1: dict(n=20_000, d=128, n_queries=100, nlist=1, nprobe=1, k=10, n_levels=8,
                decay=0.05, precision="fp32"),
        2: dict(n=1_000_000, d=960, n_queries=10_000, nlist=1024, nprobe=32, k=10,
                n_levels=16, decay=0.01, n_clusters=1024, precision="fp32"),
        3: dict(n=10_000_000, d=768, n_queries=10_000, nlist=4096, nprobe=64, k=10,
                n_levels=12, decay=0.008, precision="bf16"),
        4: dict(n=5_000_000, d=384, n_queries=65_536, nlist=2048, nprobe=(1, 128),
                k=(1, 10, 100), sizes="zipf", zipf_s=1.1, precision="bf16"),
        5: dict(n=50_000_000, d=128, nlist=16384, nprobe=(8, 64), k=10,
                precision="bf16"),
    }
    for cfg, fields in exp.items():
        s = synth.spec(cfg)
        for key, val in fields.items():
            assert getattr(s, key) == val, (cfg, key)
    assert synth.spec(3).level_width == 64 and synth.spec(2).level_width == 60
