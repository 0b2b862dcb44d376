"""List sharding on CPU ranks: balanced list ownership and the exact merge of
per-shard top-k results (host-side library calls; no GPU).

A search sharded by IVF lists gives every rank the index of its lists' vectors
(with all centroids, so the probes are global); each candidate lives on one
shard, so the k smallest of the union are among the shards' own k smallest.
The two-rank test builds the shards' partial results with the oracle and
checks that gathering them over torch.distributed (gloo) and merging gives
exactly the single-process top-k.
"""
import os
import socket

import numpy as np
import pytest

import paper_2510_00566_gb300 as pano


def _row_topk(d, ids, k):
    """k smallest (d, id) of one row, padded with (-1, +inf)."""
    order = np.lexsort((ids, d))[:k]
    out_i = np.full(k, -1, np.int64)
    out_d = np.full(k, np.inf, np.float32)
    out_i[:len(order)] = ids[order]
    out_d[:len(order)] = d[order]
    return out_i, out_d


def test_merge_matches_brute_force():
    rng = np.random.default_rng(7)
    n_parts, nq, k = 3, 40, 8
    ids = np.full((n_parts, nq, k), -1, np.int64)
    dists = np.full((n_parts, nq, k), np.inf, np.float32)
    for i in range(nq):
        for p in range(n_parts):
            m = int(rng.integers(0, k + 1))  # ragged: some parts have < k
            cand = rng.choice(1000, size=m, replace=False) + 1000 * p
            d = rng.integers(0, 20, size=m).astype(np.float32)  # many ties
            ids[p, i], dists[p, i] = _row_topk(d, cand, k)
    got_i, got_d = pano.panorama_merge_topk(ids, dists)
    for i in range(nq):
        v = ids[:, i].reshape(-1) >= 0
        ref_i, ref_d = _row_topk(dists[:, i].reshape(-1)[v], ids[:, i].reshape(-1)[v], k)
        assert np.array_equal(got_i[i], ref_i), i
        assert np.array_equal(got_d[i], ref_d), i


def test_merge_keeps_an_id_once_and_pads():
    ids = np.array([[[4, 9, -1]], [[4, 2, -1]]])
    dists = np.array([[[1.0, 3.0, np.inf]], [[1.0, 2.0, np.inf]]], np.float32)
    got_i, got_d = pano.panorama_merge_topk(ids, dists)
    assert got_i.tolist() == [[4, 2, 9]]
    assert got_d.tolist() == [[1.0, 2.0, 3.0]]
    got_i, got_d = pano.panorama_merge_topk(np.full((2, 1, 2), -1), np.full((2, 1, 2), np.inf))
    assert got_i.tolist() == [[-1, -1]] and np.all(np.isinf(got_d))
    with pytest.raises(pano.LibraryError):
        pano.panorama_merge_topk(np.zeros((1, 1, 0), np.int64), np.zeros((1, 1, 0), np.float32))


def test_partition_balances_zipf_lists():
    rng = np.random.default_rng(3)
    sizes = (20000 / np.arange(1, 257) ** 1.1).astype(np.int32) + rng.integers(0, 50, 256)
    for n_shards in (1, 2, 3, 8):
        owner = pano.panorama_partition_lists(sizes, n_shards)
        assert owner.min() >= 0 and owner.max() < n_shards
        load = np.bincount(owner, weights=sizes, minlength=n_shards)
        # greedy (largest first): no shard exceeds another by more than a list
        assert load.max() - load.min() <= sizes.max()
    with pytest.raises(pano.LibraryError):
        pano.panorama_partition_lists(np.array([3, -1], np.int32), 2)


def _shard_rank(rank, world, port, result_path):
    import torch.distributed as dist
    import torch
    import synth
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = synth.scaled(2, n=3000, n_queries=24, nlist=12, n_clusters=12, d=48, n_levels=4)
    w = synth.generate(s)
    X, Q = w.X.numpy(), w.Q.numpy()
    C = synth.initial_centroids(w.X, s.nlist, seed=5).numpy()
    lists, _ = oracle.assign(X, C)
    owner = pano.panorama_partition_lists(np.bincount(lists, minlength=s.nlist), world)
    probes, _ = oracle.probe(Q, C, 4)
    k = 7
    ids = np.full((len(Q), k), -1, np.int64)
    dists = np.full((len(Q), k), np.inf, np.float32)
    for i in range(len(Q)):
        mine = [c for c in probes[i] if owner[c] == rank]
        cand = np.nonzero(np.isin(lists, mine))[0]
        d = ((X[cand].astype(np.float64) - Q[i]) ** 2).sum(1).astype(np.float32)
        ids[i], dists[i] = _row_topk(d, cand, k)
    out = pano.gather_merge_topk(torch.from_numpy(ids), torch.from_numpy(dists))
    if rank == 0:
        ref_i = np.full_like(ids, -1)
        ref_d = np.full_like(dists, np.inf)
        for i in range(len(Q)):
            cand = np.nonzero(np.isin(lists, probes[i]))[0]
            d = ((X[cand].astype(np.float64) - Q[i]) ** 2).sum(1).astype(np.float32)
            ref_i[i], ref_d[i] = _row_topk(d, cand, k)
        ok = np.array_equal(out[0], ref_i) and np.array_equal(out[1], ref_d)
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    else:
        assert out is None
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_search_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    result = tmp_path / "result.txt"
    mp.start_processes(_shard_rank, args=(2, port, str(result)), nprocs=2, join=True,
                       start_method="spawn")
    assert result.read_text() == "ok"
