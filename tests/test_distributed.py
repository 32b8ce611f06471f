"""Multi-rank logic on CPU with the gloo backend (world size 2, no GPU).

The path shards by documents: each rank holds a contiguous document range,
computes its local top-k and one exchange gathers B x k candidates; the merge
keeps the first k of (score desc, global id asc).  Here every rank uses the CPU
oracle for its shard, so the test checks the exchange and the merge rule
against the unsharded oracle.  It also checks bench.py's timing reduction
(the slowest rank's time).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    docs = synth.docs(30_000, seed=2)
    qs = synth.queries(8, seed=2)
    k = 50
    cuts = [0, 13_000, docs.n]
    lo, hi = cuts[rank], cuts[rank + 1]
    shard = docs.slice(lo, hi)
    ref = oracle.OracleIndex.from_batch(shard)
    ids, sc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, k)
    ids = torch.from_numpy(ids.astype(np.int64) + lo)
    sc = torch.from_numpy(sc)
    g_ids = [torch.empty_like(ids) for _ in range(world)]
    g_sc = [torch.empty_like(sc) for _ in range(world)]
    dist.all_gather(g_ids, ids)
    dist.all_gather(g_sc, sc)
    # timing reduction: the slowest rank's time
    span = bench.reduce_max_over_ranks(0.5 + rank, dist, torch.device("cpu"))
    if rank == 0:
        all_ids = torch.cat(g_ids, dim=1).numpy()
        all_sc = torch.cat(g_sc, dim=1).numpy()
        merged_ids = np.empty((qs.n, k), np.int64)
        merged_sc = np.empty((qs.n, k))
        for q in range(qs.n):
            order = np.lexsort((all_ids[q], -all_sc[q]))[:k]
            merged_ids[q] = all_ids[q][order]
            merged_sc[q] = all_sc[q][order]
        np.save(os.path.join(out_dir, "ids.npy"), merged_ids)
        np.save(os.path.join(out_dir, "sc.npy"), merged_sc)
        np.save(os.path.join(out_dir, "span.npy"), np.array([span]))
    dist.barrier()
    dist.destroy_process_group()


def test_doc_sharded_exchange_matches_unsharded(tmp_path):
    import oracle
    import synth
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    docs = synth.docs(30_000, seed=2)
    qs = synth.queries(8, seed=2)
    ref = oracle.OracleIndex.from_batch(docs)
    ids, sc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, 50)
    assert np.array_equal(np.load(tmp_path / "ids.npy"), ids)
    assert np.array_equal(np.load(tmp_path / "sc.npy"), sc)
    assert float(np.load(tmp_path / "span.npy")[0]) == 1.5
