"""Exact top-k when a doc-tiled candidate list overflows (Sec. 4.3: every
posting is processed, the result is exact by construction).

The doc-tiled search takes a lower bound theta_q of each query's k-th score
from a sample of tiles (every R-th tile) and keeps the documents above it in
a candidate list of fixed capacity.  A collection whose sample tiles hold
none of a query's terms makes theta_q = 0, so almost every document becomes a
candidate and the list overflows.  Such queries must still get their exact
top-k: the search recomputes them (radix select of the exact k-th score over
fresh scores, then an emission pass) and only reports the overflow as an
informational flag.  Here the even queries of the batch use only even term
ids and the sample tiles hold only odd ones, so every query group mixes
overflowed and ordinary queries.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_DOCS, STRIDE = 1024, 64  # the index's default tile and the search's default sample stride


def _gs():
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    return gs


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def overflow_collection(n_docs=100_003, n_queries=64, seed=7):
    """Documents whose sample tiles (tiles j * STRIDE) carry odd term ids only;
    even queries use even term ids, odd queries odd ones."""
    docs = synth.docs(n_docs, seed=seed)
    qs = synth.queries(n_queries, seed=seed)
    terms = qs.terms.copy()
    for q in range(qs.n):
        a, b = int(qs.indptr[q]), int(qs.indptr[q + 1])
        terms[a:b] = (terms[a:b] & ~1) if q % 2 == 0 else (terms[a:b] | 1)
    qs = synth.SparseBatch(qs.indptr.copy(), terms, qs.weights.copy(), qs.vocab)
    indptr, out_t, out_w = [0], [], []
    for d in range(docs.n):
        t, w = docs.row(d)
        if (d // T_DOCS) % STRIDE == 0:
            keep = (t & 1) == 1
            t, w = t[keep], w[keep]
            if t.size == 0:
                t, w = np.array([1], np.int32), np.array([1.0], np.float32)
        out_t.append(t)
        out_w.append(w)
        indptr.append(indptr[-1] + t.size)
    docs = synth.SparseBatch(np.asarray(indptr, np.int64), np.concatenate(out_t).astype(np.int32),
                             np.concatenate(out_w).astype(np.float32), docs.vocab)
    return docs, qs


@pytest.fixture(scope="module")
def coll():
    return overflow_collection()


@pytest.mark.parametrize("impact,use_head", [("f32", 0), ("f32", -1), ("f32", 2), ("u8", 0), ("u8", 1),
                                             ("u8", -1), ("f16", 0), ("bf16", -1)])
@pytest.mark.parametrize("k", [10, 100])
def test_overflowed_queries_are_exact(coll, impact, use_head, k):
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
    try:
        q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
        opts = gs.make_opts("doc_tiled", use_head=use_head)
        plan = idx.plan(q.batch, q.nnz, k, opts)
        assert (plan.tile_docs, plan.sample_stride) == (T_DOCS, STRIDE)
        assert plan.cand_capacity < docs.n // 2  # the even queries cannot fit their candidates
        ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts)
        ids, sc = gs.gs_search(idx, q, k, opts, ws)
        flags = gs.gs_search_flags(ws)
        # the overflow did happen, and it is the only flag raised
        assert flags == gs.GS_FLAG_CAND_OVERFLOW, flags
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        ref = oracle.OracleIndex.from_batch(docs, impact)
        rid, rsc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, k)
        if impact == "u8":
            check.check_u8(ids, sc, rid, rsc)
        else:
            check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids, sc, rid, rsc, docs.n)
        # a second search on the same workspace (recovery state left behind) gives the same result
        ids2, sc2 = gs.gs_search(idx, q, k, opts, ws)
        torch.cuda.synchronize()
        if impact == "u8":
            assert np.array_equal(ids2.cpu().numpy(), ids) and np.array_equal(sc2.cpu().numpy(), sc)
    finally:
        idx.free()


@pytest.mark.parametrize("impact", ["f32", "u8"])
def test_overflow_recovery_on_a_regrouped_batch(coll, impact):
    """The recovery passes work on the regrouped batch (query groups and the
    recovery list in the regrouped order, results written at each query's own
    row): regrouping puts the even queries, whose lists all overflow, together."""
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    k = 100
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
    try:
        q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
        opts = gs.make_opts("doc_tiled", query_order=1)
        assert idx.plan(q.batch, q.nnz, k, opts).query_order == 1
        ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts)
        ids, sc = gs.gs_search(idx, q, k, opts, ws)
        assert gs.gs_search_flags(ws) == gs.GS_FLAG_CAND_OVERFLOW
        perm = gs.gs_search_query_order(idx, q, k, opts, ws).cpu().numpy()
        assert not np.array_equal(perm, np.arange(qs.n))  # the batch was regrouped
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        ref = oracle.OracleIndex.from_batch(docs, impact)
        rid, rsc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, k)
        if impact == "u8":
            check.check_u8(ids, sc, rid, rsc)
        else:
            check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids, sc, rid, rsc, docs.n)
    finally:
        idx.free()


def test_ordinary_batch_raises_no_overflow(coll):
    """The odd queries alone (their terms appear in the sample) do not overflow."""
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    odd = [q for q in range(qs.n) if q % 2 == 1]
    indptr = [0]
    t, w = [], []
    for q in odd:
        a, b = qs.row(q)
        t.append(a)
        w.append(b)
        indptr.append(indptr[-1] + a.size)
    sub = synth.SparseBatch(np.asarray(indptr, np.int64), np.concatenate(t), np.concatenate(w), qs.vocab)
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, "u8")
    try:
        q = gs.Queries.from_numpy(sub.indptr, sub.terms, sub.weights, dev)
        opts = gs.make_opts("doc_tiled")
        ws = gs.alloc_workspace(idx, q.batch, q.nnz, 100, opts)
        ids, sc = gs.gs_search(idx, q, 100, opts, ws)
        assert gs.gs_search_flags(ws) == 0
        ref = oracle.OracleIndex.from_batch(docs, "u8")
        rid, rsc, _ = ref.topk(sub.indptr, sub.terms, sub.weights, 100)
        check.check_u8(ids.cpu().numpy(), sc.cpu().numpy(), rid, rsc)
    finally:
        idx.free()
