"""The doc-tiled search regroups a batch by shared tail terms (gs_search_opts.query_order).

Scores and top-k lists must not depend on the order of the batch (Sec. 4.1 Eq. 4
scores every query on its own): a regrouped search writes each query's result at
the query's own row, equal to the search in the caller's order (uint8 impacts:
bit for bit) and to the oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gs():
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    return gs


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _index(gs, docs, impact, dev):
    return gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                             torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)


def _search(gs, idx, q, k, **kw):
    opts = gs.make_opts("doc_tiled", **kw)
    ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts)
    ids, sc = gs.gs_search(idx, q, k, opts, ws)
    assert gs.gs_search_flags(ws) == 0
    return ids.cpu().numpy(), sc.cpu().numpy()


@pytest.fixture(scope="module")
def coll():
    # 100K documents; 600 queries of the uneven-batch mixture (up to 300 terms),
    # with empty queries mixed in: two ordering blocks (512 + 88 queries) and a
    # ragged last group
    docs = synth.docs(100_003, seed=5)
    qs = synth.queries(600, seed=5, law=synth.MIXTURE_LAW)
    rows = [tuple(map(list, qs.row(i))) for i in range(qs.n)]
    for i in (3, 17, 250, 599):
        rows[i] = ([], [])
    indptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    batch = synth.SparseBatch(indptr, np.array(sum([list(r[0]) for r in rows], []), np.int32),
                              np.array(sum([list(r[1]) for r in rows], []), np.float32))
    return docs, batch


@pytest.mark.parametrize("kw", [{"query_order": 1}, {"query_order": 1, "use_head": -1},
                                {"query_order": 1, "use_head": -1, "group_queries": 8}, {"query_order": 1, "use_head": 1}])
def test_regrouped_u8_equals_caller_order(coll, kw):
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    idx = _index(gs, docs, "u8", dev)
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    for k in (10, 1000):
        assert idx.plan(q.batch, q.nnz, k, gs.make_opts("doc_tiled", **kw)).query_order == 1
        off = dict(kw, query_order=-1)
        assert idx.plan(q.batch, q.nnz, k, gs.make_opts("doc_tiled", **off)).query_order == 0
        a_ids, a_sc = _search(gs, idx, q, k, **kw)
        b_ids, b_sc = _search(gs, idx, q, k, **off)
        assert np.array_equal(a_ids, b_ids) and np.array_equal(a_sc, b_sc)
    # against the oracle on the first block's ragged rows and the second block
    ref = oracle.OracleIndex.from_batch(docs, "u8")
    sub = qs.slice(480, 600)
    rid, rsc, _ = ref.topk(sub.indptr, sub.terms, sub.weights, 100)
    ids, sc = _search(gs, idx, q, 100, **kw)
    check.check_u8(ids[480:600], sc[480:600], rid, rsc)
    idx.free()


def test_regrouped_float_matches_oracle(coll):
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    sub = qs.slice(0, 160)  # 10 groups of 16
    idx = _index(gs, docs, "f32", dev)
    q = gs.Queries.from_numpy(sub.indptr, sub.terms, sub.weights, dev)
    ref = oracle.OracleIndex.from_batch(docs, "f32")
    for k in (10, 1000):
        assert idx.plan(q.batch, q.nnz, k, gs.make_opts("doc_tiled", query_order=1)).query_order == 1
        rid, rsc, _ = ref.topk(sub.indptr, sub.terms, sub.weights, k)
        ids, sc = _search(gs, idx, q, k, query_order=1)
        check.check_float(ref, sub.indptr, sub.terms, sub.weights, ids, sc, rid, rsc, docs.n)
    idx.free()


def test_small_groups_and_single_group_keep_the_order(coll):
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    idx = _index(gs, docs, "u8", dev)
    on = gs.make_opts("doc_tiled", query_order=1)
    assert idx.plan(600, qs.nnz, 10, gs.make_opts("doc_tiled", use_head=-1, group_queries=4, query_order=1)).query_order == 0
    assert idx.plan(16, 400, 10, on).query_order == 0
    assert idx.plan(32, 800, 10, on).query_order == 1
    # the default regroups only where the saving outweighs the regrouping: not over 100K documents
    assert idx.plan(600, qs.nnz, 10, gs.make_opts("doc_tiled")).query_order == 0
    idx.free()


def test_regrouping_keeps_a_bad_row_pointer_flagged():
    """A row pointer that ends past q_nnz: the batch keeps its order and the search
    raises GS_FLAG_BAD_INDPTR, reading only the first q_nnz entries."""
    gs = _gs()
    dev = _dev()
    docs = synth.docs(20_000, seed=12)
    qs = synth.queries(40, seed=12)
    idx = _index(gs, docs, "f32", dev)
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    L = gs.load()
    k = 5
    opts = gs.make_opts("doc_tiled", query_order=1)
    short = qs.nnz - 3
    assert idx.plan(qs.n, short, k, opts).query_order == 1
    ws = gs.alloc_workspace(idx, qs.n, short, k, opts)
    ids = torch.empty((qs.n, k), dtype=torch.int32, device=dev)
    sc = torch.empty((qs.n, k), dtype=torch.float32, device=dev)
    st = L.gs_search(idx.handle, ctypes.c_void_p(q.indptr.data_ptr()), ctypes.c_void_p(q.terms.data_ptr()),
                     ctypes.c_void_p(q.weights.data_ptr()), qs.n, short, k, ctypes.c_void_p(ids.data_ptr()),
                     ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(opts),
                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gs.GS_OK
    assert gs.gs_search_flags(ws) & gs.GS_FLAG_BAD_INDPTR
    idx.free()


def test_query_order_groups_queries_by_shared_tail_terms(coll):
    """gs_search_query_order returns the grouping the search used: a permutation of
    the batch whose groups load fewer tail postings per tile (the sum over groups of
    the list lengths of their distinct tail terms) than the caller's consecutive groups."""
    gs = _gs()
    dev = _dev()
    docs, qs = coll
    idx = _index(gs, docs, "f32", dev)
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    k = 100
    opts = gs.make_opts("doc_tiled", query_order=1)
    plan = idx.plan(q.batch, q.nnz, k, opts)
    G, H = plan.group_queries, plan.head_terms
    ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts)
    gs.gs_search(idx, q, k, opts, ws)
    perm = gs.gs_search_query_order(idx, q, k, opts, ws).cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(qs.n))
    df = np.bincount(docs.terms, minlength=docs.vocab)
    head = set(np.lexsort((np.arange(docs.vocab), -df))[:H].tolist())

    def tail_postings(order):
        tot = 0
        for g0 in range(0, qs.n, G):
            terms = set()
            for qq in order[g0:g0 + G]:
                terms.update(t for t in qs.row(int(qq))[0].tolist() if t not in head)
            tot += int(df[list(terms)].sum()) if terms else 0
        return tot

    assert tail_postings(perm) < 0.9 * tail_postings(np.arange(qs.n))
    with pytest.raises(gs.GsError) as e:
        gs.gs_search_query_order(idx, q, k, gs.make_opts("doc_tiled", query_order=-1), ws)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED
    idx.free()
