"""gs_search_static: the search entry point that allocates nothing.

It is for callers that cannot call cudaMalloc (another allocator owns the
device memory, or a request path must not synchronise the device); its scratch
is the library's fixed device array.  Its results must equal those of
gs_search with a caller workspace, on two calls in a row (the second call finds
the first call's leftovers in the shared array).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same_topk(ids, sc, ref_ids, ref_sc, exact):
    """The static-scratch result against the workspace result of the same search."""
    if exact:
        assert np.array_equal(ids, ref_ids) and np.array_equal(sc, ref_sc)
        return
    # float paths: the tolerance the parity tests use, 1e-5 relative + 1e-6
    # (weights and impacts are positive here, so |score| is the sum of |w x|)
    for q in range(ids.shape[0]):
        smap = dict(zip(ids[q].tolist(), sc[q].tolist()))
        rmap = dict(zip(ref_ids[q].tolist(), ref_sc[q].tolist()))
        for d in set(smap) & set(rmap):
            assert abs(smap[d] - rmap[d]) <= 1e-5 * abs(rmap[d]) + 1e-6, (q, d)
        kth = float(ref_sc[q, -1])
        band = 2 * (1e-5 * abs(kth) + 1e-6)
        # a document in only one of the two lists must score at the k-th place
        for d in set(smap) - set(rmap):
            assert abs(smap[d] - kth) <= band, (q, d, smap[d], kth)
        for d in set(rmap) - set(smap):
            assert abs(rmap[d] - kth) <= band, (q, d, rmap[d], kth)


def test_static_scratch_search_matches_workspace_search():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26441_gb300 import gpusparse as gs
    L = gs.load()
    dev = torch.device("cuda:0")
    docs = synth.docs(100_003, seed=0)
    qs = synth.queries(64, seed=0)
    for impact in ("u8", "f32"):
        idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                                torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
        q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
        ref = oracle.OracleIndex.from_batch(docs, impact)
        for algo in ("doc_tiled", "term_parallel"):
            opts = gs.make_opts(algo)
            for k in (10, 100):
                ref_ids, ref_sc = gs.gs_search(idx, q, k, opts)
                torch.cuda.synchronize()
                ref_ids, ref_sc = ref_ids.cpu().numpy(), ref_sc.cpu().numpy()
                for _call in range(2):
                    out_ids = torch.full((q.batch, k), -7, dtype=torch.int32, device=dev)
                    out_sc = torch.zeros((q.batch, k), dtype=idx.score_dtype, device=dev)
                    st = L.gs_search_static(idx.handle, ctypes.c_void_p(q.indptr.data_ptr()),
                                            ctypes.c_void_p(q.terms.data_ptr()),
                                            ctypes.c_void_p(q.weights.data_ptr()), q.batch, q.nnz, k,
                                            ctypes.c_void_p(out_ids.data_ptr()), ctypes.c_void_p(out_sc.data_ptr()),
                                            ctypes.byref(opts), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
                    assert st == gs.GS_OK
                    torch.cuda.synchronize()
                    ids, sc = out_ids.cpu().numpy(), out_sc.cpu().numpy()
                    _same_topk(ids, sc, ref_ids, ref_sc, impact == "u8")
                    # and the oracle's acceptance check, as in the parity tests
                    rid, rsc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, k)
                    if impact == "u8":
                        check.check_u8(ids, sc, rid, rsc)
                    else:
                        check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids, sc, rid, rsc, docs.n)
                    assert gs.gs_search_static_flags() == 0
        idx.free()


def test_static_scratch_rejects_oversized_batches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26441_gb300 import gpusparse as gs
    L = gs.load()
    dev = torch.device("cuda:0")
    docs = synth.docs(300_000, seed=1)
    qs = synth.queries(64, seed=1)
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, "f32")
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    opts = gs.make_opts("term_parallel")  # 64 dense rows of 300K scores: 77 MB of scratch
    assert idx.workspace_size(q.batch, q.nnz, 10, opts) > gs.GS_STATIC_SCRATCH_BYTES
    out_ids = torch.empty((q.batch, 10), dtype=torch.int32, device=dev)
    out_sc = torch.empty((q.batch, 10), dtype=torch.float32, device=dev)
    st = L.gs_search_static(idx.handle, ctypes.c_void_p(q.indptr.data_ptr()), ctypes.c_void_p(q.terms.data_ptr()),
                            ctypes.c_void_p(q.weights.data_ptr()), q.batch, q.nnz, 10,
                            ctypes.c_void_p(out_ids.data_ptr()), ctypes.c_void_p(out_sc.data_ptr()),
                            ctypes.byref(opts), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gs.GS_ERR_WORKSPACE
    idx.free()


def test_static_scratch_flags():
    """gs_search_static_flags reads the flag word of the fixed scratch array: a query term
    id outside the vocabulary is skipped and flagged, and the next clean call clears it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26441_gb300 import gpusparse as gs
    dev = torch.device("cuda:0")
    docs = synth.docs(20_000, seed=2)
    qs = synth.queries(8, seed=2)
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, "u8")
    bad_terms = qs.terms.copy()
    bad_terms[0] = docs.vocab + 5
    ref = oracle.OracleIndex.from_batch(docs, "u8")
    for terms, want in ((bad_terms, gs.GS_FLAG_BAD_TERM), (qs.terms, 0)):
        q = gs.Queries.from_numpy(qs.indptr, terms, qs.weights, dev)
        ids, sc = gs.gs_search_static(idx, q, 10)
        assert gs.gs_search_static_flags() == want
        rid, rsc, _ = ref.topk(qs.indptr, terms, qs.weights, 10)
        check.check_u8(ids.cpu().numpy(), sc.cpu().numpy(), rid, rsc)
    idx.free()
