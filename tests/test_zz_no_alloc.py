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

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same_topk(ids, sc, ref_ids, ref_sc, exact):
    if exact:
        assert np.array_equal(ids, ref_ids) and np.array_equal(sc, ref_sc)
        return
    # float paths: the tolerance the parity tests use, 1e-5 relative + 1e-6
    tol = 1e-5 * np.abs(ref_sc) + 1e-6
    assert np.all(np.abs(sc - ref_sc) <= tol)
    for q in range(ids.shape[0]):
        diff = set(ids[q].tolist()) ^ set(ref_ids[q].tolist())
        for d in diff:  # only near-equal scores at the k-th place may trade places
            assert abs(float(ref_sc[q, -1]) - float(sc[q, -1])) <= tol[q, -1]
        same = ids[q] == ref_ids[q]
        assert np.all(np.abs(sc[q][~same] - ref_sc[q][~same]) <= tol[q][~same])


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
                    _same_topk(out_ids.cpu().numpy(), out_sc.cpu().numpy(), ref_ids, ref_sc, impact == "u8")
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
