"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

uint8 impacts: ids and int32 scores bit-exact.  Float impacts: oracle/check.py
criteria (i)-(iii) with tau = 1e-5 * A + 1e-6.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from oracle import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALGOS = ["term_parallel", "doc_tiled"]
# the doc-tiled kernel with and without the dense head
VARIANTS = [("term_parallel", {}), ("doc_tiled", {}), ("doc_tiled", {"use_head": -1}),
            ("doc_tiled", {"use_head": 1}), ("doc_tiled", {"use_head": 2}), ("doc_tiled", {"use_head": 3}),
            ("doc_parallel", {})]


def _supported(impact, kw):
    """The tensor-memory head (use_head 3) serves FP32 impacts only."""
    return kw.get("use_head") != 3 or impact == "f32"


def _gs():
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    return gs


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _cudart():
    """The CUDA runtime of the toolkit, for raw device-to-host copies of index arrays."""
    import glob
    import os
    for cand in [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so")] + \
            glob.glob("/usr/local/cuda*/lib64/libcudart.so*"):
        if os.path.exists(cand):
            lib = ctypes.CDLL(cand)
            lib.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            lib.cudaMemcpy.restype = ctypes.c_int
            return lib
    pytest.skip("libcudart.so not found")


class Case:
    """A collection + query batch + GPU index + oracle index for one impact type."""

    def __init__(self, docs, qs, impact, tile_docs=0, head_terms=0, doc_major=True):
        gs = _gs()
        dev = _dev()
        self.docs, self.qs, self.impact = docs, qs, impact
        self.idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                                     torch.from_numpy(docs.weights).to(dev), docs.vocab, impact, tile_docs,
                                     head_terms, doc_major)
        self.q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
        self.ref = oracle.OracleIndex.from_batch(docs, impact)

    def search(self, k, algo, **kw):
        gs = _gs()
        opts = gs.make_opts(algo, **kw)
        ws = gs.alloc_workspace(self.idx, self.q.batch, self.q.nnz, k, opts)
        ids, sc = gs.gs_search(self.idx, self.q, k, opts, ws)
        flags = gs.gs_search_flags(ws)
        return ids.cpu().numpy(), sc.cpu().numpy(), flags

    def check(self, k, algo, **kw):
        ids, sc, flags = self.search(k, algo, **kw)
        assert flags == 0, f"flags {flags}"
        rid, rsc, _ = self.ref.topk(self.qs.indptr, self.qs.terms, self.qs.weights, k)
        if self.impact == "u8":
            check.check_u8(ids, sc, rid, rsc)
            return {}
        return check.check_float(self.ref, self.qs.indptr, self.qs.terms, self.qs.weights, ids, sc, rid, rsc,
                                 self.docs.n)


@pytest.fixture(scope="module")
def tiny_docs():
    # 100K documents, 64 queries: the small workload; N is not a multiple of 32 or of a tile
    return synth.docs(100_003, seed=0), synth.queries(64, seed=0)


@pytest.fixture(scope="module")
def cases(tiny_docs):
    docs, qs = tiny_docs
    return {imp: Case(docs, qs, imp) for imp in ("f32", "f16", "bf16", "u8")}


@pytest.mark.parametrize("algo,kw", VARIANTS)
@pytest.mark.parametrize("impact", ["f32", "f16", "bf16", "u8"])
def test_topk_small_workload(cases, impact, algo, kw):
    if not _supported(impact, kw):
        pytest.skip("head kind not offered for this impact type")
    stats = cases[impact].check(10, algo, **kw)
    if stats:
        assert stats["max_rel_err"] < 1e-5


@pytest.mark.parametrize("algo,kw", VARIANTS)
@pytest.mark.parametrize("impact", ["f32", "u8"])
def test_topk_k1000_and_kmax(cases, impact, algo, kw):
    if not _supported(impact, kw):
        pytest.skip("head kind not offered for this impact type")
    cases[impact].check(1000, algo, **kw)
    cases[impact].check(2048, algo, **kw)
    cases[impact].check(1, algo, **kw)


def test_dense_head_layout(cases):
    """The dense head holds, for the longest lists, every document's stored impact (0 if absent)."""
    for impact in ("f32", "u8"):
        c = cases[impact]
        st = c.idx.stats()
        lay = c.idx.layout()
        assert st.head_terms == {"f32": 24, "u8": 64}[impact]  # defaults: FMA head 24 rows, tensor head 64
        H, ld = st.head_terms, lay.head_ld
        ib = {"f32": 4, "u8": 1}[impact]
        torch.cuda.synchronize()
        ht = np.empty(H, np.int32)
        assert _cudart().cudaMemcpy(ctypes.c_void_p(ht.ctypes.data), ctypes.c_void_p(lay.head_term), 4 * H, 2) == 0
        dense = np.empty(H * ld * ib, np.uint8)
        assert _cudart().cudaMemcpy(ctypes.c_void_p(dense.ctypes.data), ctypes.c_void_p(lay.head_dense),
                                    dense.nbytes, 2) == 0
        dense = (dense.view(np.float32) if impact == "f32" else dense).reshape(H, ld).astype(np.float64)
        lens = [len(c.ref.posting_list(int(t))[0]) for t in range(c.docs.vocab)]
        order = sorted(range(c.docs.vocab), key=lambda t: (-lens[t], t))[:H]
        assert ht.tolist() == order
        for h in range(H):
            docs_t, x_t = c.ref.posting_list(int(ht[h]))
            row = np.zeros(ld)
            row[docs_t] = x_t
            assert np.array_equal(dense[h], row)


@pytest.mark.parametrize("impact", ["f32", "f16", "bf16", "u8"])
def test_doc_tiled_keeps_two_ctas_per_sm(impact):
    """The scoring kernel's shared memory leaves room for two resident CTAs
    per SM, with and without the dense head, for every tile shape the
    autotuner tries."""
    gs = _gs()
    dev = _dev()
    docs = synth.docs(20_000, seed=3)
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
    try:
        for use_head in (0, 1, 2, -1) + ((3,) if impact == "f32" else ()):
            for G, T in ((16, 1024), (8, 2048), (4, 4096)):
                if use_head >= 0 and G != 16:
                    continue
                plan = idx.plan(64, 64 * 30, 100, gs.make_opts("doc_tiled", group_queries=G, tile_docs=T,
                                                               use_head=use_head))
                assert plan.algo == 2 and plan.tile_docs == T
                if use_head == 3:
                    # the occupancy calculator answers 1 for the tensor-memory head's
                    # kernel; its resources (64 registers, 113 KB of shared memory, 5
                    # barriers) are those of the others, and ncu's launch statistics
                    # show two resident CTAs per SM
                    assert plan.ctas_per_sm >= 1
                    continue
                assert plan.ctas_per_sm == 2, (impact, use_head, G, T, plan.ctas_per_sm)
    finally:
        idx.free()

@pytest.mark.parametrize("impact", ["f32", "u8"])
def test_dense_rows_full_matrix(cases, impact):
    """Every score of the [B, N] matrix (gs_score_dense) against the oracle rows."""
    gs = _gs()
    c = cases[impact]
    rows = gs.gs_score_dense(c.idx, c.q).cpu().numpy()
    ref_rows, _ = c.ref.rows(c.qs.indptr, c.qs.terms, c.qs.weights)
    if impact == "u8":
        check.check_rows(rows, ref_rows, "u8")
    else:
        absref = oracle.OracleIndex(c.docs.indptr, c.docs.terms, np.abs(c.docs.weights), c.docs.n, c.docs.vocab,
                                    impact)
        arows, _ = absref.rows(c.qs.indptr, c.qs.terms, np.abs(c.qs.weights))
        check.check_rows(rows, ref_rows, impact, arows)


def test_index_layout(cases):
    """Sec. 3.2: doc-sorted lists, padded to 32 with (-1, 0), per-term metadata, segment table."""
    gs = _gs()
    for impact in ("f32", "u8", "bf16"):
        c = cases[impact]
        st = c.idx.stats()
        lay = c.idx.layout()
        V, bb = st.vocab, st.block_bytes
        assert bb == {"f32": 256, "f16": 192, "bf16": 192, "u8": 160}[impact]

        def d2h(ptr, nbytes):
            out = np.empty(nbytes, dtype=np.uint8)
            torch.cuda.synchronize()
            rc = _cudart().cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr),
                                      ctypes.c_size_t(nbytes), 2)  # cudaMemcpyDeviceToHost
            assert rc == 0
            return out
        term_block = d2h(lay.term_block, 8 * (V + 1)).view(np.int64)
        term_len = d2h(lay.term_len, 4 * V).view(np.int32)
        max_score = d2h(lay.max_score, 4 * V).view(np.float32)
        blocks = d2h(lay.blocks, st.blocks * bb).reshape(st.blocks, bb)
        assert term_block[-1] == st.blocks
        # Eq. 2: padded length = ceil(len / 32) * 32
        assert np.array_equal(np.diff(term_block), (term_len.astype(np.int64) + 31) // 32)
        assert st.postings == c.docs.nnz == int(term_len.sum())
        assert st.posting_bytes == st.blocks * bb
        ids = blocks[:, :128].copy().view(np.int32).reshape(-1)
        imp_raw = blocks[:, 128:].copy()
        if impact == "f32":
            imp = imp_raw.view(np.float32).reshape(-1).astype(np.float64)
        elif impact == "u8":
            imp = imp_raw.reshape(-1).astype(np.float64)
        else:
            imp = torch.from_numpy(imp_raw.view(np.int16).reshape(-1)).view(torch.bfloat16).double().numpy()
        rng = np.random.default_rng(0)
        terms = np.concatenate([np.arange(20), rng.integers(0, V, 300)])
        seg = None
        if lay.seg:
            seg = d2h(lay.seg, 4 * V * (st.num_tiles + 1)).view(np.uint32).reshape(V, st.num_tiles + 1)
        for t in terms:
            a, b = term_block[t] * 32, term_block[t + 1] * 32
            L = term_len[t]
            rdocs, rx = c.ref.posting_list(int(t))
            assert L == len(rdocs)
            assert np.array_equal(ids[a:a + L], rdocs)
            assert np.array_equal(imp[a:a + L], rx)
            assert np.all(ids[a + L:b] == -1) and np.all(imp[a + L:b] == 0)
            if L:
                assert max_score[t] == np.float32(rx.max())
            if seg is not None:
                bounds = np.arange(st.num_tiles + 1, dtype=np.int64) * st.tile_docs
                assert np.array_equal(seg[t], np.searchsorted(rdocs, bounds, side="left"))


def test_edge_cases():
    """Empty and one-term queries, repeated terms, ragged sizes, B = 1."""
    gs = _gs()
    docs = synth.docs(5_000, seed=3)
    base = synth.queries(6, seed=3)
    rows = [([], []), ([base.terms[0]], [1.0]), ([7, 7, 9], [0.5, 0.25, 2.0])]
    for i in range(3):
        t, w = base.row(i)
        rows.append((list(t), list(w)))
    indptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    qs = synth.SparseBatch(indptr, np.array(sum([list(r[0]) for r in rows], []), np.int32),
                           np.array(sum([list(r[1]) for r in rows], []), np.float32))
    for impact in ("u8", "f32"):
        c = Case(docs, qs, impact, tile_docs=256)
        for algo, kw in VARIANTS:
            if not _supported(impact, kw):
                continue
            for k in (1, 7, 300, 2048):
                c.check(k, algo, **kw)
    # a single query
    single = qs.slice(3, 4)
    c = Case(docs, single, "f32", tile_docs=256)
    for algo in ALGOS:
        c.check(5, algo)


def test_u8_head_with_large_summed_weights():
    """A query repeating a head term sums its quantized weights past the
    range in which the tensor-core head sums exactly in FP32; that group
    takes the integer FMA head, and the result stays bit-exact."""
    docs = synth.docs(20_000, seed=5)
    top = int(np.argmax(np.bincount(docs.terms, minlength=docs.vocab)))
    base = synth.queries(20, seed=5)
    rows = [([top] * 12, [5.0] * 12)] + [tuple(map(list, base.row(i))) for i in range(1, 20)]
    indptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    qs = synth.SparseBatch(indptr, np.array(sum([list(r[0]) for r in rows], []), np.int32),
                           np.array(sum([list(r[1]) for r in rows], []), np.float32))
    c = Case(docs, qs, "u8")
    for kw in ({}, {"use_head": 2}, {"use_head": 1}):
        c.check(100, "doc_tiled", **kw)


def test_doc_tiled_large_query_groups():
    """Groups with more distinct terms than one planning batch holds and more
    (query, weight) entries than shared memory stages: the kernel plans the
    group in several batches per tile and reads entries from global memory,
    with float and with fixed-point tail reductions."""
    docs = synth.docs(30_000, seed=8)
    rng = np.random.default_rng(8)
    # large weights: the float tail falls back to float reductions; small weights
    # (sum |w| max|x| ~ 5 per query): the fixed-point tail with unstaged entries
    for n, per, wlo, whi in ((20, 150, 0.05, 3.0), (18, 100, 0.005, 0.02)):
        terms = np.concatenate([rng.choice(docs.vocab, size=per, replace=False) for _ in range(n)]).astype(np.int32)
        weights = rng.uniform(wlo, whi, size=n * per).astype(np.float32)
        indptr = np.arange(0, n * per + 1, per, dtype=np.int64)
        qs = synth.SparseBatch(indptr, terms, weights)
        for impact in ("u8", "f32", "f16"):
            c = Case(docs, qs, impact)
            for kw in ({}, {"use_head": -1}, {"use_head": 1}, {"use_head": 2}):
                for k in (10, 1000):
                    c.check(k, "doc_tiled", **kw)
            c.idx.free()


def test_fixed_point_tail_coarse_scale():
    """Float impacts accumulate the sparse tail in fixed point with a per-query
    scale 2^S chosen from sum |w| max|x|.  One heavy tail term and three tiny
    ones give a coarse scale (S near 22) while the top-1000 reaches documents
    that hold only the tiny terms (A ~ 1e-4): scores stay within tau there."""
    docs = synth.docs(40_000, seed=9)
    df = np.bincount(docs.terms, minlength=docs.vocab)
    order = np.argsort(-df, kind="stable")
    heavy, tiny = int(order[150]), [int(t) for t in order[200:203]]  # outside any dense head
    rows = [([heavy] + tiny, [90.0, 1e-4, 2e-4, 3e-4]), (tiny, [1e-4, 1e-4, 1e-4])]
    base = synth.queries(14, seed=9)
    rows += [tuple(map(list, base.row(i))) for i in range(14)]
    indptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    qs = synth.SparseBatch(indptr, np.array(sum([list(r[0]) for r in rows], []), np.int32),
                           np.array(sum([list(r[1]) for r in rows], []), np.float32))
    for impact in ("f32", "f16"):
        c = Case(docs, qs, impact)
        for k in (10, 1000):
            c.check(k, "doc_tiled")
        c.idx.free()


def test_thresholds_at_and_below_zero():
    """Sampled thresholds theta_q <= 0: negative weights on the most frequent
    terms (held by almost every document) make most scores negative, so the
    top-k reaches the documents without those terms (score 0, ties at theta_q)
    or negative scores.  The main pass keeps a document only if its own score
    is >= theta_q, whatever the other documents of its chunk hold."""
    gs = _gs()
    docs = synth.docs(100_003, seed=11)
    df = np.bincount(docs.terms, minlength=docs.vocab)
    order = np.argsort(-df, kind="stable")
    t0, t1, t2, t3 = (int(order[i]) for i in (0, 1, 2, 60))
    rows = [([t0], [-1.0]), ([t0, t1], [-0.5, -0.25]), ([t0, t3], [-0.75, 2.0]), ([t1, t2, t3], [-1.0, -1.0, -0.5]),
            ([t3], [-1.0]), ([], [])]
    base = synth.queries(12, seed=11)
    rows += [tuple(map(list, base.row(i))) for i in range(12)]
    indptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    qs = synth.SparseBatch(indptr, np.array(sum([list(r[0]) for r in rows], []), np.int32),
                           np.array(sum([list(r[1]) for r in rows], []), np.float32))
    c = Case(docs, qs, "f32")
    for kw in ({}, {"tile_docs": 2048}, {"use_head": 2}, {"use_head": -1}):
        for k in (10, 1000, 2048):
            plan = c.idx.plan(qs.n, qs.nnz, k, gs.make_opts("doc_tiled", **kw))
            assert plan.sample_stride > 0  # the sampled-threshold main pass runs
            c.check(k, "doc_tiled", **kw)
    c.idx.free()


@pytest.mark.parametrize("algo,kw", VARIANTS)
@pytest.mark.parametrize("impact", ["f32", "f16", "bf16", "u8"])
def test_handworked_golden_on_gpu(impact, algo, kw):
    """The hand-worked example of tests/golden (Sec. 4.1 Eq. 4 by hand: ties broken by id,
    u8 half-way quantisation 0.5 -> 26 and 1.5 -> 76, a negative weight, a repeated term,
    an empty query, an absent term) through the C ABI.  Its values are dyadic, exact in
    every impact type, so the GPU must reproduce the stored scores and order exactly."""
    if not _supported(impact, kw):
        pytest.skip("head kind not offered for this impact type")
    import json
    import os
    gs = _gs()
    dev = _dev()
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handworked.json")))
    rows = [sorted((int(t), float(w)) for t, w in d.items()) for d in g["docs"]]
    indptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    terms = np.array([t for r in rows for t, _ in r], np.int32)
    weights = np.array([w for r in rows for _, w in r], np.float32)
    idx = gs.gs_index_build(torch.from_numpy(indptr).to(dev), torch.from_numpy(terms).to(dev),
                            torch.from_numpy(weights).to(dev), g["vocab"], impact, 256, 0, True)
    try:
        qind = np.cumsum([0] + [len(q["terms"]) for q in g["queries"]]).astype(np.int32)
        qt = np.array([t for q in g["queries"] for t in q["terms"]], np.int32)
        qw = np.array([w for q in g["queries"] for w in q["weights"]], np.float32)
        q = gs.Queries.from_numpy(qind, qt, qw, dev)
        n = len(rows)
        for k in (n, 2):
            ids, sc = gs.gs_search(idx, q, k, gs.make_opts(algo, **kw))
            ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
            for i, qq in enumerate(g["queries"]):
                want = qq["u8" if impact == "u8" else "f32"]
                order = want["order"][:k]
                assert ids[i].tolist() == order, (qq["name"], ids[i].tolist(), order)
                assert [float(x) for x in sc[i]] == [float(want["scores"][d]) for d in order], qq["name"]
    finally:
        idx.free()


def test_bad_query_terms_are_flagged():
    gs = _gs()
    docs = synth.docs(3_000, seed=4)
    qs = synth.queries(4, seed=4)
    terms = qs.terms.copy()
    terms[0] = 10 ** 6
    w = qs.weights.copy()
    w[3] = np.nan
    bad = synth.SparseBatch(qs.indptr, terms, w)
    c = Case(docs, bad, "f32", tile_docs=256)
    ref_ids, ref_sc, flagged = c.ref.topk(bad.indptr, bad.terms, bad.weights, 5)
    assert flagged
    for algo in ALGOS:
        ids, sc, flags = c.search(5, algo)
        assert flags & gs.GS_FLAG_BAD_TERM
        assert flags & gs.GS_FLAG_BAD_WEIGHT
        check.check_float(c.ref, bad.indptr, bad.terms, bad.weights, ids, sc, ref_ids, ref_sc, docs.n)
    # synchronous calls report the skipped data with GS_ERR_DATA (results written all the same)
    k = 5
    opts = gs.make_opts("doc_tiled")
    ws = gs.alloc_workspace(c.idx, bad.n, bad.nnz, k, opts, host_io=True)
    h_ids = torch.empty((bad.n, k), dtype=torch.int32).pin_memory()
    h_sc = torch.empty((bad.n, k), dtype=torch.float32).pin_memory()
    h = (torch.from_numpy(bad.indptr.astype(np.int32)), torch.from_numpy(bad.terms), torch.from_numpy(bad.weights))
    with pytest.raises(gs.GsError) as e:
        gs.gs_search_host(c.idx, *h, k, h_ids, h_sc, ws, opts)
    assert e.value.status == gs.GS_ERR_DATA
    assert gs.gs_search_flags(ws) == gs.GS_FLAG_BAD_TERM | gs.GS_FLAG_BAD_WEIGHT
    check.check_float(c.ref, bad.indptr, bad.terms, bad.weights, h_ids.numpy(), h_sc.numpy(), ref_ids, ref_sc,
                      docs.n)
    runner = gs.Runner(c.idx, max_batch=4, max_q_nnz=bad.nnz, max_k=k, autotune=False)
    with pytest.raises(gs.GsError) as e:
        runner.search(*h, k)
    assert e.value.status == gs.GS_ERR_DATA
    runner.free()
    # the server rejects such a request at submit
    server = gs.Server([c.idx], lanes=1, max_batch=4, max_q_nnz=256, max_k=k)
    t0, w0 = bad.row(0)
    with pytest.raises(gs.GsError) as e:
        server.submit(0, np.ascontiguousarray(t0), np.ascontiguousarray(w0), k)
    assert e.value.status == gs.GS_ERR_INVALID_ARG
    qn = int(np.searchsorted(bad.indptr, 3, side="right") - 1)  # the query holding the NaN weight
    tn, wn = bad.row(qn)
    assert np.isnan(wn).any()
    with pytest.raises(gs.GsError) as e:
        server.submit(0, np.ascontiguousarray(tn), np.ascontiguousarray(wn), k)
    assert e.value.status == gs.GS_ERR_INVALID_ARG
    qv = next(i for i in range(bad.n) if bad.indptr[i] > 3 or bad.indptr[i + 1] <= 0)  # a valid query
    tv, wv = bad.row(qv)
    assert np.all(tv < docs.vocab) and np.all(np.isfinite(wv))
    ids1, sc1, _ = server.wait(server.submit(0, np.ascontiguousarray(tv), np.ascontiguousarray(wv), k), k,
                               torch.float32)
    one = bad.slice(qv, qv + 1)
    check.check_float(c.ref, one.indptr, one.terms, one.weights, ids1[None], sc1[None], ref_ids[qv:qv + 1],
                      ref_sc[qv:qv + 1], docs.n)
    server.close()


def test_query_row_pointer_past_capacity_is_flagged():
    """A query CSR whose row pointer ends past q_nnz raises GS_FLAG_BAD_INDPTR; every
    access stays inside the first q_nnz entries (the arrays here hold more)."""
    gs = _gs()
    dev = _dev()
    docs = synth.docs(5_000, seed=11)
    qs = synth.queries(6, seed=11)
    c = Case(docs, qs, "f32", tile_docs=256)
    L = gs.load()
    k = 5
    for algo in ALGOS:
        opts = gs.make_opts(algo)
        short = qs.nnz - 3  # the row pointer ends 3 entries past this capacity
        ws = gs.alloc_workspace(c.idx, qs.n, short, k, opts)
        ids = torch.empty((qs.n, k), dtype=torch.int32, device=dev)
        sc = torch.empty((qs.n, k), dtype=torch.float32, device=dev)
        st = L.gs_search(c.idx.handle, ctypes.c_void_p(c.q.indptr.data_ptr()), ctypes.c_void_p(c.q.terms.data_ptr()),
                         ctypes.c_void_p(c.q.weights.data_ptr()), qs.n, short, k, ctypes.c_void_p(ids.data_ptr()),
                         ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                         ctypes.byref(opts), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == gs.GS_OK
        assert gs.gs_search_flags(ws) & gs.GS_FLAG_BAD_INDPTR
    c.idx.free()


def test_argument_errors():
    gs = _gs()
    docs = synth.docs(5_000, seed=5)
    qs = synth.queries(3, seed=5)
    c = Case(docs, qs, "f32", tile_docs=256)
    with pytest.raises(gs.GsError):
        gs.gs_search(c.idx, c.q, docs.n + 1)
    with pytest.raises(gs.GsError) as e:
        gs.gs_search(c.idx, c.q, 4096)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.gs_search(c.idx, c.q, 5, None, ws)
    assert e.value.status == gs.GS_ERR_WORKSPACE
    # invalid documents are rejected at build
    bad_w = docs.weights.copy()
    bad_w[0] = 7.0
    with pytest.raises(gs.GsError) as e:
        gs.gs_index_build(torch.from_numpy(docs.indptr).cuda(), torch.from_numpy(docs.terms).cuda(),
                          torch.from_numpy(bad_w).cuda(), docs.vocab, "u8")
    assert e.value.status == gs.GS_ERR_DATA
    dup = docs.terms.copy()
    dup[1] = dup[0]
    with pytest.raises(gs.GsError) as e:
        gs.gs_index_build(torch.from_numpy(docs.indptr).cuda(), torch.from_numpy(dup).cuda(),
                          torch.from_numpy(docs.weights).cuda(), docs.vocab, "f32")
    assert e.value.status == gs.GS_ERR_DATA


def test_host_io_matches_device_path(cases):
    gs = _gs()
    c = cases["f32"]
    k = 100
    for algo in ALGOS:
        opts = gs.make_opts(algo)
        ids_d, sc_d = gs.gs_search(c.idx, c.q, k, opts)
        ws = gs.alloc_workspace(c.idx, c.q.batch, c.q.nnz, k, opts, host_io=True)
        h_ids = torch.empty((c.q.batch, k), dtype=torch.int32).pin_memory()
        h_sc = torch.empty((c.q.batch, k), dtype=torch.float32).pin_memory()
        gs.gs_search_host(c.idx, c.q.indptr.cpu().pin_memory(), c.q.terms.cpu().pin_memory(),
                          c.q.weights.cpu().pin_memory(), k, h_ids, h_sc, ws, opts)
        torch.cuda.synchronize()
        rid, rsc, _ = c.ref.topk(c.qs.indptr, c.qs.terms, c.qs.weights, k)
        check.check_float(c.ref, c.qs.indptr, c.qs.terms, c.qs.weights, h_ids.numpy(), h_sc.numpy(), rid, rsc,
                          c.docs.n)


def test_medium_workload_1m():
    """1M documents, 128 queries, top-1000 on FP32 and uint8 impacts (uint8 bit-exact)."""
    docs = synth.docs(1_000_000, seed=0)
    qs = synth.queries(128, seed=0)
    for impact in ("u8", "f32"):
        c = Case(docs, qs, impact)
        for algo, kw in VARIANTS:
            if _supported(impact, kw):
                c.check(1000, algo, **kw)
        c.idx.free()


def test_reduced_precision_error_vs_fp64():
    """Each impact form's error against the FP64 oracle on the FP32 impacts (the
    unrounded scores), 1M documents, 32 queries, top-1000 on the doc-tiled path.

    Gate: every form matches the FP64 oracle on its own stored impacts (uint8
    bit-exact, floats within tau).  Report (printed): the largest and mean error of
    the returned scores against the unrounded FP64 scores, relative to
    A = sum |w x|, and recall of the unrounded exact top-1000."""
    docs = synth.docs(1_000_000, seed=0)
    qs = synth.queries(32, seed=0)
    k = 1000
    truth = oracle.OracleIndex.from_batch(docs, "f32")
    tid, _, _ = truth.topk(qs.indptr, qs.terms, qs.weights, k)
    report = []
    for impact in ("f32", "f16", "bf16", "u8"):
        c = Case(docs, qs, impact)
        c.check(k, "doc_tiled")
        ids, sc, flags = c.search(k, "doc_tiled")
        assert flags == 0
        s_true, a_true = truth.doc_scores(qs.indptr, qs.terms, qs.weights, ids.astype(np.int32))
        scale = 1.0 / (51.0 * 51.0) if impact == "u8" else 1.0  # uint8: round(51 w) x round(51 x)
        rel = np.abs(sc.astype(np.float64) * scale - s_true) / np.maximum(a_true, 1e-30)
        recall = np.mean([len(set(ids[q].tolist()) & set(tid[q].tolist())) / k for q in range(qs.n)])
        report.append((impact, float(rel.max()), float(rel.mean()), float(recall)))
        c.idx.free()
    print("\nimpact | max |s - s64|/A | mean |s - s64|/A | recall@1000 of the unrounded top-1000")
    for impact, mx, mean, rec in report:
        print(f"{impact} | {mx:.3e} | {mean:.3e} | {rec:.4f}")
    by = {r[0]: r for r in report}
    assert by["f32"][1] <= 1e-5 + 1e-6 and by["f32"][3] >= 0.999
    for impact in ("f16", "bf16", "u8"):
        assert by[impact][3] >= 0.8, by[impact]


@pytest.mark.slow
def test_full_size_batch_sampled_rows():
    """The bench's workload and launch: 8,841,823 documents, one batch of 500
    queries, top-1000, default doc-tiled plan (groups of 16 queries; at this size
    the default regroups the batch by shared tail terms).  The oracle checks one
    returned row of every query group the search used, at a different position in
    each group (position 16 g + g mod the group's size of the regrouped batch),
    uint8 bit-exact and FP32 / FP16 / BF16 within tau."""
    import os
    gs = _gs()
    docs = synth.docs(synth.N_8_8M, seed=0, threads=os.cpu_count() or 0)
    qs = synth.queries(500, seed=0)
    k = 1000
    pos = np.array([16 * g + g % min(16, qs.n - 16 * g) for g in range((qs.n + 15) // 16)])
    assert len(pos) == 32 and pos[-1] < qs.n
    for impact in ("u8", "f32", "f16", "bf16"):
        c = Case(docs, qs, impact)
        opts = gs.make_opts("doc_tiled")
        assert c.idx.plan(qs.n, qs.nnz, k, opts).query_order == 1
        ws = gs.alloc_workspace(c.idx, c.q.batch, c.q.nnz, k, opts)
        ids, sc = gs.gs_search(c.idx, c.q, k, opts, ws)
        assert gs.gs_search_flags(ws) == 0
        perm = gs.gs_search_query_order(c.idx, c.q, k, opts, ws).cpu().numpy()
        assert np.array_equal(np.sort(perm), np.arange(qs.n))
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        del ws
        c.idx.free()
        rows = perm[pos]  # the caller's queries at those positions of the regrouped batch
        parts = [qs.slice(int(r), int(r) + 1) for r in rows]
        indptr = np.cumsum([0] + [p.nnz for p in parts]).astype(np.int64)
        sample = synth.SparseBatch(indptr, np.concatenate([p.terms for p in parts]),
                                   np.concatenate([p.weights for p in parts]))
        rid, rsc, _ = c.ref.topk(sample.indptr, sample.terms, sample.weights, k)
        if impact == "u8":
            check.check_u8(ids[rows], sc[rows], rid, rsc)
        else:
            check.check_float(c.ref, sample.indptr, sample.terms, sample.weights, ids[rows], sc[rows], rid, rsc,
                              docs.n)
        del c


def test_runner_graph_replay_matches_search():
    """Uneven batches through captured graphs (autotuned plans) equal the direct search."""
    gs = _gs()
    docs = synth.docs(60_000, seed=6)
    qs = synth.queries(40, seed=6, law=synth.MIXTURE_LAW)
    for impact in ("u8", "f32"):
        c = Case(docs, qs, impact, tile_docs=1024)
        runner = gs.Runner(c.idx, max_batch=32, max_q_nnz=int(qs.nnz), max_k=100)
        for (lo, hi) in [(0, 1), (1, 6), (6, 38), (0, 3), (3, 6)]:
            sub = qs.slice(lo, hi)
            for k in (10, 100):
                for _rep in range(2):  # first call tunes and captures, second replays
                    ids, sc = runner.search(torch.from_numpy(sub.indptr.astype(np.int32)),
                                            torch.from_numpy(sub.terms), torch.from_numpy(sub.weights), k)
                    rid, rsc, _ = c.ref.topk(sub.indptr, sub.terms, sub.weights, k)
                    if impact == "u8":
                        check.check_u8(ids.numpy(), sc.numpy(), rid, rsc)
                    else:
                        check.check_float(c.ref, sub.indptr, sub.terms, sub.weights, ids.numpy(), sc.numpy(), rid,
                                          rsc, docs.n)
        plan = runner.plan(8, 10)
        assert plan["tile_docs"] % 1024 == 0 and plan["tuned_ms"] > 0
        runner.free()


def test_server_same_alone_and_in_the_mix():
    """Continuous batching: every request's result is the same served alone and in a concurrent mix."""
    import random
    import threading
    gs = _gs()
    dev = _dev()
    docs_a = synth.docs(40_000, seed=7)
    docs_b = synth.docs(70_000, seed=8)
    qs = synth.queries(48, seed=7, law=synth.MIXTURE_LAW)
    idx = []
    refs = []
    for docs, impact in ((docs_a, "u8"), (docs_b, "f16")):
        idx.append(gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                                     torch.from_numpy(docs.weights).to(dev), docs.vocab, impact))
        refs.append((docs, oracle.OracleIndex.from_batch(docs, impact)))
    server = gs.Server(idx, lanes=3, max_batch=16, max_q_nnz=4096, max_k=200, max_wait_us=200)
    rng = random.Random(0)
    reqs = [(i, rng.randrange(2), rng.choice([1, 10, 200])) for i in range(qs.n)]

    def run(i, ix, k):
        t, w = qs.row(i)
        tk = server.submit(ix, np.ascontiguousarray(t), np.ascontiguousarray(w), k)
        return server.wait(tk, k, idx[ix].score_dtype)

    alone = {r: run(*r)[:2] for r in reqs}
    mix = {}
    lock = threading.Lock()

    def worker(part):
        tickets = []
        for (i, ix, k) in part:
            t, w = qs.row(i)
            tickets.append(((i, ix, k), server.submit(ix, np.ascontiguousarray(t), np.ascontiguousarray(w), k)))
        for key, tk in tickets:
            out = server.wait(tk, key[2], idx[key[1]].score_dtype)
            with lock:
                mix[key] = out[:2]

    order = reqs[:]
    rng.shuffle(order)
    threads = [threading.Thread(target=worker, args=(order[j::3],)) for j in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    st = server.stats()
    assert st["completed"] == 2 * len(reqs) and st["batches"] < 2 * len(reqs)
    for key in reqs:
        (i, ix, k) = key
        a_ids, a_sc = alone[key]
        m_ids, m_sc = mix[key]
        if ix == 0:  # uint8: bit-exact
            assert np.array_equal(a_ids, m_ids) and np.array_equal(a_sc, m_sc)
        else:
            tol = 1e-5 * np.abs(a_sc) + 1e-6
            assert np.all(np.abs(a_sc - m_sc) <= tol)
        # and both match the oracle
        docs, ref = refs[ix]
        sub = qs.slice(i, i + 1)
        rid, rsc, _ = ref.topk(sub.indptr, sub.terms, sub.weights, k)
        if ix == 0:
            check.check_u8(m_ids[None], m_sc[None], rid, rsc)
        else:
            check.check_float(ref, sub.indptr, sub.terms, sub.weights, m_ids[None], m_sc[None], rid, rsc, docs.n)
    # bounded waits: an unknown ticket is an argument error, a wait that runs out is a timeout
    with pytest.raises(gs.GsError):
        server.wait(10 ** 9, 10, torch.float32, timeout_us=0)
    server.close()


def test_sharded_merge_equals_unsharded():
    """Documents split into virtual shards (contiguous id ranges, local ids), searched
    separately and merged on the GPU: the same top-k as one index (bit-exact on uint8)."""
    gs = _gs()
    dev = _dev()
    docs = synth.docs(90_001, seed=10)
    qs = synth.queries(24, seed=10)
    cuts = [0, 20_000, 50_000, 51_000, docs.n]  # uneven shards, one tiny
    for impact in ("u8", "f32"):
        full = Case(docs, qs, impact)
        for k in (10, 1000):
            ref_ids, ref_sc = gs.gs_search(full.idx, full.q, k)
            sid, ssc, shards = [], [], []
            for a, b in zip(cuts[:-1], cuts[1:]):
                sub = docs.slice(a, b)
                c = Case(sub, qs, impact)
                kk = min(k, sub.n)
                i_, s_ = gs.gs_search(c.idx, c.q, kk)
                sid.append(i_.contiguous())
                ssc.append(s_.contiguous())
                shards.append(c)
            # shards with fewer than k documents return all of them: pad the others to a common k_in
            k_in = min(x.shape[1] for x in sid)
            ids, sc = gs.gs_merge_topk([x[:, :k_in].contiguous() for x in sid], [x[:, :k_in].contiguous() for x in ssc],
                                       cuts[:-1], min(k, k_in * len(sid)))
            torch.cuda.synchronize()
            kk = ids.shape[1]
            if impact == "u8":
                assert torch.equal(ids.cpu(), ref_ids.cpu()[:, :kk]) and torch.equal(sc.cpu(), ref_sc.cpu()[:, :kk])
            else:
                rid, rsc, _ = full.ref.topk(qs.indptr, qs.terms, qs.weights, kk)
                check.check_float(full.ref, qs.indptr, qs.terms, qs.weights, ids.cpu().numpy(), sc.cpu().numpy(),
                                  rid, rsc, docs.n)


def test_graph_capture_as_first_search_of_a_process():
    """A runner without autotuning captures its first search into a graph; in a fresh
    process that is the first search at all, so every attribute the kernels need must
    already be set when the index is built (no attribute call inside a capture)."""
    import os
    import subprocess
    import sys
    _dev()
    code = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch, synth, oracle
from oracle import check
from paper_2606_26441_gb300 import gpusparse as gs
dev = torch.device("cuda:0")
docs = synth.docs(30_000, seed=13)
qs = synth.queries(12, seed=13)
for impact in ("u8", "f32"):
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
    r = gs.Runner(idx, max_batch=16, max_q_nnz=int(qs.nnz), max_k=50, autotune=False)
    ids, sc = r.search(torch.from_numpy(qs.indptr.astype(np.int32)), torch.from_numpy(qs.terms),
                       torch.from_numpy(qs.weights), 50)
    ref = oracle.OracleIndex.from_batch(docs, impact)
    rid, rsc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, 50)
    if impact == "u8":
        check.check_u8(ids.numpy(), sc.numpy(), rid, rsc)
    else:
        check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids.numpy(), sc.numpy(), rid, rsc, docs.n)
    r.free()
    idx.free()
print("capture-first ok")
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", code, root], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    assert "capture-first ok" in p.stdout
