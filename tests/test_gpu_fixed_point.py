"""The doc-tiled tail in fixed point and in float, side by side in one batch
(Sec. 4.1 Eq. 4 scores, exact within the float tolerance).

With float impacts the tail adds each product w x as an integer
round(w x 2^S_q) when the rounding error of every query q of the group,
n_q 2^-(S_q + 1) for n_q tail entries, stays within 0.9e-6; 2^S_q is the
largest power of two with 2^S_q U_q <= 2^31 - 2^10 - n_q, U_q = sum over the
tail entries of |w| max|x|.  A group with one query that fails the test keeps
float reductions.  Groups hold 16 queries.  Here the even groups have queries
16 g + 4 i + 1 with their weights multiplied by 100 (n_q U_q about 100 times
over the bound: float groups), and every query of the odd groups has its
weights multiplied by 1/100 (about 100 times under it: fixed-point groups).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import check

torch = pytest.importorskip("torch")

N_DOCS, N_Q, SEED, GROUP = 100_003, 64, 5, 16


def _gs():
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    return gs


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _factor(q):
    if (q // GROUP) % 2 == 1:
        return 0.01
    return 100.0 if q % 4 == 1 else 1.0


def mixed_batch():
    docs = synth.docs(N_DOCS, seed=SEED)
    qs = synth.queries(N_Q, seed=SEED)
    w = qs.weights.astype(np.float64).copy()
    for q in range(qs.n):
        a, b = int(qs.indptr[q]), int(qs.indptr[q + 1])
        w[a:b] *= _factor(q)
    qs = synth.SparseBatch(qs.indptr.copy(), qs.terms.copy(), w.astype(np.float32), qs.vocab)
    return docs, qs


def test_the_batch_holds_both_kinds_of_group():
    """Host check of the premise (no GPU): with all of a query's terms in the
    tail, the scaled-up queries exceed the rounding bound many times over and
    the scaled-down ones stay far below it.  Head terms only lower n_q U_q, and
    the scaled-up queries keep far more than a 1/100 share of it in the tail."""
    docs, qs = mixed_batch()
    mx = np.zeros(docs.vocab)
    np.maximum.at(mx, docs.terms, np.abs(docs.weights).astype(np.float64))
    for q in range(qs.n):
        t, w = qs.row(q)
        ratio = len(t) * float(np.sum(np.abs(w) * mx[t])) / 2.0 ** 32 / 0.9e-6
        if _factor(q) > 1:
            assert ratio > 10.0, (q, ratio)
        elif _factor(q) < 1:
            assert ratio < 0.1, (q, ratio)


@pytest.fixture(scope="module")
def batch():
    return mixed_batch()


@pytest.mark.gpu
@pytest.mark.parametrize("impact,use_head", [("f32", 0), ("f32", -1), ("f32", 2), ("f32", 3), ("f16", 0),
                                             ("f16", 1), ("bf16", 0), ("bf16", -1)])
@pytest.mark.parametrize("k", [10, 1000])
def test_float_and_fixed_point_groups_are_exact(batch, impact, use_head, k):
    gs = _gs()
    dev = _dev()
    docs, qs = batch
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, impact)
    try:
        q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
        opts = gs.make_opts("doc_tiled", use_head=use_head)
        ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts)
        ids, sc = gs.gs_search(idx, q, k, opts, ws)
        assert gs.gs_search_flags(ws) & ~gs.GS_FLAG_CAND_OVERFLOW == 0
        ref = oracle.OracleIndex.from_batch(docs, impact)
        rid, rsc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, k)
        check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids.cpu().numpy(), sc.cpu().numpy(), rid, rsc,
                          docs.n)
    finally:
        idx.free()
