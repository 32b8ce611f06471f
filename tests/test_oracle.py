"""Pins for the CPU oracle (no GPU).

The oracle is the plain definition of Sec. 4.1, Eq. 4 with exact top-k by
(score desc, doc id asc).  It is pinned here against things other than itself:
a hand-worked example, pure-Python brute force with library rounding,
numpy's dense matrix product, closed forms and invariants.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _batch_from_dicts(rows, vocab):
    indptr, terms, w = [0], [], []
    for r in rows:
        items = sorted((int(t), float(v)) for t, v in r.items())
        terms += [t for t, _ in items]
        w += [v for _, v in items]
        indptr.append(len(terms))
    return synth.SparseBatch(np.array(indptr, np.int64), np.array(terms, np.int32),
                             np.array(w, np.float32), vocab)


def _queries(qs, vocab):
    indptr, terms, w = [0], [], []
    for q in qs:
        terms += q["terms"]
        w += q["weights"]
        indptr.append(len(terms))
    return synth.SparseBatch(np.array(indptr, np.int64), np.array(terms, np.int32),
                             np.array(w, np.float32), vocab)


@pytest.mark.parametrize("impact", ["f32", "u8"])
def test_handworked_golden(impact):
    g = json.load(open(os.path.join(GOLDEN, "handworked.json")))
    docs = _batch_from_dicts(g["docs"], g["vocab"])
    qs = _queries(g["queries"], g["vocab"])
    ix = oracle.OracleIndex.from_batch(docs, impact)
    rows, bad = ix.rows(qs.indptr, qs.terms, qs.weights)
    assert not bad
    ids, sc, _ = ix.topk(qs.indptr, qs.terms, qs.weights, docs.n)
    for i, q in enumerate(g["queries"]):
        exp = q[impact]
        assert rows[i].tolist() == [float(v) for v in exp["scores"]], q["name"]
        assert ids[i].tolist() == exp["order"], q["name"]
        assert sc[i].tolist() == [float(exp["scores"][d]) for d in exp["order"]]


SMALL_DOC_LAW = synth.NnzLaw(((1.0, "poisson", 30, 0),), 1, 60)
SMALL_QUERY_LAW = synth.NnzLaw(((1.0, "poisson", 12, 0),), 1, 40)


def _tiny(seed, n=600, vocab=300, B=12):
    """Small collections keep the laws' shape at a vocabulary small enough for brute force."""
    docs = synth.docs(n, seed=seed, vocab=vocab, law=SMALL_DOC_LAW)
    qs = synth.queries(B, seed=seed, vocab=vocab, law=SMALL_QUERY_LAW)
    return docs, qs


@pytest.mark.parametrize("impact", ["f32", "f16", "bf16", "u8"])
def test_against_python_bruteforce(impact):
    docs, qs = _tiny(3)
    ix = oracle.OracleIndex.from_batch(docs, impact)
    rows, bad = ix.rows(qs.indptr, qs.terms, qs.weights)
    assert not bad
    ref = bf.score_rows(docs, qs, impact)
    # same per-document addition order (query-term order) -> identical doubles
    assert np.array_equal(rows, np.array(ref))
    k = 37
    ids, sc, _ = ix.topk(qs.indptr, qs.terms, qs.weights, k)
    rids, rsc = bf.topk(ref, k)
    assert ids.tolist() == rids
    assert sc.tolist() == rsc


def test_against_numpy_dense_matmul():
    """Library special case: dense FP64 Q @ D^T then lexsort by (-score, id)."""
    docs, qs = _tiny(5, n=1500, vocab=400, B=16)
    D = np.zeros((docs.n, docs.vocab))
    for d in range(docs.n):
        t, w = docs.row(d)
        D[d, t] = w.astype(np.float64)
    Q = np.zeros((qs.n, qs.vocab))
    for q in range(qs.n):
        t, w = qs.row(q)
        np.add.at(Q[q], t, w.astype(np.float64))
    S = Q @ D.T
    A = np.abs(Q) @ np.abs(D).T
    ix = oracle.OracleIndex.from_batch(docs)
    rows, _ = ix.rows(qs.indptr, qs.terms, qs.weights)
    tol = 64 * 2.0 ** -52 * A + 1e-300
    assert np.all(np.abs(rows - S) <= tol)
    k = 50
    ids, sc, _ = ix.topk(qs.indptr, qs.terms, qs.weights, k)
    for q in range(qs.n):
        order = np.lexsort((np.arange(docs.n), -S[q]))[:k]
        # identical except where two scores are within rounding of each other
        diff = set(order.tolist()) ^ set(ids[q].tolist())
        theta = S[q][order[-1]]
        for d in diff:
            assert abs(S[q][d] - theta) <= 2 * tol[q].max()
        assert np.all(np.diff(sc[q]) <= 0)


def test_closed_forms():
    docs, qs = _tiny(7, n=800, vocab=200, B=4)
    ix = oracle.OracleIndex.from_batch(docs)
    # one-term query, weight 1: scores are the term's stored impacts, the rest 0
    for t in [0, 1, 17, 150]:
        plist_docs, plist_x = ix.posting_list(t)
        ids, sc, _ = ix.topk(np.array([0, 1]), np.array([t], np.int32), np.array([1.0], np.float32), docs.n)
        nz = len(plist_docs)
        order = sorted(range(nz), key=lambda i: (-plist_x[i], plist_docs[i]))
        assert ids[0][:nz].tolist() == [int(plist_docs[i]) for i in order]
        assert sc[0][:nz].tolist() == [float(plist_x[i]) for i in order]
        rest = sorted(set(range(docs.n)) - set(plist_docs.tolist()))
        assert ids[0][nz:].tolist() == rest
        assert np.all(sc[0][nz:] == 0.0)
    # empty query: ids 0..k-1, zero scores
    ids, sc, _ = ix.topk(np.array([0, 0]), np.zeros(0, np.int32), np.zeros(0, np.float32), 25)
    assert ids[0].tolist() == list(range(25)) and np.all(sc == 0)
    # k = N is a full sort: a permutation of all documents
    ids, sc, _ = ix.topk(qs.indptr, qs.terms, qs.weights, docs.n)
    for q in range(qs.n):
        assert sorted(ids[q].tolist()) == list(range(docs.n))


def test_posting_lists_layout_rules():
    """Lists are doc-sorted and hold exactly the documents that carry the term (Sec. 3.2)."""
    docs, _ = _tiny(9, n=700, vocab=150, B=1)
    ix = oracle.OracleIndex.from_batch(docs)
    assert ix.postings == docs.nnz
    for t in range(docs.vocab):
        d, x = ix.posting_list(t)
        assert np.all(np.diff(d) > 0)
        for di, xi in zip(d[:5], x[:5]):
            tt, ww = docs.row(int(di))
            assert float(ww[list(tt).index(t)]) == xi


@pytest.mark.parametrize("impact", ["f32", "u8"])
def test_term_order_permutation(impact):
    docs, qs = _tiny(11)
    ix = oracle.OracleIndex.from_batch(docs, impact)
    rng = np.random.default_rng(0)
    perm_terms, perm_w = qs.terms.copy(), qs.weights.copy()
    for q in range(qs.n):
        a, b = qs.indptr[q], qs.indptr[q + 1]
        p = rng.permutation(b - a)
        perm_terms[a:b] = qs.terms[a:b][p]
        perm_w[a:b] = qs.weights[a:b][p]
    r1, _ = ix.rows(qs.indptr, qs.terms, qs.weights)
    r2, _ = ix.rows(qs.indptr, perm_terms, perm_w)
    if impact == "u8":
        assert np.array_equal(r1, r2)
    else:
        assert np.allclose(r1, r2, rtol=1e-13, atol=1e-300)


def test_linearity_and_scaling():
    docs, qs = _tiny(13, B=2)
    ix = oracle.OracleIndex.from_batch(docs)
    t, w = qs.row(0)
    h = len(t) // 2
    parts = [(t[:h], w[:h]), (t[h:], w[h:])]
    rows = []
    for pt, pw in parts + [(t, w)]:
        r, _ = ix.rows(np.array([0, len(pt)]), pt, pw)
        rows.append(r[0])
    assert np.allclose(rows[0] + rows[1], rows[2], rtol=1e-13, atol=1e-12)
    # scaling every query weight by 2 doubles every FP64 score exactly
    r1, _ = ix.rows(qs.indptr, qs.terms, qs.weights)
    r2, _ = ix.rows(qs.indptr, qs.terms, qs.weights * 2)
    assert np.array_equal(2 * r1, r2)


def test_u8_quantisation_pins():
    # round(w * 255 / 5) with half-to-even, clamped
    cases = {0.0: 0, 0.01: 1, 0.5: 26, 1.0: 51, 1.5: 76, 2.5: 128, 4.99: 254, 5.0: 255, 7.0: 255, -1.0: 0}
    for w, v in cases.items():
        assert oracle.quant_u8(w) == v, w
    rng = np.random.default_rng(1)
    w = rng.uniform(0, 5, 20000).astype(np.float32)
    ref = [min(max(round(51 * float(x)), 0), 255) for x in w]
    assert oracle.stored_impacts(w, "u8").tolist() == [float(v) for v in ref]


def test_f16_bf16_rounding_pins():
    rng = np.random.default_rng(2)
    w = np.concatenate([
        rng.lognormal(-0.5, 0.8, 50000),
        rng.uniform(-70000, 70000, 2000),
        rng.uniform(-1e-4, 1e-4, 5000),  # binary16 subnormals
        np.array([65504.0, 65519.0, 65520.0, 6.1035156e-05, 5.96e-08, 2.98e-08, 1.0 + 2 ** -11,
                  1.0 + 3 * 2 ** -11, 2049.0, 2051.0])]).astype(np.float32)
    with np.errstate(over="ignore"):
        ref16 = w.astype(np.float16).astype(np.float64)
    assert np.array_equal(oracle.stored_impacts(w, "f16"), ref16)
    import torch
    wb = np.concatenate([w, np.array([3.0e38, 1e-40, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8], np.float32)])
    ref = torch.from_numpy(wb).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.stored_impacts(wb, "bf16"), ref)


def test_data_errors():
    docs, qs = _tiny(15, B=3)
    ix = oracle.OracleIndex.from_batch(docs)
    bad_t = qs.terms.copy()
    bad_t[0] = docs.vocab + 5
    _, _, bad = ix.topk(qs.indptr, bad_t, qs.weights, 5)
    assert bad
    bad_w = qs.weights.copy()
    bad_w[1] = np.nan
    _, _, bad = ix.topk(qs.indptr, qs.terms, bad_w, 5)
    assert bad
    # repeated term inside a document is rejected at build
    t = docs.terms.copy()
    t[1] = t[0]
    with pytest.raises(oracle.OracleError):
        oracle.OracleIndex(docs.indptr, t, docs.weights, docs.n, docs.vocab)
    w = docs.weights.copy()
    w[0] = 6.0
    with pytest.raises(oracle.OracleError):
        oracle.OracleIndex(docs.indptr, docs.terms, w, docs.n, docs.vocab, "u8")
    w[0] = 1e6
    with pytest.raises(oracle.OracleError):
        oracle.OracleIndex(docs.indptr, docs.terms, w, docs.n, docs.vocab, "f16")


def test_doc_major_recomputation_matches_term_walk():
    docs, qs = _tiny(17)
    for impact in ["f32", "u8", "bf16"]:
        ix = oracle.OracleIndex.from_batch(docs, impact)
        ids, sc, _ = ix.topk(qs.indptr, qs.terms, qs.weights, 40)
        s, a = ix.doc_scores(qs.indptr, qs.terms, qs.weights, ids)
        assert np.allclose(s, sc, rtol=1e-13, atol=1e-12)
        assert np.all(a >= np.abs(s) - 1e-9)
