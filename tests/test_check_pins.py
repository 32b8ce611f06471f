"""Pins of the acceptance checks themselves (oracle/check.py): every float and
uint8 parity test passes or fails through them, so each must be shown to
reject a wrong answer.  Each case plants one mistake in an otherwise correct
result (taken from the oracle) and expects the check to fail for that reason;
the unmodified result, and a swap of two tied documents at the k-th place,
must pass.  Criteria (Sec. 4.1 Eq. 4 scores, Sec. 4.3 exactness, ordered by
score desc, id asc): (i) k distinct in-range ids in order, (ii) every score
within tau = 1e-5 A + 1e-6 of FP64, (iii) ids in only one of the two lists lie
within 2 tau of the k-th score.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import check

K = 10


@pytest.fixture(scope="module")
def setup():
    docs = synth.docs(3_000, seed=21)
    # documents 100 and 101 are copies of document 7: equal scores for every query
    rows = [docs.row(i) for i in range(docs.n)]
    rows[100] = rows[7]
    rows[101] = rows[7]
    indptr = np.cumsum([0] + [len(t) for t, _ in rows]).astype(np.int64)
    docs = synth.SparseBatch(indptr, np.concatenate([t for t, _ in rows]).astype(np.int32),
                             np.concatenate([w for _, w in rows]).astype(np.float32), docs.vocab)
    qs = synth.queries(4, seed=21)
    out = {}
    for impact in ("f32", "u8"):
        ref = oracle.OracleIndex.from_batch(docs, impact)
        ids, sc, _ = ref.topk(qs.indptr, qs.terms, qs.weights, K)
        full, _ = ref.rows(qs.indptr, qs.terms, qs.weights)
        out[impact] = (ref, ids, sc, full)
    return docs, qs, out


def _float(setup, ids, sc):
    docs, qs, out = setup
    ref, rid, rsc, _ = out["f32"]
    return check.check_float(ref, qs.indptr, qs.terms, qs.weights, ids, sc, rid, rsc, docs.n)


def _gpu_like(setup):
    """A correct result as the GPU returns it: float32 scores of the oracle's top-k."""
    _, _, out = setup
    _, rid, rsc, _ = out["f32"]
    return rid.copy(), rsc.astype(np.float32)


def test_correct_result_passes(setup):
    ids, sc = _gpu_like(setup)
    st = _float(setup, ids, sc)
    assert st["boundary_swaps"] == 0


def test_tied_swap_at_the_boundary_passes(setup):
    """Documents 7, 100 and 101 are identical: with query q placing them at the
    k-th place, any of them may fill it, provided the ids stay ordered."""
    docs, qs, out = setup
    ref, rid, rsc, full = out["f32"]
    ids, sc = _gpu_like(setup)
    for q in range(qs.n):
        if rid[q, -1] == 7:  # 7 at rank k, 100 and 101 just below: give rank k to 100
            ids[q, -1] = 100
            assert _float(setup, ids, sc)["boundary_swaps"] == 1
            return
    # the seed does not put document 7 at rank k: build a query that does
    t, w = docs.row(7)
    one = synth.SparseBatch(np.array([0, len(t)], np.int64), t.copy(), w.copy(), docs.vocab)
    rid1, rsc1, _ = ref.topk(one.indptr, one.terms, one.weights, 2)
    assert rid1[0].tolist() == [7, 100]  # ties ordered by id
    gpu = np.array([[7, 101]], np.int32)
    st = check.check_float(ref, one.indptr, one.terms, one.weights, gpu, rsc1.astype(np.float32), rid1, rsc1,
                           docs.n)
    assert st["boundary_swaps"] == 1


@pytest.mark.parametrize("mistake,message", [
    ("duplicate id", "duplicate ids"),
    ("reversed order", "not ordered"),
    ("id out of range", "out of range"),
    ("score off by 3 tau", "tau"),
    ("wrong document far below the k-th score", "far from the boundary"),
    ("best document dropped", "far from the boundary"),
])
def test_float_check_rejects(setup, mistake, message):
    docs, qs, out = setup
    ref, rid, rsc, full = out["f32"]
    ids, sc = _gpu_like(setup)
    q = 1
    if mistake == "duplicate id":
        ids[q, 1] = ids[q, 0]
        sc[q, 1] = sc[q, 0]
    elif mistake == "reversed order":
        ids[q] = ids[q][::-1].copy()
        sc[q] = sc[q][::-1].copy()
    elif mistake == "id out of range":
        ids[q, -1] = docs.n
    elif mistake == "score off by 3 tau":
        a = ref.doc_scores(qs.indptr, qs.terms, np.abs(qs.weights), ids.astype(np.int32))[1][q, 0]
        sc[q, 0] = np.float32(float(rsc[q, 0]) + 3 * (1e-5 * a + 1e-6))
    elif mistake == "wrong document far below the k-th score":
        far = int(np.argsort(full[q])[0])  # the lowest-scoring document, with its exact score
        assert full[q, far] < rsc[q, -1] - 1e-3
        ids[q, -1] = far
        sc[q, -1] = np.float32(full[q, far])
    elif mistake == "best document dropped":
        # rank 1 removed, the (k+1)-th document appended: sorted, scores exact, set wrong
        order = np.lexsort((np.arange(docs.n), -full[q]))
        nxt = int(order[K])
        assert full[q, order[0]] - full[q, nxt] > 1e-3
        ids[q] = np.concatenate([ids[q, 1:], [nxt]])
        sc[q] = np.concatenate([sc[q, 1:], [np.float32(full[q, nxt])]])
    with pytest.raises(AssertionError, match=message):
        _float(setup, ids, sc)


@pytest.mark.parametrize("mistake", ["swapped ranks", "score off by one", "other document"])
def test_u8_check_rejects(setup, mistake):
    _, _, out = setup
    _, rid, rsc, full = out["u8"]
    ids, sc = rid.copy(), rsc.astype(np.int32)
    check.check_u8(ids, sc, rid, rsc)  # control
    q = 2
    if mistake == "swapped ranks":
        ids[q, [0, 1]] = ids[q, [1, 0]]
    elif mistake == "score off by one":
        sc[q, 3] += 1
    else:
        ids[q, -1] = int(np.argsort(full[q])[0])
    with pytest.raises(AssertionError):
        check.check_u8(ids, sc, rid, rsc)
