"""The seeded input generator: determinism and the stated laws (no GPU)."""
import numpy as np

import synth


def test_deterministic_and_thread_independent():
    a = synth.docs(20000, seed=4, threads=1)
    b = synth.docs(20000, seed=4, threads=4)
    assert np.array_equal(a.indptr, b.indptr)
    assert np.array_equal(a.terms, b.terms)
    assert np.array_equal(a.weights, b.weights)
    c = synth.docs(20000, seed=5)
    assert not np.array_equal(a.terms[:1000], c.terms[:1000])


def test_queries_do_not_depend_on_collection_size():
    q1 = synth.queries(50, seed=0)
    q2 = synth.queries(80, seed=0)
    assert np.array_equal(q1.indptr, q2.indptr[:51])
    assert np.array_equal(q1.terms, q2.terms[:q1.nnz])


def test_document_law():
    d = synth.docs(50000, seed=0)
    nnz = np.diff(d.indptr)
    assert nnz.min() >= 1 and nnz.max() <= 400
    assert abs(nnz.mean() - 120) < 0.5
    assert d.weights.min() > 0 and d.weights.max() <= 5.0
    # lognormal(-0.5, 0.8) median exp(-0.5)
    assert abs(np.median(d.weights) - np.exp(-0.5)) < 0.01
    for i in range(0, 50000, 997):
        t, _ = d.row(i)
        assert np.all(np.diff(t) > 0)  # sorted, no repeats
    # Zipf ranks: the rank-1 term sits in (almost) every document
    perm = synth.vocab_perm()
    df = np.bincount(d.terms, minlength=synth.VOCAB) / d.n
    assert df[perm[0]] > 0.99
    assert df[perm[0]] >= df[perm[10]] >= df[perm[100]] >= df[perm[1000]]


def test_query_laws():
    q = synth.queries(20000, seed=0)
    nnz = np.diff(q.indptr)
    assert nnz.min() >= 1 and nnz.max() <= 64 and abs(nnz.mean() - 24) < 0.3
    for i in range(0, 20000, 499):
        t, _ = q.row(i)
        assert len(set(t.tolist())) == len(t)
    m = synth.queries(20000, seed=0, law=synth.MIXTURE_LAW)
    nnz = np.diff(m.indptr)
    assert nnz.min() >= 1 and nnz.max() <= 300
    frac_long = np.mean(nnz >= 150)
    assert 0.03 < frac_long < 0.07
    expected_mean = 0.7 * 20 + 0.25 * 60 + 0.05 * 225
    assert abs(nnz.mean() - expected_mean) < 1.5


def test_documents_and_queries_share_the_vocabulary_permutation():
    """Queries drawn with another seed still put their frequent terms on frequent document terms."""
    d = synth.docs(20000, seed=3)
    df = np.bincount(d.terms, minlength=synth.VOCAB)
    for seed in (0, 5, 11):
        q = synth.queries(200, seed=seed)
        assert df[q.terms].mean() > 0.2 * d.n
