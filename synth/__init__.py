"""Seeded synthetic inputs for exact sparse scoring (documents and query batches).

This package only draws inputs; it holds no scoring arithmetic.  The CPU oracle
(``oracle/``) and the GPU library (``paper_2606_26441_gb300``) both take its
output and share nothing else.

The synthetic laws stand in for the paper's SPLADE vectors on MS MARCO
(Sec. 6.1: documents with ~127 non-zeros, queries with ~50, V = 30,522); the
workload sizes follow the paper's scaling experiment (Table 4: 100K to 8.8M
passages, batch 500, top-1000).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_libsynth.so")
_lib = None

VOCAB = 30522  # BERT WordPiece vocabulary (Sec. 6.1)
N_8_8M = 8_841_823  # full MS MARCO passage collection size used in Sec. 6.4


def build(force: bool = False) -> str:
    """Compile gen.c into an in-tree shared library (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_counts.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_int]
        lib.synth_counts.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_vocab_perm.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p]
        lib.synth_vocab_perm.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass(frozen=True)
class NnzLaw:
    """Mixture of up to 4 components, clamped to [lo, hi].

    Each component is (weight, kind, a, b): kind "poisson" uses a = lambda;
    kind "uniform" draws an integer uniformly in [a, b].
    """
    components: tuple
    lo: int
    hi: int

    def packed(self) -> np.ndarray:
        rows = []
        for (w, kind, a, b) in self.components:
            rows.append([float(w), 0.0 if kind == "poisson" else 1.0, float(a), float(b)])
        return np.ascontiguousarray(np.array(rows, dtype=np.float64).reshape(-1))


DOC_LAW = NnzLaw((( 1.0, "poisson", 120, 0),), 1, 400)
QUERY_LAW = NnzLaw(((1.0, "poisson", 24, 0),), 1, 64)
# uneven batches: 70% Poisson(20), 25% Poisson(60), 5% uniform[150, 300]
MIXTURE_LAW = NnzLaw(((0.70, "poisson", 20, 0), (0.25, "poisson", 60, 0), (0.05, "uniform", 150, 300)),
                     1, 300)

STREAM_DOCS = 1
STREAM_QUERIES = 2


@dataclass
class SparseBatch:
    """CSR rows of sparse vectors: row i has terms[indptr[i]:indptr[i+1]]."""
    indptr: np.ndarray  # int64[n + 1]
    terms: np.ndarray   # int32[nnz]
    weights: np.ndarray  # float32[nnz]
    vocab: int = VOCAB

    @property
    def n(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row(self, i: int):
        a, b = int(self.indptr[i]), int(self.indptr[i + 1])
        return self.terms[a:b], self.weights[a:b]

    def slice(self, lo: int, hi: int) -> "SparseBatch":
        a, b = int(self.indptr[lo]), int(self.indptr[hi])
        return SparseBatch(self.indptr[lo:hi + 1] - a, self.terms[a:b], self.weights[a:b], self.vocab)


def generate(n: int, law: NnzLaw, *, vocab: int = VOCAB, zipf_s: float = 1.1, mu: float = -0.5,
             sigma: float = 0.8, wmax: float = 5.0, seed: int = 0, stream: int = STREAM_DOCS,
             sort_terms: bool = True, threads: int = 0, perm_seed: int = 0) -> SparseBatch:
    """Draw n sparse vectors (see gen.c for the laws).

    seed selects the draws; perm_seed the vocabulary permutation shared by the
    documents and queries of one collection.
    """
    lib = _load()
    comp = law.packed()
    nnz = np.empty(n, dtype=np.int32)
    rc = lib.synth_counts(n, seed, stream, len(law.components), comp.ctypes.data, law.lo, law.hi,
                          nnz.ctypes.data, threads)
    if rc != 0:
        raise ValueError(f"synth_counts failed ({rc})")
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nnz, out=indptr[1:])
    total = int(indptr[-1])
    terms = np.empty(total, dtype=np.int32)
    w = np.empty(total, dtype=np.float32)
    rc = lib.synth_fill(n, vocab, zipf_s, mu, sigma, wmax, seed, perm_seed, stream, indptr.ctypes.data,
                        1 if sort_terms else 0, terms.ctypes.data, w.ctypes.data, threads)
    if rc != 0:
        raise ValueError(f"synth_fill failed ({rc})")
    return SparseBatch(indptr, terms, w, vocab)


def vocab_perm(vocab: int = VOCAB, perm_seed: int = 0) -> np.ndarray:
    """Zipf rank (0-based) -> term id, as used by generate()."""
    out = np.empty(vocab, dtype=np.int32)
    if _load().synth_vocab_perm(vocab, perm_seed, out.ctypes.data) != 0:
        raise ValueError("synth_vocab_perm failed")
    return out


def docs(n: int, seed: int = 0, vocab: int = VOCAB, law: NnzLaw = DOC_LAW, threads: int = 0) -> SparseBatch:
    """Document vectors: rows sorted by term id."""
    return generate(n, law, vocab=vocab, seed=seed, stream=STREAM_DOCS, sort_terms=True, threads=threads)


def queries(n: int, seed: int = 0, vocab: int = VOCAB, law: NnzLaw = QUERY_LAW,
            threads: int = 0) -> SparseBatch:
    """Query vectors: rows keep draw order; independent of the number of documents."""
    return generate(n, law, vocab=vocab, seed=seed, stream=STREAM_QUERIES, sort_terms=False,
                    threads=threads)


@dataclass(frozen=True)
class Workload:
    """One named workload: sizes of the collection and of the query batch."""
    name: str
    n_docs: int
    batch: int
    k: int
    impacts: tuple = ("f32",)
    query_law: NnzLaw = QUERY_LAW
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    # 100K docs, 64 queries, top-10 (oracle finishes in seconds)
    "docs100k_b64_top10": Workload("docs100k_b64_top10", 100_000, 64, 10, ("f32",)),
    # 1M docs, 128 queries, top-1000; FP32 and uint8 impacts
    "docs1m_b128_top1000": Workload("docs1m_b128_top1000", 1_000_000, 128, 1000, ("f32", "u8")),
    # 8.84M docs, 500 queries, top-1000; FP32 / FP16 / BF16 / uint8 impacts
    "docs8.8m_b500_top1000": Workload("docs8.8m_b500_top1000", N_8_8M, 500, 1000,
                                      ("f32", "f16", "bf16", "u8")),
    # uneven batches over 8.84M docs: mixture query law, several batch sizes and k
    "docs8.8m_uneven": Workload("docs8.8m_uneven", N_8_8M, 1024, 1000, ("f32",), MIXTURE_LAW,
                                {"batches": (1, 8, 64, 256, 1024), "ks": (10, 100, 1000)}),
    # serving: 1M and 8.84M documents resident (FP16), Poisson arrivals at several rates
    "serving_1m_8.8m": Workload("serving_1m_8.8m", N_8_8M, 256, 1000, ("f16",), MIXTURE_LAW,
                                {"rates": (200, 1000, 2000, 5000, 10000, 20000), "seconds": 3.0}),
    # document sparsity sweep: 500K docs with exactly n terms each, 64 queries, top-1000
    "sparsity_500k_b64": Workload("sparsity_500k_b64", 500_000, 64, 1000, ("f32",), QUERY_LAW,
                                  {"doc_nnz": (10, 50, 100, 200, 500)}),
}
