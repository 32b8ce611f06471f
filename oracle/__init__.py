"""CPU oracle for exact batched sparse scoring -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2606_26441_gb300``): the C source ``oracle.c`` builds its own
term -> postings lists, walks them in FP64 (int64 on the uint8 path) and fully
sorts each score row by (score desc, document id asc).

Definition followed: Sec. 4.1, Eq. 4 (score = sum_i w_i * s_d(t_i)) evaluated
as the scatter-adds of Eq. 5; exactness by construction (Sec. 4.3); padding
never contributes (Sec. 3.2).  Pins: ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

IMPACTS = {"f32": 0, "f16": 1, "bf16": 2, "u8": 3}
OR_OK, OR_ERR_ARG, OR_ERR_NOMEM, OR_ERR_DATA = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, OpenMP) in-tree."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    P, I64, I32, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    L.oracle_quant_u8.argtypes = [ctypes.c_float]
    L.oracle_quant_u8.restype = I32
    L.oracle_round_f16.argtypes = [ctypes.c_float]
    L.oracle_round_f16.restype = ctypes.c_double
    L.oracle_round_bf16.argtypes = [ctypes.c_float]
    L.oracle_round_bf16.restype = ctypes.c_double
    L.oracle_index_build.argtypes = [I64, I32, P, P, P, I, ctypes.POINTER(P)]
    L.oracle_index_build.restype = I
    L.oracle_index_free.argtypes = [P]
    L.oracle_index_free.restype = None
    L.oracle_index_postings.argtypes = [P]
    L.oracle_index_postings.restype = I64
    L.oracle_index_list.argtypes = [P, I32, I64, P, P]
    L.oracle_index_list.restype = I64
    L.oracle_topk.argtypes = [P, I32, P, P, P, I32, P, P, ctypes.POINTER(I), I]
    L.oracle_topk.restype = I
    L.oracle_rows.argtypes = [P, I32, P, P, P, P, ctypes.POINTER(I), I]
    L.oracle_rows.restype = I
    L.oracle_doc_scores.argtypes = [I64, I32, P, P, P, I, I32, P, P, P, I32, P, P, P, I]
    L.oracle_doc_scores.restype = I
    L.oracle_stored_array.argtypes = [I, I64, P, P]
    L.oracle_stored_array.restype = I
    L.oracle_query_array.argtypes = [I, I64, P, P]
    L.oracle_query_array.restype = I
    _lib = L
    return L


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def stored_impacts(w, impact: str) -> np.ndarray:
    """Dequantised impact values the index stores for weights w (FP64)."""
    w = _c(w, np.float32)
    out = np.empty(w.shape, dtype=np.float64)
    rc = _load().oracle_stored_array(IMPACTS[impact], w.size, w.ctypes.data, out.ctypes.data)
    if rc:
        raise OracleError(rc, "stored_impacts")
    return out


def query_weights(w, impact: str) -> np.ndarray:
    w = _c(w, np.float32)
    out = np.empty(w.shape, dtype=np.float64)
    rc = _load().oracle_query_array(IMPACTS[impact], w.size, w.ctypes.data, out.ctypes.data)
    if rc:
        raise OracleError(rc, "query_weights")
    return out


def quant_u8(w: float) -> int:
    return int(_load().oracle_quant_u8(float(w)))


class OracleIndex:
    """The oracle's own inverted index over a document CSR batch."""

    def __init__(self, indptr, terms, weights, n_docs: int, vocab: int, impact: str = "f32"):
        self._indptr = _c(indptr, np.int64)
        self._terms = _c(terms, np.int32)
        self._w = _c(weights, np.float32)
        self.n_docs, self.vocab, self.impact = int(n_docs), int(vocab), impact
        h = ctypes.c_void_p()
        rc = _load().oracle_index_build(self.n_docs, self.vocab, self._indptr.ctypes.data,
                                        self._terms.ctypes.data, self._w.ctypes.data, IMPACTS[impact],
                                        ctypes.byref(h))
        if rc:
            raise OracleError(rc, "oracle_index_build")
        self._h = h

    @classmethod
    def from_batch(cls, docs, impact: str = "f32") -> "OracleIndex":
        return cls(docs.indptr, docs.terms, docs.weights, docs.n, docs.vocab, impact)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.oracle_index_free(h)
            self._h = None

    @property
    def postings(self) -> int:
        return int(_load().oracle_index_postings(self._h))

    def posting_list(self, t: int):
        L = _load()
        n = L.oracle_index_list(self._h, int(t), 0, None, None)
        docs = np.empty(max(n, 0), dtype=np.int32)
        x = np.empty(max(n, 0), dtype=np.float64)
        L.oracle_index_list(self._h, int(t), n, docs.ctypes.data, x.ctypes.data)
        return docs, x

    def topk(self, q_indptr, q_terms, q_w, k: int, threads: int = 0):
        """Returns (ids int32[B,k], scores float64[B,k], data_error bool)."""
        qi, qt, qw = _c(q_indptr, np.int64), _c(q_terms, np.int32), _c(q_w, np.float32)
        B = qi.shape[0] - 1
        ids = np.empty((B, k), dtype=np.int32)
        sc = np.empty((B, k), dtype=np.float64)
        bad = ctypes.c_int(0)
        rc = _load().oracle_topk(self._h, B, qi.ctypes.data, qt.ctypes.data, qw.ctypes.data, k,
                                 ids.ctypes.data, sc.ctypes.data, ctypes.byref(bad), threads)
        if rc:
            raise OracleError(rc, "oracle_topk")
        return ids, sc, bool(bad.value)

    def rows(self, q_indptr, q_terms, q_w, threads: int = 0):
        """Full score rows float64[B, N] and the data-error flag."""
        qi, qt, qw = _c(q_indptr, np.int64), _c(q_terms, np.int32), _c(q_w, np.float32)
        B = qi.shape[0] - 1
        rows = np.empty((B, self.n_docs), dtype=np.float64)
        bad = ctypes.c_int(0)
        rc = _load().oracle_rows(self._h, B, qi.ctypes.data, qt.ctypes.data, qw.ctypes.data,
                                 rows.ctypes.data, ctypes.byref(bad), threads)
        if rc:
            raise OracleError(rc, "oracle_rows")
        return rows, bool(bad.value)

    def doc_scores(self, q_indptr, q_terms, q_w, docs_ids, threads: int = 0):
        """Doc-major recomputation of (score, A) for the given [B, m] document ids."""
        return doc_scores(self._indptr, self._terms, self._w, self.n_docs, self.vocab, self.impact,
                          q_indptr, q_terms, q_w, docs_ids, threads)


def doc_scores(indptr, terms, weights, n_docs, vocab, impact, q_indptr, q_terms, q_w, docs_ids,
               threads: int = 0):
    ip, tt, ww = _c(indptr, np.int64), _c(terms, np.int32), _c(weights, np.float32)
    qi, qt, qw = _c(q_indptr, np.int64), _c(q_terms, np.int32), _c(q_w, np.float32)
    ids = _c(docs_ids, np.int32)
    B, m = ids.shape
    s = np.empty((B, m), dtype=np.float64)
    a = np.empty((B, m), dtype=np.float64)
    rc = _load().oracle_doc_scores(int(n_docs), int(vocab), ip.ctypes.data, tt.ctypes.data, ww.ctypes.data,
                                   IMPACTS[impact], B, qi.ctypes.data, qt.ctypes.data, qw.ctypes.data, m,
                                   ids.ctypes.data, s.ctypes.data, a.ctypes.data, threads)
    if rc:
        raise OracleError(rc, "oracle_doc_scores")
    return s, a
