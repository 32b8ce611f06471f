"""Thin Python binding of libgpusparse (include/gpusparse.h) over ctypes.

Argument marshalling only: every step of index build and search runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  The
names mirror the C entry points; `Index` is a small convenience owner of a
gs_index handle.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpusparse.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_OUT_OF_MEMORY, GS_ERR_CUDA = 0, 1, 2, 3
GS_ERR_UNSUPPORTED, GS_ERR_DATA, GS_ERR_TIMEOUT, GS_ERR_WORKSPACE = 4, 5, 6, 7
IMPACTS = {"f32": 0, "f16": 1, "bf16": 2, "u8": 3}
ALGOS = {"auto": 0, "term_parallel": 1, "doc_tiled": 2, "doc_parallel": 3}
GS_FLAG_BAD_TERM, GS_FLAG_BAD_WEIGHT, GS_FLAG_CAND_OVERFLOW = 1, 2, 4
GS_FLAG_TIMEOUT, GS_FLAG_BAD_INDPTR = 8, 16
GS_MAX_K = 2048
GS_STATIC_SCRATCH_BYTES = 64 << 20

EXPORTED = (
    "gs_index_build", "gs_index_build_ex", "gs_index_info", "gs_index_get_layout", "gs_index_free",
    "gs_search_workspace_size", "gs_search", "gs_search_host", "gs_score_dense", "gs_search_flags",
    "gs_search_plan", "gs_search_query_order", "gs_search_static", "gs_search_static_flags", "gs_runner_create",
    "gs_runner_search", "gs_runner_plan",
    "gs_runner_free", "gs_server_create", "gs_server_submit", "gs_server_wait", "gs_server_stats_get",
    "gs_server_destroy", "gs_merge_topk",
    "gs_status_str", "gs_last_cuda_error", "gs_version", "gs_kernel_launches",
)
GS_NUM_STAGE_EVENTS = 6


class GsError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _lib
        msg = lib.gs_status_str(status).decode() if lib is not None else str(status)
        if status == GS_ERR_CUDA and lib is not None:
            msg += f" ({lib.gs_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg}")
        self.status = status


class gs_build_opts(ctypes.Structure):
    _fields_ = [("tile_docs", ctypes.c_int32), ("head_terms", ctypes.c_int32), ("doc_major", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class gs_index_stats(ctypes.Structure):
    _fields_ = [("num_docs", ctypes.c_int64), ("postings", ctypes.c_int64), ("padded_postings", ctypes.c_int64),
                ("blocks", ctypes.c_int64), ("posting_bytes", ctypes.c_int64), ("meta_bytes", ctypes.c_int64),
                ("vocab", ctypes.c_int32), ("impact", ctypes.c_int32), ("block_bytes", ctypes.c_int32),
                ("tile_docs", ctypes.c_int32), ("num_tiles", ctypes.c_int32), ("score_is_int", ctypes.c_int32),
                ("head_terms", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("head_bytes", ctypes.c_int64)]


class gs_index_layout(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_void_p), ("term_block", ctypes.c_void_p), ("term_len", ctypes.c_void_p),
                ("max_score", ctypes.c_void_p), ("seg", ctypes.c_void_p), ("head_term", ctypes.c_void_p),
                ("head_dense", ctypes.c_void_p), ("head_ld", ctypes.c_int64), ("doc_indptr", ctypes.c_void_p),
                ("doc_terms", ctypes.c_void_p), ("doc_impacts", ctypes.c_void_p)]


class gs_search_opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("group_queries", ctypes.c_int32), ("tile_docs", ctypes.c_int32),
                ("chunk_blocks", ctypes.c_int32), ("sample_stride", ctypes.c_int32),
                ("use_head", ctypes.c_int32), ("stage_events", ctypes.POINTER(ctypes.c_void_p)),
                ("query_order", ctypes.c_int32)]


class gs_plan_info(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("group_queries", ctypes.c_int32), ("tile_docs", ctypes.c_int32),
                ("sample_stride", ctypes.c_int32), ("num_groups", ctypes.c_int32), ("num_tiles", ctypes.c_int32),
                ("sample_tiles", ctypes.c_int32), ("chunk_blocks", ctypes.c_int32),
                ("cand_capacity", ctypes.c_int64), ("head_terms", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("query_order", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


class gs_server_config(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_q_nnz", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("max_wait_us", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("workspace_budget_bytes", ctypes.c_int64), ("opts", gs_search_opts)]


class gs_server_stats(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_in_flight", ctypes.c_int32), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("batched_queries", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("lane_workspace_bytes", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library; fails loudly when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2606_26441_gb300._build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(path)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.gs_index_build.argtypes = [P, P, P, I64, I64, I32, ctypes.c_int, P, ctypes.POINTER(P)]
    L.gs_index_build.restype = ctypes.c_int
    L.gs_index_build_ex.argtypes = [P, P, P, I64, I64, I32, ctypes.c_int, ctypes.POINTER(gs_build_opts), P,
                                    ctypes.POINTER(P)]
    L.gs_index_build_ex.restype = ctypes.c_int
    L.gs_index_info.argtypes = [P, ctypes.POINTER(gs_index_stats)]
    L.gs_index_info.restype = ctypes.c_int
    L.gs_index_get_layout.argtypes = [P, ctypes.POINTER(gs_index_layout)]
    L.gs_index_get_layout.restype = ctypes.c_int
    L.gs_index_free.argtypes = [P]
    L.gs_index_free.restype = None
    L.gs_search_workspace_size.argtypes = [P, I32, I64, I32, ctypes.POINTER(gs_search_opts), I32,
                                           ctypes.POINTER(SZ)]
    L.gs_search_workspace_size.restype = ctypes.c_int
    L.gs_search.argtypes = [P, P, P, P, I32, I64, I32, P, P, P, SZ, ctypes.POINTER(gs_search_opts), P]
    L.gs_search.restype = ctypes.c_int
    L.gs_search_host.argtypes = [P, P, P, P, I32, I64, I32, P, P, P, SZ, ctypes.POINTER(gs_search_opts), P]
    L.gs_search_host.restype = ctypes.c_int
    L.gs_score_dense.argtypes = [P, P, P, P, I32, I64, P, P, SZ, P]
    L.gs_score_dense.restype = ctypes.c_int
    L.gs_search_plan.argtypes = [P, I32, I64, I32, ctypes.POINTER(gs_search_opts), ctypes.POINTER(gs_plan_info)]
    L.gs_search_plan.restype = ctypes.c_int
    L.gs_search_static.argtypes = [P, P, P, P, I32, I64, I32, P, P, ctypes.POINTER(gs_search_opts), P]
    L.gs_search_static.restype = ctypes.c_int
    L.gs_search_static_flags.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
    L.gs_search_static_flags.restype = ctypes.c_int
    L.gs_runner_create.argtypes = [P, I32, I64, I32, ctypes.POINTER(gs_search_opts), I32, ctypes.POINTER(P)]
    L.gs_runner_create.restype = ctypes.c_int
    L.gs_runner_search.argtypes = [P, P, P, P, I32, I32, P, P, P]
    L.gs_runner_search.restype = ctypes.c_int
    L.gs_runner_plan.argtypes = [P, I32, I32, ctypes.POINTER(gs_search_opts), ctypes.POINTER(ctypes.c_float)]
    L.gs_runner_plan.restype = ctypes.c_int
    L.gs_runner_free.argtypes = [P]
    L.gs_runner_free.restype = None
    L.gs_server_create.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(gs_server_config), ctypes.POINTER(P)]
    L.gs_server_create.restype = ctypes.c_int
    L.gs_server_submit.argtypes = [P, I32, P, P, I32, I32, ctypes.POINTER(I64)]
    L.gs_server_submit.restype = ctypes.c_int
    L.gs_server_wait.argtypes = [P, I64, P, P, I64, ctypes.POINTER(ctypes.c_double)]
    L.gs_server_wait.restype = ctypes.c_int
    L.gs_server_stats_get.argtypes = [P, ctypes.POINTER(gs_server_stats)]
    L.gs_server_stats_get.restype = ctypes.c_int
    L.gs_server_destroy.argtypes = [P]
    L.gs_server_destroy.restype = None
    L.gs_merge_topk.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I64), I32, I32, I32, I32, I32,
                                P, P, P]
    L.gs_merge_topk.restype = ctypes.c_int
    L.gs_search_query_order.argtypes = [P, I32, I64, I32, ctypes.POINTER(gs_search_opts), P, SZ, P, P]
    L.gs_search_query_order.restype = ctypes.c_int
    L.gs_search_flags.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint32)]
    L.gs_search_flags.restype = ctypes.c_int
    L.gs_status_str.argtypes = [ctypes.c_int]
    L.gs_status_str.restype = ctypes.c_char_p
    L.gs_last_cuda_error.argtypes = []
    L.gs_last_cuda_error.restype = ctypes.c_char_p
    L.gs_version.argtypes = []
    L.gs_version.restype = I32
    L.gs_kernel_launches.argtypes = []
    L.gs_kernel_launches.restype = I64
    _lib = L
    return L


def _check(status: int, what: str):
    if status != GS_OK:
        raise GsError(status, what)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_opts(algo="auto", group_queries=0, tile_docs=0, chunk_blocks=0, sample_stride=0, use_head=0,
              stage_events=None, query_order=0) -> gs_search_opts:
    """gs_search_opts (0 = the library's default for each field).

    algo: "auto", "term_parallel", "doc_tiled" or "doc_parallel"; use_head: 0 = auto (FMA head for
    FP32 impacts, warp-level tensor-core head otherwise), 1 = FMA head, 2 = warp-level tensor-core head (mma.sync),
    3 = tensor-memory head (tcgen05, FP32 impacts), -1 = none;
    sample_stride 1 = no sample (every document a candidate).  stage_events: None or
    GS_NUM_STAGE_EVENTS torch.cuda.Event objects (recorded at stage boundaries).  query_order: 1 = the
    doc-tiled search regroups the batch by shared tail terms (results stay at each query's own row),
    0 = regroup where the library's cost model predicts a gain, -1 = keep the caller's order."""
    o = gs_search_opts()
    o.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    o.group_queries, o.tile_docs = group_queries, tile_docs
    o.chunk_blocks, o.sample_stride = chunk_blocks, sample_stride
    o.use_head = use_head
    o.query_order = query_order
    if stage_events is not None:
        assert len(stage_events) == GS_NUM_STAGE_EVENTS
        arr = (ctypes.c_void_p * GS_NUM_STAGE_EVENTS)(*[ctypes.c_void_p(e.cuda_event) for e in stage_events])
        o._events_keepalive = arr
        o.stage_events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
    return o


@dataclass
class Queries:
    """A query batch as device CSR tensors (int32 indptr/terms, float32 weights)."""
    indptr: torch.Tensor
    terms: torch.Tensor
    weights: torch.Tensor

    @property
    def batch(self) -> int:
        return int(self.indptr.numel() - 1)

    @property
    def nnz(self) -> int:
        return int(self.terms.numel())

    @staticmethod
    def from_numpy(indptr, terms, weights, device="cuda") -> "Queries":
        return Queries(torch.as_tensor(indptr).to(device=device, dtype=torch.int32),
                       torch.as_tensor(terms).to(device=device, dtype=torch.int32),
                       torch.as_tensor(weights).to(device=device, dtype=torch.float32))


class Index:
    """Owner of a gs_index handle (device-resident inverted index)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        self._L = load()

    @staticmethod
    def build(doc_indptr: torch.Tensor, doc_terms: torch.Tensor, doc_w: torch.Tensor, vocab: int,
              impact: str = "f32", tile_docs: int = 0, head_terms: int = 0, doc_major: bool = False,
              stream=None) -> "Index":
        return gs_index_build(doc_indptr, doc_terms, doc_w, vocab, impact, tile_docs, head_terms, doc_major, stream)

    @property
    def handle(self):
        return self._h

    def stats(self) -> gs_index_stats:
        s = gs_index_stats()
        _check(self._L.gs_index_info(self._h, ctypes.byref(s)), "gs_index_info")
        return s

    def layout(self) -> gs_index_layout:
        lay = gs_index_layout()
        _check(self._L.gs_index_get_layout(self._h, ctypes.byref(lay)), "gs_index_get_layout")
        return lay

    @property
    def score_dtype(self):
        return torch.int32 if self.stats().score_is_int else torch.float32

    def workspace_size(self, batch: int, q_nnz: int, k: int, opts: gs_search_opts | None = None,
                       host_io: bool = False) -> int:
        n = ctypes.c_size_t(0)
        _check(self._L.gs_search_workspace_size(self._h, batch, q_nnz, k, ctypes.byref(opts) if opts else None,
                                                1 if host_io else 0, ctypes.byref(n)),
               "gs_search_workspace_size")
        return int(n.value)

    def plan(self, batch: int, q_nnz: int, k: int, opts: gs_search_opts | None = None) -> gs_plan_info:
        out = gs_plan_info()
        _check(self._L.gs_search_plan(self._h, batch, q_nnz, k, ctypes.byref(opts) if opts else None,
                                      ctypes.byref(out)), "gs_search_plan")
        return out

    def search(self, q: Queries, k: int, opts: gs_search_opts | None = None, workspace: torch.Tensor | None = None,
               out_ids: torch.Tensor | None = None, out_scores: torch.Tensor | None = None, stream=None):
        return gs_search(self, q, k, opts, workspace, out_ids, out_scores, stream)

    def score_dense(self, q: Queries, workspace=None, stream=None) -> torch.Tensor:
        return gs_score_dense(self, q, workspace, stream)

    def free(self):
        if self._h is not None and self._h.value:
            self._L.gs_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gs_index_build(doc_indptr, doc_terms, doc_w, vocab: int, impact: str = "f32", tile_docs: int = 0,
                   head_terms: int = 0, doc_major: bool = False, stream=None) -> Index:
    """Builds the index from device CSR tensors (int64 indptr, int32 terms, float32 weights).

    head_terms: 0 = default (24 for FP32 impacts, 64 otherwise), -1 = no dense head."""
    L = load()
    assert doc_indptr.dtype == torch.int64 and doc_terms.dtype == torch.int32 and doc_w.dtype == torch.float32
    h = ctypes.c_void_p()
    o = gs_build_opts()
    o.tile_docs = tile_docs
    o.head_terms = head_terms
    o.doc_major = 1 if doc_major else 0
    _check(L.gs_index_build_ex(_ptr(doc_indptr), _ptr(doc_terms), _ptr(doc_w), doc_indptr.numel() - 1,
                               doc_terms.numel(), vocab, IMPACTS[impact], ctypes.byref(o), _stream(stream),
                               ctypes.byref(h)), "gs_index_build")
    return Index(h)


def alloc_workspace(index: Index, batch: int, q_nnz: int, k: int, opts=None, host_io=False, device=None):
    n = index.workspace_size(batch, q_nnz, k, opts, host_io)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device or torch.device("cuda"))


def gs_search(index: Index, q: Queries, k: int, opts=None, workspace=None, out_ids=None, out_scores=None,
              stream=None):
    """Exact top-k: returns (ids int32[B,k], scores float32|int32[B,k]) on the device (asynchronous)."""
    L = load()
    B = q.batch
    dev = q.indptr.device
    if workspace is None:
        workspace = alloc_workspace(index, B, q.nnz, k, opts, device=dev)
    if out_ids is None:
        out_ids = torch.empty((B, k), dtype=torch.int32, device=dev)
    if out_scores is None:
        out_scores = torch.empty((B, k), dtype=index.score_dtype, device=dev)
    _check(L.gs_search(index.handle, _ptr(q.indptr), _ptr(q.terms), _ptr(q.weights), B, q.nnz, k, _ptr(out_ids),
                       _ptr(out_scores), _ptr(workspace), workspace.numel(), ctypes.byref(opts) if opts else None,
                       _stream(stream)), "gs_search")
    return out_ids, out_scores


def gs_search_static(index: Index, q: Queries, k: int, opts=None, out_ids=None, out_scores=None, stream=None):
    """gs_search with the library's fixed scratch array instead of a workspace (no allocation inside)."""
    L = load()
    B = q.batch
    dev = q.indptr.device
    if out_ids is None:
        out_ids = torch.empty((B, k), dtype=torch.int32, device=dev)
    if out_scores is None:
        out_scores = torch.empty((B, k), dtype=index.score_dtype, device=dev)
    _check(L.gs_search_static(index.handle, _ptr(q.indptr), _ptr(q.terms), _ptr(q.weights), B, q.nnz, k,
                              _ptr(out_ids), _ptr(out_scores), ctypes.byref(opts) if opts else None,
                              _stream(stream)), "gs_search_static")
    return out_ids, out_scores


def gs_search_host(index: Index, h_indptr, h_terms, h_w, k: int, out_ids, out_scores, workspace, opts=None,
                   stream=None):
    """Host-memory queries and results (tensors on the CPU, ideally pinned); synchronous.

    Raises GsError(GS_ERR_DATA) when the device skipped invalid query data; the results are
    written all the same (gs_search_flags(workspace) tells which flags were raised)."""
    L = load()
    B = h_indptr.numel() - 1
    _check(L.gs_search_host(index.handle, _ptr(h_indptr), _ptr(h_terms), _ptr(h_w), B, h_terms.numel(), k,
                            _ptr(out_ids), _ptr(out_scores), _ptr(workspace), workspace.numel(),
                            ctypes.byref(opts) if opts else None, _stream(stream)), "gs_search_host")
    return out_ids, out_scores


def gs_score_dense(index: Index, q: Queries, workspace=None, stream=None) -> torch.Tensor:
    """Dense [B, N] score rows (Eq. 4) from the term-parallel scatter-add."""
    L = load()
    st = index.stats()
    dev = q.indptr.device
    o = make_opts("term_parallel")
    if workspace is None:
        workspace = alloc_workspace(index, q.batch, q.nnz, 1, o, device=dev)
    rows = torch.empty((q.batch, st.num_docs), dtype=index.score_dtype, device=dev)
    _check(L.gs_score_dense(index.handle, _ptr(q.indptr), _ptr(q.terms), _ptr(q.weights), q.batch, q.nnz,
                            _ptr(rows), _ptr(workspace), workspace.numel(), _stream(stream)), "gs_score_dense")
    return rows


def gs_search_static_flags(stream=None) -> int:
    """Synchronises the stream and returns the GS_FLAG_* bits of the last gs_search_static on this device."""
    L = load()
    f = ctypes.c_uint32(0)
    _check(L.gs_search_static_flags(_stream(stream), ctypes.byref(f)), "gs_search_static_flags")
    return int(f.value)


def gs_search_query_order(index: Index, q: Queries, k: int, opts, workspace: torch.Tensor, stream=None) -> torch.Tensor:
    """The regrouped order of the last doc-tiled search on this workspace: perm[p] = the caller's query at
    position p (group g = positions [g G, g G + G)).  Raises GsError(GS_ERR_UNSUPPORTED) when the search
    did not regroup."""
    L = load()
    perm = torch.empty(q.batch, dtype=torch.int32, device=workspace.device)
    _check(L.gs_search_query_order(index.handle, q.batch, q.nnz, k, ctypes.byref(opts) if opts else None,
                                   _ptr(workspace), workspace.numel(), _ptr(perm), _stream(stream)),
           "gs_search_query_order")
    return perm


def gs_search_flags(workspace: torch.Tensor, stream=None) -> int:
    """Synchronises the stream and returns the GS_FLAG_* bits of the last call on this workspace."""
    L = load()
    f = ctypes.c_uint32(0)
    _check(L.gs_search_flags(_ptr(workspace), _stream(stream), ctypes.byref(f)), "gs_search_flags")
    return int(f.value)


class Runner:
    """Uneven batches from captured CUDA graphs, tile shapes autotuned per batch bucket (gs_runner_*)."""

    def __init__(self, index: Index, max_batch: int, max_q_nnz: int, max_k: int, opts=None, autotune=True):
        self._L = load()
        self.index = index  # keeps the index alive
        h = ctypes.c_void_p()
        _check(self._L.gs_runner_create(index.handle, max_batch, max_q_nnz, max_k,
                                        ctypes.byref(opts) if opts else None, 1 if autotune else 0,
                                        ctypes.byref(h)), "gs_runner_create")
        self._h = h
        self.max_batch, self.max_k = max_batch, max_k

    def search(self, h_indptr, h_terms, h_w, k: int, out_ids=None, out_scores=None, stream=None):
        """Host tensors in (int32 indptr/terms, float32 weights), host tensors out; synchronous."""
        B = h_indptr.numel() - 1
        if out_ids is None:
            out_ids = torch.empty((B, k), dtype=torch.int32)
        if out_scores is None:
            out_scores = torch.empty((B, k), dtype=self.index.score_dtype)
        _check(self._L.gs_runner_search(self._h, _ptr(h_indptr), _ptr(h_terms), _ptr(h_w), B, k, _ptr(out_ids),
                                        _ptr(out_scores), _stream(stream)), "gs_runner_search")
        return out_ids, out_scores

    def plan(self, batch: int, k: int):
        o = gs_search_opts()
        ms = ctypes.c_float(0)
        _check(self._L.gs_runner_plan(self._h, batch, k, ctypes.byref(o), ctypes.byref(ms)), "gs_runner_plan")
        return {"algo": o.algo, "tile_docs": o.tile_docs, "group_queries": o.group_queries,
                "sample_stride": o.sample_stride, "use_head": o.use_head, "chunk_blocks": o.chunk_blocks,
                "query_order": o.query_order, "tuned_ms": ms.value}

    def free(self):
        if self._h is not None and self._h.value:
            self._L.gs_runner_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over resident indexes (gs_server_*)."""

    def __init__(self, indexes, lanes=4, max_batch=256, max_q_nnz=16384, max_k=1000, max_wait_us=0,
                 workspace_budget_bytes=0, opts=None):
        self._L = load()
        self.indexes = list(indexes)  # kept alive
        arr = (ctypes.c_void_p * len(self.indexes))(*[ix.handle.value for ix in self.indexes])
        cfg = gs_server_config()
        cfg.lanes, cfg.max_batch, cfg.max_q_nnz, cfg.max_k = lanes, max_batch, max_q_nnz, max_k
        cfg.max_wait_us, cfg.workspace_budget_bytes = max_wait_us, workspace_budget_bytes
        if opts is not None:
            cfg.opts = opts
        h = ctypes.c_void_p()
        _check(self._L.gs_server_create(arr, len(self.indexes), ctypes.byref(cfg), ctypes.byref(h)),
               "gs_server_create")
        self._h = h
        self.max_k = max_k

    def submit(self, index_id: int, terms, weights, k: int) -> int:
        """terms: int32 numpy array, weights: float32 numpy array (host)."""
        t = ctypes.c_int64(0)
        _check(self._L.gs_server_submit(self._h, index_id, terms.ctypes.data, weights.ctypes.data, len(terms), k,
                                        ctypes.byref(t)), "gs_server_submit")
        return t.value

    def wait(self, ticket: int, k: int, score_dtype, timeout_us: int = 10_000_000):
        """Returns (ids, scores, latency_us); raises GsError (GS_ERR_TIMEOUT) when the wait runs out."""
        import numpy as np
        ids = np.empty(k, np.int32)
        sc = np.empty(k, np.int32 if score_dtype == torch.int32 else np.float32)
        lat = ctypes.c_double(0)
        _check(self._L.gs_server_wait(self._h, ticket, ids.ctypes.data, sc.ctypes.data, timeout_us, ctypes.byref(lat)),
               "gs_server_wait")
        return ids, sc, lat.value

    def stats(self) -> dict:
        st = gs_server_stats()
        _check(self._L.gs_server_stats_get(self._h, ctypes.byref(st)), "gs_server_stats_get")
        return {f: getattr(st, f) for f, _ in gs_server_stats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            self._L.gs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_merge_topk(shard_ids, shard_scores, doc_offsets, k: int, stream=None):
    """Global top-k from per-shard [B, k_in] device results; doc_offsets: first global id of each shard."""
    L = load()
    S = len(shard_ids)
    B, k_in = shard_ids[0].shape
    ids = (ctypes.c_void_p * S)(*[t.data_ptr() for t in shard_ids])
    scs = (ctypes.c_void_p * S)(*[t.data_ptr() for t in shard_scores])
    offs = (ctypes.c_int64 * S)(*[int(o) for o in doc_offsets])
    is_int = shard_scores[0].dtype == torch.int32
    out_ids = torch.empty((B, k), dtype=torch.int32, device=shard_ids[0].device)
    out_sc = torch.empty((B, k), dtype=shard_scores[0].dtype, device=shard_ids[0].device)
    _check(L.gs_merge_topk(ids, scs, offs, S, B, k_in, k, 1 if is_int else 0, _ptr(out_ids), _ptr(out_sc),
                           _stream(stream)), "gs_merge_topk")
    return out_ids, out_sc


def gs_version() -> int:
    return int(load().gs_version())


def gs_kernel_launches() -> int:
    return int(load().gs_kernel_launches())
