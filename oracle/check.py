"""Acceptance checks of GPU top-k results against the oracle (test infrastructure).

uint8 path: ids and int32 scores equal the oracle's exactly.
Float paths, per query, with tau(d) = 1e-5 * A(q, d) + 1e-6 and
A(q, d) = sum_i |w_i x_d(t_i)| (FP64, recomputed from the document vectors):
  (i)   k distinct ids in [0, N), ordered by (GPU score desc, id asc);
  (ii)  |s_gpu(d) - s64(d)| <= tau(d) for every returned d;
  (iii) with theta the oracle's k-th score and tau* the largest tau over the
        union of both id sets, every id in only one of the two sets has
        |s64(d) - theta| <= 2 tau*.
"""
from __future__ import annotations

import numpy as np

REL_TOL = 1e-5
ABS_TOL = 1e-6


def check_u8(gpu_ids, gpu_scores, ref_ids, ref_scores):
    gpu_ids, gpu_scores = np.asarray(gpu_ids), np.asarray(gpu_scores)
    if not np.array_equal(gpu_ids, ref_ids):
        bad = np.argwhere(gpu_ids != ref_ids)
        q, j = bad[0]
        raise AssertionError(f"u8 ids differ at query {q} rank {j}: gpu {gpu_ids[q, j]} oracle {ref_ids[q, j]} "
                             f"({len(bad)} mismatches)")
    if not np.array_equal(gpu_scores.astype(np.int64), ref_scores.astype(np.int64)):
        raise AssertionError("u8 scores differ")


def check_float(index, q_indptr, q_terms, q_w, gpu_ids, gpu_scores, ref_ids, ref_scores, n_docs):
    """index: oracle.OracleIndex of the same documents and impact type."""
    gpu_ids = np.asarray(gpu_ids).astype(np.int64)
    gpu_scores = np.asarray(gpu_scores).astype(np.float64)
    B, k = gpu_ids.shape
    # (i)
    assert gpu_ids.min() >= 0 and gpu_ids.max() < n_docs, "id out of range"
    for q in range(B):
        assert len(set(gpu_ids[q].tolist())) == k, f"duplicate ids in query {q}"
        s, d = gpu_scores[q], gpu_ids[q]
        ok = (s[:-1] > s[1:]) | ((s[:-1] == s[1:]) & (d[:-1] < d[1:]))
        assert np.all(ok), f"query {q}: not ordered by (score desc, id asc)"
    # (ii)
    s64, a64 = index.doc_scores(q_indptr, q_terms, q_w, gpu_ids.astype(np.int32))
    tau = REL_TOL * a64 + ABS_TOL
    err = np.abs(gpu_scores - s64)
    if not np.all(err <= tau):
        q, j = np.argwhere(err > tau)[0]
        raise AssertionError(f"query {q} rank {j}: |gpu - fp64| = {err[q, j]:.3e} > tau {tau[q, j]:.3e}")
    # (iii)
    r64, ra = index.doc_scores(q_indptr, q_terms, q_w, np.asarray(ref_ids, dtype=np.int32))
    rtau = REL_TOL * ra + ABS_TOL
    swaps = 0
    for q in range(B):
        theta = float(ref_scores[q, -1])
        tstar = max(float(tau[q].max()), float(rtau[q].max()))
        g, o = set(gpu_ids[q].tolist()), set(np.asarray(ref_ids[q]).tolist())
        only_g = g - o
        only_o = o - g
        gmap = dict(zip(gpu_ids[q].tolist(), s64[q].tolist()))
        omap = dict(zip(np.asarray(ref_ids[q]).tolist(), r64[q].tolist()))
        for d in only_g:
            assert abs(gmap[d] - theta) <= 2 * tstar, f"query {q}: gpu-only doc {d} far from the boundary"
        for d in only_o:
            assert abs(omap[d] - theta) <= 2 * tstar, f"query {q}: oracle-only doc {d} far from the boundary"
        swaps += len(only_g)
    return {"max_abs_err": float(err.max()), "max_rel_err": float((err / np.maximum(a64, 1e-300)).max()),
            "boundary_swaps": swaps}


def check_rows(gpu_rows, ref_rows, index_impact, abs_rows=None):
    """Full [B, N] rows: exact on u8; within tau on float paths (abs_rows = A)."""
    gpu_rows = np.asarray(gpu_rows)
    if index_impact == "u8":
        assert np.array_equal(gpu_rows.astype(np.int64), ref_rows.astype(np.int64)), "u8 rows differ"
        return {"max_abs_err": 0.0}
    err = np.abs(gpu_rows.astype(np.float64) - ref_rows)
    tau = REL_TOL * abs_rows + ABS_TOL
    assert np.all(err <= tau), f"rows: max err {err.max():.3e}"
    return {"max_abs_err": float(err.max())}
