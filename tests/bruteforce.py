"""Pure-Python brute force for tiny inputs (test helper).

score(q, d) = sum_i w_i * s_d(t_i)  (Sec. 4.1, Eq. 4), evaluated per (query,
document) pair from the document's own term -> weight map, adding the query
terms in query order.  Stored impacts come from library conversions that are
independent of the oracle's C code: numpy float16 (IEEE binary16,
nearest-even), torch bfloat16 (nearest-even) and Python's round() (half to
even) for round(w * 255 / 5).
"""
import numpy as np


def stored(w: float, impact: str) -> float:
    if impact == "f32":
        return float(np.float32(w))
    if impact == "f16":
        return float(np.float16(np.float32(w)))
    if impact == "bf16":
        import torch
        return float(torch.tensor([float(np.float32(w))], dtype=torch.float32).to(torch.bfloat16).float()[0])
    if impact == "u8":
        v = round(51 * float(np.float32(w)))  # exact product in double; round() is half-to-even
        return float(min(max(v, 0), 255))
    raise ValueError(impact)


def query_weight(w: float, impact: str) -> float:
    if impact == "u8":
        return stored(w, "u8")
    return float(np.float32(w))


def doc_maps(docs, impact):
    maps = []
    for d in range(docs.n):
        t, w = docs.row(d)
        maps.append({int(a): stored(float(b), impact) for a, b in zip(t, w)})
    return maps


def score_rows(docs, queries, impact="f32"):
    maps = doc_maps(docs, impact)
    rows = []
    for q in range(queries.n):
        qt, qw = queries.row(q)
        pairs = [(int(a), query_weight(float(b), impact)) for a, b in zip(qt, qw)]
        row = []
        for d in range(docs.n):
            m = maps[d]
            s = 0.0
            for t, w in pairs:
                x = m.get(t)
                if x is not None:
                    s += w * x
            row.append(s)
        rows.append(row)
    return rows


def topk(rows, k):
    ids, scores = [], []
    for row in rows:
        order = sorted(range(len(row)), key=lambda d: (-row[d], d))[:k]
        ids.append(order)
        scores.append([row[d] for d in order])
    return ids, scores
