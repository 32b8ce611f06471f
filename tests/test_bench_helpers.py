"""bench.py's accounting helpers on the CPU: the kernel-source digest that keys
the recorded DRAM traffic, the recorded-traffic lookup, and the algorithmic and
naive byte counts of the roofline (checked against direct counts)."""
import os
import shutil
import types

import numpy as np
import pytest

import bench
import synth


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_2606_26441_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2606_26441_gb300", "csrc", f), csrc / f)
    return root, csrc


def test_kernel_digest_ignores_comments_not_code(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.kernel_source_digest()
    src = (csrc / "gs_doctiled.cu").read_text()
    (csrc / "gs_doctiled.cu").write_text("// a new comment\n/* and a block\n comment */\n" + src.replace("\n", "\n  "))
    assert bench.kernel_source_digest() == d0
    (csrc / "gs_doctiled.cu").write_text(src.replace("kDefaultSampleStride = 64", "kDefaultSampleStride = 63"))
    assert bench.kernel_source_digest() != d0


def test_recorded_traffic_only_for_its_workload_and_source(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = tmp_path / "traffic.md"
    rec.write_text("# record\n\n- workload: w1\n- form: f32:doc_tiled\n"
                   f"- kernel source sha256: {bench.kernel_source_digest()}\n"
                   "- dram bytes per main-pass launch: 12345\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.recorded_traffic("w1", "f32:doc_tiled") == 12345
    assert bench.recorded_traffic("w2", "f32:doc_tiled") is None
    assert bench.recorded_traffic("w1", "u8:doc_tiled") is None
    (csrc / "gs_topk.cuh").write_text((csrc / "gs_topk.cuh").read_text() + "\nint changed_code;\n")
    assert bench.recorded_traffic("w1", "f32:doc_tiled") is None


def test_byte_counts_against_direct_counts():
    docs = synth.docs(3_000, seed=11)
    qs = synth.queries(20, seed=11)
    df = np.bincount(docs.terms, minlength=docs.vocab).astype(np.int64)
    # naive stream: every (query, term) reads the whole list, plus 8 B per score cell
    direct = sum(int(df[t]) for t in qs.terms) * (4 + 4) + 8 * qs.n * docs.n
    assert bench.naive_stream_bytes(docs, qs, "f32", df) == direct
    # doc-tiled: per group of G queries, each distinct term once, outside the sample tiles
    T, R, ns = 256, 4, 2
    sdf = bench.sample_term_counts(docs, T, R, ns)
    sample_docs = set()
    for j in range(ns):
        sample_docs.update(range(j * R * T, min(docs.n, j * R * T + T)))
    main_df = np.zeros(docs.vocab, np.int64)
    for d in range(docs.n):
        if d not in sample_docs:
            t, _ = docs.row(d)
            main_df[t] += 1
    assert np.array_equal(df - sdf, main_df)
    plan = types.SimpleNamespace(group_queries=8)
    got, extra = bench.algorithmic_bytes(plan, docs, qs, "u8", "doc_tiled", {"df": df, "sample_df": sdf})
    want = 0
    for g0 in range(0, qs.n, 8):
        a, e = int(qs.indptr[g0]), int(qs.indptr[min(qs.n, g0 + 8)])
        want += int(sum(main_df[t] for t in set(qs.terms[a:e].tolist())))
    assert extra["postings"] == want and got == want * (4 + 1)
    # a regrouped batch: the groups are consecutive positions of the given order
    order = np.random.default_rng(3).permutation(qs.n)
    got_o, extra_o = bench.algorithmic_bytes(plan, docs, qs, "u8", "doc_tiled", {"df": df, "sample_df": sdf}, order)
    want_o = 0
    for g0 in range(0, qs.n, 8):
        terms = set()
        for q in order[g0:g0 + 8]:
            terms.update(qs.row(int(q))[0].tolist())
        want_o += int(sum(main_df[t] for t in terms))
    assert extra_o["postings"] == want_o and got_o == want_o * (4 + 1)
    ident = bench.algorithmic_bytes(plan, docs, qs, "u8", "doc_tiled", {"df": df, "sample_df": sdf}, np.arange(qs.n))
    assert ident[0] == got


def test_compute_work_against_direct_counts():
    """Tail reductions = (query, posting) pairs of non-head terms outside the sample
    tiles; head FLOPs = 2 x 16 queries x the group's distinct head terms x main documents."""
    docs = synth.docs(3_000, seed=12)
    qs = synth.queries(20, seed=12)
    df = np.bincount(docs.terms, minlength=docs.vocab).astype(np.int64)
    T, R, ns, H, G = 256, 4, 2, 5, 8
    sdf = bench.sample_term_counts(docs, T, R, ns)
    plan = types.SimpleNamespace(group_queries=G, sample_tiles=ns, tile_docs=T)
    tail, head_flops = bench.compute_work(plan, docs, qs, df, sdf, H)
    head = sorted(range(docs.vocab), key=lambda t: (-df[t], t))[:H]
    want_tail, rows = 0, 0
    for g0 in range(0, qs.n, G):
        a, e = int(qs.indptr[g0]), int(qs.indptr[min(qs.n, g0 + G)])
        for t in qs.terms[a:e].tolist():
            if t not in head:
                want_tail += int(df[t] - sdf[t])
        rows += len({t for t in qs.terms[a:e].tolist() if t in head})
    assert tail == want_tail
    assert head_flops == 2 * 16 * rows * (docs.n - ns * T)


def test_microbench_rates_parse(tmp_path, monkeypatch):
    f = tmp_path / "mb.md"
    f.write_text("# probe\n\n- red.shared.add.s32 random cells, lanes per clk per SM: 12.5\n"
                 "- ffma, FMA lanes per clk per SM: 127.9 (at 2070 MHz)\n- not a number: n/a\n")
    monkeypatch.setattr(bench, "MICROBENCH_FILE", str(f))
    r = bench.microbench_rates()
    assert r["red.shared.add.s32 random cells, lanes per clk per SM"] == 12.5
    assert r["ffma, FMA lanes per clk per SM"] == 127.9
    assert "not a number" not in r
