#!/usr/bin/env python
"""Exact top-k sparse retrieval benchmark on GB300 (one JSON line on rank 0).

Metric: exact top-1000 QPS and p50/p99 batch latency at 8.84M documents,
batch 500 (the paper's scaling workload, Table 4), next to the plain FP32
batched form (term-parallel scatter-add + dense top-k) on the same GPU, plus
the HBM-roofline fraction of the dominant kernel.  A step = one gs_search of
the whole batch: query prep, scoring, exact top-k.  Index build is outside the
timed region (Sec. 3.2 builds it once).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank serves its own batch on its own GPU
(replicas; no data-path collective); value = all ranks' queries / the slowest
rank's time.  --impl reference times the CPU oracle (the reference arm of this
benchmark) on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "exact top-1000 QPS & p50/p99 ms @8.8M docs vs plain FP32 batch; % HBM peak"
BYTES_PER_IMPACT = {"f32": 4, "f16": 2, "bf16": 2, "u8": 1}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="docs8.8m_b500_top1000", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--headline", default="f32:doc_tiled", help="impact:algo of the reported value")
    ap.add_argument("--forms", default="f32:term_parallel,u8:doc_tiled,f16:doc_tiled,bf16:doc_tiled",
                    help="other impact:algo[:opt=v;opt=v] forms measured beside the headline ('' = none); "
                         "opts are gs_search_opts fields, e.g. f32:doc_tiled:use_head=2")
    ap.add_argument("--cpu-queries", type=int, default=0, help="oracle sample size (0 = one per core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the serving and uneven-batch legs")
    ap.add_argument("--microbench", action="store_true",
                    help="build and run the rate microbenchmarks (paper_2606_26441_gb300/microbench/rates.cu)")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers

def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_dt_tile_kernel_docs8.8m_b500_top1000.md")
KERNEL_SOURCES = ("gs_doctiled.cu", "gs_doctiled.cuh", "gs_internal.cuh", "gs_topk.cuh", "gs_tc05.cuh", "gs_order.cu")


def kernel_source_digest():
    """sha256 over the doc-tiled kernel's source files (in KERNEL_SOURCES order), with
    comments and whitespace removed: a digest of the code, not of its comments."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_26441_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()


def recorded_traffic(workload, form):
    """DRAM bytes (read + write) per main-pass launch from the committed ncu capture,
    or None when that capture is of another workload or form, or the kernel source has
    changed since it was taken."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    rec = {}
    for line in open(TRAFFIC_FILE):
        if line.startswith("- ") and ": " in line:
            key, val = line[2:].split(": ", 1)
            rec[key.strip()] = val.strip().strip("`")
    try:
        if rec.get("workload") != workload or rec.get("form") != form:
            return None
        if rec.get("kernel source sha256") != kernel_source_digest():
            return None
        return int(rec["dram bytes per main-pass launch"])
    except (KeyError, ValueError, OSError):
        return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(statistics.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's value (replicas: the job ends when the last rank does)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------- reference arm (CPU oracle)

def run_reference(args, w, docs, qs):
    import oracle
    c = cores()
    per_step = args.cpu_queries or c
    t0 = time.perf_counter()
    ref = oracle.OracleIndex.from_batch(docs, "f32")
    build_s = time.perf_counter() - t0
    times = []
    n_q = qs.n
    for step in range(args.warmup + args.steps):
        lo = (step * per_step) % max(1, n_q - per_step + 1)
        sub = qs.slice(lo, lo + per_step)
        t = time.perf_counter()
        ref.topk(sub.indptr, sub.terms, sub.weights, w.k, threads=c)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    qps = per_step * len(times) / total
    ms = [t * 1e3 for t in times]
    return {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "QPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)),
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, "f32", "oracle (CPU, FP64 term walk + full sort)"),
        "cpu_baseline": {"value": qps, "unit": "QPS", "cores": c, "kind": "oracle",
                         "sample": f"{per_step} queries per step of the {w.batch}-query batch, full "
                                   f"{w.n_docs}-doc collection; oracle index build {build_s:.1f}s untimed"},
        "e2e": {"value": qps, "unit": "QPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def workload_config(w, impact, algo):
    return {"workload": w.name, "n_docs": w.n_docs, "batch": w.batch, "k": w.k, "impact": impact, "algo": algo,
            "vocab": synth.VOCAB, "doc_nnz": "Poisson(120) in [1,400]", "query_nnz": "Poisson(24) in [1,64]",
            "terms": "Zipf(1.1) over a seeded vocabulary permutation", "weights": "lognormal(-0.5,0.8) clipped (0,5]",
            "l2": "no flush: the posting index (GBs) is far larger than the 129 MB L2",
            "parallelism": "replicas"}


# --------------------------------------------------------------------------- GPU arm

def naive_stream_bytes(docs, qs, impact, df):
    """Every query reading its own terms' posting lists, plus FP32 score rows written once
    and read once (8 B per query and document)."""
    return int(df[qs.terms].sum()) * (4 + BYTES_PER_IMPACT[impact]) + 8 * qs.n * docs.n


def group_terms(qs, order, g0, G):
    """Query terms of the group at positions [g0, g0 + G) of `order` (None: the caller's order)."""
    if order is None:
        a, e = int(qs.indptr[g0]), int(qs.indptr[min(qs.n, g0 + G)])
        return qs.terms[a:e]
    rows = [qs.terms[int(qs.indptr[q]):int(qs.indptr[q + 1])] for q in order[g0:g0 + G]]
    return np.concatenate(rows) if rows else qs.terms[:0]


def algorithmic_bytes(plan, docs, qs, impact, algo, layout_info, order=None):
    """Algorithmic bytes of the dominant kernel per launch.

    doc_tiled main pass : sum over groups of sum over the group's distinct terms
                          of the term's postings outside the sample tiles,
                          times (4 + impact bytes); the groups are those the
                          search used (`order`: the regrouped batch);
    term_parallel scatter: sum over (query, term) of the term's postings times
                          (4 + impact bytes), plus 4 B per score-row element
                          (each row is updated in place once it is zeroed).
    """
    b = 4 + BYTES_PER_IMPACT[impact]
    df = layout_info["df"]
    if algo == "term_parallel":
        post = int(df[qs.terms].sum())
        return post * b + 4 * qs.n * docs.n, {"postings": post}
    G = plan.group_queries
    main_df = df - layout_info["sample_df"]
    post = 0
    for g0 in range(0, qs.n, G):
        u = np.unique(group_terms(qs, order, g0, G))
        post += int(main_df[u].sum())
    return post * b, {"postings": post}


MICROBENCH_FILE = os.path.join(ROOT, "profiles", "microbench_shared_red_ffma_l2_red.md")


def microbench_rates():
    """Measured rates committed in the microbenchmark summary: {name: per-clock-per-SM value}."""
    out = {}
    if not os.path.exists(MICROBENCH_FILE):
        return out
    for line in open(MICROBENCH_FILE):
        if line.startswith("- ") and ": " in line:
            key, val = line[2:].split(": ", 1)
            try:
                out[key.strip()] = float(val.strip().split()[0])
            except ValueError:
                pass
    return out


def compute_work(plan, docs, qs, df, sample_df, head_terms, order=None):
    """Work of the doc-tiled main pass that is not HBM traffic: shared-memory
    reductions of the sparse tail (one per (query, posting) of a non-head term
    outside the sample tiles) and FMAs of the dense head (16 queries x the
    group's active head rows x every document of the main tiles)."""
    H = head_terms
    head = set(np.argsort(-df, kind="stable")[:H].tolist()) if H > 0 else set()
    main_df = df - sample_df
    n_main = docs.n - plan.sample_tiles * plan.tile_docs
    G = plan.group_queries
    tail = 0
    head_rows = 0
    for g0 in range(0, qs.n, G):
        t = group_terms(qs, order, g0, G)
        in_head = np.isin(t, list(head)) if head else np.zeros(t.shape, bool)
        tail += int(main_df[t[~in_head]].sum())
        head_rows += len(np.unique(t[in_head]))
    head_flops = 2 * 16 * head_rows * n_main if H > 0 else 0
    return tail, head_flops


def sample_term_counts(docs, T, R, n_sample):
    """Postings of every term inside the sample tiles (tiles j * R, j < n_sample)."""
    cnt = np.zeros(docs.vocab, dtype=np.int64)
    if R <= 0 or n_sample <= 0:
        return cnt
    for j in range(n_sample):
        d0 = j * R * T
        a, e = int(docs.indptr[d0]), int(docs.indptr[min(docs.n, d0 + T)])
        cnt += np.bincount(docs.terms[a:e], minlength=docs.vocab)
    return cnt


def check_flags(gs, flags, when):
    bad = flags & (gs.GS_FLAG_BAD_TERM | gs.GS_FLAG_BAD_WEIGHT | gs.GS_FLAG_BAD_INDPTR)
    if bad:
        raise RuntimeError(f"search raised data flags {bad} ({when})")


def time_form(gs, torch, idx, q, k, algo, steps, warmup, dist, device_index, sample_clocks=False, opts_kw=None):
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(gs.GS_NUM_STAGE_EVENTS)] for _ in range(steps)]
    for e in ev:  # torch creates the CUDA event on its first record; the library re-records it
        for x in e:
            x.record()
    torch.cuda.synchronize()
    kw = opts_kw or {}
    opts_plain = gs.make_opts(algo, **kw)
    opts_t = [gs.make_opts(algo, stage_events=e, **kw) for e in ev]
    ws = gs.alloc_workspace(idx, q.batch, q.nnz, k, opts_plain)
    out_ids = torch.empty((q.batch, k), dtype=torch.int32, device=q.indptr.device)
    out_sc = torch.empty((q.batch, k), dtype=idx.score_dtype, device=q.indptr.device)
    for _ in range(warmup):
        gs.gs_search(idx, q, k, opts_plain, ws, out_ids, out_sc)
    check_flags(gs, gs.gs_search_flags(ws), "warm-up")
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = None
    launches0 = gs.gs_kernel_launches()
    sampler = ClockSampler(device_index) if sample_clocks else None
    if sampler:
        sampler.__enter__()
    t0 = time.perf_counter()
    for i in range(steps):
        gs.gs_search(idx, q, k, opts_t[i], ws, out_ids, out_sc)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if sampler:
        sampler.__exit__()
        clocks = sampler.summary()
    launches = gs.gs_kernel_launches() - launches0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the flag word of the last timed search: invalid query data fails the run;
    # a candidate overflow (results exact, recomputed) is reported
    flags = gs.gs_search_flags(ws)
    check_flags(gs, flags, "timed steps")
    per_step = [e[0].elapsed_time(e[-1]) for e in ev]
    span = ev[0][0].elapsed_time(ev[-1][-1])
    stages = np.array([[e[j].elapsed_time(e[j + 1]) for j in range(len(e) - 1)] for e in ev])
    return {"span_ms": span, "per_step_ms": per_step, "stage_ms": stages.mean(axis=0).tolist(), "wall_s": wall,
            "launches": launches, "clocks": clocks, "ids": out_ids, "scores": out_sc, "ws": ws,
            "cand_overflow": bool(flags & gs.GS_FLAG_CAND_OVERFLOW)}


def e2e_form(gs, torch, idx, qs, k, algo, steps, warmup):
    """Same metric through gs_search_host: pinned host queries in, host results out, copies timed."""
    opts = gs.make_opts(algo)
    B = qs.n
    h_indptr = torch.from_numpy(qs.indptr.astype(np.int32)).pin_memory()
    h_terms = torch.from_numpy(qs.terms).pin_memory()
    h_w = torch.from_numpy(qs.weights).pin_memory()
    h_ids = torch.empty((B, k), dtype=torch.int32).pin_memory()
    h_sc = torch.empty((B, k), dtype=idx.score_dtype).pin_memory()
    ws = gs.alloc_workspace(idx, B, qs.nnz, k, opts, host_io=True)
    for _ in range(warmup):
        gs.gs_search_host(idx, h_indptr, h_terms, h_w, k, h_ids, h_sc, ws, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        gs.gs_search_host(idx, h_indptr, h_terms, h_w, k, h_ids, h_sc, ws, opts)
    dt = time.perf_counter() - t0
    h2d = h_indptr.numel() * 4 + h_terms.numel() * 4 + h_w.numel() * 4
    d2h = B * k * 8
    return {"value": B * steps / dt, "unit": "QPS", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt / steps * 1e3, "api": "gs_search_host"}


def run_gpu(args, w, docs, qs, world, rank, local):
    import torch
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    k = w.k
    d_indptr = torch.from_numpy(docs.indptr).to(dev)
    d_terms = torch.from_numpy(docs.terms).to(dev)
    d_w = torch.from_numpy(docs.weights).to(dev)
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    df = np.bincount(docs.terms, minlength=docs.vocab).astype(np.int64)

    head_imp, head_algo = args.headline.split(":")
    forms = [args.headline] + [f for f in args.forms.split(",") if f]
    indexes = {}
    results = {}
    for form in forms:
        imp, algo, *rest = form.split(":")
        kw = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in rest[0].split(";")} if rest else {}
        if imp not in indexes:
            indexes[imp] = gs.gs_index_build(d_indptr, d_terms, d_w, docs.vocab, imp)
        idx = indexes[imp]
        r = time_form(gs, torch, idx, q, k, algo, args.steps, args.warmup, dist, local,
                      sample_clocks=form == args.headline, opts_kw=kw)
        plan = idx.plan(q.batch, q.nnz, k, gs.make_opts(algo, **kw))
        # the groups the doc-tiled search used (it regroups the batch by shared tail terms)
        r["order"] = (gs.gs_search_query_order(idx, q, k, gs.make_opts(algo, **kw), r["ws"]).cpu().numpy()
                      if algo == "doc_tiled" and plan.query_order else None)
        results[form] = (r, plan, idx)

    # headline
    r, plan, idx = results[args.headline]
    span_s = reduce_max_over_ranks(r["span_ms"] / 1e3, dist, dev)
    value = w.batch * args.steps * world / span_s
    st = idx.stats()
    # dominant kernel: the scoring stage (stage 3 -> 4)
    stage_names = ["query_prep", "sample_scoring" if head_algo == "doc_tiled" else "zero_rows",
                   "sample_topk", "scoring", "final_topk"]
    T, R, ns = plan.tile_docs, plan.sample_stride, plan.sample_tiles
    layout_info = {"df": df, "sample_df": sample_term_counts(docs, T, R, ns) if head_algo == "doc_tiled" else 0}
    alg_bytes, extra = algorithmic_bytes(plan, docs, qs, head_imp, head_algo, layout_info, r["order"])
    kern_ms = r["stage_ms"][3]
    peak, peak_src = load_peaks()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    # (query, posting) updates the scoring kernel performs
    upd_df = df - layout_info["sample_df"] if head_algo == "doc_tiled" else df
    updates = int(upd_df[qs.terms].sum())
    forms_out = {}
    for form, (rr, pl, ix) in results.items():
        algo = form.split(":")[1]
        ms = rr["per_step_ms"]
        forms_out[form] = {
            "qps": w.batch * len(ms) / (rr["span_ms"] / 1e3), "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "per_query_ms": float(np.mean(ms)) / w.batch,
            "stage_ms": dict(zip(stage_names if algo == "doc_tiled" else
                                 ["query_prep", "zero_rows", "-", "scoring", "topk"], rr["stage_ms"])),
            "index_bytes": int(ix.stats().posting_bytes), "meta_bytes": int(ix.stats().meta_bytes),
            "cand_overflow": rr["cand_overflow"]}
    plain = forms_out.get("f32:term_parallel")
    out = {
        "metric": METRIC, "value": value, "unit": "QPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(r["per_step_ms"])), "p50_ms": float(np.percentile(r["per_step_ms"], 50)),
        "p99_ms": float(np.percentile(r["per_step_ms"], 99)), "per_query_ms": float(np.mean(r["per_step_ms"])) / w.batch,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head_imp, "data": "synthetic",
        "config": workload_config(w, head_imp, head_algo),
        "plan": {"group_queries": plan.group_queries, "tile_docs": plan.tile_docs, "sample_stride": plan.sample_stride,
                 "sample_tiles": plan.sample_tiles, "cand_capacity": int(plan.cand_capacity),
                 "query_order": "regrouped by shared tail terms" if r["order"] is not None else "caller's order"},
        "vs_plain_fp32": (value / plain["qps"]) if plain and (head_imp, head_algo) != ("f32", "term_parallel") else None,
        "forms": forms_out,
        "roofline": {"bound": "hbm", "kernel": "dt_tile_kernel (main pass)" if head_algo == "doc_tiled"
                     else "tp_scatter_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                     "traffic": recorded_traffic(w.name, args.headline), "algorithmic_bytes": alg_bytes,
                     "algorithmic_bytes_caller_order": algorithmic_bytes(plan, docs, qs, head_imp, head_algo,
                                                                         layout_info)[0],
                     "kernel_ms": kern_ms,
                     "postings_read": extra["postings"], "scatter_updates": updates,
                     "naive_stream_bytes": naive_stream_bytes(docs, qs, head_imp, df),
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "updates_per_s": updates / (kern_ms / 1e3)},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    rf = out["roofline"]
    if rf["traffic"]:
        # measured DRAM bytes over the same launch time: how much of HBM the pass really uses
        rf["dram_gbs"] = rf["traffic"] / (kern_ms / 1e3) / 1e9
        rf["dram_frac"] = rf["dram_gbs"] / peak
    if head_algo == "doc_tiled":
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (r["clocks"] or {}).get("sm_mhz") or 2070.0
        rates = microbench_rates()
        tail, head_flops = compute_work(plan, docs, qs, df, layout_info["sample_df"], st.head_terms, r["order"])
        comp = {"sm_mhz": mhz, "sms": sms, "tail_reductions": tail,
                "tail_reductions_per_s": tail / (kern_ms / 1e3), "head_flops": head_flops,
                "head_tflops": head_flops / (kern_ms / 1e3) / 1e12,
                "source": os.path.relpath(MICROBENCH_FILE, ROOT)}
        red = rates.get("red.shared.add.s32 random cells, lanes per clk per SM")
        if red:
            comp["red_shared_peak_per_s"] = red * sms * mhz * 1e6
            comp["tail_frac"] = comp["tail_reductions_per_s"] / comp["red_shared_peak_per_s"]
        ffma = rates.get("ffma, FMA lanes per clk per SM")
        if ffma:
            comp["ffma_peak_tflops"] = 2 * ffma * sms * mhz * 1e6 / 1e12
            comp["head_frac"] = comp["head_tflops"] / comp["ffma_peak_tflops"]
        rf["compute"] = comp
    if not args.no_e2e:
        out["e2e"] = e2e_form(gs, torch, idx, qs, k, head_algo, max(3, args.steps // 2), 2)
    if not args.no_legs and world == 1:
        out["serving"] = serving_leg(gs, torch, dev, docs, d_indptr, d_terms, d_w, indexes, forms_out)
        out["uneven"] = uneven_leg(gs, torch, indexes.get("f32") or idx, docs)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def uneven_point(gs, torch, idx, runner, qs, B, k, steps, max_nnz):
    """One (batch size, k) point of the uneven-batch suite: the same host batches through
    plain per-batch gs_search_host calls (default plan, no graph) and through the
    runner's autotuned, graph-replayed plan.  Host queries in, host results out."""
    subs = [qs.slice(i * B, (i + 1) * B) for i in range(steps + 1)]
    host = [(torch.from_numpy(sb.indptr.astype(np.int32)).pin_memory(), torch.from_numpy(sb.terms).pin_memory(),
             torch.from_numpy(sb.weights).pin_memory()) for sb in subs]
    opts = gs.make_opts("auto")
    ws = gs.alloc_workspace(idx, B, max_nnz, k, opts, host_io=True)
    hid = torch.empty((B, k), dtype=torch.int32).pin_memory()
    hsc = torch.empty((B, k), dtype=idx.score_dtype).pin_memory()
    t_plain = []
    for i, (a, b, c) in enumerate(host):
        t = time.perf_counter()
        gs.gs_search_host(idx, a, b, c, k, hid, hsc, ws, opts)
        if i:
            t_plain.append((time.perf_counter() - t) * 1e3)
    del ws
    t_graph = []
    for i, (a, b, c) in enumerate(host):
        t = time.perf_counter()
        runner.search(a, b, c, k, hid, hsc)
        if i:  # the first call tunes and captures
            t_graph.append((time.perf_counter() - t) * 1e3)
    row = {"batch": B, "k": k}
    for name, ts in (("plain", t_plain), ("graph_tuned", t_graph)):
        row[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                     "qps": B * len(ts) / (sum(ts) / 1e3)}
    row["plan"] = runner.plan(B, k)
    row["speedup"] = row["plain"]["p50_ms"] / row["graph_tuned"]["p50_ms"]
    return row


UNEVEN_LAW = "70% Poisson(20), 25% Poisson(60), 5% uniform[150,300], clamped [1,300]"


def uneven_suite(gs, torch, idx, points, steps):
    batches = sorted({B for B, _ in points})
    need = max(batches) * (steps + 2)
    qs = synth.queries(need, seed=0, law=synth.MIXTURE_LAW)
    max_nnz = max(int(qs.indptr[i + max(batches)] - qs.indptr[i])
                  for i in range(0, need - max(batches) + 1, max(batches)))
    runner = gs.Runner(idx, max_batch=max(batches), max_q_nnz=max_nnz, max_k=max(k for _, k in points))
    rows = []
    for B, k in points:
        rows.append(uneven_point(gs, torch, idx, runner, qs, B, k, steps, max_nnz))
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    runner.free()
    return rows


def uneven_leg(gs, torch, idx, docs):
    """Bounded leg of the default run: batch 1 (k = 10) and batch 64 (k = 1000) of
    mixture-law queries on the headline's FP32 index."""
    t0 = time.perf_counter()
    rows = uneven_suite(gs, torch, idx, [(1, 10), (64, 1000)], steps=8)
    return {"metric": "p50/p99 batch latency, graph-replayed autotuned plans vs plain per-batch launches "
            "(host queries in, host results out)", "n_docs": docs.n, "impact": "f32", "query_nnz": UNEVEN_LAW,
            "steps_per_point": 8, "results": rows, "wall_s": time.perf_counter() - t0}


def run_uneven(args, w):
    """Uneven batches (mixture query law): captured-graph runner with autotuned plans vs plain launches."""
    import torch
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    dev = torch.device("cuda:0")
    docs = synth.docs(w.n_docs, seed=0, threads=cores())
    steps = max(3, min(args.steps, 8))
    idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                            torch.from_numpy(docs.weights).to(dev), docs.vocab, "f32")
    points = [(B, k) for B in w.extra["batches"] for k in w.extra["ks"]]
    results = uneven_suite(gs, torch, idx, points, steps)
    return {"suite": "uneven", "metric": "p50/p99 batch latency and QPS, graph-replayed autotuned plans vs plain "
            "per-batch launches (host queries in, host results out)", "workload": w.name, "n_docs": w.n_docs,
            "query_nnz": UNEVEN_LAW, "steps_per_point": steps, "results": results}


def serve_rates(gs, server, idx, rates, seconds, qs, rng, max_requests=20_000):
    """Poisson arrivals at each offered rate; per-request latency from submit to completion."""
    import threading
    out = []
    qi = 0
    for rate in rates:
        n = int(min(rate * seconds, max_requests))
        gaps = rng.exponential(1.0 / rate, n)
        ks = rng.choice([10, 100, 1000], n)
        which = rng.integers(0, len(idx), n)
        rows = [qs.row((qi + i) % qs.n) for i in range(n)]
        qi += n
        rows = [(np.ascontiguousarray(t), np.ascontiguousarray(wt)) for t, wt in rows]
        tickets = [None] * n
        lat = np.zeros(n)

        def waiter():
            for i in range(n):
                while tickets[i] is None:
                    time.sleep(0.0001)
                lat[i] = server.wait(tickets[i], int(ks[i]), idx[which[i]].score_dtype, timeout_us=60_000_000)[2]

        th = threading.Thread(target=waiter)
        st0 = server.stats()
        th.start()
        t0 = time.perf_counter()
        due = t0
        for i in range(n):
            due += gaps[i]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 0.002:
                    time.sleep(due - now - 0.001)
            tickets[i] = server.submit(int(which[i]), rows[i][0], rows[i][1], int(ks[i]))
        th.join()
        elapsed = time.perf_counter() - t0
        st1 = server.stats()
        nb = st1["batches"] - st0["batches"]
        out.append({"offered_qps": rate, "requests": n, "sustained_qps": n / elapsed,
                    "p50_ms": float(np.percentile(lat, 50) / 1e3), "p99_ms": float(np.percentile(lat, 99) / 1e3),
                    "batches": nb, "mean_batch": (st1["batched_queries"] - st0["batched_queries"]) / max(nb, 1)})
        print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    return out


SERVER_CFG = {"lanes": 4, "max_batch": 256, "max_q_nnz": 256 * 64, "max_k": 1000, "max_wait_us": 500}


def serving_leg(gs, torch, dev, docs, d_indptr, d_terms, d_w, indexes, forms_out):
    """Bounded leg of the default run: continuous batching over two resident FP16
    indexes (1M documents and the headline's 8.84M), Poisson arrivals at two rates,
    against the plain FP32 batch-500 form timed above."""
    t0 = time.perf_counter()
    big = indexes.get("f16") or gs.gs_index_build(d_indptr, d_terms, d_w, docs.vocab, "f16")
    small_docs = synth.docs(1_000_000, seed=1, threads=cores())
    small = gs.gs_index_build(torch.from_numpy(small_docs.indptr).to(dev), torch.from_numpy(small_docs.terms).to(dev),
                              torch.from_numpy(small_docs.weights).to(dev), small_docs.vocab, "f16")
    idx = [small, big]
    server = gs.Server(idx, **SERVER_CFG)
    qs = synth.queries(40_000, seed=9, law=synth.MIXTURE_LAW)
    pts = serve_rates(gs, server, idx, (2000, 10000), 2.0, qs, np.random.default_rng(0))
    stats = server.stats()
    server.close()
    small.free()
    plain = forms_out.get("f32:term_parallel")
    return {"metric": "per-request p50/p99 latency (submit to completion) and sustained QPS, Poisson arrivals, "
            "continuous batching", "indexes": ["1M docs f16", f"{docs.n} docs f16"], "k": "uniform over {10,100,1000}",
            "target_index": "uniform over the two", "query_nnz": UNEVEN_LAW,
            "server": dict(SERVER_CFG, lanes_created=stats["lanes"], max_in_flight=stats["max_in_flight"]),
            "plain_fp32_batch500": ({"qps": plain["qps"], "p50_ms": plain["p50_ms"], "p99_ms": plain["p99_ms"]}
                                    if plain else None),
            "results": pts, "wall_s": time.perf_counter() - t0}


def run_serving(args, w):
    """Poisson arrivals over two resident FP16 indexes (1M and 8.84M docs), continuous batching."""
    import torch
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    dev = torch.device("cuda:0")
    big = synth.docs(synth.N_8_8M, seed=0, threads=cores())
    small = synth.docs(1_000_000, seed=1, threads=cores())
    idx = []
    for d in (small, big):
        idx.append(gs.gs_index_build(torch.from_numpy(d.indptr).to(dev), torch.from_numpy(d.terms).to(dev),
                                     torch.from_numpy(d.weights).to(dev), d.vocab, "f16"))
    # the plain FP32 batch-500 form on the 8.84M collection, same GPU, same run
    f32 = gs.gs_index_build(torch.from_numpy(big.indptr).to(dev), torch.from_numpy(big.terms).to(dev),
                            torch.from_numpy(big.weights).to(dev), big.vocab, "f32")
    qb = synth.queries(500, seed=5)
    q = gs.Queries.from_numpy(qb.indptr, qb.terms, qb.weights, dev)
    o = gs.make_opts("term_parallel")
    ws = gs.alloc_workspace(f32, 500, q.nnz, 1000, o)
    ts = []
    for i in range(4):
        t0 = time.perf_counter()
        gs.gs_search(f32, q, 1000, o, ws)
        torch.cuda.synchronize()
        if i:
            ts.append((time.perf_counter() - t0) * 1e3)
    plain = {"form": "term-parallel FP32, batch 500, 8.84M docs, k=1000", "batch_ms": float(np.median(ts)),
             "qps": 500 / (np.median(ts) / 1e3)}
    del ws, f32
    torch.cuda.empty_cache()
    server = gs.Server(idx, **SERVER_CFG)
    qs = synth.queries(60_000, seed=9, law=w.query_law)
    out = serve_rates(gs, server, idx, w.extra["rates"], w.extra["seconds"], qs, np.random.default_rng(0))
    stats = server.stats()
    server.close()
    return {"suite": "serving", "metric": "per-request p50/p99 latency (submit to completion) and sustained QPS "
            "under Poisson arrivals, continuous batching over two resident FP16 indexes",
            "indexes": ["1M docs f16", "8.84M docs f16"], "k": "uniform over {10,100,1000}",
            "query_nnz": "mixture law", "server": dict(SERVER_CFG, max_in_flight=stats["max_in_flight"]),
            "plain_fp32_batch500": plain, "results": out}


def run_sweep(args, w):
    """Document sparsity sweep (the paper's Table 5 set-up): term-parallel vs doc-tiled vs doc-parallel."""
    import torch
    from paper_2606_26441_gb300 import gpusparse as gs
    gs.load()
    dev = torch.device("cuda:0")
    qs = synth.queries(w.batch, seed=0)
    q = gs.Queries.from_numpy(qs.indptr, qs.terms, qs.weights, dev)
    out = []
    for nnz in w.extra["doc_nnz"]:
        law = synth.NnzLaw(((1.0, "uniform", nnz, nnz),), nnz, nnz)
        docs = synth.docs(w.n_docs, seed=0, law=law, threads=cores())
        idx = gs.gs_index_build(torch.from_numpy(docs.indptr).to(dev), torch.from_numpy(docs.terms).to(dev),
                                torch.from_numpy(docs.weights).to(dev), docs.vocab, "f32", doc_major=True)
        row = {"doc_nnz": nnz, "postings": docs.nnz}
        for algo in ("term_parallel", "doc_tiled", "doc_parallel"):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(gs.GS_NUM_STAGE_EVENTS)]
            for e in ev:
                e.record()
            o = gs.make_opts(algo, stage_events=ev)
            ws = gs.alloc_workspace(idx, q.batch, q.nnz, w.k, o)
            ts = []
            for i in range(4):
                gs.gs_search(idx, q, w.k, o, ws)
                torch.cuda.synchronize()
                if i:
                    ts.append(ev[0].elapsed_time(ev[-1]))
            row[algo + "_ms"] = float(np.median(ts))
            del ws
        out.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        idx.free()
    return {"suite": "sparsity", "metric": "batch latency (ms) vs document non-zeros, top-1000",
            "n_docs": w.n_docs, "batch": w.batch, "k": w.k, "results": out}


def run_microbench():
    """Builds paper_2606_26441_gb300/microbench/rates.cu (nvcc, sm_103a) and prints its rates as the
    '- name: value' lines that microbench_rates() reads."""
    src = os.path.join(ROOT, "paper_2606_26441_gb300", "microbench", "rates.cu")
    exe = os.path.join(tempfile.mkdtemp(), "rates")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe, src],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(out, end="")
    names = {"red.shared.add.s32 distinct banks": "red.shared.add.s32 distinct banks, lanes per clk per SM",
             "red.shared.add.s32 random cells": "red.shared.add.s32 random cells, lanes per clk per SM",
             "red.shared.add.f32 distinct banks": "red.shared.add.f32 distinct banks, lanes per clk per SM",
             "red.shared.add.f32 random cells": "red.shared.add.f32 random cells, lanes per clk per SM",
             "red.shared.add.u64 distinct": "red.shared.add.u64 distinct banks, lanes per clk per SM",
             "red.shared.add.u64 random cells": "red.shared.add.u64 random cells, lanes per clk per SM"}
    for line in out.splitlines():
        for pre, key in names.items():
            if line.startswith(pre + " "):
                print(f"- {key}: {float(line.split('lanes/s')[1].split()[0]):.2f}")
        if line.startswith("ffma"):
            print(f"- ffma, FMA lanes per clk per SM: {float(line.split('TFLOP/s')[1].split()[0]):.2f}")
            print(f"- ffma, TFLOP/s: {float(line.split('ms')[1].split()[0]):.2f}")
        if line.startswith("red.global.add.f32"):
            print(f"- red.global.add.f32 random cells (L2), G per s: {float(line.split('ms')[1].split()[0]):.1f}")


def main():
    args = parse()
    if args.microbench:
        run_microbench()
        return
    world, rank, local = dist_setup(args)
    w = synth.WORKLOADS[args.workload]
    if w.extra.get("batches"):
        if rank == 0:
            print(json.dumps(run_uneven(args, w)), flush=True)
        return
    if w.extra.get("doc_nnz"):
        if rank == 0:
            print(json.dumps(run_sweep(args, w)), flush=True)
        return
    if w.extra.get("rates"):
        if rank == 0:
            print(json.dumps(run_serving(args, w)), flush=True)
        return
    t0 = time.perf_counter()
    docs = synth.docs(w.n_docs, seed=0, threads=cores())
    qs = synth.queries(w.batch, seed=rank, law=w.query_law)
    gen_s = time.perf_counter() - t0
    if args.impl == "reference":
        if rank != 0:
            return
        out = run_reference(args, w, docs, qs)
        print(json.dumps(out), flush=True)
        return
    out = run_gpu(args, w, docs, qs, world, rank, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        c = cores()
        nq = args.cpu_queries or c
        ref = oracle.OracleIndex.from_batch(docs, args.headline.split(":")[0])
        sub = qs.slice(0, nq)
        t = time.perf_counter()
        ref.topk(sub.indptr, sub.terms, sub.weights, w.k, threads=c)
        dt = time.perf_counter() - t
        # one query on one thread: the oracle's per-query cost without parallelism
        one = qs.slice(0, 1)
        t1 = time.perf_counter()
        ref.topk(one.indptr, one.terms, one.weights, w.k, threads=1)
        dt1 = time.perf_counter() - t1
        out["cpu_baseline"] = {"value": nq / dt, "unit": "QPS", "cores": c, "kind": "oracle",
                               "sample": f"first {nq} of the {w.batch} queries over the full {w.n_docs}-doc "
                                         f"collection ({dt:.1f}s wall on {c} threads)",
                               "single_thread_ms_per_query": dt1 * 1e3}
    out["setup_s"] = {"generate": gen_s}
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
