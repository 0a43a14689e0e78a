"""Benchmark: Gedges/s of y = x A on the BV-delta layout (uncompressed edges m
per second), beside the plain CSR product on the same GPU and the seconds of
PageRank to L1 < 1e-8, on a synthetic web-like graph of n = 862,664 nodes and
~19.2 M edges (copying model; stands in for a web crawl of that size).

One step = one product y = x A through the C ABI (push-chain kernel + push-
gather kernel), inputs resident in HBM, L2 flushed (256 MiB write) before
every timed step. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bv|reference] [--k K]

--impl reference times the CPU oracle (the plain FP64 compressed product of
Sec. 4 in C, single thread) on the same workload.
Under torchrun each rank runs its own replica (weak scaling, no collective
on the data path); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gedges/s of x·A on BV layout vs CSR SpMV on GB300; PageRank s to L1<1e-8"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="bv", choices=["bv", "reference"])
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-graph batch leg")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--no-krhs", action="store_true", help="skip the k = 32 leg")
    ap.add_argument("--config3", action="store_true", help="(the default) the k = 32 leg on the web-like graph "
                                                           "n = 7.4 M, 194 M edges")
    ap.add_argument("--no-config3", action="store_true", help="run the k = 32 leg on the bench graph instead")
    ap.add_argument("--no-variants", action="store_true", help="skip the A^T-pull and social-graph legs")
    ap.add_argument("--config5", action="store_true", help="(the default) the BV-vs-CSR crossover on the social "
                                                           "graph n = 5.4 M and the web graph n = 22.7 M (k = 8)")
    ap.add_argument("--no-config5", action="store_true", help="skip the n = 5.4 M and n = 22.7 M graphs")
    ap.add_argument("--no-high-compression", action="store_true", help="skip the m/m' >= 5 web graph leg")
    ap.add_argument("--window-sweep", action="store_true",
                    help="encode the bench graph (and one copying among 31 rows) with window W in {1, 3, 7, 15, 31} "
                         "and chain bound R, W * R <= 32: compression and both products' speed")
    ap.add_argument("--config4", action="store_true",
                    help="train the warm-start network on 200 generated graphs (n log-uniform in [1e5, 1e6]) and "
                         "evaluate it on the web-like graph n = 18.5 M")
    a = ap.parse_args()
    a.config3 = not a.no_config3
    a.config5 = not a.no_config5
    return a


def workload_spec():
    import synth
    return synth.web_862k()


def workload_name(g):
    return f"web-like copying model n={g.n:,} m={g.m:,} (row copy p=0.8, window 7)"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.dev = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


class FlushL2:
    """Evicts the L2 before a timed step: a 256 MiB write (twice the L2), then
    a 256 MiB read of another buffer, so that the write's dirty lines are
    written back to HBM before the step starts instead of during it (the
    step then reads its inputs from HBM into an L2 of clean lines)."""

    def __init__(self, torch):
        self.a = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.b = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.sink = torch.empty(1, dtype=torch.float32, device="cuda")

    def fill_(self, v):
        self.a.fill_(v)
        self.sink.copy_(self.b.amax().reshape(1))
        return self


def copy_floor(torch, flush, nbytes, steps):
    """CUDA-event time of a plain device copy moving the same bytes (half read,
    half written) after the same flush: what a streaming kernel of this size
    attains on this GPU, launch included."""
    half = max(4, int(nbytes) // 8)
    src = torch.ones(half, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        flush.fill_(1.0)
        dst.copy_(src)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2.0e6 * min(500.0, 20.0 + 2.0 * steps)))
    for a, b in evs:
        flush.fill_(1.0)
        a.record(stream)
        dst.copy_(src)
        b.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    us = 1e3 * float(np.median(ms))
    return {"bytes": 8 * half, "us": us, "gbs": 8 * half / (us * 1e-6) / 1e9,
            "what": "torch copy_ of the same bytes (half read, half written), same flush, median"}


def gpu_id_for_smi():
    import torch
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis or "0"


# ----------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel: str, source_digest: str, k: int = 1):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source, for this kernel family and k (line
    'traffic_bytes_per_launch: <B> source: <digest> kernel: <family> k: <k>')."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    pat = re.compile(r"\s*traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source:\s*([0-9a-f]+)"
                     r"\s+kernel:\s*(\S+)\s+k:\s*(\d+)")
    for fn in sorted(os.listdir(d)):
        if not fn.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(d, fn)):
            m = pat.match(line)
            if m and m.group(2) == source_digest and m.group(3) == kernel and int(m.group(4)) == k:
                return float(m.group(1))
    return None


# Sources that define or launch the product kernels; a change to any of them
# retires the DRAM traffic recorded under profiles/.
PRODUCT_SOURCES = ("kernels.cuh", "device_common.cuh", "bvg_internal.h", "api.cu", "fused.cuh", "pull_fused.cuh")


def code_only(text: str) -> str:
    """C/CUDA source without its comments and blank lines (string literals in
    these files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_digest():
    """Digest of the product's CUDA code; a comment-only edit keeps it."""
    import hashlib
    h = hashlib.sha256()
    for fn in PRODUCT_SOURCES:
        h.update(code_only(open(os.path.join(ROOT, "paper_1708_07271_gb300", "csrc", fn)).read()).encode())
    return h.hexdigest()[:16]


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------- CPU oracle
def cpu_oracle_prepare(g, k):
    """Inputs of the oracle's compressed product: its own references and x."""
    import oracle
    import synth
    ref, _ = oracle.choose_refs(g.row_ptr, g.col)
    x = synth.rhs(g.n, k, synth.seed_for(2, 1)).astype(np.float64)
    return ref, x


def cpu_oracle_run(g, prep, seconds, max_runs=None):
    """Times the oracle's compressed product (Sec. 4 push form, FP64, 1 thread)."""
    import oracle
    ref, x = prep
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.bv_xA(g.row_ptr, g.col, ref, x)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= seconds and len(times) >= 3:
            break
        if max_runs and len(times) >= max_runs:
            break
    return times


def run_reference(args):
    import synth
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    g = synth.copying_model(workload_spec())
    prep = cpu_oracle_prepare(g, args.k)
    # each step is one full product of the oracle
    for _ in range(max(0, args.warmup)):
        cpu_oracle_run(g, prep, 0.0, max_runs=1)
    times = []
    for _ in range(args.steps):
        times += cpu_oracle_run(g, prep, 0.0, max_runs=1)
    t = float(np.sum(times))
    val = g.m * args.k * args.steps / t / 1e9
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gedges/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(g), "k": args.k, "parallelism": "single CPU thread"},
        "cpu_baseline": {"value": val, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full products of the oracle's compressed x A (FP64, C, 1 thread)"},
        "e2e": {"value": val, "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- extra legs
def transpose_csr(row_ptr, col, n):
    """CSR of A^T (rows sorted, no duplicates) from the CSR of A."""
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col, np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    order = np.lexsort((src, ci))
    tp = np.zeros(n + 1, np.int64)
    tp[1:] = np.cumsum(np.bincount(ci, minlength=n))
    return tp, src[order].astype(np.int32)


def variants_leg(args, bvg, synth, torch, timed, dg, g, cg):
    """Two comparisons on the bench graph and a social-shaped one:
    x A as the pull on an encoding of A^T (the paper's own choice for its
    PageRank) against the push on A's encoding; and BV against CSR on a graph
    with power-law out-degree and random ids (weak locality, little
    compression), where the paper expects the compressed product to lose."""
    x = torch.from_numpy(synth.rhs(g.n, 1, synth.seed_for(2, 1))).cuda().reshape(-1)
    y = torch.empty_like(x)
    y2 = torch.empty_like(x)
    tp, tc = transpose_csr(g.row_ptr, g.col, g.n)
    hgT = bvg.bvg_encode(tp, tc)
    stT = bvg.bvg_stats(hgT)
    dgT = bvg.bvg_upload(hgT)

    def warm_timed(fn):
        for _ in range(args.warmup):
            fn()
        return timed(fn, args.steps)

    push = warm_timed(lambda: bvg.bvg_spmv_xA(dg, x, y))
    pullT = warm_timed(lambda: bvg.bvg_spmv_Ax(dgT, x, y2))
    torch.cuda.synchronize()
    rel = float(((y - y2).abs().max() / y.abs().max()).item())
    # and the other way round: A x^T as the push (x A^T) on A^T's encoding
    pull = warm_timed(lambda: bvg.bvg_spmv_Ax(dg, x, y))
    pushT = warm_timed(lambda: bvg.bvg_spmv_xA(dgT, x, y2))
    torch.cuda.synchronize()
    relT = float(((y - y2).abs().max() / y.abs().max()).item())
    gd = lambda m, ms: m * len(ms) / (np.sum(ms) * 1e-3) / 1e9  # noqa: E731
    out = {"xA_push_on_A_gedges_s": gd(g.m, push), "xA_pull_on_AT_gedges_s": gd(g.m, pullT),
           "AT_m_over_words": stT["m"] / max(1, stT["words"]), "max_rel_diff_push_vs_pull": rel,
           "Ax_pull_on_A_gedges_s": gd(g.m, pull), "Ax_push_on_AT_gedges_s": gd(g.m, pushT),
           "max_rel_diff_pull_vs_push_on_AT": relT}

    def biclique_leg(gs, xs, ys, k):
        """The biclique format (Sec. 6) on the same graph: its words and both
        products on the device."""
        t0 = time.perf_counter()
        bd = bvg.bvg_biclique_upload(gs.row_ptr, gs.col)
        enc_s = time.perf_counter() - t0
        r = {"words": bd.info["words"], "m_over_words": gs.m / max(1, bd.info["words"]),
             "bicliques": bd.info["bicliques"], "edges_in_bicliques": bd.info["biclique_edges"],
             "encode_upload_seconds": enc_s}
        for name, fn in (("xA", lambda: bvg.bvg_biclique_spmv_xA(bd, xs, ys)),
                         ("Ax", lambda: bvg.bvg_biclique_spmv_Ax(bd, xs, ys))):
            r[name + "_gedges_s"] = gd(gs.m * k, warm_timed(fn))
        del bd
        return r

    def stream_leg(gs, budget, k):
        """A·xᵀ with the structure streamed from page-locked host memory through
        two device slots of half the stated budget each (the resident pull
        beside it)."""
        t0 = time.perf_counter()
        sm = bvg.bvg_stream_create(gs.row_ptr, gs.col, budget)
        create_s = time.perf_counter() - t0
        info = bvg.bvg_stream_info(sm)
        xs = torch.from_numpy(synth.rhs(gs.n, k, synth.seed_for(5, 9))).cuda()
        if k == 1:
            xs = xs.reshape(-1)
        ys = torch.empty_like(xs)
        ms = warm_timed(lambda: bvg.bvg_stream_spmv(sm, xs, ys))
        sec = float(np.mean(ms)) * 1e-3
        del sm
        return {"budget_bytes": budget, "k": k, "blocks": info["blocks"], "image_bytes": info["image_bytes"],
                "slot_bytes": info["slot_bytes"], "create_seconds": create_s, "Ax_gedges_s": gs.m * k / sec / 1e9,
                "ms_per_product": sec * 1e3, "host_to_device_gbs": info["image_bytes"] / sec / 1e9}

    def crossover(spec, k, with_biclique=False, stream_budget=None):
        gs = synth.copying_model(spec)
        hs = bvg.bvg_encode(gs.row_ptr, gs.col)
        st = bvg.bvg_stats(hs)
        ds = bvg.bvg_upload(hs)
        cs = bvg.bvg_csr_upload(gs.row_ptr, gs.col)
        xs = torch.from_numpy(synth.rhs(gs.n, k, synth.seed_for(5, 1))).cuda()
        if k == 1:
            xs = xs.reshape(-1)
        ys = torch.empty_like(xs)
        r = {"n": gs.n, "m": gs.m, "k": k, "m_over_mprime": st["m"] / max(1, st["nnz_diff"]),
             "m_over_words": st["m"] / max(1, st["words"])}
        for name, fn in (("bv_xA", lambda: bvg.bvg_spmv_xA(ds, xs, ys)), ("csr_xA", lambda: bvg.bvg_csr_spmv_xA(cs, xs, ys)),
                         ("cusparse_xA", lambda: bvg.bvg_csr_cusparse_xA(cs, xs, ys)),
                         ("bv_Ax", lambda: bvg.bvg_spmv_Ax(ds, xs, ys)), ("csr_Ax", lambda: bvg.bvg_csr_spmv_Ax(cs, xs, ys)),
                         ("cusparse_Ax", lambda: bvg.bvg_csr_cusparse_Ax(cs, xs, ys))):
            r[name + "_gedges_s"] = gd(gs.m * k, warm_timed(fn))
        r["bv_over_best_csr_xA"] = r["bv_xA_gedges_s"] / max(r["csr_xA_gedges_s"], r["cusparse_xA_gedges_s"])
        r["bv_over_best_csr_Ax"] = r["bv_Ax_gedges_s"] / max(r["csr_Ax_gedges_s"], r["cusparse_Ax_gedges_s"])
        del ds, cs
        if with_biclique:
            r["biclique"] = biclique_leg(gs, xs, ys, k)
        if stream_budget:
            r["stream"] = stream_leg(gs, stream_budget, k)
        return r

    out["social"] = crossover(synth.replace(synth.social_5m4(), n=g.n), 1, with_biclique=True)
    xb = torch.from_numpy(synth.rhs(g.n, 1, synth.seed_for(2, 1))).cuda().reshape(-1)
    out["biclique_bench_graph"] = biclique_leg(g, xb, torch.empty_like(xb), 1)
    out["stream_bench_graph"] = [stream_leg(g, 16 << 20, kk) for kk in (1, 32)]
    if not args.no_high_compression:
        out["high_compression"] = crossover(synth.web_862k_hc(), 1)
        out["high_compression"]["graph"] = ("web-like copying model, exact copies with probability 0.93 "
                                            "(m/m' >= 5, the paper's 'compressed 5x or more' regime)")
    # column blocks (Sec. 6): a graph whose rows link into two regions of ids
    # with independent prototypes, A encoded whole and split into 2 and 4
    # blocks of consecutive columns (each block its own references)
    g2 = synth.two_region((g.n // 2) // 1024 * 1024, synth.seed_for(6, 1))  # regions of whole 1024-column tiles
    x2 = torch.from_numpy(synth.rhs(g2.n, 1, synth.seed_for(6, 2))).cuda().reshape(-1)
    y2 = torch.empty_like(x2)
    sc2 = torch.empty_like(x2)
    cols = {"graph": "two regions of ids (n = %d rows, the second half empty), each region's links from its own "
                     "web-like copying model" % g2.n, "n": g2.n, "m": g2.m, "blocks": []}
    for nb in (1, 2, 4):
        cb = bvg.bvg_colblocks_create(g2.row_ptr, g2.col, cuts=bvg.aligned_cuts(g2.n, nb))
        st2 = cb.stats()
        r = {"nblocks": nb, "m_over_mprime": g2.m / max(1, st2["nnz_diff"]), "m_over_words": g2.m / max(1, st2["words"]),
             "bits_per_edge": st2["bits_per_edge"]}
        r["xA_gedges_s"] = gd(g2.m, warm_timed(lambda: bvg.bvg_spmv_xA_colblocks(cb, x2, y2, scratch=sc2)))
        r["Ax_gedges_s"] = gd(g2.m, warm_timed(lambda: bvg.bvg_spmv_Ax_colblocks(cb, x2, y2, scratch=sc2)))
        cols["blocks"].append(r)
        del cb
    out["column_blocks"] = cols
    if args.config5:
        out["social_5m4"] = crossover(synth.social_5m4(), 1)
        out["web_22m7_k8"] = crossover(synth.web_22m7(), 8, stream_budget=512 << 20)
    return out


def window_sweep_leg(args, bvg, torch, timed, g):
    """The reference window W (Sec. 4; wider windows are the paper's future
    work, Sec. 6) and the chain bound R against compression and speed, with
    W * R <= 32 (one 32-bit descendant mask per row): the bench graph, whose
    rows copy prototypes among the previous 7 rows, and the same model with
    prototypes among the previous 31 rows; x A and A x^T at k = 1, L2 flushed
    before each product."""
    import synth
    out = {}
    for label, gg in (("copy_window_7", g), ("copy_window_31", synth.copying_model(synth.replace(
            synth.web_862k(), window=31)))):
        x = torch.from_numpy(synth.rhs(gg.n, 1, synth.seed_for(2, 1))).cuda().reshape(-1)
        y = torch.empty_like(x)
        rows = []
        for w in (1, 3, 7, 15, 31):
            for r in (1, 2, 3):
                if w * r > 32 or (w == 1 and r > 1):
                    continue
                hs = bvg.bvg_encode(gg.row_ptr, gg.col, window=w, max_chain=r)
                st = bvg.bvg_stats(hs)
                ds = bvg.bvg_upload(hs)
                res = {"window": w, "max_chain": r, "m_over_mprime": st["m"] / max(1, st["nnz_diff"]),
                       "m_over_words": st["m"] / max(1, st["words"]), "bits_per_edge": st["bits_per_edge"]}
                for name, fn in (("xA", lambda: bvg.bvg_spmv_xA(ds, x, y)), ("Ax", lambda: bvg.bvg_spmv_Ax(ds, x, y))):
                    for _ in range(args.warmup):
                        fn()
                    ms = timed(fn, args.steps)
                    res[name + "_gedges_s"] = gg.m * len(ms) / (np.sum(ms) * 1e-3) / 1e9
                rows.append(res)
                del ds
        out[label] = {"m": gg.m, "sweep": rows}
    return out


def krhs_leg(args, bvg, synth, torch, flush, timed, dg, g, k=32):
    """k = 32 right-hand sides in one product (row-major n x 32, one walk of
    the structure): x A and A x^T, Gedges/s counted as m * k per step; and
    personalized PageRank for 32 one-hot teleport vectors at once (seed nodes
    drawn uniformly), to L1 < 1e-8 in every column."""
    if args.config3:
        g = synth.copying_model(synth.web_7m4())
        dg = bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col))
    x = torch.from_numpy(synth.rhs(g.n, k, synth.seed_for(3, 1))).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        bvg.bvg_spmv_xA(dg, x, y)
        bvg.bvg_spmv_Ax(dg, x, y)
    push = timed(lambda: bvg.bvg_spmv_xA(dg, x, y), args.steps)
    pull = timed(lambda: bvg.bvg_spmv_Ax(dg, x, y), args.steps)
    # the push kernels against the HBM roofline (per-kernel CUDA events, a separate pass)
    from paper_1708_07271_gb300 import bytemodel
    bvg.bvg_trace_enable(dg, True)
    bvg.bvg_trace_read(dg)
    timed(lambda: bvg.bvg_spmv_xA(dg, x, y), args.steps)
    tr = bvg.bvg_trace_read(dg)
    bvg.bvg_trace_enable(dg, False)
    L = bvg.bvg_dev_layout(dg)
    peak, peak_kind = measured_peaks()
    kernels = {}
    for name, (cnt, ms) in tr.items():
        if name in bytemodel.KERNELS:
            b = bytemodel.KERNELS[name](L, k)
            sec = ms / cnt * 1e-3
            kernels[name] = {"avg_us": sec * 1e6, "algorithmic_bytes": b, "achieved_gbs": b / sec / 1e9,
                             "frac": b / sec / 1e9 / peak,
                             "traffic": None if args.config3 else profile_traffic(name, kernel_source_digest(), k)}
    seeds = synth.nodes(k, g.n, synth.seed_for(3, 2)).astype(np.int64)
    out = torch.empty((g.n, k), dtype=torch.float32, device="cuda")

    def median_solve(solve):
        solve()  # captures the update graph for this teleport form
        runs = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it_, res_, rc_ = solve()
            runs.append((time.perf_counter() - t0, it_, float(np.max(res_)), rc_))
        runs.sort()
        return runs[len(runs) // 2]

    s_, it, res, rc = median_solve(lambda: bvg.bvg_pagerank_seeds(dg, seeds, tol=1e-8, max_iter=1000, out=out))
    # the same one-hot vectors written out densely (n x k floats read every update)
    p0 = torch.zeros((g.n, k), dtype=torch.float32, device="cuda")
    p0[torch.from_numpy(seeds).cuda(), torch.arange(k, device="cuda")] = 1.0
    s_dense, it_dense, _, _ = median_solve(lambda: bvg.bvg_pagerank(dg, p0=p0, tol=1e-8, max_iter=1000, out=out))
    del p0
    # the same personalized solves one vector at a time (the first two seeds)
    singles = []
    for c in range(2):
        o1 = torch.empty((g.n, 1), dtype=torch.float32, device="cuda")
        bvg.bvg_pagerank_seeds(dg, seeds[c:c + 1], tol=1e-8, max_iter=1000, out=o1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it1, _, _ = bvg.bvg_pagerank_seeds(dg, seeds[c:c + 1], tol=1e-8, max_iter=1000, out=o1)
        singles.append((time.perf_counter() - t0, it1))
    per_vector = float(np.mean([t for t, _ in singles]))
    gd = lambda ms: g.m * k * len(ms) / (np.sum(ms) * 1e-3) / 1e9  # noqa: E731
    return {"k": k, "graph": workload_name(g), "xA_gedges_s": gd(push), "xA_ms_per_step": float(np.mean(push)),
            "Ax_gedges_s": gd(pull), "Ax_ms_per_step": float(np.mean(pull)),
            "push_roofline": {"peak_gbs": peak, "peak_kind": f"{peak_kind} HBM copy", "kernels": kernels},
            "ppr": {"vectors": k, "seconds": s_, "iterations": it, "max_l1_resid": res, "status": rc,
                    "teleport": "one-hot seed nodes (bvg_pagerank_seeds)",
                    "dense_teleport_seconds": s_dense, "dense_teleport_iterations": it_dense,
                    "one_vector_seconds": per_vector,
                    "one_vector_iterations": [i for _, i in singles],
                    "speedup_vs_one_at_a_time": k * per_vector / s_}}


def batch_leg(args, bvg, synth, torch, flush, timed, world, rank, shard):
    """64 copying-model graphs, n log-uniform in [1e3, 1e6], k = 1: one
    batched product (two launches from one CUDA graph) against the same
    products one graph at a time. Under torchrun the graphs are split across
    ranks (longest first by edges); the figure is all edges over the max time."""
    sizes = synth.multi_graph_sizes(count=64, lo=1e3, hi=1e6, seed=synth.seed_for(3, 7))
    specs = [synth.web_small(int(n), synth.seed_for(3, 100 + i)) for i, n in enumerate(sizes)]
    est_edges = [int(n) * 20 for n in sizes]  # the generator's mean degree, for the split
    mine = shard.assign_graphs(est_edges, world)[rank]
    gs = [synth.copying_model(specs[i]) for i in mine]
    dgs = [bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col)) for g in gs]
    b = bvg.bvg_batch_create(dgs)
    xs = [torch.from_numpy(synth.rhs(g.n, 1, synth.seed_for(3, 200 + i))).cuda().reshape(-1)
          for i, g in zip(mine, gs)]
    ys = [torch.empty_like(x) for x in xs]
    m_local = sum(g.m for g in gs)

    def seq():
        for d, x, y in zip(dgs, xs, ys):
            bvg.bvg_spmv_xA(d, x, y)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        bvg.bvg_batch_spmv_xA(b, xs, ys)
        seq()
    t_b = float(np.sum(timed(lambda: bvg.bvg_batch_spmv_xA(b, xs, ys), args.steps)))
    t_s = float(np.sum(timed(seq, args.steps)))
    tb, m_all = shard.reduce_timing(t_b, m_local * args.steps, device="cuda")
    ts, _ = shard.reduce_timing(t_s, 0.0, device="cuda")
    return {"graphs": len(sizes), "n_total": int(sum(int(v) for v in sizes)),
            "m_total": int(shard.reduce_timing(0.0, m_local, device="cuda")[1]),
            "gedges_s": m_all / (tb * 1e-3) / 1e9, "ms_per_step": tb / args.steps,
            "one_graph_at_a_time_ms_per_step": ts / args.steps, "speedup_vs_one_at_a_time": ts / tb,
            "launches_per_step": 2, "split": f"graphs split over {world} rank(s), longest first"}


def warmstart_leg(args, bvg, synth, torch, dg, g, pr_s, pr_it):
    """The learned warm start on the bench graph: the network is trained on
    PageRank vectors that bvg_pagerank computes on eight generated graphs
    (n log-uniform in [1e5, 3e5]), then PageRank on the bench graph starts
    from its prediction. Time includes the features and the prediction.
    With --config4: 200 training graphs, n log-uniform in [1e5, 1e6], and the
    evaluation on the web-like graph n = 18.5 M (its uniform-start solve
    timed here too)."""
    count, hi = (200, 1e6) if args.config4 else (8, 3e5)
    sizes = synth.multi_graph_sizes(count=count, lo=1e5, hi=hi, seed=synth.seed_for(4, 7))
    train, pstars = [], []
    for i, n in enumerate(sizes):
        gt = synth.copying_model(synth.web_small(int(n), synth.seed_for(4, 100 + i)))
        d = bvg.bvg_upload(bvg.bvg_encode(gt.row_ptr, gt.col))
        p, _, _, _ = bvg.bvg_pagerank(d, tol=1e-10, max_iter=1000)
        train.append(d)
        pstars.append(p)
    net = bvg.bvg_mlp_create(7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = bvg.bvg_warmstart_train(net, train, pstars, epochs=10, lr=3e-3, batch=16384)
    train_s = time.perf_counter() - t0
    del train
    if args.config4:
        g = synth.copying_model(synth.web_18m5())
        dg = bvg.bvg_upload(bvg.bvg_encode(g.row_ptr, g.col))
        pu = torch.empty(g.n, device="cuda")
        bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000, out=pu)
        uruns = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, uit, _, _ = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000, out=pu)
            uruns.append((time.perf_counter() - t0, uit))
        uruns.sort()
        pr_s, pr_it = uruns[1]
    p = torch.empty(g.n, device="cuda")
    p_init = torch.empty(g.n, device="cuda")
    bvg.bvg_warmstart_predict(net, dg, out=p_init)
    bvg.bvg_pagerank(dg, p_init=p_init, tol=1e-8, max_iter=1000, out=p)
    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bvg.bvg_warmstart_predict(net, dg, out=p_init)
        _, it, res, rc = bvg.bvg_pagerank(dg, p_init=p_init, tol=1e-8, max_iter=1000, out=p)
        runs.append((time.perf_counter() - t0, it, float(res[0]), rc))
    runs.sort()
    s, it, res, rc = runs[len(runs) // 2]
    # the prediction alone (features, network, normalisation), against the
    # time of one update, and the net effect on the solve
    pts = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bvg.bvg_warmstart_predict(net, dg, out=p_init)
        torch.cuda.synchronize()
        pts.append(time.perf_counter() - t0)
    predict_s = float(np.median(pts))
    per_update = pr_s / max(pr_it, 1)
    saved = pr_it - it
    break_even = predict_s / per_update
    if s >= pr_s:
        finding = (f"negative result: the learned start saves {saved} of {pr_it} updates, but its features and "
                   f"prediction take as long as {break_even:.1f} updates, so the solve is {1e3 * (s - pr_s):.2f} ms "
                   f"slower; the error left after the first updates lies in long-wavelength modes along the id order, "
                   f"which per-node features do not see")
    else:
        finding = (f"the learned start saves {saved} of {pr_it} updates and costs {break_even:.1f} updates' time: "
                   f"{1e3 * (pr_s - s):.2f} ms faster")
    return {"graph": workload_name(g), "seconds": s, "iterations": it, "l1_resid": res, "status": rc,
            "uniform_seconds": pr_s, "uniform_iterations": pr_it, "predict_seconds": predict_s,
            "updates_saved": saved, "break_even_updates": break_even, "finding": finding,
            "train_seconds": train_s, "train_loss": loss,
            "train_graphs": len(sizes), "train_nodes": int(sum(int(v) for v in sizes))}


# ----------------------------------------------------------------- GPU arm
def run_bv(args):
    import torch
    import synth
    import paper_1708_07271_gb300 as bvg
    from paper_1708_07271_gb300 import bytemodel

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_1708_07271_gb300 import shard

    def max_over_ranks(v):
        return shard.reduce_timing(v, 0.0, device="cuda")[0]

    k = args.k
    g = synth.copying_model(workload_spec())
    hg = bvg.bvg_encode(g.row_ptr, g.col)
    st = bvg.bvg_stats(hg)
    dg = bvg.bvg_upload(hg)
    L = bvg.bvg_dev_layout(dg)
    cg = bvg.bvg_csr_upload(g.row_ptr, g.col)
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(synth.rhs(g.n, k, synth.seed_for(2, 1))).cuda()
    if k == 1:
        x = x.reshape(-1)
    y = torch.empty_like(x)
    flush = FlushL2(torch)

    def timed(fn, steps):
        """Per-step CUDA-event time (ms) with an L2 flush before each step. The
        steps are queued behind a sleep kernel so the host runs ahead and the
        events time the device work, not host launch gaps."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        torch.cuda._sleep(int(2.0e6 * min(500.0, 20.0 + 2.0 * steps)))
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    xa = lambda: bvg.bvg_spmv_xA(dg, x, y)  # noqa: E731
    for _ in range(args.warmup):
        flush.fill_(1.0)
        xa()
    torch.cuda.synchronize()
    L = bvg.bvg_dev_layout(dg)  # again: the first product may have built the point columns

    # ---- timed region: K steps of x A
    sampler = ClockSampler(gpu_id_for_smi()) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier()
    step_ms = timed(xa, args.steps)
    barrier()
    # per-kernel durations: the same steps again with CUDA events around each
    # kernel launch (events between launches stop the launch overlap, so this
    # pass is kept apart from the step timing above)
    bvg.bvg_trace_enable(dg, True)
    bvg.bvg_trace_read(dg)
    timed(xa, args.steps)
    trace = bvg.bvg_trace_read(dg)
    bvg.bvg_trace_enable(dg, False)
    clocks = sampler.stop() if sampler else None
    t_total = max_over_ranks(float(np.sum(step_ms)))
    value = world * g.m * k * args.steps / (t_total * 1e-3) / 1e9
    launches = sum(v[0] for v in trace.values())  # launches per timed region (same count in both passes)

    # ---- roofline of the dominant kernel (largest share of the step)
    peak, peak_kind = measured_peaks()
    dom = max(trace.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    dom_bytes = bytemodel.KERNELS[dom_name](L, k)
    dom_avg_s = dom_ms / dom_launches * 1e-3
    achieved = dom_bytes / dom_avg_s / 1e9
    traffic = profile_traffic(dom_name, kernel_source_digest(), k)
    floor = copy_floor(torch, flush, dom_bytes, max(5, args.steps))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom_name, "algorithmic_bytes": dom_bytes,
                "avg_launch_us": dom_avg_s * 1e6, "peak_kind": f"{peak_kind} HBM copy",
                "share": dom_ms / sum(v[1] for v in trace.values()),
                "kernels": {kk: {"launches": vv[0], "avg_us": 1e3 * vv[1] / vv[0]} for kk, vv in trace.items()},
                "copy_floor": floor, "frac_of_copy_floor": achieved / floor["gbs"]}

    # ---- same protocol (W warm-up calls, then K timed steps): CSR baseline, pull product
    def warm_timed(fn):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            fn()
        return timed(fn, args.steps)

    csr_ms = warm_timed(lambda: bvg.bvg_csr_spmv_xA(cg, x, y))
    cusp_ms = warm_timed(lambda: bvg.bvg_csr_cusparse_xA(cg, x, y))
    pull_ms = warm_timed(lambda: bvg.bvg_spmv_Ax(dg, x, y))
    bvg.bvg_trace_enable(dg, True)
    bvg.bvg_trace_read(dg)
    bvg.bvg_spmv_Ax(dg, x, y)
    pull_kernels = sorted(bvg.bvg_trace_read(dg))
    bvg.bvg_trace_enable(dg, False)
    pull_roofline = None
    if pull_kernels == ["pull_fused"]:  # one launch per product: its time is the step's
        pb = bytemodel.pull_fused(L, k)
        pull_gbs = pb / (float(np.mean(pull_ms)) * 1e-3) / 1e9
        pull_roofline = {"kernel": "pull_fused", "algorithmic_bytes": pb, "avg_us": 1e3 * float(np.mean(pull_ms)),
                         "achieved_gbs": pull_gbs, "frac": pull_gbs / peak,
                         "traffic": profile_traffic("pull_fused", kernel_source_digest(), k)}
    csr_ax_ms = warm_timed(lambda: bvg.bvg_csr_spmv_Ax(cg, x, y))
    cusp_ax_ms = warm_timed(lambda: bvg.bvg_csr_cusparse_Ax(cg, x, y))
    gedges = lambda ms: g.m * k * len(ms) / (np.sum(ms) * 1e-3) / 1e9  # noqa: E731

    # ---- end to end through the C ABI with host buffers (pinned)
    hx = torch.from_numpy(synth.rhs(g.n, k, synth.seed_for(2, 1))).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    for _ in range(2):
        bvg.bvg_spmv_xA_host(dg, hx, hy)
    e2e_s = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bvg.bvg_spmv_xA_host(dg, hx, hy)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(float(np.sum(e2e_s)))
    e2e = {"value": world * g.m * k * args.steps / e2e_total / 1e9, "unit": "Gedges/s",
           "h2d_bytes_per_step": int(hx.numel() * 4), "d2h_bytes_per_step": int(hy.numel() * 4),
           "path": "bvg_spmv_xA_host on page-locked buffers (copy to device scratch, product, copy back, "
                   "synchronise), host wall clock per call"}

    # ---- PageRank to L1 < 1e-8, uniform start, single vector
    pr_runs = []
    p = torch.empty(g.n, device="cuda")
    bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000, out=p)
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, iters, res, rc = bvg.bvg_pagerank(dg, tol=1e-8, max_iter=1000, out=p)
        pr_runs.append((time.perf_counter() - t0, iters, float(res[0]), rc))
    pr_runs.sort()
    pr_s, pr_it, pr_res, pr_rc = pr_runs[len(pr_runs) // 2]

    variants = None if args.no_variants else variants_leg(args, bvg, synth, torch, timed, dg, g, cg)
    krhs = None if args.no_krhs else krhs_leg(args, bvg, synth, torch, flush, timed, dg, g)
    batch = None if args.no_batch else batch_leg(args, bvg, synth, torch, flush, timed, world, rank, shard)
    warm = None if args.no_warmstart else warmstart_leg(args, bvg, synth, torch, dg, g, pr_s, pr_it)
    wsweep = window_sweep_leg(args, bvg, torch, timed, g) if args.window_sweep else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times = cpu_oracle_run(g, cpu_oracle_prepare(g, k), args.cpu_seconds)
        cpu = {"value": g.m * k / float(np.mean(times)) / 1e9, "unit": "Gedges/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(times)} full products of the oracle's compressed x A (FP64, C, 1 thread) on the "
                         f"same graph, {np.sum(times):.1f} s; host has {os.cpu_count()} cores"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(g), "k": k,
                       "l2": "flushed before every timed step: a 256 MiB write, then a 256 MiB read of another "
                             "buffer (the write's dirty lines reach HBM before the step)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "csr_gedges_s": gedges(csr_ms), "cusparse_gedges_s": gedges(cusp_ms),
            "bv_over_csr": float(np.sum(csr_ms) / np.sum(step_ms)),
            "bv_over_best_csr": float(min(np.sum(csr_ms), np.sum(cusp_ms)) / np.sum(step_ms)),
            "pull_gedges_s": gedges(pull_ms), "csr_Ax_gedges_s": gedges(csr_ax_ms),
            "cusparse_Ax_gedges_s": gedges(cusp_ax_ms),
            "pull_over_best_csr": float(min(np.sum(csr_ax_ms), np.sum(cusp_ax_ms)) / np.sum(pull_ms)),
            "pull_kernels": pull_kernels, "pull_roofline": pull_roofline,
            "pagerank": {"seconds": pr_s, "iterations": pr_it, "l1_resid": pr_res, "status": pr_rc,
                         "start": "uniform", "k": 1},
            "k_rhs": krhs, "batch": batch, "warm_start": warm, "variants": variants, "window_sweep": wsweep,
            "compression": {"m_over_mprime": st["m"] / max(1, st["nnz_diff"]),
                            "m_over_words": st["m"] / max(1, st["words"]), "bits_per_edge": st["bits_per_edge"],
                            "structure_MB": L["structure_bytes"] / 1e6},
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_bv(args)


if __name__ == "__main__":
    main()
