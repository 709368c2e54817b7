"""Benchmark of the relocalization hot path (render candidates + NCC + argmax).

Workload (one "step" = one query through the whole path): the driving-scale
street -- 2M Gaussians, SH degree 3, FP32 attributes, 20 m blocks; each query
selects the blocks within 40 m of its coarse pose (~280k-320k Gaussians), renders
64 candidate poses (4 x 4 x 4 grid, 0.5 m / 2 deg) at 1408x376, scores each
against the query image by NCC, takes the argmax and exports the winner's RGB
and depth.  Metric: candidate views rendered + NCC-scored per second.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the slow plain restatement of
the method) on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica on its own
queries (the path has no exchange step: "replicas only"), value = all ranks'
candidates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate views rendered+NCC-scored/s at 1408x376"
UNIT = "candidates/s"
N_GAUSS = 2_000_000
GRID = (4, 4, 4, 0.5, 2.0)
RADIUS = 40.0
N_QUERIES = 4
# FP32 operations per evaluated (pixel, Gaussian) pair, plus one exponential:
# the quadratic form and the threshold (~8), alpha with its clamp (~3), the
# transmittance update and stop test (~3), the weighted colour (3 FMAs, 6)
# and the weight (~2) -- the algorithmic count of the method, not of any
# particular kernel's instruction mix
FLOPS_PER_EVAL = 22
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this
# workload's 64-view k_blend<16,16,1,false> launch of query 0 (2174.55 MB +
# 14.79 MB); to be re-taken whenever that kernel changes (None: not taken)
BLEND_DRAM_BYTES_PER_LAUNCH = 2_189_346_816
WORKLOAD = ("driving street: 2M Gaussians SH3 FP32, 20 m blocks, 40 m radius (~280k-320k/query), "
            "1408x376 fx=fy=552, 64 candidates (4x4x4 grid 0.5 m / 2 deg), 16x16 tiles")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def stage_rooflines(stage_ms, S, V, n_vis, n_inst, n_eval_per_view, fp32_peak, ex2_peak_gops, hbm_gbs):
    """Per-stage achieved fractions from algorithmic work (not from what the
    kernels happen to move).  S subset Gaussians, V views, n_vis visible
    (view, Gaussian) pairs, n_inst tile instances.
      project     HBM: attributes read once per Gaussian (236 B, SH3 FP32) +
                  the depth key of every (view, Gaussian) pair (4 B; culled
                  pairs marked) + the tile rectangle and 48-byte record of
                  each visible pair (56 B)
      depth_sort  HBM: the first pass reads the key of every pair twice (count
                  and scatter, 8 B) and writes the visible pairs (8 B); three
                  more passes read the key for counting and key + value for
                  scattering and write key + value (20 B per visible pair each)
      tile_count  HBM: depth-ordered index (4 B) and rectangle (8 B) read,
      + tile_emit rectangle written (8 B), read back with the index (12 B),
                  each instance written once (4 B)
      blend       FP32: 22 operations per evaluated (pixel, Gaussian) pair
                  (oracle count), against the measured FP32 FMA peak; plus one
                  exponential per pair against the measured ex2 rate"""
    gb = lambda nbytes, ms: nbytes / (ms * 1e-3) / 1e9
    out = {}
    b = S * 236 + S * V * 4 + n_vis * 56
    out["project"] = {"bound": "hbm", "bytes": b, "achieved_gbs": gb(b, stage_ms["project"])}
    b = S * V * 8 + n_vis * 8 + 3 * 20 * n_vis
    out["depth_sort"] = {"bound": "hbm", "bytes": b, "achieved_gbs": gb(b, stage_ms["depth_sort"])}
    b = n_vis * (4 + 8 + 8 + 12) + n_inst * 4
    ms = stage_ms["tile_count"] + stage_ms["tile_emit"]
    out["tile_binning"] = {"bound": "hbm", "bytes": b, "achieved_gbs": gb(b, ms)}
    for k in ("project", "depth_sort", "tile_binning"):
        out[k]["peak_gbs"] = hbm_gbs
        out[k]["frac"] = out[k]["achieved_gbs"] / hbm_gbs if hbm_gbs else None
    flops = n_eval_per_view * V * FLOPS_PER_EVAL
    t = stage_ms["blend"] * 1e-3
    out["blend"] = {"bound": "alu", "flop": flops, "achieved_tflops": flops / t / 1e12, "peak_tflops": fp32_peak,
                    "frac": flops / t / 1e12 / fp32_peak,
                    "ex2_frac": n_eval_per_view * V / t / 1e9 / ex2_peak_gops}
    return out


class ClockSampler:
    """nvidia-smi sampling during the timed region (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def batch_queries(ctx, cam, n, seed, dev):
    """Batching workload: n queries along the street, candidate grids with 8..128
    candidates (nx, ny in 2..4, nyaw in 2..8) and block radii 15..95 m (subsets of
    about 50k..800k Gaussians); query images rendered at the hidden poses."""
    import torch
    import scenegen as sg
    r = sg.Rng(seed)
    hidden, seeds = sg.street_queries(n, seed=seed)
    out = []
    for i in range(n):
        nx = int(r.uniform(1, 2, 5)[0]); ny = int(r.uniform(1, 2, 5)[0]); nyaw = int(r.uniform(1, 2, 9)[0])
        radius = float(r.uniform(1, 15.0, 95.0)[0])
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], radius)
        img = torch.empty((1, 3, cam.height, cam.width), device=dev)
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(1000 + i, cam.height, cam.width), device=dev)).contiguous()
        out.append((img, sg.pose_from_xyz_yaw(*seeds[i]), radius, (nx, ny, nyaw, 0.5, 2.0)))
    return out


def run_batch_leg(ctx, cam, dev, stream, n_queries=256):
    """One graph-captured reloc_localize_batch over n_queries queries (autotuned)."""
    import tempfile
    import torch
    qs = batch_queries(ctx, cam, n_queries, 21, dev)
    table = os.path.join(tempfile.gettempdir(), "reloc_tune_table.txt")
    tune = ctx.autotune(qs[:4], cam, table, force=True, stream=stream)
    ctx.set_batch_options(use_graph=True, mem_budget=24 << 30)
    ctx.localize_batch(qs, cam, stream=stream, want_scores=False)       # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res, _ = ctx.localize_batch(qs, cam, stream=stream, want_scores=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c = ctx.last_counts()
    n_cand = sum(q[3][0] * q[3][1] * q[3][2] for q in qs)
    subs = [r.n_gauss for r in res]
    ctx.set_batch_options(use_graph=False, mem_budget=16 << 30)
    # the same queries as separate reloc_localize calls, same stream
    for q in qs[:4]:
        ctx.localize(q[0], q[1], q[2], q[3], cam, stream=stream, want_scores=False)
    e0.record(stream)
    for q in qs:
        ctx.localize(q[0], q[1], q[2], q[3], cam, stream=stream, want_scores=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_sep = e0.elapsed_time(e1)
    return {"queries": n_queries, "candidates": int(n_cand), "ms": ms,
            "candidates_per_s": n_cand / (ms / 1e3), "queries_per_s": n_queries / (ms / 1e3),
            "separate_calls_ms": ms_sep, "speedup_vs_separate_calls": ms_sep / ms,
            "subset_min": int(min(subs)), "subset_max": int(max(subs)), "kernel_launches": c.kernel_launches,
            "cuda_graph": True, "tuned": {"tile": [tune.tile_w, tune.tile_h], "rpl": tune.blend_rpl,
                                          "configs_timed": tune.n_tried}}


WEIGHTS = os.path.join(ROOT, "paper_2403_11367_gb300", "weights", "proposal_street.bin")


def run_learned_leg(ctx, cam, dev, stream, g_map, n_queries=256):
    """Learned proposal (top-k + margin fallback) vs the plain 64-candidate
    sweep on the same queries: queries/s of both, recall of the plain winner;
    and the learned + batched + BF16-storage form against the plain FP32
    per-query path."""
    import numpy as np
    import torch
    import scenegen as sg
    if not os.path.exists(WEIGHTS):
        return {"available": False, "reason": "no trained weights (run paper_2403_11367_gb300.train_proposal)"}
    with open(os.path.splitext(WEIGHTS)[0] + ".json") as f:
        meta = json.load(f)
    ctx.proposal_init(0)
    ctx.proposal_set_params(np.fromfile(WEIGHTS, dtype="<f4"))
    hidden, seeds = sg.street_queries(n_queries, seed=33)
    qs = []
    for i in range(n_queries):
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], RADIUS)
        img = torch.empty((1, 3, cam.height, cam.width), device=dev)
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(2000 + i, cam.height, cam.width), device=dev)).contiguous()
        qs.append((img, sg.pose_from_xyz_yaw(*seeds[i]), RADIUS, GRID))
    out = {"available": True, "queries": n_queries, "top_k": meta["top_k"], "tau": meta["tau"],
           "trained_on": meta["samples"], "recall_heldout_4096": meta.get("recall_heldout")}
    ctx.set_batch_options(use_graph=True, mem_budget=24 << 30)
    best = {}
    for mode in ("plain", "learned"):
        ctx.set_proposal(mode == "learned", meta["top_k"], meta["tau"])
        ctx.localize_batch(qs, cam, stream=stream, want_scores=False)       # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, _ = ctx.localize_batch(qs, cam, stream=stream, want_scores=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best[mode] = [r.best_index for r in res]
        out[f"queries_per_s_{mode}"] = n_queries / (ms / 1e3)
        out[f"candidates_scored_per_query_{mode}"] = float(np.mean([r.n_scored for r in res]))
    ctx.set_proposal(False, meta["top_k"], meta["tau"])
    ctx.set_batch_options(use_graph=False, mem_budget=16 << 30)
    out["recall_vs_full_sweep"] = float(np.mean(np.array(best["plain"]) == np.array(best["learned"])))
    out["speedup"] = out["queries_per_s_learned"] / out["queries_per_s_plain"]

    # the three patterns together -- learned proposal, one batched graph-captured
    # call, BF16 attribute storage -- against the plain FP32 method run per query
    # (one reloc_localize call per query, full 64-candidate sweep)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for q in qs[:4]:
        ctx.localize(q[0], q[1], q[2], q[3], cam, stream=stream, want_scores=False)
    e0.record(stream)
    per_query = [ctx.localize(q[0], q[1], q[2], q[3], cam, stream=stream, want_scores=False)[0].best_index
                 for q in qs]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    from paper_2403_11367_gb300 import reloc as R
    cb = R.Context(R.reloc_default_config())
    cb.load_map(g_map, R.BF16)
    cb.proposal_init(0)
    cb.proposal_set_params(np.fromfile(WEIGHTS, dtype="<f4"))
    cb.set_batch_options(use_graph=True, mem_budget=24 << 30)
    cb.set_proposal(True, meta["top_k"], meta["tau"])
    cb.localize_batch(qs, cam, stream=stream, want_scores=False)
    torch.cuda.synchronize()
    e0.record(stream)
    res, _ = cb.localize_batch(qs, cam, stream=stream, want_scores=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_comb = e0.elapsed_time(e1)
    cb.close()
    out["combined"] = {
        "form": "learned top-k + margin fallback, one batched graph-captured call, BF16 attribute storage",
        "baseline": "plain FP32, one reloc_localize per query (64-candidate sweep)",
        "queries_per_s": n_queries / (ms_comb / 1e3), "queries_per_s_plain_fp32_per_query": n_queries / (ms_plain / 1e3),
        "speedup": ms_plain / ms_comb,
        "candidates_scored_per_query": float(np.mean([r.n_scored for r in res])),
        "winner_agreement_vs_plain_fp32": float(np.mean(np.array([r.best_index for r in res]) == np.array(per_query)))}
    return out


# the proposal network's layers: (C_in, C_out, H_out, W_out) of the five 3x3
# stride-2 convolutions, then the two fully connected layers (in, out)
PROPOSAL_CONVS = [(2, 32, 24, 88), (32, 64, 12, 44), (64, 64, 6, 22), (64, 128, 3, 11), (128, 128, 2, 6)]
PROPOSAL_FCS = [(1536, 1024), (1024, 64)]


def proposal_train_flop_per_sample():
    """Algorithmic FLOPs of one training sample's contractions: forward, the
    weight gradient (the same products) and the input gradient (all layers but
    the first), 2 per multiply-add, without the GEMMs' K padding."""
    fwd = [2 * ho * wo * co * 9 * ci for ci, co, ho, wo in PROPOSAL_CONVS] + [2 * i * o for i, o in PROPOSAL_FCS]
    return 2 * sum(fwd) + sum(fwd[1:])


def run_gemm_leg(ctx, dev, stream, batch=256, steps=10):
    """The tensor-core GEMM (tcgen05, TMA-fed, BF16 in, FP32 accumulate):
    proposal training throughput (samples/s and the contraction TFLOP/s of the
    steps, against the sustained BF16 peak), and single launches timed alone on
    the network's largest GEMM at a large batch and on a square GEMM (TFLOP/s
    against the burst BF16 peak)."""
    import torch
    from paper_2403_11367_gb300 import reloc as R
    pk = _peaks()
    out = {}
    gen = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn((batch, R.PROPOSAL_H, R.PROPOSAL_W, 2), generator=gen).to(torch.bfloat16).to(dev).contiguous()
    y = torch.randint(0, R.PROPOSAL_CLASSES, (batch,), generator=gen, dtype=torch.int32).to(dev)
    ctx.proposal_init(3)
    for _ in range(3):
        ctx.proposal_train_step(x, y, 1e-4, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.proposal_train_step(x, y, 1e-4, stream=stream)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    fl = proposal_train_flop_per_sample() * batch
    out["proposal_training"] = {"batch": batch, "ms_per_step": dt * 1e3, "samples_per_s": batch / dt,
                                "gemm_tflops": fl / dt / 1e12, "flop_per_step": fl,
                                "peak_tflops": pk.get("bf16_tflops_sustained"),
                                "frac": fl / dt / 1e12 / pk["bf16_tflops_sustained"] if pk.get("bf16_tflops_sustained")
                                else None,
                                "note": "host-synchronised steps (loss read back), many small launches"}
    for name, (M, N, K) in (("fc1_batch8192", (8192, 1024, 1536)), ("square8192", (8192, 8192, 8192))):
        A = torch.randn((M, K), generator=gen).to(torch.bfloat16).to(dev)
        B = torch.randn((N, K), generator=gen).to(torch.bfloat16).to(dev)
        C = torch.empty((M, N), device=dev)
        for _ in range(3):
            ctx.gemm_bf16(A, B, C, stream=stream)
        ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.gemm_bf16(A, B, C, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = min(ms) / 1e3
        tf = 2.0 * M * N * K / t / 1e12
        out[name] = {"M": M, "N": N, "K": K, "ms": t * 1e3, "tflops": tf, "peak_tflops": pk.get("bf16_tflops"),
                     "frac": tf / pk["bf16_tflops"] if pk.get("bf16_tflops") else None}
        del A, B, C
    return out


PAPER_GRID = (15, 15, 36, 2.0, 10.0)   # 2 m x 10 deg over (-15, 15) m and a full turn: 8100 cells
SEARCH_FRACTION, SEARCH_BATCH, SEARCH_STOP = 0.2, 64, 0.8


def run_random_leg(ctx, cam, dev, stream, n_queries=8):
    """Random search with early stop (Sec. IV-A) on the paper's grid: coarse
    poses off the hidden pose by x, y ~ U(-10, 10) m and yaw ~ U(-90, 90) deg;
    20% of the 8100 cells visited in batches of 64, stop at NCC >= 0.8.
    Reports candidates/s, queries/s, cells scored per query, early stops and
    how often the best cell is the hidden pose's nearest cell or a neighbour
    (within one grid step in x, y and yaw)."""
    import numpy as np
    import torch
    import scenegen as sg
    hidden, _ = sg.street_queries(n_queries, seed=51)
    r = sg.Rng(52)
    off = np.stack([r.uniform(n_queries, -10, 10), r.uniform(n_queries, -10, 10),
                    r.uniform(n_queries, -np.pi / 2, np.pi / 2)], 1)
    nx, ny, nyaw, sxy, syaw = PAPER_GRID
    jobs = []
    for i in range(n_queries):
        h = hidden[i]
        runs, _, _ = ctx.select_block(h[0], h[1], RADIUS)
        img = torch.empty((1, 3, cam.height, cam.width), device=dev)
        ctx.render(runs, sg.pose_from_xyz_yaw(*h)[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(3000 + i, cam.height, cam.width), device=dev)).contiguous()
        jobs.append((img, sg.pose_from_xyz_yaw(h[0] + off[i, 0], h[1] + off[i, 1], h[2], h[3] + off[i, 2])))
    ctx.localize_random(jobs[0][0], jobs[0][1], RADIUS, PAPER_GRID, cam, fraction=0.02, batch=SEARCH_BATCH,
                        stream=stream, want_scores=False)                 # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = [ctx.localize_random(img, pose, RADIUS, PAPER_GRID, cam, fraction=SEARCH_FRACTION, ncc_stop=SEARCH_STOP,
                               batch=SEARCH_BATCH, seed=100 + i, stream=stream, want_scores=False)[0]
           for i, (img, pose) in enumerate(jobs)]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    near = 0
    for i, rr in enumerate(res):
        ix, iy, iyaw = rr.best_index % nx, (rr.best_index // nx) % ny, rr.best_index // (nx * ny)
        # the hidden pose's offset from the coarse pose, in grid steps
        fx = -off[i, 0] / sxy + 0.5 * (nx - 1)
        fy = -off[i, 1] / sxy + 0.5 * (ny - 1)
        fyaw = -np.degrees(off[i, 2]) / syaw + 0.5 * (nyaw - 1)
        near += int(abs(ix - fx) <= 1 and abs(iy - fy) <= 1 and abs(iyaw - fyaw) <= 1)
    scored = sum(rr.n_scored for rr in res)
    # the early stop at thresholds the synthetic street reaches (its best NCC
    # over 20% of the paper grid is ~0.70-0.75, below the 0.8 above)
    sweep = {}
    for thr in (0.72, 0.7, 0.65):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rs = [ctx.localize_random(img, pose, RADIUS, PAPER_GRID, cam, fraction=SEARCH_FRACTION, ncc_stop=thr,
                                  batch=SEARCH_BATCH, seed=100 + i, stream=stream, want_scores=False)[0]
              for i, (img, pose) in enumerate(jobs)]
        torch.cuda.synchronize()
        d1 = time.perf_counter() - t1
        sc1 = sum(x.n_scored for x in rs)
        sweep[str(thr)] = {"stopped_early": sum(x.stopped_early for x in rs), "mean_scored_per_query": sc1 / n_queries,
                           "queries_per_s": n_queries / d1, "candidates_per_s": sc1 / d1,
                           "best_equal_to_full_20pct": sum(int(x.best_index == y.best_index) for x, y in zip(rs, res))}
    return {"grid": "15 x 15 x 36 cells, 2 m / 10 deg (8100)", "fraction": SEARCH_FRACTION,
            "ncc_stop": SEARCH_STOP, "batch": SEARCH_BATCH, "queries": n_queries, "candidates_scored": scored,
            "candidates_per_s": scored / dt, "queries_per_s": n_queries / dt,
            "mean_scored_per_query": scored / n_queries, "stopped_early": sum(rr.stopped_early for rr in res),
            "best_within_one_cell_of_hidden": near, "best_ncc": [round(rr.best_score, 4) for rr in res],
            "stop_at_reachable_thresholds": sweep}


def _stand_in_pairs(W_render, W_query, cam, depth, alpha, gen, step=8, noise=0.5, outliers=0.1):
    """Matcher stand-in for the refinement leg (the paper's learned matcher is
    not available): render pixels on a grid with alpha >= 0.95, their points
    from the rendered depth, projected into the query's true pose, with
    Gaussian pixel noise and a share of random outliers."""
    import torch
    H, W = cam.height, cam.width
    ys, xs = torch.meshgrid(torch.arange(step // 2, H - 1, step, device=depth.device),
                            torch.arange(step // 2, W - 1, step, device=depth.device), indexing="ij")
    ys, xs = ys.reshape(-1), xs.reshape(-1)
    a = alpha[ys, xs].double()
    keep = a >= 0.95
    ys, xs, a = ys[keep], xs[keep], a[keep]
    z = depth[ys, xs].double() / a
    u, v = xs.double() + 0.5, ys.double() + 0.5
    Pc = torch.stack([z * (u - cam.cx) / cam.fx, z * (v - cam.cy) / cam.fy, z], 1)
    X = (Pc - torch.tensor(W_render[:3, 3], device=depth.device)) @ torch.tensor(W_render[:3, :3], device=depth.device)
    P = X @ torch.tensor(W_query[:3, :3], device=depth.device).T + torch.tensor(W_query[:3, 3], device=depth.device)
    q = torch.stack([cam.fx * P[:, 0] / P[:, 2] + cam.cx, cam.fy * P[:, 1] / P[:, 2] + cam.cy], 1)
    q = q + noise * torch.randn(q.shape, device=depth.device, dtype=torch.float64, generator=gen)
    n_out = int(outliers * q.shape[0])
    idx = torch.randperm(q.shape[0], device=depth.device, generator=gen)[:n_out]
    q[idx, 0] = torch.rand(n_out, device=depth.device, dtype=torch.float64, generator=gen) * W
    q[idx, 1] = torch.rand(n_out, device=depth.device, dtype=torch.float64, generator=gen) * H
    ok = (P[:, 2] > 0.1) & (q[:, 0] >= 0) & (q[:, 0] < W) & (q[:, 1] >= 0) & (q[:, 1] < H)
    return torch.stack([u, v, q[:, 0], q[:, 1]], 1)[ok].float().contiguous()


def _pose_error(A, B):
    import numpy as np
    ca, cb = -A[:3, :3].T @ A[:3, 3], -B[:3, :3].T @ B[:3, 3]
    Rd = A[:3, :3] @ B[:3, :3].T
    s = 0.5 * np.linalg.norm([Rd[2, 1] - Rd[1, 2], Rd[0, 2] - Rd[2, 0], Rd[1, 0] - Rd[0, 1]])
    return float(np.linalg.norm(ca - cb)), math.degrees(math.atan2(s, (np.trace(Rd) - 1.0) / 2.0))


def run_refine_leg(ctx, cam, dev, stream, n_queries=8, iters=3):
    """Refinement after the 64-candidate sweep (Sec. III-C.2): per iteration the
    library renders depth + alpha at the current pose (1 view) and solves PnP
    on the stand-in matcher's pairs; reports pose errors before and after and
    the library's time per iteration (matcher time excluded)."""
    import numpy as np
    import torch
    import scenegen as sg
    hidden, seeds = sg.street_queries(n_queries, seed=71)
    H, W = cam.height, cam.width
    gen = torch.Generator(device=dev)
    gen.manual_seed(72)
    before, after, lib_ms, n_pairs = [], [], [], []
    render_ms, pnp_ms = [], []
    for i in range(n_queries):
        Wh = sg.pose_from_xyz_yaw(*hidden[i])
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], RADIUS)
        img = torch.empty((1, 3, H, W), device=dev)
        ctx.render(runs, Wh[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(4000 + i, H, W), device=dev)).contiguous()
        d1 = torch.empty((1, H, W), device=dev)
        a1 = torch.empty((1, H, W), device=dev)
        res, _ = ctx.localize(img, sg.pose_from_xyz_yaw(*seeds[i]), RADIUS, GRID, cam, best_depth=d1[0],
                              best_alpha=a1[0], stream=stream, want_scores=False)
        Wk = np.array(res.best_pose).reshape(4, 4)
        before.append(_pose_error(Wk, Wh))
        for it in range(iters):
            t0 = time.perf_counter()
            if it > 0:
                ctx.render(runs, Wk[None], cam, depth=d1, alpha=a1, stream=stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pairs = _stand_in_pairs(Wk, Wh, cam, d1[0], a1[0], gen)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            out = ctx.refine_pnp(Wk, cam, d1[0], a1[0], pairs, stream=stream)
            t3 = time.perf_counter()
            Wk = np.array(out.pose).reshape(4, 4)
            if it > 0:
                lib_ms.append(1e3 * ((t1 - t0) + (t3 - t2)))
                render_ms.append(1e3 * (t1 - t0))
            pnp_ms.append(1e3 * (t3 - t2))
            n_pairs.append(int(pairs.shape[0]))
        after.append(_pose_error(Wk, Wh))
    b, a = np.array(before), np.array(after)
    return {"queries": n_queries, "iterations": iters, "matcher": "stand-in (true pose + rendered depth, "
            "0.5 px noise, 10% outliers)", "pairs_per_iteration": float(np.mean(n_pairs)),
            "error_before_m_deg": [float(np.median(b[:, 0])), float(np.median(b[:, 1]))],
            "error_after_m_deg": [float(np.median(a[:, 0])), float(np.median(a[:, 1]))],
            "max_error_after_m_deg": [float(a[:, 0].max()), float(a[:, 1].max())],
            "library_ms_per_iteration": float(np.mean(lib_ms)) if lib_ms else None,
            "render_ms_per_iteration": float(np.mean(render_ms)) if render_ms else None,
            "pnp_ms_per_solve": float(np.mean(pnp_ms)) if pnp_ms else None}


def run_ascent_leg(cam, dev, stream, n_queries=4, iters=15):
    """Direct pose ascent on NCC from the 64-candidate sweep's winner (the
    paper's future direction) on the street map with SH degree 0: per
    iteration one gradient evaluation (reloc_score_grad, 1 view) and a line
    search of 8 step lengths along the scaled gradient scored in one batched
    call; a step is taken only if it raises NCC.  Reports NCC and pose error
    before and after, and milliseconds per iteration."""
    import numpy as np
    import torch
    from paper_2403_11367_gb300 import reloc as R
    import scenegen as sg
    g = sg.street_gaussians(N_GAUSS, seed=11, sh_degree=0)
    ctx = R.Context(R.reloc_default_config(), device=dev.index or 0)
    ctx.load_map(g)
    hidden, seeds = sg.street_queries(n_queries, seed=81)
    H, W = cam.height, cam.width
    scale = np.array([0.05, 0.05, 0.05, math.radians(0.5), math.radians(0.5), math.radians(0.5)])
    fracs = 2.0 ** -np.arange(8)
    out = {"queries": n_queries, "iterations": iters, "ncc_before": [], "ncc_after": [], "err_before_m_deg": [],
           "err_after_m_deg": []}
    ms = []
    for i in range(n_queries):
        Wh = sg.pose_from_xyz_yaw(*hidden[i])
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], RADIUS)
        img = torch.empty((1, 3, H, W), device=dev)
        ctx.render(runs, Wh[None], cam, rgb=img)
        q = (img[0] + torch.tensor(sg.image_noise(5000 + i, H, W), device=dev)).contiguous()
        res, _ = ctx.localize(q, sg.pose_from_xyz_yaw(*seeds[i]), RADIUS, GRID, cam, want_scores=False)
        Wk = np.array(res.best_pose).reshape(4, 4)
        runs, _, _ = ctx.select_block(*(-Wk[:3, :3].T @ Wk[:3, 3])[:2], RADIUS)
        out["ncc_before"].append(res.best_score)
        out["err_before_m_deg"].append(_pose_error(Wk, Wh))
        ncc = res.best_score
        for it in range(iters):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, gr = ctx.score_grad(runs, Wk[None], cam, q, stream=stream)
            d = gr[0] * scale * scale
            d = d / max(1e-30, np.sqrt(np.sum((d / scale) ** 2)))          # unit step in scaled units
            trials = np.stack([_apply_left(Wk, f * d) for f in fracs])
            sc, _ = ctx.score(runs, trials, cam, q, stream=stream)
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t0))
            k = int(np.argmax(sc))
            if sc[k] <= ncc:
                break
            Wk, ncc = trials[k], float(sc[k])
        out["ncc_after"].append(ncc)
        out["err_after_m_deg"].append(_pose_error(Wk, Wh))
    ctx.close()
    out["ms_per_iteration"] = float(np.mean(ms))
    return out


def run_train_leg(cam, dev, stream, n_views=16, steps=20, warmup=3):
    """Map training (Sec. III-B.3, Eq. 6 with lambda 0.2, w_photo = w_reproj
    = 1) on the street map with SH degree 0: a 16-frame driving sequence (1 m
    apart along the street), targets rendered from the map, the start map the
    same Gaussians with seeded colour and opacity noise; one step = forward
    render of the 16 views (with depth and alpha), L1 + D-SSIM of the renders
    and of the re-projected pairs, backward blend, chain rule to the 14
    parameters of every Gaussian and one Adam step.  Reports milliseconds per
    step (CUDA events on the stream), views per second, the forward stages'
    share, and the loss before and after."""
    import numpy as np
    import torch
    from paper_2403_11367_gb300 import reloc as R
    import scenegen as sg
    g = sg.street_gaussians(N_GAUSS, seed=11, sh_degree=0)
    H, W = cam.height, cam.width
    hidden, _ = sg.street_queries(1, seed=91)
    x, y, z, yaw = hidden[0]
    poses = np.stack([sg.pose_from_xyz_yaw(x + k * math.cos(yaw), y + k * math.sin(yaw), z, yaw)
                      for k in range(n_views)])
    ctx = R.Context(R.reloc_default_config(), device=dev.index or 0)
    ctx.load_map(g)
    mid = (x + 0.5 * n_views * math.cos(yaw), y + 0.5 * n_views * math.sin(yaw))
    runs, n_sub, _ = ctx.select_block(mid[0], mid[1], RADIUS + n_views / 2)
    targets = torch.empty((n_views, 3, H, W), device=dev)
    ctx.render(runs, poses, cam, rgb=targets, stream=stream)
    r = sg.Rng(17)
    noisy = sg.Gaussians(g.mean, g.scale, g.quat,
                         np.clip(g.opacity + r.normal(g.n, 0.0, 0.1), 0.02, 0.98).astype(np.float32),
                         np.clip(g.sh + r.normal(3 * g.n, 0.0, 0.1).reshape(g.n, 1, 3), 0.0, 1.0).astype(np.float32),
                         0)
    ctx.load_map(noisy)
    runs, n_sub, _ = ctx.select_block(mid[0], mid[1], RADIUS + n_views / 2)
    losses = [ctx.train_step(runs, poses, cam, targets, stream=stream) for _ in range(warmup)]
    ctx.set_profiling(True)
    st = torch.cuda.Stream(device=dev) if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        losses.append(ctx.train_step(runs, poses, cam, targets, stream=st))
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stage_ms, calls = ctx.stage_times()
    fwd = sum(v / max(1, calls[k]) for k, v in stage_ms.items() if k not in ("score",))
    ctx.close()
    return {"views": n_views, "image": [W, H], "subset_gaussians": int(n_sub), "steps": steps,
            "ms_per_step": ms, "views_per_s": n_views * 1e3 / ms,
            "forward_ms_per_step": fwd, "loss_first": losses[0], "loss_last": losses[-1],
            "loss": "0.8 L1 + 0.2 D-SSIM of the 16 renders + the same of the 15 re-projected pairs"}


def _apply_left(W, delta):
    """[Exp(phi) R | Exp(phi) t + rho] for delta = (rho, phi)."""
    import numpy as np
    phi = delta[3:]
    th = float(np.linalg.norm(phi))
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    E = np.eye(3) + (math.sin(th) / th if th > 1e-12 else 1.0) * K + \
        ((1 - math.cos(th)) / th ** 2 if th > 1e-12 else 0.5) * K @ K
    out = np.eye(4)
    out[:3, :3] = E @ W[:3, :3]
    out[:3, 3] = E @ W[:3, 3] + delta[:3]
    return out


def run_precision_leg(g, cam, dev, stream, queries, seed_poses, ref_scores, ref_best, orc0=None):
    """FP32 / FP16 / BF16 attribute storage on the driving workload:
    candidates/s, deviation of every NCC score and winner from the FP32 path,
    and each storage's error against the FP64 oracle of the FP32 map: all 64
    NCC scores of query 0, and every pixel of the FP32 winner's view of query 0
    (RGB max-abs over all pixels and over the pixels the oracle does not flag
    as threshold-adjacent)."""
    import numpy as np
    import torch
    import oracle
    from paper_2403_11367_gb300 import reloc as R
    out = {}
    V = GRID[0] * GRID[1] * GRID[2]
    pix_ref = None
    if orc0 is not None:
        _, _, _, _, oscores, sub, poses, _ = orc0
        wpose = poses[ref_best[0]][None]
        pix_ref = oracle.render_views(sub, wpose, cam)
    for name, prec in (("fp32", R.FP32), ("fp16", R.FP16), ("bf16", R.BF16)):
        ctx = R.Context(R.reloc_default_config())
        ctx.load_map(g, prec)
        dev_sc, agree = 0.0, 0
        scores0 = None
        for k in range(len(queries)):
            res, sc = ctx.localize(queries[k], seed_poses[k], RADIUS, GRID, cam, stream=stream)
            dev_sc = max(dev_sc, float(np.abs(sc - ref_scores[k]).max()))
            agree += int(res.best_index == ref_best[k])
            if k == 0:
                scores0 = sc
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(8):
            ctx.localize(queries[k % len(queries)], seed_poses[k % len(queries)], RADIUS, GRID, cam, stream=stream,
                         want_scores=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"candidates_per_s": 8 * V / (e0.elapsed_time(e1) / 1e3), "max_ncc_dev_vs_fp32": dev_sc,
                     "winner_agreement_vs_fp32": agree / len(queries),
                     "map_bytes_per_gaussian": 12 + (4 if prec == R.FP32 else 2) * (8 + 3 * 16)}
        if pix_ref is not None:
            runs, _, _ = ctx.select_block(seeds_xy(seed_poses[0])[0], seeds_xy(seed_poses[0])[1], RADIUS)
            rgb = torch.empty((1, 3, cam.height, cam.width), device=dev)
            ctx.render(runs, wpose, cam, rgb=rgb, stream=stream)
            torch.cuda.synchronize()
            e = np.abs(rgb.cpu().numpy().astype(np.float64) - pix_ref["rgb"]).max(axis=1)
            mask = pix_ref["flags"] == 0
            out[name]["vs_fp64_oracle"] = {
                "ncc_max_abs_err_64_views": float(np.abs(scores0 - oscores).max()),
                "winner_equal": bool(int(np.argmax(scores0)) == int(oracle.argmax(oscores))),
                "rgb_max_abs_err_unflagged": float(e[mask].max(initial=0)),
                "rgb_max_abs_err_all": float(e.max()), "flagged_fraction": float(1 - mask.mean()),
                "view": "query 0, the FP32 winner's pose, 1408x376"}
        ctx.close()
    return out


def seeds_xy(pose):
    """Camera centre (x, y) of a world-to-camera pose."""
    import numpy as np
    c = -np.asarray(pose)[:3, :3].T @ np.asarray(pose)[:3, 3]
    return float(c[0]), float(c[1])


def rank_queries(rank: int = 0):
    """This replica's queries: the rank-th run of N_QUERIES draws of one seeded
    query stream, so the ranks' queries are disjoint and rank 0's are the
    single-GPU workload's."""
    import scenegen as sg
    hidden, seeds = sg.street_queries(N_QUERIES * (rank + 1), seed=12)
    return hidden[N_QUERIES * rank:], seeds[N_QUERIES * rank:]


def make_workload(rank: int = 0):
    import scenegen as sg
    g = sg.street_gaussians(N_GAUSS, seed=11, sh_degree=3)
    cam = sg.street_camera()
    hidden, seeds = rank_queries(rank)
    return g, cam, hidden, seeds


def max_over_ranks(dist, x: float, device) -> float:
    """The largest x over all ranks (the slowest replica's time); x itself
    without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, slowest_s: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's time."""
    return world * units_per_rank / slowest_s


# ---------------------------------------------------------------- oracle ----

def oracle_sample(g, cam, hidden, seeds, n_cand: int, query_index: int = 0, images=False):
    """Oracle (FP64, OpenMP over views) on the first n_cand grid candidates of
    one query: block select, render, NCC.  Returns (seconds of the render and
    NCC, threads, per-view counts (n_vis, n_inst, n_eval), seconds of the block
    selection and query render, scores, the subset, the poses, the query)."""
    import numpy as np

    import oracle
    import scenegen as sg
    oracle.build()
    h, s = hidden[query_index], seeds[query_index]
    seed_pose = sg.pose_from_xyz_yaw(*s)
    t0 = time.perf_counter()
    idx, nb = oracle.block_select(g.mean, 20.0, s[0], s[1], RADIUS)
    sub = g.subset(idx)
    q = oracle.render(sub, sg.pose_from_xyz_yaw(*h), cam)["rgb"] + sg.image_noise(13 + query_index, cam.height,
                                                                                    cam.width)
    t1 = time.perf_counter()
    poses = oracle.grid_poses(seed_pose, *GRID)[:n_cand]
    out = oracle.render_views(sub, poses, cam, query=q, images=images, flags=images)
    oracle.argmax(out["scores"])
    t2 = time.perf_counter()
    return t2 - t1, oracle.max_threads(), out["counts"], t1 - t0, np.asarray(out["scores"]), sub, poses, q


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, cam, hidden, seeds = make_workload(0)
    n_cand = 16
    for _ in range(args.warmup):
        oracle_sample(g, cam, hidden, seeds, n_cand, 0)
    total, cores = 0.0, 1
    for k in range(args.steps):
        dt, cores, *_ = oracle_sample(g, cam, hidden, seeds, n_cand, k % N_QUERIES)
        total += dt
    value = n_cand * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded street scene standing in for KITTI-360)",
            "config": {"workload": WORKLOAD, "sample": f"{n_cand} of 64 candidates per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_cand} of the 64 candidates of one query per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours ---

def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc as R
    import scenegen as sg

    g, cam, hidden, seeds = make_workload(rank)
    ctx = R.Context(R.reloc_default_config(), device=local)
    ctx.load_map(g)
    V = GRID[0] * GRID[1] * GRID[2]
    H, W = cam.height, cam.width
    stream = torch.cuda.current_stream(dev)

    # query images: rendered on the GPU at the hidden pose (+ seeded noise)
    queries, seed_poses = [], []
    n_runs = max(len(ctx.select_block(s_[0], s_[1], RADIUS)[0]) for s_ in seeds[:N_QUERIES])
    for qi in range(N_QUERIES):
        runs, _, _ = ctx.select_block(hidden[qi][0], hidden[qi][1], RADIUS)
        img = torch.empty((1, 3, H, W), device=dev)
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[qi])[None], cam, rgb=img)
        img = img[0] + torch.tensor(sg.image_noise(13 + qi, H, W), device=dev)
        queries.append(img.contiguous())
        seed_poses.append(sg.pose_from_xyz_yaw(*seeds[qi]))
    brgb = torch.empty((3, H, W), device=dev)
    bdep = torch.empty((H, W), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step(k):
        res, _ = ctx.localize(queries[k % N_QUERIES], seed_poses[k % N_QUERIES], RADIUS, GRID, cam, brgb, bdep,
                              stream=stream, want_scores=False)
        return res

    peaks = R.reloc_measure_peaks(local)          # roofline denominators, this GPU, before the timed region
    for k in range(args.warmup):
        step(k)
    ctx.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    best = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            res = step(k)
            ev[k][1].record(stream)
            launches += ctx.last_counts().kernel_launches
            best.append(res.best_index)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    stage_ms, stage_calls = ctx.stage_times()
    counts = ctx.last_counts()
    S_sub = counts.n_gauss
    ctx.set_profiling(False)
    total_ms = max_over_ranks(dist, total_ms, dev)
    value = job_throughput(world, V * args.steps, total_ms / 1e3)

    # e2e: the host-buffer entry point, pinned host query and winner buffers
    qh = [q.cpu().pin_memory() for q in queries]
    rgb_h = torch.empty((3, H, W), pin_memory=True)
    dep_h = torch.empty((H, W), pin_memory=True)
    for k in range(2):
        ctx.localize_host(qh[k % N_QUERIES], seed_poses[k % N_QUERIES], RADIUS, GRID, cam, rgb_h, dep_h, stream=stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e2e_s = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        a = time.perf_counter()
        ctx.localize_host(qh[k % N_QUERIES], seed_poses[k % N_QUERIES], RADIUS, GRID, cam, rgb_h, dep_h,
                          stream=stream)
        e2e_s += time.perf_counter() - a
    e2e_s = max_over_ranks(dist, e2e_s, dev)

    # FP32 reference scores of the bench queries for the precision leg
    ref_scores, ref_best = [], []
    for k in range(N_QUERIES):
        res, sc = ctx.localize(queries[k], seed_poses[k], RADIUS, GRID, cam, stream=stream)
        ref_scores.append(sc)
        ref_best.append(res.best_index)

    # the oracle on exactly the timed views: all 64 candidates of each query
    # (the algorithmic counts of the roofline); query 0's render is also the
    # CPU baseline sample
    orc = [oracle_sample(g, cam, hidden, seeds, V, k) for k in range(N_QUERIES)] if rank == 0 else None
    precision = run_precision_leg(g, cam, dev, stream, queries, seed_poses, ref_scores, ref_best,
                                  orc[0] if orc else None) if not args.no_batch else None
    batch = run_batch_leg(ctx, cam, dev, stream) if not args.no_batch else None
    learned = run_learned_leg(ctx, cam, dev, stream, g) if not args.no_batch else None
    random_search = run_random_leg(ctx, cam, dev, stream) if not args.no_batch else None
    refine = run_refine_leg(ctx, cam, dev, stream) if not args.no_batch else None
    ascent = run_ascent_leg(cam, dev, stream) if not args.no_batch else None
    train = run_train_leg(cam, dev, stream) if not args.no_batch else None
    gemm = run_gemm_leg(ctx, dev, stream) if not args.no_batch else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    blend_ms = stage_ms["blend"] / max(1, stage_calls["blend"])
    # algorithmic work of the blend over the timed steps: evaluated (pixel,
    # Gaussian) pairs of every view, counted exactly by the oracle for the
    # views each step rendered (step k: query k mod 4, all 64 candidates)
    cpu_s, cores = orc[0][0], orc[0][1]
    n_eval_q = [float(o[2][:, 2].sum()) for o in orc]
    n_eval_steps = sum(n_eval_q[k % N_QUERIES] for k in range(args.steps))
    n_eval_per_view = n_eval_steps / (args.steps * V)
    flops = n_eval_steps * FLOPS_PER_EVAL / args.steps
    peak = max(peaks["fp32_scalar_tflops"], peaks["fp32_packed_tflops"])
    achieved = flops / (blend_ms / 1e3) / 1e12
    per_stage = {k: v / max(1, stage_calls[k]) for k, v in stage_ms.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded street scene standing in for KITTI-360)",
        "config": {"workload": WORKLOAD, "queries": N_QUERIES, "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas{world}"},
        "queries_per_s": job_throughput(world, args.steps, total_ms / 1e3),
        "e2e": {"value": job_throughput(world, V * args.steps, e2e_s), "unit": UNIT,
                # query image + candidate view parameters + block runs in; winner RGB + depth
                # + per-view counts/scores + flags out
                "h2d_bytes_per_step": 3 * H * W * 4 + 64 * V + 16 * (n_runs + 1),
                "d2h_bytes_per_step": 4 * H * W * 4 + 20 * V + 24},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_blend", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": BLEND_DRAM_BYTES_PER_LAUNCH,
                     "traffic_gbs": (BLEND_DRAM_BYTES_PER_LAUNCH / (blend_ms / 1e3) / 1e9
                                     if BLEND_DRAM_BYTES_PER_LAUNCH else None),
                     "peak_source": "measured on this GPU before the timed region: register-resident "
                                    "FP32 FMA microbenchmark (reloc_measure_peaks), the larger of scalar "
                                    f"{peaks['fp32_scalar_tflops']:.1f} and packed f32x2 "
                                    f"{peaks['fp32_packed_tflops']:.1f} TFLOP/s",
                     "work": f"{n_eval_per_view:.6g} evaluated pixel-Gaussian pairs/view (oracle count over the "
                             f"timed steps' views: queries {N_QUERIES} x {V} candidates, step k = query k mod "
                             f"{N_QUERIES}) x {V} views x {FLOPS_PER_EVAL} flop",
                     "n_eval_per_query": n_eval_q, "flop_per_launch": flops,
                     "launch_ms": blend_ms,
                     "recompute": "achieved = flop_per_launch / (launch_ms / 1e3) / 1e12; launch_ms = "
                                  "stage_ms.blend (query statistics + the scoring blend, mean over the timed steps)"},
        "stage_ms": per_stage,
        "stage_roofline": {**stage_rooflines(per_stage, S_sub, V, counts.n_visible, counts.n_instances,
                                             n_eval_per_view, peak, peaks["ex2_gops"], _peaks().get("hbm_gbs")),
                           **({"k_gemm_bf16": {"bound": "tensor", "unit": "TFLOP/s",
                                               "achieved_tflops": gemm["square8192"]["tflops"],
                                               "peak_tflops": gemm["square8192"]["peak_tflops"],
                                               "frac": gemm["square8192"]["frac"],
                                               "work": "8192^3 BF16 GEMM, 2 M N K flop, one launch timed alone "
                                                       "(burst peak)"}} if gemm else {})},
        "counts": {"n_gauss": counts.n_gauss, "n_visible": counts.n_visible, "n_instances": counts.n_instances},
        "batch": batch,
        "learned": learned,
        "random_search": random_search,
        "refine": refine,
        "pose_ascent": ascent,
        "map_training": train,
        "tensor_gemm": gemm,
        "precision": precision,
        "cpu_baseline": {"value": V / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"the {V} candidates of query 0 (FP64 render + NCC)"},
        "clocks": clocks,
        "peaks": {"hbm_gbs": _peaks().get("hbm_gbs"), "bf16_tflops": _peaks().get("bf16_tflops"), **peaks},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_small_case(leg, dev, stream):
    """Small cases for ncu captures of one kernel.  blend_small: three
    16-candidate localize calls of the driving workload's query 0 (its
    scoring blend is the second k_blend launch).  gemm_small: one 4096^3
    tensor-core GEMM after one warm-up launch."""
    import torch
    from paper_2403_11367_gb300 import reloc as R
    import scenegen as sg
    if leg == "gemm_small":
        ctx = R.Context()
        gen = torch.Generator(device="cpu").manual_seed(3)
        A = torch.randn((4096, 4096), generator=gen).to(torch.bfloat16).to(dev)
        B = torch.randn((4096, 4096), generator=gen).to(torch.bfloat16).to(dev)
        C = torch.empty((4096, 4096), device=dev)
        for _ in range(2):
            ctx.gemm_bf16(A, B, C, stream=stream)
        torch.cuda.synchronize()
        return {"gemm": [4096, 4096, 4096], "c00": float(C[0, 0])}
    g, cam, hidden, seeds = make_workload(0)
    ctx = R.Context(R.reloc_default_config())
    ctx.load_map(g)
    runs, _, _ = ctx.select_block(hidden[0][0], hidden[0][1], RADIUS)
    img = torch.empty((1, 3, cam.height, cam.width), device=dev)
    ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[0])[None], cam, rgb=img, stream=stream)
    q = (img[0] + torch.tensor(sg.image_noise(13, cam.height, cam.width), device=dev)).contiguous()
    best = []
    for _ in range(3):
        res, _ = ctx.localize(q, sg.pose_from_xyz_yaw(*seeds[0]), RADIUS, (4, 2, 2, 0.5, 2.0), cam, stream=stream,
                              want_scores=False)
        best.append(res.best_index)
    torch.cuda.synchronize()
    return {"views": 16, "best": best}


def run_leg(args):
    import torch
    from paper_2403_11367_gb300.build import build
    build()
    import scenegen as sg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cam = sg.street_camera()
    stream = torch.cuda.current_stream(dev)
    if args.leg == "map_training":
        out = run_train_leg(cam, dev, stream, steps=args.steps, warmup=args.warmup)
    elif args.leg in ("blend_small", "gemm_small"):
        out = run_small_case(args.leg, dev, stream)
    else:
        out = run_ascent_leg(cam, dev, stream)
    print(json.dumps({"leg": args.leg, **out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batching, learned-proposal and precision legs")
    ap.add_argument("--leg", choices=["map_training", "pose_ascent", "blend_small", "gemm_small"],
                    help="run one self-contained leg alone on cuda:0 and print its JSON object "
                         "(blend_small, gemm_small: small cases for ncu captures)")
    args = ap.parse_args()
    if args.leg:
        run_leg(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
