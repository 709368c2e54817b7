"""Winner agreement of the learned proposal with the FP64 oracle's own full
sweep, on held-out driving queries the CPU can afford.

For each query (a hidden pose along the 2M-Gaussian street not used in
training, a coarse pose within +-1 m / +-3 deg, the render at the hidden pose
plus seeded N(0, 0.02^2) noise) the GPU runs the plain 64-candidate sweep and
the learned top-k + margin fallback (the shipped weights and threshold); the
oracle runs its own sweep (block selection around the coarse pose, FP64
render and NCC of all 64 candidates on the same noisy image).  Run as a
script for the 64-query sample:

    python tests/proposal_oracle_check.py 64
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

GRID = (4, 4, 4, 0.5, 2.0)
RADIUS = 40.0
WEIGHTS = os.path.join(ROOT, "paper_2403_11367_gb300", "weights", "proposal_street.bin")


def learned_vs_oracle(n_queries: int, seed: int = 34):
    import torch

    import oracle
    import scenegen as sg
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc as R

    with open(os.path.splitext(WEIGHTS)[0] + ".json") as f:
        meta = json.load(f)
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    dev = torch.device("cuda:0")
    ctx = R.Context()
    ctx.load_map(g)
    ctx.proposal_init(0)
    ctx.proposal_set_params(np.fromfile(WEIGHTS, dtype="<f4"))
    hidden, seeds = sg.street_queries(n_queries, seed=seed)
    qs, q_host = [], []
    for i in range(n_queries):
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], RADIUS)
        img = torch.empty((1, 3, cam.height, cam.width), device=dev)
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(5000 + i, cam.height, cam.width), device=dev)).contiguous()
        qs.append((img, sg.pose_from_xyz_yaw(*seeds[i]), RADIUS, GRID))
        q_host.append(img.cpu().numpy().astype(np.float64))
    plain, _ = ctx.localize_batch(qs, cam, want_scores=False)
    ctx.set_proposal(True, meta["top_k"], meta["tau"])
    learned, _ = ctx.localize_batch(qs, cam, want_scores=False)
    ctx.set_proposal(False, meta["top_k"], meta["tau"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w_or, margin = [], []
    for i in range(n_queries):
        s = seeds[i]
        idx, _ = oracle.block_select(g.mean, 20.0, s[0], s[1], RADIUS)
        poses = oracle.grid_poses(sg.pose_from_xyz_yaw(*s), *GRID)
        r = oracle.render_views(g.subset(idx), poses, cam, query=q_host[i], images=False, flags=False)
        sc = np.sort(r["scores"])
        w_or.append(oracle.argmax(r["scores"]))
        margin.append(float(sc[-1] - sc[-2]))
    ctx.close()
    return {
        "queries": n_queries, "top_k": meta["top_k"], "tau": meta["tau"], "oracle_s": time.perf_counter() - t0,
        "oracle_winner": w_or, "oracle_top2_margin": margin,
        "gpu_sweep_winner": [r.best_index for r in plain], "learned_winner": [r.best_index for r in learned],
        "learned_scored": [r.n_scored for r in learned],
        "gpu_sweep_vs_oracle": float(np.mean([r.best_index == w for r, w in zip(plain, w_or)])),
        "learned_vs_oracle": float(np.mean([r.best_index == w for r, w in zip(learned, w_or)])),
        "learned_fallbacks": int(sum(r.n_scored > meta["top_k"] for r in learned)),
    }


if __name__ == "__main__":
    out = learned_vs_oracle(int(sys.argv[1]) if len(sys.argv) > 1 else 64)
    print(json.dumps(out), flush=True)
