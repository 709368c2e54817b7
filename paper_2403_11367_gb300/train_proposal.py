"""Train the learned candidate proposal on the driving street and evaluate it.

    python -m paper_2403_11367_gb300.train_proposal --samples 40000 --heldout 4096 \
        --out paper_2403_11367_gb300/weights/proposal_street.bin

Every step runs through the C ABI on the GPU:
  data     per sample, a hidden pose along the street and a coarse pose within
           +-1 m / +-3 deg of it; the query is the render at the hidden pose
           plus N(0, 0.02^2) noise, the second input channel the render at the
           coarse pose; the label is the full 64-candidate sweep's NCC winner
           (reloc_localize_batch without the proposal);
  training softmax cross-entropy, Adam, cosine learning-rate decay
           (reloc_proposal_train_step: tcgen05 BF16 GEMMs, FP32 accumulation);
  eval     recall of the full sweep's winner when only the top-k cells are
           scored and the sweep runs below the margin threshold; the threshold
           is chosen on the first half of the held-out set (recall >= target;
           and at least the --fallback-quantile quantile of the margins, so the
           sweep also runs on the queries the network is least sure of) and
           reported on the second half, with the recall of the top-k cells
           alone; throughput learned vs plain (--eval-only: the held-out
           evaluation of the weights in --out, without training);
  curve    (--curve n1,n2,...) the same network trained from scratch on
           nested subsets of the training set, held-out recall and top-1 of
           each: how recall grows with the number of renders.
Writes the flat FP32 parameters (include/reloc.h layout) to --out and a JSON
summary beside it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GRID = (4, 4, 4, 0.5, 2.0)
RADIUS = 40.0


def make_samples(ctx, R, cam, n, seed, chunk=64, noise_std=0.02):
    """Inputs [n][47][176][2] (BF16 bits, device) and labels [n] (int32, device)."""
    import torch
    import scenegen as sg
    dev = torch.device("cuda:0")
    hidden, seeds = sg.street_queries(n, seed=seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    H, W = cam.height, cam.width
    inputs = torch.empty((n, 47, 176, 2), dtype=torch.int16, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    coarse = torch.empty((1, 3, H, W), device=dev)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        qs = []
        for i in range(c0, c1):
            runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], RADIUS)
            img = torch.empty((1, 3, H, W), device=dev)
            ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
            img = (img[0] + noise_std * torch.randn((3, H, W), device=dev, generator=gen)).contiguous()
            seed_pose = sg.pose_from_xyz_yaw(*seeds[i])
            runs_c, _, _ = ctx.select_block(seeds[i][0], seeds[i][1], RADIUS)
            ctx.render(runs_c, seed_pose[None], cam, rgb=coarse)
            ctx.proposal_make_input(img, coarse[0], cam, inputs[i])
            qs.append((img, seed_pose, RADIUS, GRID))
        res, _ = ctx.localize_batch(qs, cam, want_scores=False)
        labels[c0:c1] = torch.tensor([r.best_index for r in res], dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    return inputs, labels, hidden, seeds


def train(ctx, x_tr, y_tr, n_samples, epochs, batch, lr0, seed):
    """Adam with cosine learning-rate decay over `epochs` passes of the first
    n_samples samples; returns the mean loss of each epoch."""
    import torch
    n = n_samples - n_samples % batch
    steps_per_epoch = n // batch
    total = steps_per_epoch * epochs
    gen = torch.Generator(device="cuda:0")
    gen.manual_seed(seed)
    losses, step = [], 0
    for ep in range(epochs):
        perm = torch.randperm(n_samples, device="cuda:0", generator=gen)[:n]
        ep_loss = []
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            lr = 0.5 * lr0 * (1 + math.cos(math.pi * step / total)) + 1e-5
            ep_loss.append(ctx.proposal_train_step(x_tr[idx].contiguous(), y_tr[idx].contiguous(), lr))
            step += 1
        losses.append(float(np.mean(ep_loss)))
    return losses


def heldout_logits(ctx, x_te):
    import torch
    n = x_te.shape[0]
    logits = torch.empty((n, 64), device="cuda:0")
    for b in range(0, n, 256):
        e = min(n, b + 256)
        ctx.proposal_forward(x_te[b:e].contiguous(), logits[b:e])
    torch.cuda.synchronize()
    return logits.cpu().numpy().astype(np.float64)


def recall_at(logits, labels, k, tau):
    """Fraction of queries whose full-sweep winner is found: scored within the
    top-k cells, or the margin p1 - p2 is below tau (full sweep)."""
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    order = np.argsort(-logits, axis=1, kind="stable")
    topk = order[:, :k]
    ps = np.sort(p, axis=1)
    margin = ps[:, -1] - ps[:, -2]
    hit = (topk == labels[:, None]).any(axis=1)
    found = hit | (margin < tau)
    return float(found.mean()), float((margin < tau).mean())


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=40000)
    ap.add_argument("--heldout", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--top-k", type=int, default=8)
    ap.add_argument("--target-recall", type=float, default=1.0)
    ap.add_argument("--curve", default="", help="comma-separated training-set sizes for the recall curve")
    ap.add_argument("--fallback-quantile", type=float, default=0.01,
                    help="tau is at least this quantile of the tuning half's top-two margins")
    ap.add_argument("--eval-only", action="store_true", help="evaluate the weights in --out (no training)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2403_11367_gb300", "weights", "proposal_street.bin"))
    args = ap.parse_args(argv)

    import torch
    import scenegen as sg
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc as R

    t0 = time.time()
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    ctx = R.Context()
    ctx.load_map(g)
    ctx.set_batch_options(use_graph=True, mem_budget=24 << 30)
    ctx.proposal_init(seed=args.seed)

    t1 = time.time()
    prev = None
    if args.eval_only:
        with open(os.path.splitext(args.out)[0] + ".json") as f:
            prev = json.load(f)
        ctx.proposal_set_params(np.fromfile(args.out, dtype="<f4"))
    else:
        x_tr, y_tr, _, _ = make_samples(ctx, R, cam, args.samples, seed=31)
    x_te, y_te, h_te, s_te = make_samples(ctx, R, cam, args.heldout, seed=32)
    t2 = time.time()
    print(f"data: {0 if args.eval_only else args.samples} + {args.heldout} samples in {t2 - t1:.1f} s", flush=True)
    lab = y_te.cpu().numpy()
    half = args.heldout // 2

    curve = []
    for n_sub in [int(v) for v in args.curve.split(",") if v] if (args.curve and not args.eval_only) else []:
        if n_sub >= args.samples:
            continue
        ctx.proposal_init(seed=args.seed)
        train(ctx, x_tr, y_tr, n_sub, args.epochs, args.batch, args.lr, args.seed)
        z = heldout_logits(ctx, x_te)
        r, _ = recall_at(z, lab, args.top_k, -1.0)
        curve.append({"samples": n_sub, "recall_topk": r, "top1": float((z.argmax(axis=1) == lab).mean())})
        print("curve", curve[-1], flush=True)

    if args.eval_only:
        losses = prev["epoch_loss"]
        curve = [c for c in prev.get("recall_curve", []) if c["samples"] != args.samples]
    else:
        ctx.proposal_init(seed=args.seed)
        losses = train(ctx, x_tr, y_tr, args.samples, args.epochs, args.batch, args.lr, args.seed)
    for ep, l in enumerate(losses):
        print(f"epoch {ep}: loss {l:.4f}", flush=True)
    t3 = time.time()

    z = heldout_logits(ctx, x_te)
    r_all, _ = recall_at(z, lab, args.top_k, -1.0)
    curve.append({"samples": args.samples, "recall_topk": r_all, "top1": float((z.argmax(axis=1) == lab).mean())})
    taus = np.concatenate([[-1.0], np.linspace(0, 1, 1001)])
    tau = 1.0
    for t in taus:
        r, _ = recall_at(z[:half], lab[:half], args.top_k, t)
        if r >= args.target_recall:
            tau = float(t)
            break
    # ... and at least the given quantile of the tuning half's margins
    zt = z[:half] - z[:half].max(axis=1, keepdims=True)
    pt = np.exp(zt)
    pt = np.sort(pt / pt.sum(axis=1, keepdims=True), axis=1)
    tau = max(tau, float(np.quantile(pt[:, -1] - pt[:, -2], args.fallback_quantile)))
    rec, fb = recall_at(z[half:], lab[half:], args.top_k, tau)
    rec_topk, _ = recall_at(z[half:], lab[half:], args.top_k, -1.0)
    top1 = float((z[half:].argmax(axis=1) == lab[half:]).mean())
    print(f"held-out: tau {tau:.3f} recall {rec:.4f} fallback {fb:.3f} top-k alone {rec_topk:.4f} top-1 {top1:.3f}",
          flush=True)

    # throughput learned vs plain on 256 held-out queries (device-resident inputs)
    import scenegen as sg2
    qs = []
    dev = torch.device("cuda:0")
    for i in range(256):
        runs, _, _ = ctx.select_block(h_te[i][0], h_te[i][1], RADIUS)
        img = torch.empty((1, 3, cam.height, cam.width), device=dev)
        ctx.render(runs, sg2.pose_from_xyz_yaw(*h_te[i])[None], cam, rgb=img)
        qs.append((img[0].contiguous(), sg2.pose_from_xyz_yaw(*s_te[i]), RADIUS, GRID))
    timing = {}
    for mode in ("plain", "learned"):
        ctx.set_proposal(mode == "learned", args.top_k, tau)
        ctx.localize_batch(qs, cam, want_scores=False)
        torch.cuda.synchronize()
        a = time.perf_counter()
        res, _ = ctx.localize_batch(qs, cam, want_scores=False)
        torch.cuda.synchronize()
        timing[mode] = (time.perf_counter() - a, [r.best_index for r in res], [r.n_scored for r in res])
    ctx.set_proposal(False, args.top_k, tau)
    agree = float(np.mean(np.array(timing["plain"][1]) == np.array(timing["learned"][1])))
    summary = {
        "samples": args.samples, "heldout": args.heldout, "epochs": args.epochs, "batch": args.batch,
        "lr": args.lr, "top_k": args.top_k, "tau": tau, "target_recall": args.target_recall,
        "fallback_quantile": args.fallback_quantile,
        "recall_heldout": rec, "fallback_rate": fb, "recall_topk_alone_heldout": rec_topk,
        "top1_heldout": top1, "epoch_loss": losses, "recall_curve": curve,
        "queries_per_s_plain": 256 / timing["plain"][0], "queries_per_s_learned": 256 / timing["learned"][0],
        "agreement_256": agree, "mean_scored_learned": float(np.mean(timing["learned"][2])),
        "data_s": prev["data_s"] if prev else t2 - t1, "train_s": prev["train_s"] if prev else t3 - t2,
        "total_s": prev["total_s"] if prev else time.time() - t0,
    }
    print(json.dumps(summary), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    if not args.eval_only:
        ctx.proposal_get(0).astype("<f4").tofile(args.out)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
