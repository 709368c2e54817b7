"""The learned candidate proposal on the GPU (tcgen05 BF16 GEMMs, FP32
accumulation) against the FP64 CNN oracle run on the same BF16-rounded
weights and inputs.

The GPU network stores its activations in BF16 (8 significand bits) and
carries every backward signal as two BF16 terms (hi + lo, ~16 bits).  The
oracle's act_bf16 mode stores the activations the same way (the BF16
network's definition) and is FP64 otherwise: against it, logits within 2e-3
relative L2 and every gradient tensor at cosine >= 0.999 and relative L2
<= 1e-2 (FP32 accumulation and the odd activation rounded the other way at
a tie).  Against the pure FP64 network (activations not rounded) the BF16
storage itself shows: logits within 3e-2, gradients at cosine >= 0.998 and
relative L2 <= 0.1 (the stored activations are rounded six layers deep and a
weight gradient sums up to 540,672 products with strong cancellation for
random labels).  A step along the GPU gradient must lower the oracle's loss.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


def rounded_params(flat):
    """Oracle parameters equal to what the GPU computes with: BF16 weights,
    FP32 biases."""
    p = flat.astype(np.float64).copy()
    for wo, bo, shape in oracle.cnn_offsets():
        p[wo:bo] = torch.tensor(flat[wo:bo]).to(torch.bfloat16).float().numpy()
    return p


def inputs(B, seed):
    x = sg.Rng(seed).uniform(B * 47 * 176 * 2).reshape(B, 47, 176, 2).astype(np.float32)
    t = torch.tensor(x).to(torch.bfloat16)
    return t.cuda().view(torch.int16), t.float().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def cosine(a, b):
    return float(np.dot(a, b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


def test_forward_matches_oracle(R):
    ctx = R.Context()
    ctx.proposal_init(seed=5)
    p = rounded_params(ctx.proposal_get(0))
    xi, x = inputs(64, 7)
    logits = torch.empty((64, 64), device="cuda:0")
    ctx.proposal_forward(xi, logits)
    torch.cuda.synchronize()
    got = logits.cpu().numpy().astype(np.float64)
    e = rel_l2(got, oracle.cnn_forward(p, x, act_bf16=True))
    e64 = rel_l2(got, oracle.cnn_forward(p, x))
    print("forward logits rel L2: BF16-activation oracle", e, "FP64 network", e64)
    assert e <= 2e-3
    assert e64 <= 3e-2


def test_gradients_match_oracle(R):
    ctx = R.Context()
    ctx.proposal_init(seed=6)
    p = rounded_params(ctx.proposal_get(0))
    xi, x = inputs(64, 8)
    labels = (sg.Rng(9).u64(64) % np.uint64(64)).astype(np.int32)
    loss = ctx.proposal_train_step(xi, torch.tensor(labels, device="cuda:0"), 0.0, update=False)
    g = ctx.proposal_get(1).astype(np.float64)
    loss_ref, g_ref = oracle.cnn_loss_grad(p, x, labels, act_bf16=True)
    loss64, g64 = oracle.cnn_loss_grad(p, x, labels)
    print("loss", loss, "BF16-activation oracle", loss_ref, "FP64 network", loss64)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    assert abs(loss - loss64) <= 1e-2 * loss64
    for t, (wo, bo, shape) in enumerate(oracle.cnn_offsets()):
        for name, lo, hi in (("W", wo, bo), ("b", bo, bo + shape[0])):
            c, e = cosine(g[lo:hi], g_ref[lo:hi]), rel_l2(g[lo:hi], g_ref[lo:hi])
            c64, e64 = cosine(g[lo:hi], g64[lo:hi]), rel_l2(g[lo:hi], g64[lo:hi])
            print(f"layer {t} {name}: cosine {c:.6f} rel L2 {e:.3e} | FP64 network: cosine {c64:.6f} rel L2 {e64:.3e}")
            assert c >= 0.999 and e <= 1e-2, (t, name, c, e)
            assert c64 >= 0.998 and e64 <= 0.1, (t, name, c64, e64)
    # the GPU gradient is a descent direction of the oracle's loss
    eta = 1e-3 / np.linalg.norm(g)
    assert oracle.cnn_loss_grad(p - eta * g, x, labels)[0] < loss_ref


def test_adam_step_matches_oracle(R):
    ctx = R.Context()
    ctx.proposal_init(seed=10)
    p0 = ctx.proposal_get(0).astype(np.float64)
    xi, x = inputs(64, 11)
    labels = torch.tensor((np.arange(64) * 7 % 64).astype(np.int32), device="cuda:0")
    ctx.proposal_train_step(xi, labels, 1e-3, update=True)
    g = ctx.proposal_get(1).astype(np.float64)
    p1 = ctx.proposal_get(0).astype(np.float64)
    w1, _, _ = oracle.adam(p0, np.zeros_like(p0), np.zeros_like(p0), g, 1e-3, 1)
    assert np.abs(p1 - w1).max() <= 1e-6


def test_make_input_matches_oracle(R):
    ctx = R.Context()
    cam = sg.Camera(352, 94, 138.0, 138.0, 176.0, 47.0)
    a = sg.random_image(21, 3, 94, 352)
    b = sg.random_image(22, 3, 94, 352)
    out = torch.zeros((47, 176, 2), dtype=torch.int16, device="cuda:0")
    ctx.proposal_make_input(torch.tensor(a, device="cuda:0"), torch.tensor(b, device="cuda:0"), cam, out)
    got = out.view(torch.bfloat16).float().cpu().numpy()
    for ch, img in ((0, a), (1, b)):
        ref = oracle.downsample_gray(img, 2)
        assert np.abs(got[..., ch] - ref).max() <= 2.0 ** -8 * np.abs(ref).max()


def test_training_learns_a_synthetic_task(R):
    """A bright 8x5-pixel block at one of 64 places; the label is the place."""
    ctx = R.Context()
    ctx.proposal_init(seed=12)
    B = 128
    r = sg.Rng(13)
    losses = []
    for step in range(60):
        lab = (r.u64(B) % np.uint64(64)).astype(np.int32)
        x = 0.1 * r.uniform(B * 47 * 176 * 2).reshape(B, 47, 176, 2).astype(np.float32)
        for i, c in enumerate(lab):
            y0, x0 = 5 * (c // 8), 22 * (c % 8)
            x[i, y0:y0 + 5, x0:x0 + 8, 0] += 1.0
        t = torch.tensor(x).to(torch.bfloat16).cuda().view(torch.int16)
        losses.append(ctx.proposal_train_step(t, torch.tensor(lab, device="cuda:0"), 2e-3))
    print("loss", losses[0], losses[-1])
    assert losses[0] > 0.8 * math.log(64)
    assert np.mean(losses[-5:]) < 0.5


def test_learned_localize_fallback_and_topk(R):
    g = sg.street_gaussians(150_000, seed=31, sh_degree=3)
    cam = sg.Camera(352, 94, 138.0, 138.0, 176.0, 47.0)
    ctx = R.Context()
    ctx.load_map(g)
    ctx.proposal_init(seed=14)
    hidden, seeds = sg.street_queries(3, seed=32)
    qs = []
    for i in range(3):
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], 40.0)
        img = torch.empty((1, 3, 94, 352), device="cuda:0")
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
        qs.append((img[0].contiguous(), sg.pose_from_xyz_yaw(*seeds[i]), 40.0, (4, 4, 4, 0.5, 2.0)))
    plain, plain_sc = ctx.localize_batch(qs, cam)
    # margin above any p1 - p2: every query falls back to the full sweep
    ctx.set_proposal(True, 8, 2.0)
    fb, fb_sc = ctx.localize_batch(qs, cam)
    for a, b, sa, sb in zip(plain, fb, plain_sc, fb_sc):
        assert a.best_index == b.best_index and a.best_score == b.best_score and b.n_scored == 64
        assert np.array_equal(sa, sb)
    # negative margin: always the top-8 cells
    ctx.set_proposal(True, 8, -1.0)
    tk, tk_sc = ctx.localize_batch(qs, cam)
    for a, b, sa, sb in zip(plain, tk, plain_sc, tk_sc):
        assert b.n_scored == 8 and b.n_candidates == 64
        scored = ~np.isnan(sb)
        assert scored.sum() == 8 and scored[b.best_index]
        assert np.array_equal(sb[scored], sa[scored])           # same renders, same scores
        assert b.best_score == np.max(sb[scored])
    ctx.set_proposal(False, 8, 0.0)


def test_learned_winner_equals_oracle_full_sweep():
    """Eight held-out driving queries: the GPU's plain sweep and the learned
    top-k + fallback (shipped weights) pick the FP64 oracle's own full-sweep
    winner (ties within the NCC tolerance excepted)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from proposal_oracle_check import learned_vs_oracle
    r = learned_vs_oracle(8)
    print(r)
    for i in range(r["queries"]):
        if r["oracle_top2_margin"][i] < 2e-6:
            continue
        assert r["gpu_sweep_winner"][i] == r["oracle_winner"][i], i
        assert r["learned_winner"][i] == r["oracle_winner"][i], i
