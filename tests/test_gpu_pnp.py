"""reloc_refine_pnp (Sec. III-C.2 PnP refinement) against the oracle's FP64
solve on the same inputs (oracle-rendered depth and alpha, pixel pairs from
the oracle's back-projection and projection): noise-free pairs and pairs
with noise and outliers give the same pose (both solve the same FP64
problem; only summation order differs), the same number of usable pairs;
invalid calls.  End to end on the driving street: localize, then iterate
render (depth + alpha at the current pose) -> pairs -> PnP three times, the
pairs coming from a stand-in matcher (the hidden pose and the rendered depth,
0.5 px noise, 10% outliers); the pose error must shrink to the noise level."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from pnp_cases import make_pairs, pose_error, tiny_views

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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("noise,outliers", [(0.0, 0.0), (0.5, 0.25)])
def test_pnp_matches_oracle(R, noise, outliers):
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr, noise_px=noise, outlier_frac=outliers, seed=11)
    ref = oracle.refine_pnp(Wr, s.camera, depth, alpha, pairs)
    ctx = R.Context()
    res = ctx.refine_pnp(Wr, s.camera, dev(depth), dev(alpha), dev(pairs))
    P = np.array(res.pose).reshape(4, 4)
    dt, dr = pose_error(P, ref["pose"])
    print("gpu vs oracle", dt, dr, res.iters, ref["iters"], res.rms_px, ref["rms_px"])
    assert res.n_used == ref["n_used"] == len(pairs)
    assert dt < 1e-9 and dr < 1e-10
    assert abs(res.rms_px - ref["rms_px"]) <= 1e-6 * max(1.0, ref["rms_px"])


def test_pnp_many_pairs_matches_oracle(R):
    """Every pixel of the tiny view as a pair (~25k pairs, so the solve spreads
    over about a hundred blocks): the same pose as the oracle's FP64 solve."""
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr, step=1, noise_px=0.3, outlier_frac=0.1, seed=5)
    ref = oracle.refine_pnp(Wr, s.camera, depth, alpha, pairs)
    ctx = R.Context()
    res = ctx.refine_pnp(Wr, s.camera, dev(depth), dev(alpha), dev(pairs))
    dt, dr = pose_error(np.array(res.pose).reshape(4, 4), ref["pose"])
    print(len(pairs), "pairs; gpu vs oracle", dt, dr, res.iters, ref["iters"])
    assert len(pairs) > 20000 and res.n_used == ref["n_used"]
    assert dt < 1e-9 and dr < 1e-10
    assert abs(res.rms_px - ref["rms_px"]) <= 1e-6 * max(1.0, ref["rms_px"])


def test_pnp_invalid_calls(R):
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr)
    ctx = R.Context()
    with pytest.raises(R.RelocError) as e:
        ctx.refine_pnp(Wr, s.camera, dev(depth), dev(alpha), dev(pairs[:0]))
    assert e.value.status == R.EINVAL
    with pytest.raises(R.RelocError) as e:              # nothing in front of the alpha cut
        ctx.refine_pnp(Wr, s.camera, dev(depth), dev(np.zeros_like(alpha)), dev(pairs))
    assert e.value.status == R.ENUMERIC
    with pytest.raises(R.RelocError) as e:
        ctx.refine_pnp(Wr, s.camera, dev(depth), dev(alpha), dev(pairs), max_iters=-1)
    assert e.value.status == R.EINVAL
    res = ctx.refine_pnp(Wr, s.camera, dev(depth), dev(alpha), dev(pairs))   # still usable
    assert res.n_used == len(pairs)


def stand_in_pairs(W_render, W_query, cam, depth, alpha, step, noise, outliers, gen):
    """Matcher stand-in (torch, float64): render pixels on a grid with alpha >=
    0.95, their points from the rendered depth, projected into the query pose."""
    H, W = cam.height, cam.width
    ys, xs = torch.meshgrid(torch.arange(step // 2, H - 1, step, device="cuda:0"),
                            torch.arange(step // 2, W - 1, step, device="cuda:0"), indexing="ij")
    ys, xs = ys.reshape(-1), xs.reshape(-1)
    a = alpha[ys, xs].double()
    keep = a >= 0.95
    ys, xs, a = ys[keep], xs[keep], a[keep]
    z = depth[ys, xs].double() / a
    u, v = xs.double() + 0.5, ys.double() + 0.5
    Pc = torch.stack([z * (u - cam.cx) / cam.fx, z * (v - cam.cy) / cam.fy, z], 1)
    Rr = torch.tensor(W_render[:3, :3], device="cuda:0")
    tr = torch.tensor(W_render[:3, 3], device="cuda:0")
    X = (Pc - tr) @ Rr
    Rq = torch.tensor(W_query[:3, :3], device="cuda:0")
    tq = torch.tensor(W_query[:3, 3], device="cuda:0")
    P = X @ Rq.T + tq
    q = torch.stack([cam.fx * P[:, 0] / P[:, 2] + cam.cx, cam.fy * P[:, 1] / P[:, 2] + cam.cy], 1)
    q = q + noise * torch.randn(q.shape, device="cuda:0", dtype=torch.float64, generator=gen)
    n_out = int(outliers * q.shape[0])
    idx = torch.randperm(q.shape[0], device="cuda:0", generator=gen)[:n_out]
    q[idx, 0] = torch.rand(n_out, device="cuda:0", dtype=torch.float64, generator=gen) * W
    q[idx, 1] = torch.rand(n_out, device="cuda:0", dtype=torch.float64, generator=gen) * H
    ok = (P[:, 2] > 0.1) & (q[:, 0] >= 0) & (q[:, 0] < W) & (q[:, 1] >= 0) & (q[:, 1] < H)
    return torch.stack([u, v, q[:, 0], q[:, 1]], 1)[ok].float().contiguous()


def test_refinement_loop_on_the_street(R):
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    hidden, seeds = sg.street_queries(1, seed=61)
    Wh = sg.pose_from_xyz_yaw(*hidden[0])
    ctx = R.Context()
    ctx.load_map(g)
    runs, _, _ = ctx.select_block(hidden[0][0], hidden[0][1], 40.0)
    H, W = cam.height, cam.width
    img = torch.empty((1, 3, H, W), device="cuda:0")
    ctx.render(runs, Wh[None], cam, rgb=img)
    rgb = torch.empty((3, H, W), device="cuda:0")
    depth = torch.empty((H, W), device="cuda:0")
    alpha = torch.empty((H, W), device="cuda:0")
    res, _ = ctx.localize(img[0].contiguous(), sg.pose_from_xyz_yaw(*seeds[0]), 40.0, (4, 4, 4, 0.5, 2.0), cam,
                          best_rgb=rgb, best_depth=depth, best_alpha=alpha, want_scores=False)
    Wk = np.array(res.best_pose).reshape(4, 4)
    errs = [pose_error(Wk, Wh)]
    gen = torch.Generator(device="cuda:0")
    gen.manual_seed(5)
    for it in range(3):
        if it > 0:
            d1 = torch.empty((1, H, W), device="cuda:0")
            a1 = torch.empty((1, H, W), device="cuda:0")
            ctx.render(runs, Wk[None], cam, depth=d1, alpha=a1)
            depth, alpha = d1[0], a1[0]
        pairs = stand_in_pairs(Wk, Wh, cam, depth, alpha, 8, 0.5, 0.1, gen)
        out = ctx.refine_pnp(Wk, cam, depth, alpha, pairs)
        Wk = np.array(out.pose).reshape(4, 4)
        errs.append(pose_error(Wk, Wh))
    print("pose error per iteration (m, deg):", [(round(t, 4), round(math.degrees(r), 4)) for t, r in errs])
    assert errs[-1][0] < 0.02 and errs[-1][1] < math.radians(0.05)
    assert errs[-1][0] < errs[0][0] or errs[0][0] < 0.02
