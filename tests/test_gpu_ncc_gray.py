"""Gray NCC (reloc_config.ncc_gray = 1: Eq. ncc over the gray values
(R + G + B) / 3 of render and query) against the oracle with the same
option: scores within the NCC tolerance of the RGB parity tests, the same
winner and winner image through reloc_localize, and the gray score's pose
gradient (reloc_score_grad, SH degree 0) within 1e-3 of the oracle's norm."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import TOL_NCC

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


@pytest.fixture(scope="module")
def tiny(R):
    s = sg.tiny_scene()
    ctx = R.Context(R.reloc_default_config(ncc_gray=1, block_size=5.0))
    ctx.load_map(s.gaussians)
    g = s.gaussians.subset(ctx.map_order())
    q = (oracle.render(g, s.hidden_pose, s.camera)["rgb"] + s.query_noise).astype(np.float32)
    return s, ctx, g, q


def test_gray_scores_match_oracle(R, tiny):
    s, ctx, g, q = tiny
    sc, dg = ctx.score([(0, ctx.n)], s.candidate_poses, s.camera, torch.tensor(q, device="cuda:0"))
    ref = oracle.render_views(g, s.candidate_poses, s.camera, oracle.params(ncc_gray=1), query=q, images=False,
                              flags=False)["scores"]
    rgb = oracle.render_views(g, s.candidate_poses, s.camera, query=q, images=False, flags=False)["scores"]
    err = np.abs(sc - ref).max()
    print("gray ncc max err", err, "gray vs rgb", np.abs(ref - rgb).max())
    assert err <= TOL_NCC and not dg.any()
    assert np.abs(ref - rgb).max() > 1e-3                       # the option changes the score


def test_gray_localize_winner(R, tiny):
    s, ctx, g, q = tiny
    cam = s.camera
    brgb = torch.empty((3, cam.height, cam.width), device="cuda:0")
    res, sc = ctx.localize(torch.tensor(q, device="cuda:0"), s.seed_pose, 12.0, (3, 3, 2, 0.5, 3.0), cam,
                           best_rgb=brgb)
    c = -s.seed_pose[:3, :3].T @ s.seed_pose[:3, 3]
    idx, _ = oracle.block_select(s.gaussians.mean, 5.0, c[0], c[1], 12.0)
    poses = oracle.grid_poses(s.seed_pose, 3, 3, 2, 0.5, 3.0)
    ref = oracle.render_views(s.gaussians.subset(idx), poses, cam, oracle.params(ncc_gray=1), query=q)
    assert np.abs(sc - ref["scores"]).max() <= TOL_NCC
    top = np.sort(ref["scores"])[::-1]
    if top[0] - top[1] > TOL_NCC:
        assert res.best_index == oracle.argmax(ref["scores"])


def test_gray_pose_gradient_matches_oracle(R, tiny):
    s, ctx, g, q = tiny
    qd = torch.tensor(q, device="cuda:0")
    for v in (0, 7):
        W = s.candidate_poses[v]
        sc, gr = ctx.score_grad([(0, ctx.n)], W[None], s.camera, qd)
        ncc, ref = oracle.ncc_pose_grad(g, W, s.camera, q, oracle.params(ncc_gray=1))
        err = np.linalg.norm(gr[0] - ref) / np.linalg.norm(ref)
        print(v, sc[0], ncc, err)
        assert abs(sc[0] - ncc) <= TOL_NCC and err <= 1e-3
