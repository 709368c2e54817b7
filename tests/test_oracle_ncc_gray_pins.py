"""Pins of the oracle's gray NCC option (Eq. ncc with "intensity" read as
the gray value (R + G + B) / 3 per pixel instead of every RGB sample).

Against what the definition fixes: the score equals numpy's Pearson r of
the gray images of the plain oracle's renders and the query; a noise-free
query rendered at a candidate's pose scores 1 there; on a scene and query
whose three channels are equal the gray and RGB scores coincide (the RGB
vector is the gray vector three times over); on coloured scenes they differ;
the pose gradient of the gray score equals central differences of the plain
gray score with every render threshold off."""
import numpy as np
import pytest

import oracle
import scenegen as sg

SMOOTH = dict(cut=50.0, alpha_min=0.0, t_min=0.0, alpha_max=1.0)


@pytest.fixture(scope="module")
def scene():
    s = sg.tiny_scene(n=2000)
    q = oracle.render(s.gaussians, s.hidden_pose, s.camera)["rgb"] + s.query_noise
    return s, q


def test_gray_score_is_pearson_r_of_gray_images(scene):
    s, q = scene
    out = oracle.render_views(s.gaussians, s.candidate_poses, s.camera, oracle.params(ncc_gray=1), query=q,
                              images=True, flags=False)
    qg = q.mean(axis=0).ravel()
    for v in range(len(s.candidate_poses)):
        r = np.corrcoef(out["rgb"][v].mean(axis=0).ravel(), qg)[0, 1]
        assert abs(out["scores"][v] - r) < 1e-12


def test_own_pose_scores_one(scene):
    s, _ = scene
    q = oracle.render(s.gaussians, s.candidate_poses[3], s.camera)["rgb"]
    out = oracle.render_views(s.gaussians, s.candidate_poses, s.camera, oracle.params(ncc_gray=1), query=q,
                              images=False, flags=False)
    assert abs(out["scores"][3] - 1.0) < 1e-12 and oracle.argmax(out["scores"]) == 3


def test_equal_channels_give_the_rgb_score(scene):
    s, q = scene
    g = s.gaussians
    grey = sg.Gaussians(g.mean, g.scale, g.quat, g.opacity, np.repeat(g.sh[:, :, :1], 3, axis=2), 0)
    qg = np.repeat(q.mean(axis=0, keepdims=True), 3, axis=0)
    a = oracle.render_views(grey, s.candidate_poses, s.camera, oracle.params(ncc_gray=1), query=qg,
                            images=False, flags=False)["scores"]
    b = oracle.render_views(grey, s.candidate_poses, s.camera, oracle.params(), query=qg,
                            images=False, flags=False)["scores"]
    assert np.max(np.abs(a - b)) < 1e-12
    c = oracle.render_views(g, s.candidate_poses, s.camera, oracle.params(), query=q, images=False,
                            flags=False)["scores"]
    d = oracle.render_views(g, s.candidate_poses, s.camera, oracle.params(ncc_gray=1), query=q, images=False,
                            flags=False)["scores"]
    assert np.max(np.abs(c - d)) > 1e-3


def test_gray_pose_gradient_equals_central_differences(scene):
    s, q = scene
    prm = oracle.params(ncc_gray=1, **SMOOTH)
    sub = s.gaussians.subset(np.arange(0, s.gaussians.n, 5))       # 400 Gaussians (each covers every pixel)
    W = s.candidate_poses[5]
    _, g = oracle.ncc_pose_grad(sub, W, s.camera, q, prm)
    h = 1e-6
    fd = np.zeros(6)
    for k in range(6):
        d = np.zeros(6)
        d[k] = h
        fp = oracle.render_views(sub, oracle.pnp_apply(W, d)[None], s.camera, prm, query=q, images=False,
                                 flags=False)["scores"][0]
        fm = oracle.render_views(sub, oracle.pnp_apply(W, -d)[None], s.camera, prm, query=q, images=False,
                                 flags=False)["scores"][0]
        fd[k] = (fp - fm) / (2 * h)
    print(g, fd)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()
