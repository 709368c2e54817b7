"""Pins of the oracle's NCC pose gradient (forward-mode derivatives of its
own projection, compositing and NCC; SH degree 0): its NCC value equals the
plain oracle's; with every threshold switched off (no 3-sigma cut, no alpha
skip, clamp or stop, so the function is smooth) the derivatives equal central
differences of the plain oracle's NCC under the pose update; at the pose a
noise-free query was rendered from, NCC = 1 is a maximum and the gradient
vanishes; a small step along the gradient raises NCC."""
import numpy as np
import pytest

import oracle
import scenegen as sg

SMOOTH = dict(cut=50.0, alpha_min=0.0, t_min=0.0, alpha_max=1.0)


@pytest.fixture(scope="module")
def tiny():
    s = sg.tiny_scene()
    q = oracle.render(s.gaussians, s.hidden_pose, s.camera)["rgb"] + s.query_noise
    return s, q


def test_value_equals_plain_ncc(tiny):
    s, q = tiny
    for W in s.candidate_poses[:3]:
        ncc, _ = oracle.ncc_pose_grad(s.gaussians, W, s.camera, q)
        ref = oracle.render_views(s.gaussians, W[None], s.camera, query=q, images=False, flags=False)["scores"][0]
        assert abs(ncc - ref) < 1e-12


def test_smooth_gradient_equals_central_differences(tiny):
    s, q = tiny
    prm = oracle.params(**SMOOTH)
    sub = s.gaussians.subset(np.arange(0, s.gaussians.n, 25))      # 400 Gaussians: every one covers every pixel
    for W in s.candidate_poses[:2]:
        _, g = oracle.ncc_pose_grad(sub, W, s.camera, q, prm)
        h = 1e-6
        fd = np.zeros(6)
        for k in range(6):
            d = np.zeros(6); d[k] = h
            fp = oracle.render_views(sub, oracle.pnp_apply(W, d)[None], s.camera, prm, query=q,
                                     images=False, flags=False)["scores"][0]
            fm = oracle.render_views(sub, oracle.pnp_apply(W, -d)[None], s.camera, prm, query=q,
                                     images=False, flags=False)["scores"][0]
            fd[k] = (fp - fm) / (2 * h)
        print(g, fd)
        assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_gradient_vanishes_at_the_rendered_pose(tiny):
    s, _ = tiny
    q0 = oracle.render(s.gaussians, s.hidden_pose, s.camera)["rgb"]
    ncc, g = oracle.ncc_pose_grad(s.gaussians, s.hidden_pose, s.camera, q0)
    assert abs(ncc - 1.0) < 1e-12 and np.abs(g).max() < 1e-9


def test_step_along_gradient_raises_ncc(tiny):
    s, q = tiny
    W = s.candidate_poses[5]
    ncc, g = oracle.ncc_pose_grad(s.gaussians, W, s.camera, q)
    step = 1e-4 * g / np.linalg.norm(g)
    up = oracle.render_views(s.gaussians, oracle.pnp_apply(W, step)[None], s.camera, query=q, images=False,
                             flags=False)["scores"][0]
    assert up > ncc


def test_needs_sh_degree_zero():
    g = sg.street_gaussians(1000, seed=3, sh_degree=3)
    with pytest.raises(ValueError):
        oracle.ncc_pose_grad(g, np.eye(4), sg.street_camera(), np.zeros((3, 376, 1408)))
