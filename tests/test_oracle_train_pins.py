"""Pins of the oracle's map-training loss (Sec. III-B.3, the L1 part of
L_rgb) and its forward-mode derivatives along directions in the Gaussians'
parameters: its value equals the mean absolute difference of the plain
oracle's renders; with every threshold switched off and black targets
(the loss is then the mean colour, smooth in the parameters: L1 has no kink
where colours are >= 0) each directional derivative equals central
differences of the plain oracle's loss (directions in {-1, 0, 1} and step
2^-14, so every perturbed float32 parameter is exact; the differences
converge to the derivative: 2e-3 relative at 2^-8, 2e-5 at 2^-12, 2e-8 at
2^-14); derivatives are linear in the direction."""
import numpy as np
import pytest

import oracle
import scenegen as sg

SMOOTH = dict(cut=50.0, alpha_min=0.0, t_min=0.0, alpha_max=1.0)


def perturbed(g, d, h):
    """g with its parameters moved by h * d (d: [n, 14] in oracle.PARAM_ORDER)."""
    mean = (g.mean.astype(np.float64) + h * d[:, 0:3]).astype(np.float32)
    scale = (g.scale.astype(np.float64) + h * d[:, 3:6]).astype(np.float32)
    quat = (g.quat.astype(np.float64) + h * d[:, 6:10]).astype(np.float32)
    opac = (g.opacity.astype(np.float64) + h * d[:, 10]).astype(np.float32)
    sh = (g.sh.astype(np.float64) + h * d[:, None, 11:14]).astype(np.float32)
    return sg.Gaussians(mean, scale, quat, opac, sh, 0)


def l1(g, poses, cam, gt, prm):
    img = oracle.render_views(g, poses, cam, prm, images=True, flags=False)["rgb"]
    return float(np.abs(img - gt).mean())


@pytest.fixture(scope="module")
def setup():
    s = sg.tiny_scene(n=400)
    full = sg.tiny_scene()
    poses = full.candidate_poses[:2]
    # targets: the 10k-Gaussian scene's renders (the 400 Gaussians are a poor fit of them)
    gt = oracle.render_views(full.gaussians, poses, s.camera, images=True, flags=False)["rgb"]
    r = sg.Rng(21)
    dirs = (r.u64(s.gaussians.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(s.gaussians.n, 14, 6) - 1.0
    return s, poses, gt, dirs


def test_value_is_mean_absolute_difference(setup):
    s, poses, gt, dirs = setup
    L, _ = oracle.photo_loss_jvp(s.gaussians, poses, s.camera, gt, dirs)
    assert abs(L - l1(s.gaussians, poses, s.camera, gt, oracle.params())) < 1e-12


def test_smooth_directional_derivatives_equal_central_differences(setup):
    s, poses, gt, dirs = setup
    prm = oracle.params(**SMOOTH)
    gt = np.zeros_like(gt)
    _, jv = oracle.photo_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, prm)
    h = 2.0 ** -14
    for k in range(3):
        fp = l1(perturbed(s.gaussians, dirs[:, :, k], h), poses, s.camera, gt, prm)
        fm = l1(perturbed(s.gaussians, dirs[:, :, k], -h), poses, s.camera, gt, prm)
        fd = (fp - fm) / (2 * h)
        print(k, jv[k], fd)
        assert abs(jv[k] - fd) <= 1e-6 * abs(fd) + 1e-10


def test_derivative_is_linear_in_the_direction(setup):
    s, poses, gt, dirs = setup
    d2 = dirs.copy()
    d2[:, :, 2] = 2.0 * dirs[:, :, 0] - 3.0 * dirs[:, :, 1]
    _, jv = oracle.photo_loss_jvp(s.gaussians, poses, s.camera, gt, d2)
    assert abs(jv[2] - (2.0 * jv[0] - 3.0 * jv[1])) <= 1e-12 * max(1.0, abs(jv[2]))
