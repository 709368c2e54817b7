"""Pins of the oracle's SSIM (the D-SSIM term of Eq. 3; SSIM of Wang, Bovik,
Sheikh and Simoncelli 2004 with an 11 x 11 Gaussian window of standard
deviation 1.5 px, zero outside the image, C1 = 0.01^2, C2 = 0.03^2) and of
the L_rgb loss with its forward-mode derivatives.

Closed forms the definition fixes: SSIM(x, x) = 1 at every pixel; for
constant images a, b, away from the border, (2ab + C1) / (a^2 + b^2 + C1);
for y = k x (every pixel: the zero padding scales too) the luminance and
contrast-structure factors (2k mx^2 + C1)/((1 + k^2) mx^2 + C1) and
(2k sx^2 + C2)/((1 + k^2) sx^2 + C2), with the local mean and variance from
scipy's correlation under the same window; for y = x + c away from the
border the contrast-structure factor is 1; SSIM is symmetric.  The loss
value equals (1 - lambda) L1 + lambda (1 - mean SSIM) of the plain oracle's
renders; with every threshold off, its derivative along a direction equals
central differences of that value (lambda = 1: D-SSIM alone; step 2^-18,
so every perturbed float32 parameter is exact; the differences converge as
h^2: 1e-6 relative at 2^-14, 5e-9 at 2^-18)."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg

C1, C2 = 0.01 ** 2, 0.03 ** 2
SMOOTH = dict(cut=50.0, alpha_min=0.0, t_min=0.0, alpha_max=1.0)


def window():
    k = np.arange(11) - 5.0
    g = np.exp(-k ** 2 / (2 * 1.5 ** 2))
    w = np.outer(g, g)
    return w / w.sum()


def local(x):
    from scipy.ndimage import correlate
    return correlate(x, window(), mode="constant", cval=0.0)


def img(seed, h=23, w=31):
    return sg.Rng(seed).uniform(h * w).reshape(h, w)


def test_window_sums_to_one_and_is_gaussian():
    w = window()
    assert abs(w.sum() - 1.0) < 1e-15 and abs(w[5, 6] / w[5, 5] - math.exp(-1 / 4.5)) < 1e-15


def test_ssim_of_an_image_with_itself_is_one():
    x = img(1)
    assert np.max(np.abs(oracle.ssim_map(x, x) - 1.0)) < 1e-13


def test_constant_images_interior():
    a, b = 0.3, 0.7
    s = oracle.ssim_map(np.full((20, 24), a), np.full((20, 24), b))
    ref = (2 * a * b + C1) / (a * a + b * b + C1)
    assert np.max(np.abs(s[5:-5, 5:-5] - ref)) < 1e-11   # E[x^2] - mx^2 cancels to ~1e-16, over C2
    assert np.all(np.abs(s[0, :] - ref) > 1e-3)          # the zero padding shows at the border


@pytest.mark.parametrize("k", [0.5, 1.7])
def test_scaled_image_factorises(k):
    x = img(2)
    mx = local(x)
    sx = local(x * x) - mx * mx
    ref = (2 * k * mx ** 2 + C1) / ((1 + k * k) * mx ** 2 + C1) * (2 * k * sx + C2) / ((1 + k * k) * sx + C2)
    assert np.max(np.abs(oracle.ssim_map(x, k * x) - ref)) < 1e-12


def test_shifted_image_interior_is_luminance_only():
    x = img(3)
    c = 0.2
    mx = local(x)
    ref = (2 * mx * (mx + c) + C1) / (mx ** 2 + (mx + c) ** 2 + C1)
    s = oracle.ssim_map(x, x + c)
    assert np.max(np.abs(s[5:-5, 5:-5] - ref[5:-5, 5:-5])) < 1e-12


def test_symmetric():
    x, y = img(4), img(5)
    assert np.max(np.abs(oracle.ssim_map(x, y) - oracle.ssim_map(y, x))) < 1e-14


def l_rgb(g, poses, cam, gt, prm, lam):
    imgs = oracle.render_views(g, poses, cam, prm, images=True, flags=False)["rgb"]
    total = 0.0
    for v in range(len(poses)):
        l1 = np.abs(imgs[v] - gt[v]).mean()
        ss = np.mean([oracle.ssim_map(imgs[v][c], gt[v][c]).mean() for c in range(3)])
        total += (1 - lam) * l1 + lam * (1 - ss)
    return total / len(poses)


@pytest.fixture(scope="module")
def setup():
    s = sg.tiny_scene(n=400)
    full = sg.tiny_scene()
    poses = full.candidate_poses[:2]
    gt = oracle.render_views(full.gaussians, poses, s.camera, images=True, flags=False)["rgb"]
    r = sg.Rng(23)
    dirs = (r.u64(s.gaussians.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(s.gaussians.n, 14, 6) - 1.0
    return s, poses, gt, dirs


def test_loss_value_is_l1_plus_dssim(setup):
    s, poses, gt, dirs = setup
    L, _ = oracle.photo_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, lam=0.2)
    ref = l_rgb(s.gaussians, poses, s.camera, gt, oracle.params(), 0.2)
    assert abs(L - ref) < 1e-12


def test_dssim_derivatives_equal_central_differences(setup):
    from test_oracle_train_pins import perturbed
    s, poses, gt, dirs = setup
    prm = oracle.params(**SMOOTH)
    _, jv = oracle.photo_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, prm, lam=1.0)
    h = 2.0 ** -18
    for k in range(3):
        fp = l_rgb(perturbed(s.gaussians, dirs[:, :, k], h), poses, s.camera, gt, prm, 1.0)
        fm = l_rgb(perturbed(s.gaussians, dirs[:, :, k], -h), poses, s.camera, gt, prm, 1.0)
        fd = (fp - fm) / (2 * h)
        print(k, jv[k], fd, abs(jv[k] - fd) / abs(fd))
        assert abs(jv[k] - fd) <= 2e-8 * abs(fd) + 1e-12
