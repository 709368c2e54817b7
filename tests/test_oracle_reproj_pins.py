"""Pins of the oracle's re-projection loss (Sec. III-B.3, Eq. 5; the pairs
are consecutive training views, I_{t+1} re-projected into view t through
the rendered depth D / A where A >= alpha_min, bilinear sampling with pixel
centres at +0.5, pixels without a sample keep I_t).

An independent restatement pins the value: the plain oracle's depth and
alpha renders, the geometry in numpy and the bilinear sampling by scipy's
map_coordinates (order 1), L_rgb with the pinned SSIM map; the oracle's
forward-mode value equals it (lambda 0 and 0.2).  Two identical poses and
images give zero.  With every render threshold off, the derivative along a
direction equals central differences of the restatement (step 2^-18, the
float32 parameters exact; pixels whose sample crosses a bilinear cell edge
or the image edge within the step are rare and bound the agreement)."""
import numpy as np
import pytest

import oracle
import scenegen as sg

SMOOTH = dict(cut=50.0, alpha_min=0.0, t_min=0.0, alpha_max=1.0)


def reproj_plain(g, poses, cam, gt, prm, lam, alpha_min=0.5):
    from scipy.ndimage import map_coordinates
    out = oracle.render_views(g, poses, cam, prm, images=True, flags=False)
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    ray = np.stack([(xs + 0.5 - cam.cx) / cam.fx, (ys + 0.5 - cam.cy) / cam.fy, np.ones_like(xs)])
    near = prm[0]                               # near plane (the parameter vector's first entry)
    total = 0.0
    V = len(poses)
    for t in range(V - 1):
        D, A = out["depth"][t], out["alpha"][t]
        ok = A >= alpha_min
        d = np.where(ok, D / np.where(ok, A, 1.0), 0.0)
        Pc = d * ray
        Rt, tt = poses[t][:3, :3], poses[t][:3, 3]
        Rn, tn = poses[t + 1][:3, :3], poses[t + 1][:3, 3]
        X = np.einsum("ji,jhw->ihw", Rt, Pc - tt[:, None, None])
        Pn = np.einsum("ij,jhw->ihw", Rn, X) + tn[:, None, None]
        ok &= Pn[2] > near
        z = np.where(ok, Pn[2], 1.0)
        sx = cam.fx * Pn[0] / z + cam.cx - 0.5
        sy = cam.fy * Pn[1] / z + cam.cy - 0.5
        x0, y0 = np.floor(sx), np.floor(sy)
        ok &= (x0 >= 0) & (x0 <= W - 2) & (y0 >= 0) & (y0 <= H - 2)
        warped = np.empty((3, H, W))
        for c in range(3):
            smp = map_coordinates(gt[t + 1][c], [np.where(ok, sy, 0.0), np.where(ok, sx, 0.0)], order=1)
            warped[c] = np.where(ok, smp, gt[t][c])
        l1 = np.abs(warped - gt[t]).mean()
        ss = np.mean([oracle.ssim_map(warped[c], gt[t][c]).mean() for c in range(3)])
        total += (1 - lam) * l1 + lam * (1 - ss)
    return total / (V - 1)


@pytest.fixture(scope="module")
def setup():
    s = sg.tiny_scene(n=400)
    full = sg.tiny_scene()
    poses = full.candidate_poses[:3]
    gt = oracle.render_views(full.gaussians, poses, s.camera, images=True, flags=False)["rgb"]
    r = sg.Rng(29)
    dirs = (r.u64(s.gaussians.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(s.gaussians.n, 14, 6) - 1.0
    return s, poses, gt, dirs


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_value_equals_restatement(setup, lam):
    s, poses, gt, dirs = setup
    prm = oracle.params()
    L, _ = oracle.train_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, prm, lam=lam, w_photo=0.0, w_reproj=1.0)
    ref = reproj_plain(s.gaussians, poses, s.camera, gt, prm, lam)
    print(lam, L, ref)
    assert L > 1e-3 and abs(L - ref) < 1e-12


def test_value_equals_restatement_dense_depth(setup):
    # the 10k-Gaussian map: ~95% of the pixels have A >= 0.5 (7% with 400)
    s, poses, gt, dirs = setup
    full = sg.tiny_scene().gaussians
    prm = oracle.params()
    L, _ = oracle.train_loss_jvp(full, poses, s.camera, gt, np.zeros((full.n, 14, 6)), prm, lam=0.2, w_photo=0.0,
                                 w_reproj=1.0)
    ref = reproj_plain(full, poses, s.camera, gt, prm, 0.2)
    print(L, ref)
    assert L > 1e-3 and abs(L - ref) < 1e-12


def test_identical_views_give_zero(setup):
    s, poses, gt, dirs = setup
    P = np.stack([poses[0], poses[0]])
    I = np.stack([gt[0], gt[0]])
    L, _ = oracle.train_loss_jvp(s.gaussians, P, s.camera, I, dirs, lam=0.2, w_photo=0.0, w_reproj=1.0)
    assert abs(L) < 1e-12


def test_weights_combine(setup):
    s, poses, gt, dirs = setup
    Lp, jp = oracle.train_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, lam=0.2, w_photo=1.0, w_reproj=0.0)
    Lr, jr = oracle.train_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, lam=0.2, w_photo=0.0, w_reproj=1.0)
    L, j = oracle.train_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, lam=0.2, w_photo=0.7, w_reproj=1.3)
    assert abs(L - (0.7 * Lp + 1.3 * Lr)) < 1e-12
    assert np.max(np.abs(j - (0.7 * jp + 1.3 * jr))) < 1e-12 * max(1.0, np.max(np.abs(j)))


def test_derivatives_equal_central_differences(setup):
    from test_oracle_train_pins import perturbed
    s, poses, gt, dirs = setup
    prm = oracle.params(**SMOOTH)
    _, jv = oracle.train_loss_jvp(s.gaussians, poses, s.camera, gt, dirs, prm, lam=0.2, w_photo=0.0, w_reproj=1.0)
    h = 2.0 ** -18
    for k in range(3):
        fp = reproj_plain(perturbed(s.gaussians, dirs[:, :, k], h), poses, s.camera, gt, prm, 0.2)
        fm = reproj_plain(perturbed(s.gaussians, dirs[:, :, k], -h), poses, s.camera, gt, prm, 0.2)
        fd = (fp - fm) / (2 * h)
        print(k, jv[k], fd, abs(jv[k] - fd) / abs(fd))
        assert abs(jv[k] - fd) <= 1e-6 * abs(fd) + 1e-10
