"""Pins of the oracle's PnP refinement (Sec. III-C.2) against facts outside
its own code: a back-projected pixel re-projects onto itself with the same
pose; bilinear sampling is exact on an image linear in x and y; the
residual's Jacobian matches central differences of the residual under the
pose update; noise-free pairs give back the query pose exactly from a start
0.3 m / 2 deg away (up to the float32 rounding of the pixel coordinates); with a quarter of the pairs replaced by random pixels
(and 0.5 px noise on the rest) the Huber solve stays within centimetres
while a pure least-squares solve (Huber threshold 1e6 px) does not."""
import math

import numpy as np

import oracle
import scenegen as sg
from pnp_cases import make_pairs, pose_error, tiny_views


def test_backproject_reprojects_onto_itself():
    s, Wq, Wr = tiny_views()
    cam = s.camera
    rng = sg.Rng(3)
    depth = (2.0 + 3.0 * rng.uniform(cam.height * cam.width)).reshape(cam.height, cam.width).astype(np.float32)
    alpha = np.full((cam.height, cam.width), 0.8, np.float32)
    uv = np.stack([rng.uniform(50, 1, cam.width - 1), rng.uniform(50, 1, cam.height - 1)], 1)
    X, used = oracle.pnp_backproject(Wr, cam, depth, alpha, uv)
    assert used.all()
    for x, p in zip(X, uv):
        r, _ = oracle.pnp_residual(Wr, x, cam, p)
        assert np.abs(r).max() < 1e-9


def test_bilinear_exact_on_linear_image():
    s, Wq, Wr = tiny_views()
    cam = s.camera
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    depth = (3.0 + 0.01 * xs + 0.02 * ys).astype(np.float32)     # exact in float32 up to rounding
    alpha = np.ones_like(depth)
    uv = np.array([[10.3, 7.9], [100.75, 40.25], [351.6, 93.6]])
    X, used = oracle.pnp_backproject(Wr, cam, depth, alpha, uv)
    assert used.tolist() == [True, True, False]                  # last one's neighbourhood leaves the image
    for x, (u, v) in zip(X[:2], uv[:2]):
        P = Wr[:3, :3] @ x + Wr[:3, 3]
        assert abs(P[2] - (3.0 + 0.01 * (u - 0.5) + 0.02 * (v - 0.5))) < 2e-6


def test_jacobian_matches_central_differences():
    s, Wq, Wr = tiny_views()
    X = Wq[:3, :3].T @ (np.array([0.7, -0.3, 6.2]) - Wq[:3, 3])     # camera point (0.7, -0.3, 6.2)
    q = np.array([150.0, 40.0])
    r0, J = oracle.pnp_residual(Wq, X, s.camera, q)
    h = 1e-6
    for k in range(6):
        d = np.zeros(6); d[k] = h
        rp, _ = oracle.pnp_residual(oracle.pnp_apply(Wq, d), X, s.camera, q)
        rm, _ = oracle.pnp_residual(oracle.pnp_apply(Wq, -d), X, s.camera, q)
        fd = (rp - rm) / (2 * h)
        assert np.abs(fd - J[:, k]).max() <= 1e-5 * max(1.0, np.abs(J[:, k]).max())


def test_noise_free_pairs_recover_the_query_pose():
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr)
    assert len(pairs) > 200
    res = oracle.refine_pnp(Wr, s.camera, depth, alpha, pairs)
    dt, dr = pose_error(res["pose"], Wq)
    dt0, dr0 = pose_error(Wr, Wq)
    assert dt0 > 0.2 and dr0 > math.radians(1.5)
    # pairs are float32: ~1e-5 px rounding of pixel coordinates at 6 m and
    # f = 138 px moves the optimum by ~1e-7 m
    assert dt < 1e-6 and dr < 1e-7 and res["rms_px"] < 1e-4
    assert res["n_used"] == len(pairs)


def test_huber_resists_outliers():
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr, noise_px=0.5, outlier_frac=0.25, seed=7)
    robust = oracle.refine_pnp(Wr, s.camera, depth, alpha, pairs)
    plain = oracle.refine_pnp(Wr, s.camera, depth, alpha, pairs, huber_px=1e6)
    dt_r, dr_r = pose_error(robust["pose"], Wq)
    dt_p, dr_p = pose_error(plain["pose"], Wq)
    print("huber", dt_r, dr_r, "least squares", dt_p, dr_p)
    assert dt_r < 0.03 and dr_r < math.radians(0.3)
    assert dt_p > 3 * dt_r


def test_background_pixels_are_not_used():
    s, Wq, Wr = tiny_views()
    depth, alpha, pairs = make_pairs(s, Wq, Wr)
    bg = np.array([[0.5, 0.5, 10.0, 10.0]], np.float32)
    zero = np.zeros_like(alpha)
    res = oracle.refine_pnp(Wr, s.camera, depth, zero, np.concatenate([pairs, bg]))
    assert res["n_used"] == 0 and res["iters"] == 0
