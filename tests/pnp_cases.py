"""Inputs for the PnP refinement tests, built by the oracle (never from the
CUDA path): the tiny scene rendered in FP64 at a render pose (depth and
alpha as float32), render pixels on a grid where alpha is high, and their
query pixels = the oracle's projection of the back-projected points into the
query pose, optionally with seeded noise and outliers."""
import math

import numpy as np

import oracle
import scenegen as sg


def tiny_views():
    """(scene, query pose W_q, render pose W_r): W_r is W_q moved 0.3 m and 2 deg."""
    s = sg.tiny_scene()
    Wq = s.hidden_pose
    Wr = oracle.pnp_apply(Wq, np.array([0.2, -0.15, 0.1, 0.0, 0.0, math.radians(2.0)]))
    return s, Wq, Wr


def make_pairs(s, Wq, Wr, step=6, noise_px=0.0, outlier_frac=0.0, seed=1, alpha_cut=0.9):
    """depth, alpha [H, W] float32 of the render at Wr; pairs [n, 4] float32."""
    cam = s.camera
    out = oracle.render(s.gaussians, Wr, cam)
    depth, alpha = out["depth"].astype(np.float32), out["alpha"].astype(np.float32)
    ys, xs = np.mgrid[step // 2:cam.height - 1:step, step // 2:cam.width - 1:step]
    uv = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], 1)
    keep = alpha[ys.ravel(), xs.ravel()] >= alpha_cut
    uv = uv[keep]
    X, used = oracle.pnp_backproject(Wr, cam, depth, alpha, uv)
    uv, X = uv[used], X[used]
    q = np.array([oracle.pnp_residual(Wq, x, cam, np.zeros(2))[0] for x in X])
    r = sg.Rng(seed)
    q = q + noise_px * r.normal(q.size).reshape(q.shape)
    n_out = int(outlier_frac * len(q))
    if n_out:
        idx = (r.u64(n_out) % np.uint64(len(q))).astype(np.int64)
        q[idx, 0] = r.uniform(n_out, 0, cam.width)
        q[idx, 1] = r.uniform(n_out, 0, cam.height)
    pairs = np.concatenate([uv, q], 1).astype(np.float32)
    return depth, alpha, pairs


def pose_error(A, B):
    """(translation of camera centres in m, rotation angle in rad) between poses."""
    ca = -A[:3, :3].T @ A[:3, 3]
    cb = -B[:3, :3].T @ B[:3, 3]
    Rd = A[:3, :3] @ B[:3, :3].T
    # angle of Rd: atan2(|axis part|, cos part), accurate for small angles too
    s = 0.5 * np.linalg.norm([Rd[2, 1] - Rd[1, 2], Rd[0, 2] - Rd[2, 0], Rd[1, 0] - Rd[0, 1]])
    ang = math.atan2(s, (np.trace(Rd) - 1.0) / 2.0)
    return float(np.linalg.norm(ca - cb)), ang
