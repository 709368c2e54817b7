"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas: each compares it with
a closed form, an invariant, a library routine or brute force, chosen so that a
dropped term, a wrong sign or index, or a transposed operand fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def gauss(means, scales, quats, opac, cols, sh_degree=0):
    means = np.atleast_2d(np.asarray(means, np.float32))
    n = means.shape[0]
    sh = np.asarray(cols, np.float32).reshape(n, -1, 3)
    return sg.Gaussians(means, np.atleast_2d(np.asarray(scales, np.float32)),
                        np.atleast_2d(np.asarray(quats, np.float32)),
                        np.asarray(opac, np.float32).reshape(n), sh, sh_degree)


def cam(w=64, h=48, fx=50.0, fy=50.0, cx=None, cy=None):
    return sg.Camera(w, h, fx, fy, w / 2 if cx is None else cx, h / 2 if cy is None else cy)


IDENT = np.eye(4)


# ---------------------------------------------------------------- rotations --

def test_quat_to_rot_orthonormal_and_sign_invariant():
    rng = sg.Rng(7)
    for _ in range(50):
        q = rng.normal(4)
        R = oracle.quat_to_rot(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.allclose(oracle.quat_to_rot(-q), R, atol=1e-15)
        assert np.allclose(oracle.quat_to_rot(3.7 * q), R, atol=1e-14)


def test_quat_to_rot_known_rotations():
    c = math.cos(math.pi / 4)
    # 90 degrees about z maps x -> y
    assert np.allclose(oracle.quat_to_rot([c, 0, 0, c]), [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    # 90 degrees about x maps y -> z
    assert np.allclose(oracle.quat_to_rot([c, c, 0, 0]), [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-15)
    # axis-angle (Rodrigues) for a generic axis
    axis = np.array([1.0, -2.0, 0.5]); axis /= np.linalg.norm(axis)
    ang = 0.83
    q = np.r_[math.cos(ang / 2), math.sin(ang / 2) * axis]
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rr = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    assert np.allclose(oracle.quat_to_rot(q), Rr, atol=1e-14)


# ------------------------------------------------------- spherical harmonics --

def test_sh_closed_forms_low_order():
    d = np.array([0.3, -0.5, 0.81]); d /= np.linalg.norm(d)
    x, y, z = d
    Y = oracle.sh_basis(3, d)
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert abs(Y[0] - c0) < 1e-15
    # Condon-Shortley phase: Y_1,-1 = -c1 y, Y_1,0 = c1 z, Y_1,1 = -c1 x
    assert np.allclose(Y[1:4], [-c1 * y, c1 * z, -c1 * x], atol=1e-15)
    assert abs(Y[6] - math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1)) < 1e-14
    assert abs(Y[4] - 0.5 * math.sqrt(15 / math.pi) * x * y) < 1e-14


def test_sh_addition_theorem():
    # sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every unit d
    rng = sg.Rng(9)
    for _ in range(20):
        d = rng.normal(3); d /= np.linalg.norm(d)
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            s = np.sum(Y[l * l:(l + 1) ** 2] ** 2)
            assert abs(s - (2 * l + 1) / (4 * math.pi)) < 1e-13


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform in phi integrates products of
    # degree <= 6 polynomials on the sphere exactly.
    t, w = np.polynomial.legendre.leggauss(8)
    nphi = 16
    G = np.zeros((16, 16))
    for ti, wi in zip(t, w):
        st = math.sqrt(1 - ti * ti)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ti])
            G += np.outer(Y, Y) * wi * (2 * math.pi / nphi)
    assert np.allclose(G, np.eye(16), atol=1e-13)


# ---------------------------------------------------------------- projection --

def test_projection_isotropic_on_axis_closed_form():
    c = cam(64, 48, 50.0, 50.0)
    for z, s in [(4.0, 0.1), (10.0, 0.3), (2.5, 0.02)]:
        g = gauss([0, 0, z], [s, s, s], [1, 0, 0, 0], 0.5, [0.2, 0.3, 0.4])
        r = oracle.project(g, IDENT, c)[0]
        F = oracle.F
        sp = (50.0 * float(np.float32(s)) / z) ** 2
        assert r[F["visible"]] == 1
        assert abs(r[F["u"]] - 32) < 1e-12 and abs(r[F["v"]] - 24) < 1e-12
        assert abs(r[F["cov_a"]] - (sp + 0.3)) < 1e-9 * sp and abs(r[F["cov_b"]]) < 1e-12
        assert abs(r[F["con_a"]] - 1 / (sp + 0.3)) < 1e-12 and abs(r[F["con_c"]] - 1 / (sp + 0.3)) < 1e-12
        assert abs(r[F["rx"]] - 3 * math.sqrt(sp + 0.3)) < 1e-9
        assert abs(r[F["depth"]] - z) < 1e-12


def test_projection_pinhole_off_axis():
    c = cam(200, 100, 80.0, 60.0, 90.0, 45.0)
    pts = np.array([[1.0, 0.5, 5.0], [-2.0, 1.5, 7.0], [0.3, -0.4, 2.0]], np.float32)
    g = gauss(pts, [[0.1] * 3] * 3, [[1, 0, 0, 0]] * 3, [0.5] * 3, [[0.1, 0.1, 0.1]] * 3)
    recs = oracle.project(g, IDENT, c)
    F = oracle.F
    for p, r in zip(pts.astype(np.float64), recs):
        assert abs(r[F["u"]] - (80 * p[0] / p[2] + 90)) < 1e-12
        assert abs(r[F["v"]] - (60 * p[1] / p[2] + 45)) < 1e-12


def test_projection_anisotropic_rotated_on_axis():
    # on the optical axis J = diag(f/z) on x, y (third column zero), so
    # Sigma' = (f/z)^2 R2 diag(sx^2, sy^2) R2^T + eps I, exactly
    th = 0.6
    sx, sy, sz = 0.4, 0.1, 0.25
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    z, f = 6.0, 70.0
    g = gauss([0, 0, z], [sx, sy, sz], q, 0.8, [0.5, 0.5, 0.5])
    c = cam(128, 96, f, f)
    r = oracle.project(g, IDENT, c)[0]
    F = oracle.F
    sxf, syf = float(np.float32(sx)), float(np.float32(sy))
    thf = 2 * math.atan2(float(np.float32(math.sin(th / 2))), float(np.float32(math.cos(th / 2))))
    R2 = np.array([[math.cos(thf), -math.sin(thf)], [math.sin(thf), math.cos(thf)]])
    S = (f / z) ** 2 * R2 @ np.diag([sxf ** 2, syf ** 2]) @ R2.T + 0.3 * np.eye(2)
    assert np.allclose([r[F["cov_a"]], r[F["cov_b"]], r[F["cov_c"]]], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-6)
    Ci = np.linalg.inv(S)
    assert np.allclose([r[F["con_a"]], r[F["con_b"]], r[F["con_c"]]], [Ci[0, 0], Ci[0, 1], Ci[1, 1]], rtol=1e-6)


def _project_points(P, W, c):
    t = P @ W[:3, :3].T + W[:3, 3]
    return np.stack([c.fx * t[:, 0] / t[:, 2] + c.cx, c.fy * t[:, 1] / t[:, 2] + c.cy], 1)


def test_ewa_matches_monte_carlo_covariance():
    # Sigma' (eps = 0) is the first-order (Jacobian) covariance of projected
    # samples (Eq. foot_conv); the gap is O((s/z)^2) plus Monte-Carlo noise.
    c = cam(400, 300, 120.0, 90.0, 210.0, 140.0)
    W = sg.pose_from_xyz_yaw(0.5, -3.0, 1.2, 1.1)
    # add a pitch so the camera rotation has no zero entries
    a = 0.2
    Rp = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    W[:3, :3] = Rp @ W[:3, :3]
    W[:3, 3] = -W[:3, :3] @ np.array([0.5, -3.0, 1.2])
    fwd = W[2, :3]
    right = W[0, :3]
    down = W[1, :3]
    mu = np.array([0.5, -3.0, 1.2]) + 8.0 * fwd + 2.5 * right - 1.5 * down
    q = np.array([0.8, 0.3, -0.4, 0.33]); q /= np.linalg.norm(q)
    s = np.array([0.06, 0.03, 0.045])
    g = gauss(mu, s, q, 0.5, [0.2, 0.2, 0.2])
    r = oracle.project(g, W, c, oracle.params(eps2d=0.0))[0]
    F = oracle.F
    R = oracle.quat_to_rot(g.quat[0].astype(np.float64))
    M = R * g.scale[0].astype(np.float64)
    rng = sg.Rng(21)
    n = 400_000
    P = g.mean[0].astype(np.float64) + rng.normal(3 * n).reshape(n, 3) @ M.T
    uv = _project_points(P, W, c)
    cov = np.cov(uv.T)
    ref = np.array([[r[F["cov_a"]], r[F["cov_b"]]], [r[F["cov_b"]], r[F["cov_c"]]]])
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(cov - ref) / scale < 1.5e-2), (cov, ref)
    # the mean projects by the pinhole formula
    assert np.allclose([r[F["u"]], r[F["v"]]], _project_points(g.mean.astype(np.float64), W, c)[0], atol=1e-10)


def test_fov_clamp_applies_to_jacobian_only():
    c = cam(64, 48, 50.0, 50.0)
    limx = 1.3 * 32 / 50.0
    x, z = 5.0, 4.0                          # x/z = 1.25 > limx = 0.832
    s = 0.2
    g = gauss([x, 0, z], [s, s, s], [1, 0, 0, 0], 0.5, [0.1, 0.1, 0.1])
    r = oracle.project(g, IDENT, c, oracle.params(eps2d=0.0))[0]
    F = oracle.F
    J = np.array([[50 / z, 0, -50 * limx / z], [0, 50 / z, 0]])
    S = J @ (np.float32(s) ** 2 * np.eye(3)) @ J.T
    assert np.allclose([r[F["cov_a"]], r[F["cov_b"]], r[F["cov_c"]]], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-6)
    assert abs(r[F["u"]] - (50 * x / z + 32)) < 1e-9    # the mean is not clamped


def test_near_plane_and_offscreen_cull():
    c = cam()
    g = gauss([[0, 0, 0.19], [0, 0, 0.21], [0, 0, -3], [100, 0, 2]], [[0.01] * 3] * 4,
              [[1, 0, 0, 0]] * 4, [0.5] * 4, [[0.1] * 3] * 4)
    vis = oracle.project(g, IDENT, c)[:, oracle.F["visible"]]
    assert list(vis) == [0, 1, 0, 0]


# ------------------------------------------------------------ compositing --

def _single(z=5.0, s=0.1, o=0.7, col=(0.9, 0.4, 0.1)):
    return gauss([0, 0, z], [s, s, s], [1, 0, 0, 0], o, col)


def test_single_gaussian_footprint_closed_form():
    # alpha(x) = o exp(-r^2 / (2 sigma^2)) inside r <= 3 sigma, 0 outside
    c = cam(64, 48, 50.0, 50.0)
    z, s, o = 5.0, 0.1, 0.7
    out = oracle.render(_single(z, s, o), IDENT, c)
    sig2 = (50.0 * float(np.float32(s)) / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:48, 0:64]
    r2 = (xs + 0.5 - 32) ** 2 + (ys + 0.5 - 24) ** 2
    of = float(np.float32(o))
    a = of * np.exp(-0.5 * r2 / sig2)
    a[r2 > 9 * sig2] = 0
    a[a < 1 / 255] = 0
    assert np.allclose(out["alpha"], a, atol=1e-12)
    col = np.float32([0.9, 0.4, 0.1]).astype(np.float64)
    assert np.allclose(out["rgb"], col[:, None, None] * a, atol=1e-12)
    assert np.allclose(out["depth"], z * a, atol=1e-11)
    assert out["n_eval"] == int(np.sum(r2 <= 9 * sig2))


def test_footprint_boundary_at_three_sigma():
    # a wide, fully opaque-ish Gaussian: pixels just inside 3 sigma contribute,
    # just outside do not, even though o exp(-4.5) is far above 1/255
    c = cam(200, 200, 100.0, 100.0)
    z, s = 2.0, 0.12
    out = oracle.render(_single(z, s, 0.95), IDENT, c, oracle.params(eps2d=0.0))
    sig = 100.0 * float(np.float32(s)) / z
    ys, xs = np.mgrid[0:200, 0:200]
    r = np.hypot(xs + 0.5 - 100, ys + 0.5 - 100)
    assert np.all(out["alpha"][r < 3 * sig - 1e-6] > 0.95 * math.exp(-4.5) * 0.999)
    assert np.all(out["alpha"][r > 3 * sig + 1e-6] == 0)


def test_two_layer_compositing_hand_computed():
    # front-to-back: C = c1 a1 + c2 a2 (1 - a1); D likewise with depths.
    # The far Gaussian has the LOWER index: the depth sort must reorder them.
    c = cam(32, 32, 40.0, 40.0)
    g = gauss([[0, 0, 9.0], [0, 0, 4.0]], [[0.5] * 3, [0.5] * 3], [[1, 0, 0, 0]] * 2, [0.6, 0.5],
              [[0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])
    out = oracle.render(g, IDENT, c)
    # at the pixel nearest the centre the powers are tiny; evaluate exactly
    px, py = 16.5, 16.5
    rec = oracle.project(g, IDENT, c)
    F = oracle.F
    al = []
    for r in rec:
        dx, dy = px - r[F["u"]], py - r[F["v"]]
        pw = -0.5 * (r[F["con_a"]] * dx * dx + r[F["con_c"]] * dy * dy) - r[F["con_b"]] * dx * dy
        al.append(min(0.99, r[F["opacity"]] * math.exp(pw)))
    a_far, a_near = al
    Cexp = np.array([1.0, 0.0, 0.0]) * a_near + np.array([0.0, 1.0, 0.0]) * a_far * (1 - a_near)
    assert np.allclose(out["rgb"][:, 16, 16], Cexp, atol=1e-14)
    assert abs(out["depth"][16, 16] - (4.0 * a_near + 9.0 * a_far * (1 - a_near))) < 1e-13
    assert abs(out["alpha"][16, 16] - (1 - (1 - a_near) * (1 - a_far))) < 1e-14


def test_transmittance_stop_four_layers():
    # four stacked layers of alpha 0.95 at the pixel: T = 0.05, 0.0025,
    # 1.25e-4; the fourth would give 6.25e-6 < 1e-4, so it is not added.
    c = cam(16, 16, 20.0, 20.0, 8.5, 8.5)      # pixel (8, 8) centre on the axis
    zs = [2.0, 3.0, 4.0, 5.0]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]
    # the pixel centre sits on every Gaussian's projected mean (power = 0)
    g = gauss([[0, 0, z] for z in zs], [[2.0] * 3] * 4, [[1, 0, 0, 0]] * 4, [0.95] * 4, cols)
    out = oracle.render(g, IDENT, c)
    rec = oracle.project(g, IDENT, c)
    F = oracle.F
    px = py = 8.5
    T = 1.0
    Cexp = np.zeros(3)
    added = 0
    for r, col in zip(rec, cols):
        dx, dy = px - r[F["u"]], py - r[F["v"]]
        pw = -0.5 * (r[F["con_a"]] * dx * dx + r[F["con_c"]] * dy * dy) - r[F["con_b"]] * dx * dy
        a = min(0.99, r[F["opacity"]] * math.exp(pw))
        if T * (1 - a) < 1e-4:
            break
        Cexp += np.array(col) * a * T
        T *= 1 - a
        added += 1
    assert added == 3
    assert abs(T - 0.05 ** 3) < 1e-9
    assert np.allclose(out["rgb"][:, 8, 8], Cexp, atol=1e-14)
    assert abs(out["alpha"][8, 8] - (1 - T)) < 1e-14


def test_alpha_clamp_and_skip():
    c = cam(16, 16, 20.0, 20.0)
    out = oracle.render(_single(3.0, 1.0, 1.0, (1, 1, 1)), IDENT, c)
    assert abs(out["alpha"][8, 8] - 0.99) < 1e-15         # clamp
    out = oracle.render(_single(3.0, 1.0, 0.0035, (1, 1, 1)), IDENT, c)
    assert np.all(out["alpha"] == 0)                       # 0.0035 < 1/255 everywhere


def test_equal_depth_ties_follow_index_order():
    c = cam(16, 16, 20.0, 20.0)
    g = gauss([[0, 0, 3.0], [0, 0, 3.0]], [[1.0] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.5, 0.5],
              [[1, 0, 0], [0, 1, 0]])
    out = oracle.render(g, IDENT, c)
    assert out["rgb"][0, 8, 8] > out["rgb"][1, 8, 8]       # index 0 (red) in front
    g2 = g.subset(np.array([1, 0]))
    out2 = oracle.render(g2, IDENT, c)
    assert out2["rgb"][1, 8, 8] > out2["rgb"][0, 8, 8]


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_splat_equals_brute_force_bitwise(seed):
    r = sg.Rng(seed)
    n = 200
    mean = np.stack([r.uniform(n, -3, 3), r.uniform(n, -2, 2), r.uniform(n, 1.0, 9.0)], 1)
    g = sg.Gaussians(mean.astype(np.float32), np.exp(r.uniform(3 * n, -3.5, -1)).reshape(n, 3).astype(np.float32),
                     r.normal(4 * n).reshape(n, 4).astype(np.float32),
                     r.uniform(n, 0.05, 1.0).astype(np.float32), r.uniform(3 * n).reshape(n, 1, 3).astype(np.float32), 0)
    c = cam(32, 24, 20.0, 20.0)
    a = oracle.render(g, IDENT, c)
    b = oracle.render(g, IDENT, c, brute=True)
    for k in ("rgb", "depth", "alpha"):
        assert np.array_equal(a[k], b[k])
    assert a["n_eval"] == b["n_eval"]


# --------------------------------------------------------------------- NCC --

def test_ncc_invariants():
    rng = sg.Rng(5)
    a = rng.uniform(3000)
    b = 0.3 * a + rng.normal(3000, 0, 0.2)
    v, dg = oracle.ncc(a, a)
    assert abs(v - 1) < 1e-15 and not dg
    assert abs(oracle.ncc(a, 2.5 * a + 0.7)[0] - 1) < 1e-14
    assert abs(oracle.ncc(a, -0.4 * a + 3)[0] + 1) < 1e-14
    assert oracle.ncc(a, b)[0] == oracle.ncc(b, a)[0]
    # Pearson correlation from numpy's textbook routine
    assert abs(oracle.ncc(a, b)[0] - np.corrcoef(a, b)[0, 1]) < 1e-13
    for s in range(10):
        x, y = sg.Rng(100 + s).uniform(500), sg.Rng(200 + s).uniform(500)
        assert -1 <= oracle.ncc(x, y)[0] <= 1


def test_ncc_zero_variance_is_flagged():
    v, dg = oracle.ncc(np.full(100, 0.5), sg.Rng(3).uniform(100))
    assert v == 0 and dg


def test_argmax_lowest_index_on_ties():
    assert oracle.argmax([0.1, 0.5, 0.5, 0.2]) == 1
    s = sg.Rng(4).uniform(1000)
    assert oracle.argmax(s) == int(np.argmax(s))


def test_query_at_candidate_pose_selects_it():
    s = sg.tiny_scene()
    poses = s.candidate_poses
    for k in (0, 5, 11):
        q = oracle.render(s.gaussians, poses[k], s.camera)["rgb"]
        out = oracle.render_views(s.gaussians, poses, s.camera, query=q, images=False, flags=False)
        assert oracle.argmax(out["scores"]) == k
        assert abs(out["scores"][k] - 1) < 1e-12


def test_ncc_peaks_at_true_pose_and_falls_with_x_error():
    # the shape of the NCC-vs-error curves of Sec. IV-A: highest at the true
    # pose, lower as the x offset grows
    s = sg.tiny_scene()
    base = (0.0, -14.0, 2.0, math.pi / 2)
    q = oracle.render(s.gaussians, sg.pose_from_xyz_yaw(*base), s.camera)["rgb"] + s.query_noise
    offs = [0.0, 0.5, 1.5, 3.0]
    poses = np.stack([sg.pose_from_xyz_yaw(base[0] + o, base[1], base[2], base[3]) for o in offs])
    sc = oracle.render_views(s.gaussians, poses, s.camera, query=q, images=False, flags=False)["scores"]
    assert np.all(np.diff(sc) < 0), sc


# ---------------------------------------------------------- grid and blocks --

def test_grid_poses_match_independent_construction():
    seed = (3.0, -1.0, 1.6, 0.4)
    P = oracle.grid_poses(sg.pose_from_xyz_yaw(*seed), 4, 4, 4, 0.5, 2.0)
    Q = sg.street_grid_poses(seed)
    assert np.allclose(P, Q, atol=1e-12)
    for W in P:
        assert np.allclose(W[:3, :3] @ W[:3, :3].T, np.eye(3), atol=1e-14)
    # the paper's stress grid: 2 m x 10 deg over +-15 m and a full turn
    P2 = oracle.grid_poses(sg.pose_from_xyz_yaw(*seed), 15, 15, 36, 2.0, 10.0)
    assert P2.shape == (8100, 4, 4)
    centres = np.array([-W[:3, :3].T @ W[:3, 3] for W in P2])
    assert np.isclose(centres[:, 0].min(), seed[0] - 14) and np.isclose(centres[:, 0].max(), seed[0] + 14)


def test_block_select_matches_distance_scan():
    g = sg.street_gaussians(40_000, seed=5, sh_degree=0)
    B = 20.0
    for (cx, cy, R) in [(0.0, 0.0, 40.0), (-117.3, 2.0, 25.0), (240.0, -1.0, 60.0)]:
        idx, nb = oracle.block_select(g.mean, B, cx, cy, R)
        bx = np.floor(g.mean[:, 0].astype(np.float64) / B).astype(np.int64)
        by = np.floor(g.mean[:, 1].astype(np.float64) / B).astype(np.int64)
        keys = sorted(set(zip(bx.tolist(), by.tolist())))
        sel = [k for k in keys if math.hypot((k[0] + 0.5) * B - cx, (k[1] + 0.5) * B - cy) <= R]
        expect = []
        for k in sel:
            expect.extend(np.nonzero((bx == k[0]) & (by == k[1]))[0].tolist())
        assert nb == len(sel)
        assert idx.tolist() == expect


# ------------------------------------------------------- key replay and sort --

def test_stable_sort_matches_insertion_and_numpy():
    r = sg.Rng(8)
    n = 3000
    keys = (r.u64(n) % np.uint64(97)).astype(np.uint64) << np.uint64(20)
    vals = np.arange(n, dtype=np.uint32)
    k1, v1 = oracle.stable_sort(keys, vals)
    k2, v2 = oracle.stable_sort(keys, vals, insertion=True)
    o = np.argsort(keys, kind="stable")
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)
    assert np.array_equal(k1, keys[o]) and np.array_equal(v1, vals[o])


def test_tile_keys_and_ranges_match_plain_loops():
    r = sg.Rng(12)
    V, N, ntx, nty = 3, 40, 5, 4
    vis = (r.uniform(V * N) < 0.7).astype(np.uint8).reshape(V, N)
    dbits = np.frombuffer(r.uniform(V * N, 0.2, 50).astype(np.float32).tobytes(), np.uint32).reshape(V, N)
    rect = np.zeros((V, N, 4), np.int32)
    x0 = (r.uniform(V * N) * ntx).astype(int).reshape(V, N); y0 = (r.uniform(V * N) * nty).astype(int).reshape(V, N)
    rect[..., 0] = x0; rect[..., 1] = y0
    rect[..., 2] = np.minimum(ntx - 1, x0 + (r.uniform(V * N) * 3).astype(int).reshape(V, N))
    rect[..., 3] = np.minimum(nty - 1, y0 + (r.uniform(V * N) * 3).astype(int).reshape(V, N))
    keys, vals = oracle.tile_keys(vis, dbits, rect, ntx, nty)
    tb = oracle.tile_bits(ntx * nty)
    assert tb == 5
    exp = []
    for v in range(V):
        for i in range(N):
            if vis[v, i]:
                for ty in range(rect[v, i, 1], rect[v, i, 3] + 1):
                    for tx in range(rect[v, i, 0], rect[v, i, 2] + 1):
                        exp.append(((v << (32 + tb)) | ((ty * ntx + tx) << 32) | int(dbits[v, i]), i))
    assert keys.tolist() == [e[0] for e in exp] and vals.tolist() == [e[1] for e in exp]
    ks, vs = oracle.stable_sort(keys, vals)
    rg = oracle.tile_ranges(ks, V, ntx * nty)
    for v in range(V):
        for t in range(ntx * nty):
            members = [j for j, k in enumerate(ks.tolist()) if (k >> 32) == ((v << tb) | t)]
            if members:
                assert rg[v, t].tolist() == [members[0], members[-1] + 1]
            else:
                assert rg[v, t].tolist() == [0, 0]
    # within a (view, tile): depth ascending, ties by index
    for v in range(V):
        for t in range(ntx * nty):
            b, e = rg[v, t]
            seg = [(int(k) & 0xFFFFFFFF, int(i)) for k, i in zip(ks[b:e], vs[b:e])]
            assert seg == sorted(seg)


def test_counts_are_consistent():
    s = sg.tiny_scene()
    out = oracle.render_views(s.gaussians, s.candidate_poses[:2], s.camera, images=True, flags=False)
    rec = oracle.project(s.gaussians, s.candidate_poses[0], s.camera)
    F = oracle.F
    vis = rec[:, F["visible"]] == 1
    assert out["counts"][0, 0] == vis.sum()
    ninst = np.sum((rec[vis, F["tx1"]] - rec[vis, F["tx0"]] + 1) * (rec[vis, F["ty1"]] - rec[vis, F["ty0"]] + 1))
    assert out["counts"][0, 1] == ninst
    single = oracle.render(s.gaussians, s.candidate_poses[0], s.camera)
    assert out["counts"][0, 2] == single["n_eval"]
    assert np.array_equal(out["rgb"][0], single["rgb"])
