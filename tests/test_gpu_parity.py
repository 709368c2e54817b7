"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
synthetic scenes.  Each test states its bar; the helpers in parity.py hold the
tolerances and the bit-exact tile-list replay."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import TOL_NCC, compare_images, compare_rgb, replay_tile_lists, z_ref

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


def make_ctx(R, g, precision=0, **cfg):
    ctx = R.Context(R.reloc_default_config(**cfg))
    ctx.load_map(g, precision)
    return ctx


def full_range(ctx):
    return [(0, ctx.n)]


def gpu_render(ctx, ranges, poses, cam):
    V = len(poses)
    dev = torch.device("cuda:0")
    rgb = torch.empty((V, 3, cam.height, cam.width), device=dev)
    depth = torch.empty((V, cam.height, cam.width), device=dev)
    alpha = torch.empty((V, cam.height, cam.width), device=dev)
    ctx.render(ranges, poses, cam, rgb, depth, alpha)
    torch.cuda.synchronize()
    return rgb.cpu().numpy().astype(np.float64), depth.cpu().numpy().astype(np.float64), \
        alpha.cpu().numpy().astype(np.float64)


def gpu_render_rgb(ctx, ranges, poses, cam):
    """Colour only (no depth or alpha): the blend variant of the scoring
    launches, which carries no depth and weight sums."""
    rgb = torch.empty((len(poses), 3, cam.height, cam.width), device=torch.device("cuda:0"))
    ctx.render(ranges, poses, cam, rgb)
    torch.cuda.synchronize()
    return rgb.cpu().numpy().astype(np.float64)


def ordered(ctx, g):
    """The map in the library's block order (the subset order the GPU uses)."""
    return g.subset(ctx.map_order())


# exported records carry the footprint's axes scaled by sqrt(log2(e) / 2)
KAPPA2 = math.log2(math.e) / 2


def record_axes(rec):
    """Unscaled principal axes (alpha_x, alpha_y, beta_x, beta_y) of exported records, FP64."""
    return [rec[..., k].astype(np.float64) / math.sqrt(KAPPA2) for k in (4, 5, 6, 7)]


def conic_from_axes(rec):
    """Conic (a, b, c) = alpha alpha^T + beta beta^T of exported records, FP64."""
    ax, ay, bx, by = record_axes(rec)
    return np.stack([ax * ax + bx * bx, ax * ay + bx * by, ay * ay + by * by], -1)


def quad_form_error(rec, ref):
    """Largest error of the GPU's d^T Sigma'^-1 d = (alpha.d)^2 + (beta.d)^2
    against the oracle's FP64 conic at the four ends of the 3-sigma ellipse's
    principal axes (where the oracle's form equals 9): this is where a conic
    that lost the long axis's curvature is wrong by the most."""
    F = oracle.F
    a, b, c = (ref[:, F[k]] for k in ("con_a", "con_b", "con_c"))
    sxx, sxy, syy = (ref[:, F[k]] for k in ("cov_a", "cov_b", "cov_c"))
    ax, ay, bx, by = record_axes(rec)
    worst = 0.0
    for i in range(len(a)):
        lam, vec = np.linalg.eigh(np.array([[sxx[i], sxy[i]], [sxy[i], syy[i]]]))
        for j in range(2):
            for sgn in (1.0, -1.0):
                d = sgn * 3.0 * np.sqrt(lam[j]) * vec[:, j]
                q_ref = a[i] * d[0] ** 2 + 2 * b[i] * d[0] * d[1] + c[i] * d[1] ** 2
                q_gpu = (ax[i] * d[0] + ay[i] * d[1]) ** 2 + (bx[i] * d[0] + by[i] * d[1]) ** 2
                worst = max(worst, abs(q_gpu - q_ref) / 9.0)
    return worst


def export(ctx, V, S, cam, tile=(16, 16)):
    dev = torch.device("cuda:0")
    c = ctx.last_counts()
    rec = torch.empty((V, S, 12), device=dev)
    rect = torch.empty((V, S, 4), dtype=torch.int32, device=dev)
    it = torch.empty((V, c.inst_stride), dtype=torch.int32, device=dev)
    ig = torch.empty((V, c.inst_stride), dtype=torch.int32, device=dev)
    ntx = (cam.width + tile[0] - 1) // tile[0]
    nty = (cam.height + tile[1] - 1) // tile[1]
    rg = torch.empty((V, ntx * nty, 2), dtype=torch.int32, device=dev)
    cnt = ctx.export_debug(rec, rect, it, ig, rg, n_views=V)
    return (rec.cpu().numpy(), rect.cpu().numpy(), it.cpu().numpy().view(np.uint32),
            ig.cpu().numpy().view(np.uint32), cnt, rg.cpu().numpy())


@pytest.fixture(scope="module")
def tiny():
    return sg.tiny_scene()


# ------------------------------------------------------------------ tiny ----

def test_render_tiny_matches_oracle(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    g = ordered(ctx, tiny.gaussians)
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), tiny.candidate_poses, tiny.camera)
    ref = oracle.render_views(g, tiny.candidate_poses, tiny.camera)
    st = compare_images(rgb, depth, alpha, ref, z_ref(g, tiny.candidate_poses, tiny.camera))
    print("tiny render", st)
    assert st["flagged"] < 0.02
    c = ctx.last_counts()
    assert c.n_visible == ref["counts"][:, 0].sum()


def test_tile_lists_bit_exact_tiny(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    V, S = len(tiny.candidate_poses), tiny.gaussians.n
    gpu_render(ctx, full_range(ctx), tiny.candidate_poses, tiny.camera)
    rec, rect, it, ig, cnt, rg = export(ctx, V, S, tiny.camera)
    n = replay_tile_lists(rec, rect, it, ig, cnt, rg, tiny.camera.width, tiny.camera.height, 16, 16)
    assert n == ctx.last_counts().n_instances


def test_projection_records_match_oracle(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    g = ordered(ctx, tiny.gaussians)
    V, S = 4, g.n
    poses = tiny.candidate_poses[:V]
    gpu_render(ctx, full_range(ctx), poses, tiny.camera)
    rec, rect, *_ = export(ctx, V, S, tiny.camera)
    F = oracle.F
    n_boundary = 0
    for v in range(V):
        ref = oracle.project(g, poses[v], tiny.camera)
        gv = rect[v, :, 0] >= 0
        ov = ref[:, F["visible"]] == 1
        n_boundary += int((gv != ov).sum())
        both = gv & ov
        np.testing.assert_allclose(rec[v, both, 0], ref[both, F["u"]], atol=2e-4)
        np.testing.assert_allclose(rec[v, both, 1], ref[both, F["v"]], atol=2e-4)
        np.testing.assert_allclose(rec[v, both, 2], ref[both, F["depth"]], rtol=1e-6)
        # log2 of the opacity (MUFU lg2: a few ulp)
        np.testing.assert_allclose(np.exp2(rec[v, both, 3].astype(np.float64)), ref[both, F["opacity"]], rtol=2e-6)
        con = conic_from_axes(rec[v, both])
        scale = np.sqrt(np.abs(ref[both, F["con_a"]] * ref[both, F["con_c"]]))
        for k, name in enumerate(("con_a", "con_b", "con_c")):
            assert np.max(np.abs(con[:, k] - ref[both, F[name]]) / scale) < 1e-4
        assert quad_form_error(rec[v, both], ref[both]) < 1e-4
        np.testing.assert_allclose(rec[v, both, 8:11], ref[both][:, [F["r"], F["g"], F["b"]]], atol=1e-6)
        # tile rectangles: identical unless an edge is within 1e-3 px of a tile line
        rr = ref[both][:, [F["tx0"], F["ty0"], F["tx1"], F["ty1"]]].astype(np.int32)
        diff = np.any(rect[v, both] != rr, axis=1)
        if diff.any():
            u, vv = ref[both, F["u"]][diff], ref[both, F["v"]][diff]
            rx, ry = ref[both, F["rx"]][diff], ref[both, F["ry"]][diff]
            edges = np.stack([u - rx, u + rx, vv - ry, vv + ry], 1) / 16.0
            assert np.all(np.min(np.abs(edges - np.round(edges)), axis=1) * 16 < 1e-3)
    assert n_boundary <= 2


def test_scores_and_argmax_tiny(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    g = ordered(ctx, tiny.gaussians)
    q = oracle.render(g, tiny.hidden_pose, tiny.camera)["rgb"] + tiny.query_noise
    qd = torch.tensor(q, dtype=torch.float32, device="cuda:0").contiguous()
    sc, dg = ctx.score(full_range(ctx), tiny.candidate_poses, tiny.camera, qd)
    ref = oracle.render_views(g, tiny.candidate_poses, tiny.camera, query=q.astype(np.float32),
                              images=False, flags=False)
    err = np.abs(sc - ref["scores"]).max()
    print("tiny ncc max err", err)
    assert err <= TOL_NCC
    assert not dg.any()
    top = np.sort(ref["scores"])[::-1]
    if top[0] - top[1] > TOL_NCC:
        assert int(np.argmax(sc)) == oracle.argmax(ref["scores"])


def test_localize_tiny_grid(R, tiny):
    ctx = make_ctx(R, tiny.gaussians, block_size=5.0)
    g = ordered(ctx, tiny.gaussians)
    q = (oracle.render(g, tiny.hidden_pose, tiny.camera)["rgb"] + tiny.query_noise).astype(np.float32)
    qd = torch.tensor(q, device="cuda:0").contiguous()
    cam = tiny.camera
    brgb = torch.empty((3, cam.height, cam.width), device="cuda:0")
    bdep = torch.empty((cam.height, cam.width), device="cuda:0")
    bal = torch.empty((cam.height, cam.width), device="cuda:0")
    radius = 12.0
    res, sc = ctx.localize(qd, tiny.seed_pose, radius, (3, 3, 3, 0.5, 3.0), cam, brgb, bdep, bal)
    # oracle: same blocks, same grid, full sweep
    seed_c = -tiny.seed_pose[:3, :3].T @ tiny.seed_pose[:3, 3]
    idx, nb = oracle.block_select(tiny.gaussians.mean, 5.0, seed_c[0], seed_c[1], radius)
    assert res.n_blocks == nb and res.n_gauss == len(idx)
    sub = tiny.gaussians.subset(idx)
    poses = oracle.grid_poses(tiny.seed_pose, 3, 3, 3, 0.5, 3.0)
    ref = oracle.render_views(sub, poses, cam, query=q)
    assert np.abs(sc - ref["scores"]).max() <= TOL_NCC
    best = oracle.argmax(ref["scores"])
    top = np.sort(ref["scores"])[::-1]
    if top[0] - top[1] > TOL_NCC:
        assert res.best_index == best
    k = res.best_index
    assert np.allclose(np.array(res.best_pose).reshape(4, 4), poses[k], atol=1e-12)
    one = {key: ref[key][k:k + 1] for key in ("rgb", "depth", "alpha", "flags", "bound")}
    compare_images(brgb.cpu().numpy()[None].astype(np.float64), bdep.cpu().numpy()[None].astype(np.float64),
                   bal.cpu().numpy()[None].astype(np.float64), one, z_ref(sub, poses, cam))


def test_block_select_matches_oracle(R):
    g = sg.street_gaussians(60_000, seed=4, sh_degree=0)
    ctx = make_ctx(R, g)
    order = ctx.map_order()
    for (x, y, r) in [(0.0, 0.0, 40.0), (-150.0, 3.0, 30.0), (249.0, -7.0, 55.0), (0.0, 0.0, 0.0)]:
        runs, ng, nb = ctx.select_block(x, y, r)
        got = np.concatenate([order[b:e] for b, e in runs]) if runs else np.zeros(0, np.int64)
        idx, nbo = oracle.block_select(g.mean, 20.0, x, y, r)
        assert nb == nbo and ng == len(idx)
        assert np.array_equal(got, idx)


# ------------------------------------------------------------ edge cases ----

@pytest.mark.parametrize("tile", [(8, 8), (32, 8), (16, 16), (8, 16), (16, 8), (32, 16)])
def test_ragged_image_and_tile_shapes(R, tiny, tile):
    cam = sg.Camera(101, 37, 40.0, 40.0, 50.5, 18.5)
    ctx = make_ctx(R, tiny.gaussians, tile_w=tile[0], tile_h=tile[1])
    g = ordered(ctx, tiny.gaussians)
    poses = tiny.candidate_poses[:3]
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), poses, cam)
    prm = oracle.params(tile_w=tile[0], tile_h=tile[1])
    ref = oracle.render_views(g, poses, cam, prm)
    compare_images(rgb, depth, alpha, ref, z_ref(g, poses, cam))
    # colour only (the scoring launches' variant), ragged in x and y here
    compare_rgb(gpu_render_rgb(ctx, full_range(ctx), poses, cam), ref)
    rec, rect, it, ig, cnt, rg = export(ctx, 3, g.n, cam, tile)
    replay_tile_lists(rec, rect, it, ig, cnt, rg, cam.width, cam.height, tile[0], tile[1])


@pytest.mark.parametrize("width,height", [(2048, 24), (2056, 24), (120, 272), (1408, 376)])
def test_wide_rows_tile_lists(R, tiny, width, height):
    """Rows of 256 tiles of 8 x 8 (the widest the XOR-mask emission takes),
    of 257 (the emission with slot counters per column), 34 tile rows (more
    than a 32-bit row mask holds), and 176 x 47 = 8272 tiles (over 8192: the
    binning chunks double to 4096 Gaussians and the emission stages each
    chunk in two halves): tile lists bit for bit against the oracle's
    replay, images against the oracle.  The long focal length gives spans of
    up to tens of tiles, so the emission's spreading of wide spans over the
    lanes is exercised too."""
    cam = sg.Camera(width, height, 300.0, 300.0, width / 2.0, height / 2.0)
    ctx = make_ctx(R, tiny.gaussians, tile_w=8, tile_h=8)
    g = ordered(ctx, tiny.gaussians)
    poses = tiny.candidate_poses[:2]
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), poses, cam)
    ref = oracle.render_views(g, poses, cam, oracle.params(tile_w=8, tile_h=8))
    compare_images(rgb, depth, alpha, ref, z_ref(g, poses, cam))
    rec, rect, it, ig, cnt, rg = export(ctx, 2, g.n, cam, (8, 8))
    widths = (rect[..., 2] - rect[..., 0] + 1)[rect[..., 0] >= 0]
    assert widths.max() > 8
    n = replay_tile_lists(rec, rect, it, ig, cnt, rg, cam.width, cam.height, 8, 8)
    assert n == ctx.last_counts().n_instances


def test_no_dilation_uses_fp64_inverse(R, tiny):
    # eps2d = 0: tiny footprints have det(Sigma') < 1e-6 and take the FP64 path
    ctx = make_ctx(R, tiny.gaussians, eps2d=0.0)
    g = ordered(ctx, tiny.gaussians)
    poses = tiny.candidate_poses[:2]
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), poses, tiny.camera)
    ref = oracle.render_views(g, poses, tiny.camera, oracle.params(eps2d=0.0))
    compare_images(rgb, depth, alpha, ref, z_ref(g, poses, tiny.camera))


def test_empty_subset_and_nothing_visible(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    rgb, depth, alpha = gpu_render(ctx, [], tiny.candidate_poses[:2], tiny.camera)
    assert not rgb.any() and not depth.any() and not alpha.any()
    q = torch.rand((3, tiny.camera.height, tiny.camera.width), device="cuda:0")
    sc, dg = ctx.score([], tiny.candidate_poses[:2], tiny.camera, q)
    assert np.all(sc == 0) and np.all(dg == 1)
    # camera looking away from every Gaussian
    away = sg.pose_from_xyz_yaw(0.0, -14.0, 2.0, -math.pi / 2)
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), away[None], tiny.camera)
    ref = oracle.render_views(ordered(ctx, tiny.gaussians), away[None], tiny.camera)
    assert ref["counts"][0, 0] == ctx.last_counts().n_visible
    compare_images(rgb, depth, alpha, ref, 30.0)


def test_single_view_single_gaussian(R):
    g = sg.Gaussians(np.array([[0.0, 0.0, 5.0]], np.float32), np.full((1, 3), 0.3, np.float32),
                     np.array([[1, 0, 0, 0]], np.float32), np.array([0.8], np.float32),
                     np.array([[[0.2, 0.5, 0.9]]], np.float32), 0)
    cam = sg.Camera(64, 48, 50.0, 50.0, 32.0, 24.0)
    ctx = make_ctx(R, g)
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), np.eye(4)[None], cam)
    ref = oracle.render_views(g, np.eye(4)[None], cam)
    compare_images(rgb, depth, alpha, ref, 5.0)


def _rot(axis, ang):
    c, s_ = math.cos(ang), math.sin(ang)
    i, j = [(1, 2), (2, 0), (0, 1)][axis]
    m = np.eye(3)
    m[i, i] = m[j, j] = c
    m[i, j], m[j, i] = -s_, s_
    return m


def needle_scene():
    """1500 needle-like Gaussians (one long axis of 0.3-1.5 m, two of 4 mm) at
    random orientations, 3-12 m in front of a 200x120 camera (ragged 16-px
    tiles in x and y): footprints up to ~430 px long and ~1.2 px wide (the
    0.3 px^2 dilation) crossing the warp blocks at every angle, with
    Sigma''s eigenvalues up to ~2e4 apart."""
    r = sg.Rng(41)
    n = 1500
    mean = np.stack([r.uniform(n, -4.0, 4.0), r.uniform(n, -2.5, 2.5), r.uniform(n, 3.0, 12.0)], 1)
    scale = np.stack([np.exp(r.uniform(n, math.log(0.3), math.log(1.5))),
                      np.full(n, 0.004), np.full(n, 0.004)], 1)
    quat = r.normal(4 * n).reshape(n, 4)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-r.normal(n, 0.0, 1.5)))
    rgb = r.uniform(3 * n).reshape(n, 1, 3)
    g = sg.Gaussians(mean.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
                     opacity.astype(np.float32), rgb.astype(np.float32), 0)
    cam = sg.Camera(200, 120, 150.0, 150.0, 100.0, 60.0)
    poses = []
    for ax, ay, tx in ((0.0, 0.0, 0.0), (0.1, -0.15, 0.3), (-0.08, 0.2, -0.4), (0.05, 0.05, 0.1)):
        W = np.eye(4)
        W[:3, :3] = _rot(0, ax) @ _rot(1, ay)
        W[:3, 3] = (tx, 0.0, 0.0)
        poses.append(W)
    noise = sg.Rng(42).normal(3 * cam.height * cam.width, 0.0, 0.02).reshape(3, cam.height, cam.width)
    q = np.clip(noise + 0.5, 0.0, 1.0).astype(np.float32)
    return g, cam, np.stack(poses), q


def test_thin_footprints_match_oracle_across_block_shapes(R):
    """Needle-like footprints against the FP64 oracle, pixel by pixel, with
    16x16 tiles (two records per lane as well), 8x8, 32x8, 8x16 and 32x16 tiles
    (warp blocks of 16x4, 8x8, 16x4, 8x8 and 16x4 pixels; colour-only renders
    as well): RGB and alpha within 1e-4 and depth
    within 1e-4 z_ref on unflagged pixels, flagged pixels within the oracle's
    bound, NCC within 2e-6 of the oracle's.  The records' principal axes
    reproduce the oracle's quadratic form at the ends of both axes.  Besides,
    the blend keeps a record for a block only if the ellipse at the record's
    own threshold meets the box of the block's still-compositing pixels, so it
    may drop only records that no pixel of the block takes; the per-pixel
    arithmetic and the order of the records at a pixel do not depend on the
    tile shape, only the cull and the block centre the pixel offsets are taken
    from do, so the launches also agree with each other to rounding."""
    g, cam, poses, q_np = needle_scene()
    q = torch.tensor(q_np, device="cuda:0").contiguous()
    base = ref = None
    for tile, rpl in (((16, 16), 1), ((16, 16), 2), ((8, 8), 1), ((32, 8), 1), ((8, 16), 1), ((32, 16), 1)):
        ctx = make_ctx(R, g, tile_w=tile[0], tile_h=tile[1], blend_rpl=rpl)
        go = ordered(ctx, g)
        imgs = gpu_render(ctx, full_range(ctx), poses, cam)
        sc, dg = ctx.score(full_range(ctx), poses, cam, q)
        if ref is None:
            # the oracle's pixels do not depend on the tile shape
            ref = oracle.render_views(go, poses, cam, query=q_np.astype(np.float64))
            zr = z_ref(go, poses, cam)
        stats = compare_images(*imgs, ref, zr)
        rgb_only = gpu_render_rgb(ctx, full_range(ctx), poses, cam)
        compare_rgb(rgb_only, ref)
        assert np.abs(rgb_only - imgs[0]).max() <= 2e-5, (tile, rpl, float(np.abs(rgb_only - imgs[0]).max()))
        assert np.abs(sc - ref["scores"]).max() <= TOL_NCC, (tile, rpl, float(np.abs(sc - ref["scores"]).max()))
        if base is None:
            base = imgs, sc
            assert float(imgs[2].max()) > 0.9 and float((imgs[2] > 0).mean()) > 0.5
            rec, rect, *_ = export(ctx, len(poses), go.n, cam, tile)
            F = oracle.F
            for v in range(len(poses)):
                ref_rec = oracle.project(go, poses[v], cam)
                both = (rect[v, :, 0] >= 0) & (ref_rec[:, F["visible"]] == 1)
                assert quad_form_error(rec[v, both], ref_rec[both]) < 1e-4
            print("needle parity", stats)
            continue
        for i, (x, y) in enumerate(zip(imgs, base[0])):
            tol = 2e-5 * (zr if i == 1 else 1.0)            # rgb, depth (metres), alpha
            assert np.abs(x - y).max() <= tol, (tile, rpl, i, float(np.abs(x - y).max()))
        assert np.abs(sc - base[1]).max() <= TOL_NCC, (tile, rpl)


def test_overflow_grow_and_retry_is_exact(R, tiny):
    a = make_ctx(R, tiny.gaussians)
    b = make_ctx(R, tiny.gaussians, inst_capacity=64)
    ra = gpu_render(a, full_range(a), tiny.candidate_poses, tiny.camera)
    rb = gpu_render(b, full_range(b), tiny.candidate_poses, tiny.camera)
    assert b.last_counts().retries >= 1
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)


def far_scene():
    """300 Gaussians 2-12 m in front of a 64x48 camera and 60 at 15-60 km
    (scale z/40, about a pixel): depths over four and a half decades, so the
    visible depth keys differ in every byte of the float32 pattern."""
    r = sg.Rng(77)
    zn, zf = r.uniform(300, 2.0, 12.0), r.uniform(60, 15000.0, 60000.0)
    z = np.concatenate([zn, zf])
    n = len(z)
    mean = np.stack([r.uniform(n, -0.55, 0.55) * z, r.uniform(n, -0.4, 0.4) * z, z], 1)
    scale = np.concatenate([np.exp(r.uniform(3 * 300, math.log(0.05), math.log(0.4))).reshape(300, 3),
                            np.repeat((zf / 40.0)[:, None], 3, 1)])
    quat = r.normal(4 * n).reshape(n, 4)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    opacity = r.uniform(n, 0.3, 0.95)
    rgb = r.uniform(3 * n).reshape(n, 1, 3)
    g = sg.Gaussians(mean.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
                     opacity.astype(np.float32), rgb.astype(np.float32), 0)
    W = np.eye(4)
    W[:3, :3] = _rot(1, 0.05)
    W[:3, 3] = (0.3, 0.2, 0.0)
    return g, sg.Camera(64, 48, 50.0, 50.0, 32.0, 24.0), np.stack([np.eye(4), W])


def test_depths_over_four_decades(R):
    """Visible depths from 2 m to 60 km (the far Gaussians all on screen):
    images against the oracle and the tile lists bit for bit, so every byte
    of the depth sort's keys orders them."""
    g, cam, poses = far_scene()
    ctx = make_ctx(R, g)
    go = ordered(ctx, g)
    ref = oracle.render_views(go, poses, cam)
    assert ref["counts"][:, 0].min() == 360
    rgb, depth, alpha = gpu_render(ctx, full_range(ctx), poses, cam)
    compare_images(rgb, depth, alpha, ref, z_ref(go, poses, cam))
    rec, rect, it, ig, cnt, rg = export(ctx, len(poses), go.n, cam)
    replay_tile_lists(rec, rect, it, ig, cnt, rg, cam.width, cam.height, 16, 16)


def test_repeat_calls_are_deterministic(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    q = torch.rand((3, tiny.camera.height, tiny.camera.width), device="cuda:0", generator=None)
    s1, _ = ctx.score(full_range(ctx), tiny.candidate_poses, tiny.camera, q)
    s2, _ = ctx.score(full_range(ctx), tiny.candidate_poses, tiny.camera, q)
    assert np.array_equal(s1, s2)


def test_invalid_arguments_fail_cleanly(R, tiny):
    ctx = make_ctx(R, tiny.gaussians)
    with pytest.raises(R.RelocError) as e:
        ctx.render([(0, tiny.gaussians.n + 5)], tiny.candidate_poses[:1], tiny.camera)
    assert e.value.status == R.EINVAL
    bad = tiny.candidate_poses[:1].copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(R.RelocError) as e:
        ctx.render(full_range(ctx), bad, tiny.camera)
    assert e.value.status == R.ENUMERIC
    empty = R.Context()
    with pytest.raises(R.RelocError) as e:
        empty.render([], tiny.candidate_poses[:1], tiny.camera)
    assert e.value.status == R.ENOMAP
    # 4096 views of 16000 x 9000 pixels: more 64-pixel blend units than one
    # launch's work queue counts (2^29), refused before any allocation
    huge = sg.Camera(16000, 9000, 8000.0, 8000.0, 8000.0, 4500.0)
    with pytest.raises(R.RelocError) as e:
        ctx.render(full_range(ctx), np.repeat(tiny.candidate_poses[:1], 4096, axis=0), huge)
    assert e.value.status == R.EINVAL
    # the context still works after errors
    gpu_render(ctx, full_range(ctx), tiny.candidate_poses[:1], tiny.camera)


def test_bad_buffers_raise_before_any_launch(R, tiny):
    """Each wrong device buffer is rejected by the binding (ValueError) before
    the C call: a float32 score buffer where float64 is written, a query of
    another image size, an image tensor of the wrong dtype, too short outputs."""
    cam = tiny.camera
    H, W = cam.height, cam.width
    dev = torch.device("cuda:0")
    imgs = torch.rand((4, 3, H, W), device=dev)
    q = torch.rand((3, H, W), device=dev)
    sc = torch.empty(4, dtype=torch.float64, device=dev)
    dg = torch.empty(4, dtype=torch.int32, device=dev)
    bad = [dict(scores_out=torch.empty(4, dtype=torch.float32, device=dev)),
           dict(scores_out=torch.empty(3, dtype=torch.float64, device=dev)),
           dict(query=torch.rand((3, H, W + 1), device=dev)),
           dict(images=imgs.double()),
           dict(degenerate_out=torch.empty(4, dtype=torch.float32, device=dev)),
           dict(degenerate_out=torch.empty(2, dtype=torch.int32, device=dev))]
    for over in bad:
        args = dict(images=imgs, query=q, scores_out=sc, degenerate_out=dg)
        args.update(over)
        with pytest.raises(ValueError):
            R.reloc_ncc_images_noalloc(**args)
    ctx = make_ctx(R, tiny.gaussians)
    poses = tiny.candidate_poses[:2]
    with pytest.raises(ValueError):
        ctx.render(full_range(ctx), poses, cam, torch.empty((1, 3, H, W), device=dev))
    with pytest.raises(ValueError):
        ctx.render(full_range(ctx), poses, cam, None, torch.empty((2, H, W), dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        ctx.score(full_range(ctx), poses, cam, torch.rand((3, H - 1, W), device=dev))
    with pytest.raises(ValueError):
        ctx.localize(q, tiny.seed_pose, 12.0, (2, 2, 1, 0.5, 2.0), cam, best_rgb=torch.empty((3, H, W - 1), device=dev))
    # nothing was launched with a bad buffer: the good calls still agree
    R.reloc_ncc_images_noalloc(imgs, q, sc, dg)
    ref = np.array([oracle.ncc(imgs[v].cpu().numpy(), q.cpu().numpy())[0] for v in range(4)])
    assert np.abs(sc.cpu().numpy() - ref).max() <= TOL_NCC


# --------------------------------------------------------- street scenes ----

@pytest.fixture(scope="module")
def street_small():
    return sg.street_gaussians(150_000, seed=11, sh_degree=3)


def test_street_sh3_reduced_camera(R, street_small):
    # 704x188 (half resolution, ragged 16-px tiles in y), SH degree 3
    cam = sg.street_camera(704, 188, 276.0)
    hidden, seeds = sg.street_queries(2, seed=12)
    ctx = make_ctx(R, street_small)
    runs, ng, nb = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    order = ctx.map_order()
    sub = street_small.subset(np.concatenate([order[b:e] for b, e in runs]))
    poses = sg.street_grid_poses(seeds[0], 2, 2, 2, 0.5, 2.0)
    rgb, depth, alpha = gpu_render(ctx, runs, poses, cam)
    ref = oracle.render_views(sub, poses, cam)
    st = compare_images(rgb, depth, alpha, ref, z_ref(sub, poses, cam))
    print("street sh3 704x188", st)
    print("street sh3 704x188 colour only", compare_rgb(gpu_render_rgb(ctx, runs, poses, cam), ref))
    rec, rect, it, ig, cnt, rg = export(ctx, len(poses), ng, cam)
    replay_tile_lists(rec, rect, it, ig, cnt, rg, cam.width, cam.height, 16, 16)


def test_tile_lists_bit_exact_block_per_chunk(R):
    """8 views of the 2M-Gaussian street (~320k Gaussians selected) at
    704x188: over 1024 binning chunks, so the emission takes a block per
    chunk whose warps take the tile rows heaviest first; every view's tile
    lists bit for bit against the oracle's replay."""
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera(704, 188, 276.0)
    hidden, seeds = sg.street_queries(1, seed=12)
    ctx = make_ctx(R, g)
    runs, ng, nb = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    poses = sg.street_grid_poses(seeds[0], 2, 2, 2, 0.5, 2.0)
    assert len(poses) * math.ceil(ng / 2048) >= 1024
    gpu_render_rgb(ctx, runs, poses, cam)
    rec, rect, it, ig, cnt, rg = export(ctx, len(poses), ng, cam)
    n = replay_tile_lists(rec, rect, it, ig, cnt, rg, cam.width, cam.height, 16, 16)
    assert n == ctx.last_counts().n_instances


def test_blend_same_per_view_whatever_the_view_count(R, street_small):
    """The blend's work order (tiles whose lists hold 1024 records or more
    first in launches of four views or more, list order in launches of fewer)
    decides only which warp takes a unit: every view renders bit for bit the
    same alone, in threes and among eight.  32 x 16 tiles give this street
    lists longer than 1024 records."""
    cam = sg.street_camera(704, 188, 276.0)
    hidden, seeds = sg.street_queries(2, seed=12)
    ctx = make_ctx(R, street_small, tile_w=32, tile_h=16)
    runs, ng, nb = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    poses = sg.street_grid_poses(seeds[0], 2, 2, 2, 0.5, 2.0)
    rgb8, d8, a8 = gpu_render(ctx, runs, poses, cam)
    rg = export(ctx, len(poses), ng, cam, (32, 16))[5]
    assert (rg[..., 1] - rg[..., 0]).max() >= 1024
    for sel in ([0], [3], [1, 5, 6]):
        rgb, d, a = gpu_render(ctx, runs, poses[sel], cam)
        assert np.array_equal(rgb, rgb8[sel]) and np.array_equal(d, d8[sel]) and np.array_equal(a, a8[sel]), sel
    # colour only (the scoring launches' variant) too
    c8 = gpu_render_rgb(ctx, runs, poses, cam)
    for sel in ([2], [0, 4, 7]):
        assert np.array_equal(gpu_render_rgb(ctx, runs, poses[sel], cam), c8[sel]), sel


@pytest.mark.parametrize("precision", [1, 2])
def test_half_precision_storage(R, street_small, precision):
    """FP16/BF16 attribute storage (means FP32): parity with the oracle fed the
    same rounded attributes; the error against the unrounded map is reported."""
    cam = sg.street_camera(704, 188, 276.0)
    hidden, seeds = sg.street_queries(2, seed=12)
    ctx = make_ctx(R, street_small, precision)
    runs, ng, nb = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    order = ctx.map_order()
    sub = street_small.subset(np.concatenate([order[b:e] for b, e in runs]))
    dt = torch.float16 if precision == 1 else torch.bfloat16

    def rnd(a):
        return torch.tensor(a).to(dt).float().numpy()
    subr = sg.Gaussians(sub.mean, rnd(sub.scale), rnd(sub.quat), rnd(sub.opacity), rnd(sub.sh), sub.sh_degree)
    poses = sg.street_grid_poses(seeds[0], 2, 1, 1, 0.5, 2.0)
    rgb, depth, alpha = gpu_render(ctx, runs, poses, cam)
    ref = oracle.render_views(subr, poses, cam)
    st = compare_images(rgb, depth, alpha, ref, z_ref(subr, poses, cam))
    full = oracle.render_views(sub, poses, cam, flags=False)
    print("precision", precision, st, "vs unrounded map: rgb max",
          float(np.abs(rgb - full["rgb"]).max()), "mean", float(np.abs(rgb - full["rgb"]).mean()))


def test_street_full_size_sampled(R):
    """The driving configuration as the benchmark runs it: 2M Gaussians, 20 m
    blocks, 40 m radius, 1408x376, 64 candidates (4x4x4 grid, 0.5 m / 2 deg).
    Sampled views are rendered by the oracle pixel for pixel; every NCC score
    is checked against the oracle's full sweep."""
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    hidden, seeds = sg.street_queries(1, seed=12)
    ctx = make_ctx(R, g)
    order = ctx.map_order()
    seed_pose = sg.pose_from_xyz_yaw(*seeds[0])
    runs, ng, nb = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    sub = g.subset(np.concatenate([order[b:e] for b, e in runs]))
    q = (oracle.render(sub, sg.pose_from_xyz_yaw(*hidden[0]), cam)["rgb"]
         + sg.image_noise(13, cam.height, cam.width)).astype(np.float32)
    qd = torch.tensor(q, device="cuda:0")
    brgb = torch.empty((3, cam.height, cam.width), device="cuda:0")
    bdep = torch.empty((cam.height, cam.width), device="cuda:0")
    bal = torch.empty((cam.height, cam.width), device="cuda:0")
    res, sc = ctx.localize(qd, seed_pose, 40.0, (4, 4, 4, 0.5, 2.0), cam, brgb, bdep, bal)
    poses = oracle.grid_poses(seed_pose, 4, 4, 4, 0.5, 2.0)
    ref = oracle.render_views(sub, poses, cam, query=q, images=False, flags=False)
    err = np.abs(sc - ref["scores"]).max()
    print("full-size ncc max err", err, "best", res.best_index, oracle.argmax(ref["scores"]))
    assert err <= TOL_NCC
    top = np.sort(ref["scores"])[::-1]
    if top[0] - top[1] > TOL_NCC:
        assert res.best_index == oracle.argmax(ref["scores"])
    k = res.best_index
    one = oracle.render_views(sub, poses[k:k + 1], cam)
    st = compare_images(brgb.cpu().numpy()[None].astype(np.float64), bdep.cpu().numpy()[None].astype(np.float64),
                        bal.cpu().numpy()[None].astype(np.float64), one, z_ref(sub, poses[k:k + 1], cam))
    print("full-size winner image", st)
    # two more sampled views through reloc_render
    pick = [0, 63]
    rgb, depth, alpha = gpu_render(ctx, runs, poses[pick], cam)
    two = oracle.render_views(sub, poses[pick], cam)
    print("full-size sampled views", compare_images(rgb, depth, alpha, two, z_ref(sub, poses[pick], cam)))
    # the same views in colour only (the scoring launches' variant)
    print("full-size sampled views, colour only", compare_rgb(gpu_render_rgb(ctx, runs, poses[pick], cam), two))
