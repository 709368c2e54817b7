"""Map training (Sec. III-B.3) on the GPU against the oracle.

reloc_train_grad's gradient (FP32 backward blend and chain rule, per-Gaussian
sums by atomic adds) is compared with the oracle's forward-mode FP64
derivatives of the same loss (pinned to central differences by the oracle's
own tests) along seeded directions: g . d must equal the oracle's derivative
along d within 1e-3 of sum |g_i d_i| (FP32 terms each carry ~1e-6 relative
error; a pair whose inclusion test lies within rounding of its threshold may
be in one set and not the other, and a sample within rounding of its target
may take the other sign of |x|); single entries (one-hot directions at the
Gaussians with the largest gradient of each parameter) within 1e-3 relative.
The loss equals the oracle's within 1e-4 relative (FP32 render), with and
without the D-SSIM term (lambda 0, 0.2, 1), for the re-projection term alone
and for the weighted total of Eq. 6 (which does not depend on how the views
are grouped).  Adam steps
lower the loss; the map read back matches what was loaded; invalid maps and
options fail."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from train_cases import tiny_training

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L1_ONLY = dict(lambda_dssim=0.0, w_reproj=0.0)


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


@pytest.fixture(scope="module")
def case(R):
    s, g0, poses, gt = tiny_training(n_views=3)
    ctx = R.Context()
    ctx.load_map(g0)
    g = g0.subset(ctx.map_order())
    tg = torch.tensor(gt.astype(np.float32), device="cuda:0")
    grad = torch.zeros((14, g.n), device="cuda:0")
    loss = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, **L1_ONLY)
    gt32 = gt.astype(np.float32).astype(np.float64)
    return s, ctx, g, poses, gt32, tg, loss, grad.cpu().numpy().astype(np.float64)


def test_loss_matches_oracle(case):
    s, ctx, g, poses, gt32, tg, loss, G = case
    ref, _ = oracle.photo_loss_jvp(g, poses, s.camera, gt32, np.zeros((g.n, 14, 6)))
    print("loss gpu", loss, "oracle", ref)
    assert abs(loss - ref) <= 1e-4 * ref


def test_directional_derivatives_match_oracle(case):
    s, ctx, g, poses, gt32, tg, loss, G = case
    r = sg.Rng(77)
    dirs = (r.u64(g.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(g.n, 14, 6) - 1.0
    # one direction per parameter group as well: only that group's rows
    groups = [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]
    d2 = np.zeros_like(dirs)
    for k, (a, b) in enumerate(groups):
        d2[:, a:b, k] = dirs[:, a:b, k]
    d2[:, :, 5] = dirs[:, :, 5]
    for D in (dirs, d2):
        _, jv = oracle.photo_loss_jvp(g, poses, s.camera, gt32, D)
        for k in range(6):
            terms = G.T * D[:, :, k]
            mine, mass = terms.sum(), np.abs(terms).sum()
            print(k, mine, jv[k], mass)
            assert abs(mine - jv[k]) <= 1e-3 * mass + 1e-12


def test_largest_entries_match_oracle(case):
    s, ctx, g, poses, gt32, tg, loss, G = case
    picks = [(row, int(np.argmax(np.abs(G[row])))) for row in range(14)]
    for c0 in range(0, 14, 6):
        chunk = picks[c0:c0 + 6]
        D = np.zeros((g.n, 14, 6))
        for k, (row, i) in enumerate(chunk):
            D[i, row, k] = 1.0
        _, jv = oracle.photo_loss_jvp(g, poses, s.camera, gt32, D)
        for k, (row, i) in enumerate(chunk):
            print(oracle.PARAM_ORDER[row], i, G[row, i], jv[k])
            assert abs(G[row, i] - jv[k]) <= 1e-3 * abs(jv[k])


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_dssim_loss_and_derivatives_match_oracle(R, case, lam):
    s, ctx, g, poses, gt32, tg, loss, G = case
    grad = torch.zeros((14, g.n), device="cuda:0")
    mine = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, lambda_dssim=lam, w_reproj=0.0)
    Gl = grad.cpu().numpy().astype(np.float64)
    r = sg.Rng(91)
    dirs = (r.u64(g.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(g.n, 14, 6) - 1.0
    ref, jv = oracle.photo_loss_jvp(g, poses, s.camera, gt32, dirs, lam=lam)
    print("lambda", lam, "loss gpu", mine, "oracle", ref)
    assert abs(mine - ref) <= 1e-4 * ref
    for k in range(6):
        terms = Gl.T * dirs[:, :, k]
        got, mass = terms.sum(), np.abs(terms).sum()
        print(k, got, jv[k], mass)
        assert abs(got - jv[k]) <= 1e-3 * mass + 1e-12


def _check_against_oracle(ctx, g, poses, s, tg, gt32, seed, **opts):
    grad = torch.zeros((14, g.n), device="cuda:0")
    mine = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, **opts)
    Gl = grad.cpu().numpy().astype(np.float64)
    r = sg.Rng(seed)
    dirs = (r.u64(g.n * 14 * 6) % np.uint64(3)).astype(np.float64).reshape(g.n, 14, 6) - 1.0
    ref, jv = oracle.train_loss_jvp(g, poses, s.camera, gt32, dirs, lam=opts["lambda_dssim"],
                                    w_photo=opts["w_photo"], w_reproj=opts["w_reproj"])
    print(opts, "loss gpu", mine, "oracle", ref)
    assert abs(mine - ref) <= 1e-4 * ref
    for k in range(6):
        terms = Gl.T * dirs[:, :, k]
        got, mass = terms.sum(), np.abs(terms).sum()
        print(k, got, jv[k], mass)
        assert abs(got - jv[k]) <= 1e-3 * mass + 1e-12
    return mine, Gl


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_reprojection_loss_and_derivatives_match_oracle(R, case, lam):
    s, ctx, g, poses, gt32, tg, loss, G = case
    _check_against_oracle(ctx, g, poses, s, tg, gt32, 101, lambda_dssim=lam, w_photo=0.0, w_reproj=1.0)


def test_total_loss_matches_oracle_and_groups_do_not_matter(R, case):
    s, ctx, g, poses, gt32, tg, loss, G = case
    opts = dict(lambda_dssim=0.2, w_photo=0.7, w_reproj=1.3)
    L, Gl = _check_against_oracle(ctx, g, poses, s, tg, gt32, 103, **opts)
    # one view per group: each pair's two views fall in different groups
    grad = torch.zeros((14, g.n), device="cuda:0")
    L1 = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, views_per_group=1, **opts)
    G1 = grad.cpu().numpy().astype(np.float64)
    assert abs(L1 - L) <= 1e-6 * L
    assert np.abs(G1 - Gl).max() <= 1e-4 * np.abs(Gl).max()


def test_gradient_is_zero_outside_the_ranges(R, case):
    s, ctx, g, poses, gt32, tg, loss, G = case
    half = ctx.n // 2
    grad = torch.full((14, g.n), 7.0, device="cuda:0")
    ctx.train_grad([(0, half)], poses, s.camera, tg, grad, **L1_ONLY)
    gh = grad.cpu().numpy()
    assert np.all(gh[:, half:] == 0.0)
    assert np.any(gh[:, :half] != 0.0)


def test_read_map_round_trip(R):
    s = sg.tiny_scene(n=2000)
    ctx = R.Context()
    ctx.load_map(s.gaussians)
    o = ctx.map_order()
    m, sc, q, op, sh = ctx.read_map()
    g = s.gaussians
    assert np.array_equal(m, g.mean[o]) and np.array_equal(sc, g.scale[o]) and np.array_equal(q, g.quat[o])
    assert np.array_equal(op, g.opacity[o]) and np.array_equal(sh, g.sh[o])


def test_adam_steps_lower_the_loss(R):
    s, g0, poses, gt = tiny_training(n_views=8, seed=41)
    ctx = R.Context()
    ctx.load_map(g0)
    tg = torch.tensor(gt.astype(np.float32), device="cuda:0")
    losses = [ctx.train_step([(0, ctx.n)], poses, s.camera, tg, lr_mean=1e-3, **L1_ONLY) for _ in range(60)]
    print("loss", losses[0], "->", losses[-1], losses[::10])
    assert losses[-1] < 0.6 * losses[0]
    m, sc, q, op, sh = ctx.read_map()
    assert np.all(np.isfinite(m)) and np.all(sc > 0) and np.all((op > 0) & (op < 1))
    ctx.train_reset()
    ctx.train_step([(0, ctx.n)], poses, s.camera, tg, **L1_ONLY)


def test_invalid_training_calls(R):
    s, g0, poses, gt = tiny_training(n_views=1)
    tg = torch.tensor(gt.astype(np.float32), device="cuda:0")
    ctx = R.Context()
    ctx.load_map(g0, precision=R.FP16)
    grad = torch.zeros((14, g0.n), device="cuda:0")
    with pytest.raises(R.RelocError) as e:
        ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, **L1_ONLY)
    assert e.value.status == R.EINVAL
    ctx.load_map(g0)
    with pytest.raises(R.RelocError) as e:
        ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, **dict(L1_ONLY, views_per_group=0))
    assert e.value.status == R.EINVAL
    with pytest.raises(R.RelocError) as e:
        ctx.train_step([(0, ctx.n)], poses, s.camera, tg, **dict(L1_ONLY, beta1=1.0))
    assert e.value.status == R.EINVAL
    with pytest.raises(R.RelocError) as e:
        ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, reproj_alpha_min=0.0)
    assert e.value.status == R.EINVAL
    # one view: no pair, the re-projection term is 0 and the call is valid
    L0 = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, lambda_dssim=0.2, w_reproj=0.0)
    L1 = ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, grad, lambda_dssim=0.2, w_reproj=1.0)
    assert abs(L0 - L1) <= 1e-12 * L0          # FP64 atomic sums: order varies
    street = sg.street_gaussians(20000, seed=3, sh_degree=3)
    ctx.load_map(street)
    with pytest.raises(R.RelocError) as e:
        ctx.train_grad([(0, ctx.n)], poses, s.camera, tg, torch.zeros((14, street.n), device="cuda:0"), **L1_ONLY)
    assert e.value.status == R.EINVAL


def test_sub_batches_do_not_change_the_loss_or_gradient(R):
    """A 64 MiB workspace budget puts each view of a 400k-Gaussian street
    subset in its own sub-batch, so the re-projection pairs straddle
    sub-batches; loss and gradient equal those of one sub-batch (up to the
    order of the atomic sums)."""
    g = sg.street_gaussians(400_000, seed=5, sh_degree=0)
    cam = sg.street_camera(704, 188, 276.0)
    x0 = float(np.median(g.mean[:, 0]))
    poses = np.stack([sg.pose_from_xyz_yaw(x0 + k, 0.0, 1.6, 0.0) for k in range(4)])
    tg = torch.tensor(np.stack([sg.random_image(70 + k, 3, cam.height, cam.width) for k in range(4)]),
                      dtype=torch.float32, device="cuda:0")
    out = []
    for budget, vpg in ((16 << 30, 16), (64 << 20, 1)):
        ctx = R.Context()
        ctx.set_batch_options(mem_budget=budget)
        ctx.load_map(g)
        grad = torch.zeros((14, g.n), device="cuda:0")
        L = ctx.train_grad([(0, ctx.n)], poses, cam, tg, grad, views_per_group=vpg)
        out.append((L, grad.cpu().numpy()))
        ctx.close()
    (La, Ga), (Lb, Gb) = out
    print("loss", La, Lb, "max |dG|", np.abs(Ga - Gb).max(), "max |G|", np.abs(Ga).max())
    assert abs(La - Lb) <= 1e-9 * La
    # the per-Gaussian FP32 sums regroup (views per thread, atomics across groups):
    # rounding of cancelling terms reaches ~2e-5 of the largest entry; a pair lost
    # or doubled across sub-batches would be of the order of the entry itself
    assert np.abs(Ga - Gb).max() <= 1e-4 * np.abs(Ga).max()


def test_empty_subset_renders_black(R):
    """No Gaussians selected: every render is black, so L1 alone is the mean
    of the targets and the gradient is zero."""
    s, g0, poses, gt = tiny_training(n_views=2)
    tg = torch.tensor(gt.astype(np.float32), device="cuda:0")
    ctx = R.Context()
    ctx.load_map(g0)
    grad = torch.full((14, g0.n), 3.0, device="cuda:0")
    L = ctx.train_grad([], poses, s.camera, tg, grad, lambda_dssim=0.0, w_reproj=1.0)
    ref = float(np.abs(gt.astype(np.float32).astype(np.float64)).mean())
    assert abs(L - ref) <= 1e-6 * ref
    assert float(grad.abs().max()) == 0.0


def test_adam_step_matches_oracle(R):
    """One reloc_train_step from fresh Adam state equals the oracle's Adam
    step applied to the oracle's gradient, for 16 Gaussians of view 0: the
    full gradient of those Gaussians from one-hot forward-mode derivatives
    (L1 loss over 2 views).  The first step moves each latent parameter by
    lr * sign(g), so entries whose oracle gradient is within rounding of 0
    (where the FP32 sign may differ) are left out."""
    s, g0, poses, gt = tiny_training(n_views=2, seed=51)
    tg = torch.tensor(gt.astype(np.float32), device="cuda:0")
    ctx = R.Context()
    ctx.load_map(g0)
    g = g0.subset(ctx.map_order())
    recs = oracle.project(g, poses[0], s.camera)
    idx = np.nonzero(recs[:, oracle.F["visible"]] > 0)[0][::97][:16]
    assert len(idx) == 16
    opts = dict(lambda_dssim=0.0, w_reproj=0.0)
    o = R.Context.train_options(**opts)
    ctx.train_step([(0, ctx.n)], poses, s.camera, tg, **opts)
    m, sc, q, op, sh = ctx.read_map()
    after = np.concatenate([m, sc, q, op[:, None], sh[:, 0, :]], 1).astype(np.float64)[idx]
    gt32 = gt.astype(np.float32).astype(np.float64)
    G = np.zeros((len(idx), 14))
    cols = [(j, c) for j in range(len(idx)) for c in range(14)]
    for k0 in range(0, len(cols), 6):
        D = np.zeros((g.n, 14, 6))
        for k, (j, c) in enumerate(cols[k0:k0 + 6]):
            D[idx[j], c, k] = 1.0
        _, jv = oracle.train_loss_jvp(g, poses, s.camera, gt32, D, lam=0.0, w_photo=1.0, w_reproj=0.0)
        for k, (j, c) in enumerate(cols[k0:k0 + 6]):
            G[j, c] = jv[k]
    before = oracle.map_params(g)[idx]
    lr = [o.lr_mean, o.lr_scale, o.lr_quat, o.lr_opacity, o.lr_color]
    ref, _, _ = oracle.adam_step(before, G, np.zeros_like(G), np.zeros_like(G), 1, lr, o.beta1, o.beta2, o.eps)
    sure = np.abs(G) > 1e-6 * np.abs(G).max()
    err = np.abs(after - ref)
    print("checked", int(sure.sum()), "of", G.size, "max err", err[sure].max())
    assert sure.sum() > 0.8 * G.size
    assert np.all(err[sure] <= 1e-6 * np.abs(ref[sure]) + 1e-7)
