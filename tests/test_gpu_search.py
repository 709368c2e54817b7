"""reloc_localize_random (Sec. IV-A random search with early stop) against the
oracle's search on the same grid and visiting order: visited cells and the
stop batch exactly, the best cell exactly, NCC within 2e-6 (the parity bound
of a single score); the library's own seeded order against the oracle's
independent SplitMix64 / Fisher-Yates; a paper-size search (8100-cell grid,
2 m x 10 deg over +-15 m and a full turn, 20% visited) on the driving street
with sampled scores checked against the oracle; invalid options."""

import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NCC_TOL = 2e-6


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


@pytest.fixture(scope="module")
def tiny(R):
    s = sg.tiny_scene()
    ctx = R.Context()
    ctx.load_map(s.gaussians)
    g = s.gaussians.subset(ctx.map_order())        # the library's subset order
    grid = (9, 9, 8, 0.25, 2.5)
    cells = oracle.grid_poses(s.seed_pose, *grid)
    q = (oracle.render(g, s.hidden_pose, s.camera)["rgb"] + s.query_noise).astype(np.float32)
    return s, ctx, g, grid, cells, q


def run(R, ctx, s, grid, q, **kw):
    qd = torch.tensor(q, device="cuda:0")
    return ctx.localize_random(qd, s.seed_pose, 1e3, grid, s.camera, **kw)


def test_explicit_order_matches_oracle(R, tiny):
    s, ctx, g, grid, cells, q = tiny
    order = oracle.search_order(11, len(cells))[:oracle.visit_count(0.2, len(cells))]
    ref = oracle.random_search(g, cells, s.camera, q, order, 32, np.inf)
    res, sc = run(R, ctx, s, grid, q, order=order, batch=32, ncc_stop=np.inf)
    assert res.n_scored == len(order) and not res.stopped_early and res.n_candidates == len(cells)
    assert np.array_equal(np.isnan(sc), np.isnan(ref["scores"]))
    vis = ~np.isnan(sc)
    assert np.max(np.abs(sc[vis] - ref["scores"][vis])) <= NCC_TOL
    assert res.best_index == ref["best_index"]
    assert abs(res.best_score - ref["best_score"]) <= NCC_TOL


def test_early_stop_batch_matches_oracle(R, tiny):
    s, ctx, g, grid, cells, q = tiny
    order = oracle.search_order(12, len(cells))[:160]
    full = oracle.random_search(g, cells, s.camera, q, order, 32, np.inf)
    # best-so-far after each batch; a threshold between two batches' bests
    best_after = [np.max(full["scores"][order[:b + 32]]) for b in range(0, len(order), 32)]
    k = next(i for i in range(1, len(best_after)) if best_after[i] - best_after[i - 1] > 1e-4)
    tau = 0.5 * (best_after[k] + best_after[k - 1])
    ref = oracle.random_search(g, cells, s.camera, q, order, 32, tau)
    res, sc = run(R, ctx, s, grid, q, order=order, batch=32, ncc_stop=tau)
    assert ref["n_scored"] == 32 * (k + 1)
    assert res.n_scored == ref["n_scored"] and bool(res.stopped_early) == ref["stopped_early"]
    assert res.best_index == ref["best_index"]
    assert np.array_equal(np.isnan(sc), np.isnan(ref["scores"]))


def test_seeded_order_matches_oracle_generator(R, tiny):
    s, ctx, g, grid, cells, q = tiny
    for seed in (0, 7, 2**64 - 1):
        res, sc = run(R, ctx, s, grid, q, fraction=0.2, seed=seed, batch=64, ncc_stop=np.inf)
        m = oracle.visit_count(0.2, len(cells))
        assert res.n_scored == m
        assert set(np.nonzero(~np.isnan(sc))[0].tolist()) == set(oracle.search_order(seed, len(cells))[:m].tolist())


def test_winner_export_equals_its_render(R, tiny):
    s, ctx, g, grid, cells, q = tiny
    H, W = s.camera.height, s.camera.width
    rgb = torch.zeros((3, H, W), device="cuda:0")
    dep = torch.zeros((H, W), device="cuda:0")
    res, _ = run(R, ctx, s, grid, q, fraction=0.3, seed=5, batch=50, best_rgb=rgb, best_depth=dep)
    ref_rgb = torch.zeros((1, 3, H, W), device="cuda:0")
    ref_dep = torch.zeros((1, H, W), device="cuda:0")
    ctx.render([(0, ctx.n)], cells[res.best_index][None], s.camera, rgb=ref_rgb, depth=ref_dep)
    torch.cuda.synchronize()
    assert torch.equal(rgb, ref_rgb[0]) and torch.equal(dep, ref_dep[0])
    assert np.allclose(np.array(res.best_pose).reshape(4, 4), cells[res.best_index], atol=1e-12)


def test_invalid_options(R, tiny):
    s, ctx, g, grid, cells, q = tiny
    for kw in (dict(fraction=0.0), dict(fraction=1.5), dict(batch=0), dict(batch=5000),
               dict(order=[0, 1, 1]), dict(order=[len(cells)]), dict(order=[-1])):
        with pytest.raises(R.RelocError) as e:
            run(R, ctx, s, grid, q, **kw)
        assert e.value.status == R.EINVAL
    with pytest.raises(R.RelocError) as e:
        run(R, ctx, s, grid, q, ncc_stop=float("nan"))
    assert e.value.status == R.ENUMERIC
    # the context stays usable
    res, _ = run(R, ctx, s, grid, q, fraction=0.05, batch=8)
    assert res.n_scored == oracle.visit_count(0.05, len(cells))


def test_paper_size_random_search_on_the_street(R):
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    hidden, _ = sg.street_queries(1, seed=41)
    h = hidden[0]
    coarse = sg.pose_from_xyz_yaw(h[0] + 6.0, h[1] - 3.0, h[2], h[3] + 0.6)
    c = -coarse[:3, :3].T @ coarse[:3, 3]
    idx, _ = oracle.block_select(g.mean, 20.0, c[0], c[1], 40.0)
    sub = g.subset(idx)
    q = (oracle.render(sub, sg.pose_from_xyz_yaw(*h), cam)["rgb"]
         + sg.image_noise(43, cam.height, cam.width)).astype(np.float32)
    ctx = R.Context()
    ctx.load_map(g)
    grid = (15, 15, 36, 2.0, 10.0)
    res, sc = ctx.localize_random(torch.tensor(q, device="cuda:0"), coarse, 40.0, grid, cam, fraction=0.2, seed=3,
                                  batch=64)
    assert res.n_candidates == 8100 and res.n_scored == 1620 and not res.stopped_early
    assert res.n_gauss == len(idx)
    vis = np.nonzero(~np.isnan(sc))[0]
    assert len(vis) == 1620 and res.best_score == np.max(sc[vis])
    # oracle scores of the best cell and three other visited cells
    cells = oracle.grid_poses(coarse, *grid)
    pick = [res.best_index] + [int(k) for k in vis[[0, 500, 1000]]]
    out = oracle.render_views(sub, cells[pick], cam, query=q, images=False, flags=False)
    print("best", res.best_index, res.best_score, "oracle", out["scores"])
    assert np.max(np.abs(out["scores"] - sc[pick])) <= NCC_TOL
