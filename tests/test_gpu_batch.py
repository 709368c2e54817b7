"""Batched relocalization (many queries, uneven candidate counts and subsets,
one launch per stage, optional CUDA graph): results must equal those of
separate reloc_localize calls bit for bit, whatever the sub-batching, the
graph option or the capacity retries; one query is also checked against the
FP64 oracle's full sweep."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import TOL_NCC

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


@pytest.fixture(scope="module")
def street():
    g = sg.street_gaussians(200_000, seed=21, sh_degree=3)
    cam = sg.street_camera(352, 94, 138.0)
    return g, cam


def make_queries(ctx, g, cam, n, seed=22):
    """n queries along the street with uneven grids (4..27 candidates) and radii."""
    r = sg.Rng(seed)
    hidden, seeds = sg.street_queries(n, seed=seed)
    qs = []
    for i in range(n):
        nx, ny, nyaw = int(r.uniform(1, 1.0, 4.0)[0]), int(r.uniform(1, 1.0, 4.0)[0]), int(r.uniform(1, 1.0, 4.0)[0])
        radius = float(r.uniform(1, 15.0, 45.0)[0])
        runs, _, _ = ctx.select_block(hidden[i][0], hidden[i][1], radius)
        img = torch.empty((1, 3, cam.height, cam.width), device="cuda:0")
        ctx.render(runs, sg.pose_from_xyz_yaw(*hidden[i])[None], cam, rgb=img)
        img = (img[0] + torch.tensor(sg.image_noise(100 + i, cam.height, cam.width), device="cuda:0")).contiguous()
        qs.append((img, sg.pose_from_xyz_yaw(*seeds[i]), radius, (nx, ny, nyaw, 0.5, 2.0)))
    return qs


def separate(ctx, qs, cam):
    out = []
    for img, pose, radius, grid in qs:
        brgb = torch.empty((3, cam.height, cam.width), device="cuda:0")
        bdep = torch.empty((cam.height, cam.width), device="cuda:0")
        res, sc = ctx.localize(img, pose, radius, grid, cam, brgb, bdep)
        out.append((res, sc, brgb.cpu().numpy(), bdep.cpu().numpy()))
    return out


def batched(ctx, qs, cam):
    n = len(qs)
    brgb = torch.empty((n, 3, cam.height, cam.width), device="cuda:0")
    bdep = torch.empty((n, cam.height, cam.width), device="cuda:0")
    res, sc = ctx.localize_batch(qs, cam, brgb, bdep)
    torch.cuda.synchronize()
    return res, sc, brgb.cpu().numpy(), bdep.cpu().numpy()


def assert_same(sep, bat):
    res, sc, brgb, bdep = bat
    for i, (r1, s1, img1, dep1) in enumerate(sep):
        r2 = res[i]
        assert r2.best_index == r1.best_index, i
        assert r2.best_score == r1.best_score, i
        assert r2.n_gauss == r1.n_gauss and r2.n_blocks == r1.n_blocks
        assert list(r2.best_pose) == list(r1.best_pose)
        assert np.array_equal(sc[i], s1), i
        assert np.array_equal(brgb[i], img1), i
        assert np.array_equal(bdep[i], dep1), i


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_separate_calls(R, street, use_graph):
    g, cam = street
    ctx = R.Context()
    ctx.load_map(g)
    ctx.set_batch_options(use_graph=use_graph)
    qs = make_queries(ctx, g, cam, 7)
    sep = separate(ctx, qs, cam)
    bat = batched(ctx, qs, cam)
    assert_same(sep, bat)
    c = ctx.last_counts()
    assert c.n_views == sum(len(s[1]) for s in sep)


def test_batch_split_into_sub_batches(R, street):
    g, cam = street
    ctx = R.Context()
    ctx.load_map(g)
    qs = make_queries(ctx, g, cam, 6, seed=23)
    sep = separate(ctx, qs, cam)
    ctx.set_batch_options(use_graph=True, mem_budget=64 << 20)   # forces several sub-batches
    assert_same(sep, batched(ctx, qs, cam))


def test_batch_capacity_retry(R, street):
    g, cam = street
    a = R.Context()
    a.load_map(g)
    qs = make_queries(a, g, cam, 5, seed=24)
    sep = separate(a, qs, cam)
    b = R.Context(R.reloc_default_config(inst_capacity=64))
    b.load_map(g)
    bat = batched(b, qs, cam)
    assert b.last_counts().retries >= 1
    assert_same(sep, bat)


def test_batch_query_matches_oracle(R, street):
    g, cam = street
    ctx = R.Context()
    ctx.load_map(g)
    qs = make_queries(ctx, g, cam, 3, seed=25)
    res, sc, brgb, bdep = batched(ctx, qs, cam)
    k = 1
    img, pose, radius, grid = qs[k]
    c = -pose[:3, :3].T @ pose[:3, 3]
    idx, nb = oracle.block_select(g.mean, 20.0, c[0], c[1], radius)
    assert res[k].n_gauss == len(idx) and res[k].n_blocks == nb
    poses = oracle.grid_poses(pose, *grid)
    ref = oracle.render_views(g.subset(idx), poses, cam, query=img.cpu().numpy(), images=False, flags=False)
    assert np.abs(sc[k] - ref["scores"]).max() <= TOL_NCC
    top = np.sort(ref["scores"])[::-1]
    if len(top) < 2 or top[0] - top[1] > TOL_NCC:
        assert res[k].best_index == oracle.argmax(ref["scores"])


def test_batch_rejects_bad_queries(R, street):
    g, cam = street
    ctx = R.Context()
    ctx.load_map(g)
    qs = make_queries(ctx, g, cam, 2, seed=26)
    bad = list(qs)
    bad[1] = (qs[1][0], qs[1][1], qs[1][2], (0, 1, 1, 0.5, 2.0))
    with pytest.raises(R.RelocError) as e:
        ctx.localize_batch(bad, cam)
    assert e.value.status == R.EINVAL
    pose = qs[0][1].copy()
    pose[0, 3] = math.nan
    with pytest.raises(R.RelocError) as e:
        ctx.localize_batch([(qs[0][0], pose, qs[0][2], qs[0][3])], cam)
    assert e.value.status == R.ENUMERIC
    # the context still works
    batched(ctx, qs, cam)


def test_autotune_picks_and_persists(R, street, tmp_path):
    g, cam = street
    ctx = R.Context()
    ctx.load_map(g)
    qs = make_queries(ctx, g, cam, 3, seed=27)
    table = str(tmp_path / "tune.txt")
    t1 = ctx.autotune(qs, cam, table)
    assert t1.from_table == 0 and t1.n_tried >= 10 and t1.ms_per_query > 0
    ctx2 = R.Context()
    ctx2.load_map(g)
    t2 = ctx2.autotune(qs, cam, table)
    assert t2.from_table == 1
    assert (t2.tile_w, t2.tile_h, t2.blend_rpl) == (t1.tile_w, t1.tile_h, t1.blend_rpl)
    # the tuned configuration still gives the separate-call results
    assert_same(separate(ctx, qs, cam), batched(ctx, qs, cam))
