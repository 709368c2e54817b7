"""reloc_ncc_images_noalloc: NCC scoring without any device allocation.

Callers that must not allocate device memory once running (a real-time loop
that reserves everything at start-up, or a process whose device memory
belongs to another framework's pool) score images they rendered themselves
through this entry point; its only scratch is a fixed array inside the
library.  This test renders candidate views with reloc_render, scores them
with the new entry point twice in a row (different view sets, so stale
scratch from the first call would show), and checks both against the scores
of the existing entry point reloc_score for the same poses and against the
FP64 oracle's NCC of the same images, within the NCC tolerance of the parity
tests.  It also runs the largest accepted call (RELOC_NOALLOC_MAX_VIEWS
views, which fills the last scratch row), a zero-variance image (score 0,
degenerate 1) and a call without the degenerate output.  It is collected
last (file name) and needs no state from the other tests.
"""
import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_NCC = 2e-6


def test_noalloc_ncc_matches_reloc_score_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc as R

    s = sg.tiny_scene()
    cam = s.camera
    ctx = R.Context()
    ctx.load_map(s.gaussians)
    ranges = [(0, ctx.n)]
    order = ctx.map_order()
    q = (oracle.render(s.gaussians.subset(order), s.hidden_pose, cam)["rgb"] + s.query_noise).astype(np.float32)
    qd = torch.tensor(q, device="cuda:0")
    V = len(s.candidate_poses)
    imgs = torch.empty((V, 3, cam.height, cam.width), device="cuda:0")
    ctx.render(ranges, s.candidate_poses, cam, rgb=imgs)
    ref, ref_dg = ctx.score(ranges, s.candidate_poses, cam, qd)

    imgs_np = imgs.cpu().numpy()
    ref_or = np.array([oracle.ncc(imgs_np[v], q)[0] for v in range(V)])
    for sel in (np.arange(V), np.arange(V)[::-2].copy()):
        sub = imgs[torch.as_tensor(sel, device="cuda:0")].contiguous()
        scores = torch.full((len(sel),), float("nan"), dtype=torch.float64, device="cuda:0")
        dg = torch.full((len(sel),), -1, dtype=torch.int32, device="cuda:0")
        R.reloc_ncc_images_noalloc(sub, qd, scores, dg)
        torch.cuda.synchronize()
        got = scores.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref[sel]).max() <= TOL_NCC, (got, ref[sel])
        assert np.abs(got - ref_or[sel]).max() <= 1e-9, (got, ref_or[sel])
        assert np.array_equal(dg.cpu().numpy(), ref_dg[sel])

    # the largest accepted call: one view tiled to RELOC_NOALLOC_MAX_VIEWS,
    # with a zero-variance image in the last slot, no degenerate output
    n = R.NOALLOC_MAX_VIEWS
    many = imgs[3:4].expand(n, -1, -1, -1).contiguous()
    many[n - 1] = 0.25
    scores = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda:0")
    R.reloc_ncc_images_noalloc(many, qd, scores, None)
    got = scores.cpu().numpy()
    assert np.abs(got[:-1] - ref_or[3]).max() <= 1e-9
    assert got[-1] == 0.0
    dg = torch.full((2,), -1, dtype=torch.int32, device="cuda:0")
    two = torch.stack([imgs[3], many[n - 1]]).contiguous()
    scores2 = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda:0")
    R.reloc_ncc_images_noalloc(two, qd, scores2, dg)
    assert dg.cpu().numpy().tolist() == [0, 1] and scores2.cpu().numpy()[1] == 0.0

    # sizes beyond the fixed scratch are rejected before any launch
    big = torch.empty((1, 3, 2, 2), device="cuda:0")
    out = torch.empty((1,), dtype=torch.float64, device="cuda:0")
    lib_status = R.lib.reloc_ncc_images_noalloc(R._ptr(big), R.NOALLOC_MAX_VIEWS + 1, 2, 2, R._ptr(big[0]),
                                                R._ptr(out), None, R._stream(None))
    assert lib_status == R.EINVAL
    assert "RELOC_NOALLOC_MAX_VIEWS" in R.lib.reloc_last_error().decode()
    ctx.close()
