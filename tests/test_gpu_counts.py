"""Full-size check of the projection and tile binning on the driving street's
first query (64 candidates, 1408x376): the library's visible and instance
totals equal the oracle's exact counts (tests/golden/counts.json) up to the
Gaussians whose FP32 and FP64 projections fall on different sides of a
near-plane, image-edge or tile-line test -- a relative difference far below
1e-4 of the totals."""
import json
import os

import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


def test_driving_counts_match_oracle(R):
    with open(os.path.join(HERE, "golden", "counts.json")) as f:
        gold = json.load(f)["driving_q0"]
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    _, seeds = sg.street_queries(1, seed=12)
    ctx = R.Context(R.reloc_default_config())
    ctx.load_map(g)
    runs, n_gauss, _ = ctx.select_block(seeds[0][0], seeds[0][1], 40.0)
    assert n_gauss == gold["n_gauss"]
    poses = sg.street_grid_poses(seeds[0])
    assert poses.shape[0] == 64
    ctx.render(runs, poses, cam)
    c = ctx.last_counts()
    ref = np.array(gold["counts"]).sum(0)
    print("gpu", c.n_visible, c.n_instances, "oracle", ref[:2])
    assert abs(c.n_visible - ref[0]) <= 1e-4 * ref[0]
    assert abs(c.n_instances - ref[1]) <= 1e-4 * ref[1]
