"""The stored oracle counts (tests/golden/counts.json, written by
tests/golden/make_counts.py from oracle/ alone) are reproduced by the oracle
as it stands, and obey the inequalities the definitions imply: every
instance belongs to a visible Gaussian (n_inst >= n_vis) and an included
pair needs a visible Gaussian (n_vis = 0 implies n_eval = 0)."""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen as sg

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "counts.json")) as f:
        return json.load(f)


def test_tiny_counts_reproduced(golden):
    s = sg.tiny_scene()
    out = oracle.render_views(s.gaussians, s.candidate_poses, s.camera, images=False, flags=False)
    assert out["counts"].tolist() == golden["tiny"]["counts"]


def test_driving_counts_reproduced_on_four_candidates(golden):
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    _, seeds = sg.street_queries(1, seed=12)
    idx, _ = oracle.block_select(g.mean, 20.0, seeds[0][0], seeds[0][1], 40.0)
    assert len(idx) == golden["driving_q0"]["n_gauss"]
    poses = oracle.grid_poses(sg.pose_from_xyz_yaw(*seeds[0]), 4, 4, 4, 0.5, 2.0)
    pick = [0, 21, 42, 63]
    out = oracle.render_views(g.subset(idx), poses[pick], cam, images=False, flags=False)
    ref = np.array(golden["driving_q0"]["counts"])[pick]
    assert np.array_equal(out["counts"], ref)


def test_counts_consistent(golden):
    for k in ("tiny", "driving_q0"):
        c = np.array(golden[k]["counts"])
        assert (c[:, 1] >= c[:, 0]).all()
        assert ((c[:, 0] > 0) | (c[:, 2] == 0)).all()
        assert (c[:, 0] <= golden[k]["n_gauss"]).all()
