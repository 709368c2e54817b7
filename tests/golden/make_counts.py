"""Write tests/golden/counts.json: the oracle's exact algorithmic counts for the
seeded workloads, per candidate view (FP64 projection and compositing):

  n_vis   Gaussians in front of the near plane whose 3-sigma rectangle meets
          the image (Sec. III-A projection, the tile binning's input)
  n_inst  (tile, Gaussian) instances of 16x16 tiles (the rectangle's tiles)
  n_eval  evaluated (pixel, Gaussian) pairs: the pixel centre inside the
          3-sigma ellipse (power >= -4.5), up to and including the Gaussian
          at which the pixel's transmittance stops (Eq. 3 compositing); pairs
          then skipped for alpha < 1/255 are counted too, since their alpha
          had to be computed

Workloads: the tiny scene (10k Gaussians, 352x94, 16 candidates) and the
driving street's first query (2M-Gaussian map, 40 m block selection around
the seed pose, 1408x376, the 4 x 4 x 4 grid at 0.5 m / 2 deg = 64 candidates).
Only oracle/ and the seeded scene generators are used.

    python tests/golden/make_counts.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import scenegen as sg  # noqa: E402

GRID = (4, 4, 4, 0.5, 2.0)
RADIUS = 40.0


def tiny_counts():
    s = sg.tiny_scene()
    out = oracle.render_views(s.gaussians, s.candidate_poses, s.camera, images=False, flags=False)
    return {"workload": "tiny: 10k Gaussians SH0, 352x94 f=138, 16 candidates, 16x16 tiles",
            "seeds": {"scene": 1, "poses": 2}, "n_gauss": int(s.gaussians.n),
            "counts": out["counts"].tolist()}


def driving_counts():
    g = sg.street_gaussians(2_000_000, seed=11, sh_degree=3)
    cam = sg.street_camera()
    hidden, seeds = sg.street_queries(1, seed=12)
    idx, n_blocks = oracle.block_select(g.mean, 20.0, seeds[0][0], seeds[0][1], RADIUS)
    sub = g.subset(idx)
    poses = oracle.grid_poses(sg.pose_from_xyz_yaw(*seeds[0]), *GRID)
    out = oracle.render_views(sub, poses, cam, images=False, flags=False)
    return {"workload": "driving street query 0: 2M-Gaussian map SH3, 20 m blocks, 40 m radius, "
                        "1408x376 f=552, 64 candidates (4x4x4, 0.5 m / 2 deg), 16x16 tiles",
            "seeds": {"scene": 11, "queries": 12}, "n_gauss": int(sub.n), "n_blocks": int(n_blocks),
            "counts": out["counts"].tolist()}


def main():
    data = {"columns": ["n_vis", "n_inst", "n_eval"], "tiny": tiny_counts(), "driving_q0": driving_counts()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "counts.json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    for k in ("tiny", "driving_q0"):
        c = data[k]["counts"]
        print(k, data[k]["n_gauss"], [sum(r[i] for r in c) for i in range(3)])


if __name__ == "__main__":
    main()
