"""Map-training cases shared by the oracle pins and the GPU tests: the tiny
scene's Gaussians as the ground truth, a start map with seeded noise on every
parameter, and the truth rendered by the oracle as the training targets."""
import numpy as np

import oracle
import scenegen as sg


def start_map(g, seed=31, mean_std=0.03, scale_rel=0.15, quat_std=0.05, opac_std=0.5, rgb_std=0.1):
    """g with seeded noise: means (metres), log scales, quaternions, logit
    opacities, colours (clipped to [0, 1])."""
    r = sg.Rng(seed)
    n = g.n
    mean = g.mean + r.normal(3 * n, 0.0, mean_std).reshape(n, 3)
    scale = g.scale * np.exp(r.normal(3 * n, 0.0, scale_rel).reshape(n, 3))
    quat = g.quat + r.normal(4 * n, 0.0, quat_std).reshape(n, 4)
    z = np.log(g.opacity / (1 - g.opacity)) + r.normal(n, 0.0, opac_std)
    opac = 1.0 / (1.0 + np.exp(-z))
    rgb = np.clip(g.sh + r.normal(3 * n, 0.0, rgb_std).reshape(n, 1, 3), 0.0, 1.0)
    return sg.Gaussians(mean.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
                        opac.astype(np.float32), rgb.astype(np.float32), 0)


def tiny_training(n_views=4, seed=31):
    """(scene, start map, training poses [V,4,4], targets [V,3,H,W] float64)."""
    s = sg.tiny_scene()
    poses = s.candidate_poses[:n_views]
    gt = oracle.render_views(s.gaussians, poses, s.camera, images=True, flags=False)["rgb"]
    return s, start_map(s.gaussians, seed), poses, gt
