"""Seeded synthetic inputs for the relocalization hot path.

This module draws the *inputs* of the method -- Gaussian maps, camera
intrinsics, camera poses, candidate offsets and query-image noise -- from a
counter-based generator.  It holds none of the method's arithmetic (no
projection, no compositing, no NCC): both the FP64 oracle and the CUDA path
consume what it produces as plain data.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the k-th output of a stream
with seed s is mix(s + (k + 1) * 0x9E3779B97F4A7C15), so a whole array is
drawn at once.  Normal variates use the Box-Muller transform.

Workloads (they stand in for the KITTI-360 drive the paper evaluates on,
Sec. IV, which is not available here):

* ``tiny_scene``   10k Gaussians in a 20 x 20 x 4 m box, RGB colour (SH
  degree 0), 352x94 camera with fx = fy = 138, 16 jittered candidates.
* ``street_scene`` a 500 m street shaped like a LiDAR-initialised map:
  60% of the Gaussians on the ground plane (2 cm height noise), 40% on two
  facades 8 m from the centre line, anisotropic surface-aligned scales,
  SH degree 3; 1408x376 camera with fx = fy = 552.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """SplitMix64 stream: ``Rng(seed).u64(n)`` returns the next n outputs."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.seed + k * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """Doubles in [lo, hi) from the top 53 bits."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
        """Box-Muller: sqrt(-2 ln u1) cos(2 pi u2) with u1 in (0, 1]."""
        u1 = 1.0 - self.uniform(n)
        u2 = self.uniform(n)
        return mean + std * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------
# data containers
# ---------------------------------------------------------------------------

@dataclass
class Gaussians:
    """A Gaussian map as float32 arrays (the values both sides consume).

    mean  (N,3)  world position, metres
    scale (N,3)  standard deviations along the local axes (activated, > 0)
    quat  (N,4)  rotation quaternion (w, x, y, z), unit length
    opacity (N,) in (0, 1)
    sh    (N,K,3) K = (deg+1)^2 coefficients per colour channel; for degree 0
                 the single coefficient is the plain RGB colour itself.
    """
    mean: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx: np.ndarray) -> "Gaussians":
        return Gaussians(self.mean[idx], self.scale[idx], self.quat[idx],
                         self.opacity[idx], self.sh[idx], self.sh_degree)


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


@dataclass
class Scene:
    name: str
    gaussians: Gaussians
    camera: Camera
    seed_pose: np.ndarray              # (4,4) world-to-camera, float64
    hidden_pose: np.ndarray            # (4,4) world-to-camera of the query
    candidate_poses: np.ndarray        # (V,4,4)
    query_noise: np.ndarray            # (3,H,W) float32 additive noise
    extra: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# camera poses
# ---------------------------------------------------------------------------

def pose_from_xyz_yaw(x: float, y: float, z: float, yaw_rad: float) -> np.ndarray:
    """World-to-camera 4x4 (row-major, OpenCV axes: x right, y down, z forward)
    of a level camera at (x, y, z) whose optical axis points along world
    (cos yaw, sin yaw, 0); world z is up."""
    c, s = math.cos(yaw_rad), math.sin(yaw_rad)
    fwd = np.array([c, s, 0.0])
    right = np.array([s, -c, 0.0])
    down = np.array([0.0, 0.0, -1.0])
    R = np.stack([right, down, fwd])          # rows: camera axes in world
    centre = np.array([x, y, z], dtype=np.float64)
    W = np.eye(4)
    W[:3, :3] = R
    W[:3, 3] = -R @ centre
    return W


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------

def _unit_quats(rng: Rng, n: int) -> np.ndarray:
    q = rng.normal(4 * n).reshape(n, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def tiny_scene(n: int = 10_000, n_cand: int = 16, scene_seed: int = 1,
               pose_seed: int = 2, noise_seed: int = 3,
               width: int = 352, height: int = 94, focal: float = 138.0) -> Scene:
    """Small uniform-box scene with plain RGB colours (SH degree 0)."""
    r = Rng(scene_seed)
    mean = np.stack([r.uniform(n, -10, 10), r.uniform(n, -10, 10), r.uniform(n, 0, 4)], 1)
    scale = np.exp(r.uniform(3 * n, math.log(0.05), math.log(0.3))).reshape(n, 3)
    quat = _unit_quats(r, n)
    opacity = 1.0 / (1.0 + np.exp(-r.normal(n, 0.0, 1.5)))
    rgb = r.uniform(3 * n).reshape(n, 1, 3)
    g = Gaussians(mean.astype(np.float32), scale.astype(np.float32), quat.astype(np.float32),
                  opacity.astype(np.float32), rgb.astype(np.float32), 0)
    cam = Camera(width, height, focal, focal, width / 2.0, height / 2.0)
    base = (0.0, -14.0, 2.0, math.pi / 2)
    seed_pose = pose_from_xyz_yaw(*base)
    pr = Rng(pose_seed)
    off = np.stack([pr.uniform(n_cand + 1, -1, 1), pr.uniform(n_cand + 1, -1, 1),
                    pr.uniform(n_cand + 1, -math.radians(5), math.radians(5))], 1)
    cands = np.stack([pose_from_xyz_yaw(base[0] + o[0], base[1] + o[1], base[2], base[3] + o[2])
                      for o in off[:n_cand]])
    h = off[n_cand]
    hidden = pose_from_xyz_yaw(base[0] + h[0], base[1] + h[1], base[2], base[3] + h[2])
    noise = Rng(noise_seed).normal(3 * height * width, 0.0, 0.02).reshape(3, height, width)
    return Scene("tiny", g, cam, seed_pose, hidden, cands, noise.astype(np.float32),
                 {"candidate_offsets": off[:n_cand], "hidden_offset": h})


STREET_LENGTH = 500.0
STREET_HALF_WIDTH = 8.0
FACADE_HEIGHT = 10.0
CAMERA_HEIGHT = 1.6


def street_gaussians(n: int = 2_000_000, seed: int = 11, sh_degree: int = 3) -> Gaussians:
    """LiDAR-map-like street: 60% ground, 40% on the two facades y = +-8 m."""
    r = Rng(seed)
    n_ground = int(round(0.6 * n))
    n_fac = n - n_ground
    half = STREET_LENGTH / 2
    # ground plane
    gx = r.uniform(n_ground, -half, half)
    gy = r.uniform(n_ground, -STREET_HALF_WIDTH, STREET_HALF_WIDTH)
    gz = r.normal(n_ground, 0.0, 0.02)
    # facades
    fx = r.uniform(n_fac, -half, half)
    side = np.where(r.uniform(n_fac) < 0.5, -1.0, 1.0)
    fy = side * STREET_HALF_WIDTH
    fz = r.uniform(n_fac, 0.0, FACADE_HEIGHT)
    mean = np.concatenate([np.stack([gx, gy, gz], 1), np.stack([fx, fy, fz], 1)])
    # anisotropic surface-aligned scales: local z is the surface normal
    ls = r.normal(3 * n, math.log(0.12), 0.6).reshape(n, 3)
    s = np.clip(np.exp(ls), 0.03, 0.5)
    s[:, 2] *= 0.2
    # rotations: ground -> in-plane rotation about world z;
    # facade -> local z mapped onto world y (rotation of -90 deg about x),
    # then an in-plane rotation about world y.
    th = r.uniform(n, 0.0, 2 * math.pi)
    q = np.zeros((n, 4))
    q[:n_ground, 0] = np.cos(th[:n_ground] / 2)
    q[:n_ground, 3] = np.sin(th[:n_ground] / 2)
    a = th[n_ground:] / 2
    qy = np.stack([np.cos(a), np.zeros_like(a), np.sin(a), np.zeros_like(a)], 1)
    qx = np.array([math.cos(-math.pi / 4), math.sin(-math.pi / 4), 0.0, 0.0])
    q[n_ground:] = _quat_mul(qy, qx[None, :])
    opacity = 1.0 / (1.0 + np.exp(-r.normal(n, 0.0, 1.5)))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    if sh_degree == 0:
        sh[:, 0, :] = r.uniform(3 * n).reshape(n, 3)
    else:
        # DC coefficient uniform in [-sqrt(pi), sqrt(pi)] (colour spans [0, 1]
        # with the +0.5 offset); higher orders small and normal.
        sh[:, 0, :] = r.uniform(3 * n, -math.sqrt(math.pi), math.sqrt(math.pi)).reshape(n, 3)
        sh[:, 1:, :] = r.normal(3 * n * (k - 1), 0.0, 0.05).reshape(n, k - 1, 3)
    return Gaussians(mean.astype(np.float32), s.astype(np.float32), q.astype(np.float32),
                     opacity.astype(np.float32), sh.astype(np.float32), sh_degree)


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    w1, x1, y1, z1 = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    w2, x2, y2, z2 = b[:, 0], b[:, 1], b[:, 2], b[:, 3]
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def street_camera(width: int = 1408, height: int = 376, focal: float = 552.0) -> Camera:
    return Camera(width, height, focal, focal, width / 2.0, height / 2.0)


def street_queries(n_queries: int, seed: int = 12):
    """Hidden query poses along the street and a coarse (seed) pose for each,
    within +-1 m / +-3 deg of it.  Returns lists of (x, y, z, yaw) tuples."""
    r = Rng(seed)
    hx = r.uniform(n_queries, -200.0, 200.0)
    hy = r.uniform(n_queries, -3.0, 3.0)
    hyaw = r.uniform(n_queries, -math.radians(10), math.radians(10))
    dx = r.uniform(n_queries, -1.0, 1.0)
    dy = r.uniform(n_queries, -1.0, 1.0)
    dyaw = r.uniform(n_queries, -math.radians(3), math.radians(3))
    hidden = [(hx[i], hy[i], CAMERA_HEIGHT, hyaw[i]) for i in range(n_queries)]
    seeds = [(hx[i] + dx[i], hy[i] + dy[i], CAMERA_HEIGHT, hyaw[i] + dyaw[i]) for i in range(n_queries)]
    return hidden, seeds


def grid_offsets(nx: int, ny: int, nyaw: int, step_xy: float, step_yaw_deg: float) -> np.ndarray:
    """Centred grid of (dx, dy, dyaw_rad) offsets, candidate index
    ix + nx * (iy + ny * iyaw)."""
    out = np.zeros((nx * ny * nyaw, 3))
    for iyaw in range(nyaw):
        for iy in range(ny):
            for ix in range(nx):
                k = ix + nx * (iy + ny * iyaw)
                out[k] = ((ix - (nx - 1) / 2) * step_xy, (iy - (ny - 1) / 2) * step_xy,
                          math.radians((iyaw - (nyaw - 1) / 2) * step_yaw_deg))
    return out


def street_grid_poses(seed_xyzyaw, nx=4, ny=4, nyaw=4, step_xy=0.5, step_yaw_deg=2.0) -> np.ndarray:
    x, y, z, yaw = seed_xyzyaw
    off = grid_offsets(nx, ny, nyaw, step_xy, step_yaw_deg)
    return np.stack([pose_from_xyz_yaw(x + o[0], y + o[1], z, yaw + o[2]) for o in off])


def image_noise(seed: int, height: int, width: int, std: float = 0.02) -> np.ndarray:
    return Rng(seed).normal(3 * height * width, 0.0, std).reshape(3, height, width).astype(np.float32)


def random_image(seed: int, channels: int, height: int, width: int) -> np.ndarray:
    return Rng(seed).uniform(channels * height * width).reshape(channels, height, width).astype(np.float32)
