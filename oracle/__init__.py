"""FP64 CPU oracle of the 3DGS-ReLoc relocalization hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The arithmetic lives in ``reloc_oracle.c`` (plain C, IEEE FP64, OpenMP over
candidate views); this module compiles it with gcc on first use and wraps it
with numpy-facing functions.  Every function cites the passage of the paper it
follows in the C source.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reloc_oracle.c")
_SRC_CNN = os.path.join(_HERE, "cnn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# record layout (mirrors the enum in reloc_oracle.c)
REC_FIELDS = ["visible", "u", "v", "depth", "cov_a", "cov_b", "cov_c", "con_a", "con_b", "con_c",
              "rx", "ry", "r", "g", "b", "opacity", "tx0", "ty0", "tx1", "ty1",
              "det_undil", "det", "tcx", "tcy"]
F = {k: i for i, k in enumerate(REC_FIELDS)}

FLAG_POWER, FLAG_ALPHA, FLAG_T, FLAG_DEPTH = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_CNN))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-Wall", "-Wno-misleading-indentation", "-o", tmp, _SRC, _SRC_CNN, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, fp, i64p = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int64)
            u8p, u32p, u64p, i32p = (C.POINTER(C.c_uint8), C.POINTER(C.c_uint32),
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_int32))
            L.or_rec_stride.restype = C.c_int
            L.or_max_threads.restype = C.c_int
            L.or_quat_to_rot.argtypes = [dp, dp]
            L.or_sh_basis.argtypes = [C.c_int, dp, dp]
            L.or_project.argtypes = [fp, fp, fp, fp, fp, C.c_int, C.c_int64, dp, dp, dp, dp]
            L.or_render.argtypes = [dp, C.c_int64, dp, dp, dp, dp, dp, u8p, dp, C.c_int]
            L.or_render.restype = C.c_int64
            L.or_ncc.argtypes = [dp, dp, C.c_int64, C.POINTER(C.c_int)]
            L.or_ncc.restype = C.c_double
            L.or_argmax.argtypes = [dp, C.c_int]
            L.or_argmax.restype = C.c_int
            L.or_grid_poses.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp]
            L.or_pnp_apply.argtypes = [dp, dp, C.c_double, dp]
            L.or_pnp_residual.argtypes = [dp, dp, dp, dp, dp, dp]
            L.or_pnp_residual.restype = C.c_int
            L.or_refine_pnp.argtypes = [dp, dp, dp, fp, fp, fp, C.c_int64, C.c_int, C.c_double, C.c_double,
                                        C.c_double, dp]
            L.or_pnp_backproject.argtypes = [dp, dp, fp, fp, dp, C.c_int64, C.c_double, dp, u8p]
            L.or_pnp_backproject.restype = C.c_int64
            L.or_ncc_pose_grad.argtypes = [fp, fp, fp, fp, fp, C.c_int64, dp, dp, dp, dp, dp]
            L.or_train_loss_jvp.argtypes = [fp, fp, fp, fp, fp, C.c_int64, dp, dp, C.c_int, dp, dp, dp,
                                            C.c_double, C.c_double, C.c_double, C.c_double, dp]
            L.or_ssim_map.argtypes = [dp, dp, C.c_int, C.c_int, dp]
            L.or_splitmix64.argtypes = [C.c_uint64, C.c_int64, u64p]
            L.or_search_order.argtypes = [C.c_uint64, C.c_int64, i32p]
            L.or_block_select.argtypes = [fp, C.c_int64, C.c_double, C.c_double, C.c_double,
                                          C.c_double, i64p, i64p]
            L.or_block_select.restype = C.c_int64
            L.or_tile_bits.argtypes = [C.c_int]
            L.or_tile_bits.restype = C.c_int
            L.or_tile_keys.argtypes = [C.c_int, C.c_int64, u8p, u32p, i32p, C.c_int, C.c_int, u64p, u32p]
            L.or_tile_keys.restype = C.c_int64
            L.or_tile_ranges.argtypes = [u64p, C.c_int64, C.c_int, C.c_int, i64p]
            L.or_stable_sort_u64.argtypes = [u64p, u32p, C.c_int64]
            L.or_insertion_sort_u64.argtypes = [u64p, u32p, C.c_int64]
            L.or_render_views.argtypes = [fp, fp, fp, fp, fp, C.c_int, C.c_int64, dp, C.c_int, dp, dp,
                                          dp, dp, C.POINTER(C.c_int), dp, dp, dp, u8p, dp, i64p]
            L.orc_param_count.restype = C.c_int64
            L.orc_forward.argtypes = [dp, dp, C.c_int, dp]
            L.orc_forward_ex.argtypes = [dp, dp, C.c_int, dp, C.c_int]
            L.orc_loss_grad.argtypes = [dp, dp, i32p, C.c_int, dp, dp]
            L.orc_loss_grad.restype = C.c_double
            L.orc_loss_grad_ex.argtypes = [dp, dp, i32p, C.c_int, dp, dp, C.c_int]
            L.orc_loss_grad_ex.restype = C.c_double
            L.orc_bf16_round.argtypes = [C.c_double]
            L.orc_bf16_round.restype = C.c_double
            L.orc_adam.argtypes = [dp, dp, dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_int]
            L.orc_downsample_gray.argtypes = [fp, C.c_int, C.c_int, C.c_int, dp]
            L.orc_conv3x3s2.argtypes = [dp, C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, dp]
            _lib = L
    return _lib


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

DEFAULT_PARAMS = dict(near=0.2, fov_clamp=1.3, eps2d=0.3, alpha_min=1.0 / 255.0, alpha_max=0.99,
                      t_min=1e-4, cut=3.0, tile_w=16, tile_h=16,
                      flag_power=1e-5, flag_alpha=1e-5, flag_t=1e-3, flag_depth=1e-6, flag_sig=1e-5,
                      flag_pos=2e-4, ncc_gray=0)
_PORDER = ["near", "fov_clamp", "eps2d", "alpha_min", "alpha_max", "t_min", "cut", "tile_w", "tile_h",
           "flag_power", "flag_alpha", "flag_t", "flag_depth", "flag_sig", "flag_pos", "ncc_gray"]


def params(**over) -> np.ndarray:
    d = dict(DEFAULT_PARAMS)
    for k, v in over.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    out = np.zeros(16)
    for i, k in enumerate(_PORDER):
        out[i] = d[k]
    return out


def camvec(cam) -> np.ndarray:
    return np.array([cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy], dtype=np.float64)


# ---------------------------------------------------------------------------
# wrappers
# ---------------------------------------------------------------------------

def quat_to_rot(q) -> np.ndarray:
    R = np.zeros(9)
    lib().or_quat_to_rot(_p(_c(q, np.float64), C.c_double), _p(R, C.c_double))
    return R.reshape(3, 3)


def sh_basis(deg: int, d) -> np.ndarray:
    Y = np.zeros((deg + 1) ** 2)
    lib().or_sh_basis(deg, _p(_c(d, np.float64), C.c_double), _p(Y, C.c_double))
    return Y


def _gauss_ptrs(g):
    return (_c(g.mean, np.float32), _c(g.scale, np.float32), _c(g.quat, np.float32),
            _c(g.opacity, np.float32), _c(g.sh, np.float32))


def project(g, pose, cam, prm=None) -> np.ndarray:
    """Project every Gaussian of ``g`` for one world-to-camera pose.
    Returns an (N, len(REC_FIELDS)) float64 record array (fields in F)."""
    prm = params() if prm is None else prm
    m, s, q, o, sh = _gauss_ptrs(g)
    recs = np.zeros((g.n, lib().or_rec_stride()))
    lib().or_project(_p(m, C.c_float), _p(s, C.c_float), _p(q, C.c_float), _p(o, C.c_float),
                     _p(sh, C.c_float), g.sh_degree, g.n, _p(_c(pose, np.float64), C.c_double),
                     _p(camvec(cam), C.c_double), _p(_c(prm, np.float64), C.c_double), _p(recs, C.c_double))
    return recs


def render_records(recs, cam, prm=None, brute=False):
    """Composite projected records (index order = tie order).
    Returns dict(rgb (3,H,W), depth (H,W), alpha (H,W), flags (H,W) u8,
    bound (H,W): first-order bound of what a flagged decision can move, n_eval)."""
    prm = params() if prm is None else prm
    recs = _c(recs, np.float64)
    H, W = cam.height, cam.width
    rgb = np.zeros((3, H, W)); depth = np.zeros((H, W)); alpha = np.zeros((H, W))
    flags = np.zeros((H, W), np.uint8)
    bound = np.zeros((H, W))
    ne = lib().or_render(_p(recs, C.c_double), recs.shape[0], _p(camvec(cam), C.c_double),
                         _p(_c(prm, np.float64), C.c_double), _p(rgb, C.c_double), _p(depth, C.c_double),
                         _p(alpha, C.c_double), _p(flags, C.c_uint8), _p(bound, C.c_double), 1 if brute else 0)
    return dict(rgb=rgb, depth=depth, alpha=alpha, flags=flags, bound=bound, n_eval=int(ne))


def render(g, pose, cam, prm=None, brute=False):
    prm = params() if prm is None else prm
    return render_records(project(g, pose, cam, prm), cam, prm, brute)


def render_views(g, poses, cam, prm=None, query=None, images=True, flags=True):
    """Render V views (OpenMP over views); NCC against ``query`` if given.
    Returns dict(scores, degenerate, rgb, depth, alpha, flags, counts)."""
    prm = params() if prm is None else prm
    poses = _c(poses, np.float64).reshape(-1, 16)
    V = poses.shape[0]
    H, W = cam.height, cam.width
    m, s, q, o, sh = _gauss_ptrs(g)
    out = dict(counts=np.zeros((V, 3), np.int64))
    if images:
        out["rgb"] = np.zeros((V, 3, H, W)); out["depth"] = np.zeros((V, H, W)); out["alpha"] = np.zeros((V, H, W))
    if flags:
        out["flags"] = np.zeros((V, H, W), np.uint8)
        out["bound"] = np.zeros((V, H, W))
    qd = None
    if query is not None:
        qd = _c(query, np.float64).reshape(-1)
        out["scores"] = np.zeros(V); out["degenerate"] = np.zeros(V, np.int32)
    lib().or_render_views(_p(m, C.c_float), _p(s, C.c_float), _p(q, C.c_float), _p(o, C.c_float),
                          _p(sh, C.c_float), g.sh_degree, g.n, _p(poses, C.c_double), V,
                          _p(camvec(cam), C.c_double), _p(_c(prm, np.float64), C.c_double),
                          _p(qd, C.c_double), _p(out.get("scores"), C.c_double),
                          _p(out.get("degenerate"), C.c_int), _p(out.get("rgb"), C.c_double),
                          _p(out.get("depth"), C.c_double), _p(out.get("alpha"), C.c_double),
                          _p(out.get("flags"), C.c_uint8), _p(out.get("bound"), C.c_double),
                          _p(out["counts"], C.c_int64))
    return out


def ncc(a, b):
    a = _c(a, np.float64).reshape(-1)
    b = _c(b, np.float64).reshape(-1)
    dg = C.c_int(0)
    val = lib().or_ncc(_p(a, C.c_double), _p(b, C.c_double), a.size, C.byref(dg))
    return val, bool(dg.value)


def argmax(scores) -> int:
    s = _c(scores, np.float64)
    return int(lib().or_argmax(_p(s, C.c_double), s.size))


def grid_poses(seed_pose, nx, ny, nyaw, step_xy, step_yaw_deg) -> np.ndarray:
    out = np.zeros((nx * ny * nyaw, 16))
    lib().or_grid_poses(_p(_c(seed_pose, np.float64).reshape(16), C.c_double), nx, ny, nyaw,
                        step_xy, step_yaw_deg, _p(out, C.c_double))
    return out.reshape(-1, 4, 4)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 started at ``seed``."""
    out = np.zeros(count, np.uint64)
    lib().or_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, count, _p(out, C.c_uint64))
    return out


def search_order(seed: int, n: int) -> np.ndarray:
    """Visiting order of the random search (Sec. IV-A): cells 0..n-1 shuffled
    by Fisher-Yates driven by SplitMix64(seed)."""
    out = np.zeros(n, np.int32)
    lib().or_search_order(seed & 0xFFFFFFFFFFFFFFFF, n, _p(out, C.c_int32))
    return out


def visit_count(fraction: float, n_cells: int) -> int:
    """Cells a random search visits: ceil(fraction * n_cells) in double precision."""
    return min(n_cells, int(math.ceil(fraction * n_cells)))


def random_search(g, cell_poses, cam, query, order, batch, ncc_stop, prm=None):
    """Random search with early stop (Sec. IV-A), FP64: render and score the
    cells of ``order`` in consecutive batches of ``batch``; after each batch,
    stop if the best NCC so far is >= ncc_stop.  The best cell is the visited
    cell with the highest NCC, the lowest cell index on ties.
    Returns dict(best_index, best_score, n_scored, stopped_early, scores) with
    NaN scores for cells not visited."""
    order = np.asarray(order, np.int64)
    scores = np.full(len(cell_poses), np.nan)
    best, best_sc, visited, stopped = -1, -np.inf, 0, False
    for b0 in range(0, len(order), batch):
        cells = order[b0:b0 + batch]
        out = render_views(g, np.asarray(cell_poses)[cells], cam, prm, query=query, images=False, flags=False)
        for c, sc in zip(cells, out["scores"]):
            scores[c] = sc
            if sc > best_sc or (sc == best_sc and c < best):
                best, best_sc = int(c), float(sc)
        visited += len(cells)
        if best_sc >= ncc_stop:
            stopped = visited < len(order)
            break
    return dict(best_index=best, best_score=best_sc, n_scored=visited, stopped_early=stopped, scores=scores)


def ncc_pose_grad(g, pose, cam, query, prm=None):
    """NCC of the view at ``pose`` against ``query`` and its gradient with
    respect to the left pose update (rho, phi), by forward-mode
    differentiation in FP64 (SH degree 0 maps).  Returns (ncc, grad[6])."""
    if g.sh_degree != 0:
        raise ValueError("pose gradients need view-independent colour (SH degree 0)")
    prm = params() if prm is None else prm
    m, s, q, o, sh = _gauss_ptrs(g)
    out = np.zeros(7)
    lib().or_ncc_pose_grad(_p(m, C.c_float), _p(s, C.c_float), _p(q, C.c_float), _p(o, C.c_float),
                           _p(sh, C.c_float), g.n, _p(_c(pose, np.float64).reshape(16), C.c_double),
                           _p(camvec(cam), C.c_double), _p(_c(prm, np.float64), C.c_double),
                           _p(_c(query, np.float64).reshape(-1), C.c_double), _p(out, C.c_double))
    return out[0], out[1:]


PARAM_ORDER = ["mean_x", "mean_y", "mean_z", "scale_x", "scale_y", "scale_z", "quat_w", "quat_x", "quat_y",
               "quat_z", "opacity", "red", "green", "blue"]


def train_loss_jvp(g, poses, cam, gt, dirs, prm=None, lam=0.0, w_photo=1.0, w_reproj=0.0, alpha_min=0.5):
    """Map-training loss of Sec. III-B.3 (Eq. 6: w_photo L_photo + w_reproj
    L_reproj, each an L_rgb of Eq. 3: (1 - lam) mean |x - y| + lam (1 - mean
    SSIM); L_photo over the views' renders, L_reproj over consecutive view
    pairs, I_{t+1} re-projected into view t through the rendered depth D / A
    where A >= alpha_min) and its derivatives along six directions dirs
    [n, 14, 6] in the Gaussians' parameters (PARAM_ORDER), forward mode in
    FP64 (SH degree 0).  Returns (loss, jvp[6])."""
    if g.sh_degree != 0:
        raise ValueError("map training needs SH degree 0")
    prm = params() if prm is None else prm
    m, s, q, o, sh = _gauss_ptrs(g)
    poses = _c(poses, np.float64).reshape(-1, 16)
    out = np.zeros(7)
    lib().or_train_loss_jvp(_p(m, C.c_float), _p(s, C.c_float), _p(q, C.c_float), _p(o, C.c_float),
                            _p(sh, C.c_float), g.n, _p(_c(dirs, np.float64), C.c_double),
                            _p(poses, C.c_double), poses.shape[0], _p(camvec(cam), C.c_double),
                            _p(_c(prm, np.float64), C.c_double), _p(_c(gt, np.float64), C.c_double),
                            float(lam), float(w_photo), float(w_reproj), float(alpha_min), _p(out, C.c_double))
    return out[0], out[1:]


def map_params(g) -> np.ndarray:
    """The Gaussians' 14 training parameters per row, in PARAM_ORDER (FP64)."""
    if g.sh_degree != 0:
        raise ValueError("map training needs SH degree 0")
    return np.concatenate([g.mean, g.scale, g.quat, g.opacity[:, None], g.sh[:, 0, :]], 1).astype(np.float64)


def adam_step(prm, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-15, o_min=1e-6):
    """One Adam step (Kingma and Ba 2015, Algorithm 1) on 3D Gaussian
    Splatting's latent parameters of a [n, 14] parameter array (PARAM_ORDER,
    activated values): the scale through its log (s = exp(l), dL/dl = s dL/ds),
    the opacity through its logit (o = sigmoid(z), o first clamped to
    [o_min, 1 - o_min], dL/dz = o (1 - o) dL/do), mean, quaternion and colour
    as they are.  lr = (mean, scale, quaternion, opacity, colour); t = the step
    number (1 for the first).  Returns (params, m, v), FP64."""
    prm = np.asarray(prm, np.float64)
    g = np.asarray(grad, np.float64).copy()
    group = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 4, 4])
    o = np.clip(prm[:, 10], o_min, 1.0 - o_min)
    g[:, 3:6] *= prm[:, 3:6]
    g[:, 10] *= o * (1.0 - o)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    step = np.asarray(lr, np.float64)[group][None, :] * mhat / (np.sqrt(vhat) + eps)
    out = prm.copy()
    for c in (0, 1, 2, 6, 7, 8, 9, 11, 12, 13):
        out[:, c] = prm[:, c] - step[:, c]
    out[:, 3:6] = prm[:, 3:6] * np.exp(-step[:, 3:6])
    z = np.log(o / (1.0 - o)) - step[:, 10]
    out[:, 10] = 1.0 / (1.0 + np.exp(-z))
    return out, m, v


def photo_loss_jvp(g, poses, cam, gt, dirs, prm=None, lam=0.0):
    """L_photo alone (Eqs. 3-4): train_loss_jvp with w_photo = 1, w_reproj = 0."""
    return train_loss_jvp(g, poses, cam, gt, dirs, prm, lam=lam, w_photo=1.0, w_reproj=0.0)


def ssim_map(x, y):
    """SSIM of one channel at every pixel (Eq. 3's D-SSIM term): x, y [H, W]."""
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    if x.shape != y.shape or x.ndim != 2:
        raise ValueError("x and y must be equal-sized 2D arrays")
    out = np.zeros_like(x)
    lib().or_ssim_map(_p(x, C.c_double), _p(y, C.c_double), x.shape[0], x.shape[1], _p(out, C.c_double))
    return out


def pnp_apply(pose, delta, s=1.0):
    """pose updated on the left by s * delta, delta = (rho, phi)."""
    out = np.zeros(16)
    lib().or_pnp_apply(_p(_c(pose, np.float64).reshape(16), C.c_double), _p(_c(delta, np.float64), C.c_double),
                       s, _p(out, C.c_double))
    return out.reshape(4, 4)


def pnp_residual(pose, X, cam, q):
    """Reprojection residual (2) and its Jacobian (2 x 6) w.r.t. the left update
    at zero; None if the point is not in front of the camera."""
    r, J = np.zeros(2), np.zeros(12)
    ok = lib().or_pnp_residual(_p(_c(pose, np.float64).reshape(16), C.c_double),
                               _p(_c(X, np.float64), C.c_double), _p(camvec(cam), C.c_double),
                               _p(_c(q, np.float64), C.c_double), _p(r, C.c_double), _p(J, C.c_double))
    return (r, J.reshape(2, 6)) if ok else None


def pnp_backproject(pose_render, cam, depth, alpha, uv, alpha_min=0.5):
    """World points of render pixels uv [n, 2] from the view's depth D / A
    (bilinear); returns (X [n, 3], used [n] bool)."""
    uv = _c(uv, np.float64).reshape(-1, 2)
    X = np.zeros((uv.shape[0], 3))
    use = np.zeros(uv.shape[0], np.uint8)
    lib().or_pnp_backproject(_p(_c(pose_render, np.float64).reshape(16), C.c_double), _p(camvec(cam), C.c_double),
                             _p(_c(depth, np.float32), C.c_float), _p(_c(alpha, np.float32), C.c_float),
                             _p(uv, C.c_double), uv.shape[0], alpha_min, _p(X, C.c_double), _p(use, C.c_uint8))
    return X, use.astype(bool)


def refine_pnp(pose_render, cam, depth, alpha, pairs, pose_init=None, max_iters=30, huber_px=2.0,
               alpha_min=0.5, tol=1e-12):
    """PnP refinement (Sec. III-C.2) in FP64: depth, alpha [H, W] and pairs [n, 4]
    (u_r, v_r, u_q, v_q) float32.  Returns dict(pose, rms_px, cost, n_used, iters)."""
    pr = _c(pose_render, np.float64).reshape(16)
    pi = pr if pose_init is None else _c(pose_init, np.float64).reshape(16)
    d, a, p = _c(depth, np.float32), _c(alpha, np.float32), _c(pairs, np.float32)
    out = np.zeros(20)
    lib().or_refine_pnp(_p(pr, C.c_double), _p(pi, C.c_double), _p(camvec(cam), C.c_double), _p(d, C.c_float),
                        _p(a, C.c_float), _p(p, C.c_float), p.shape[0], max_iters, huber_px, alpha_min, tol,
                        _p(out, C.c_double))
    return dict(pose=out[:16].reshape(4, 4), rms_px=out[16], cost=out[17], n_used=int(out[18]), iters=int(out[19]))


def block_select(means, block_size, cx, cy, radius):
    """Original indices of the Gaussians in every block whose centre is within
    ``radius`` of (cx, cy), ordered by block key then index; and the block count."""
    m = _c(means, np.float32)
    n = m.shape[0]
    idx = np.zeros(n, np.int64)
    nb = C.c_int64(0)
    cnt = lib().or_block_select(_p(m, C.c_float), n, block_size, cx, cy, radius, _p(idx, C.c_int64),
                                C.byref(nb))
    return idx[:cnt], int(nb.value)


def tile_bits(n_tiles: int) -> int:
    return int(lib().or_tile_bits(n_tiles))


def tile_keys(vis, dbits, rect, ntx, nty):
    """vis (V,N) u8, dbits (V,N) u32, rect (V,N,4) i32 -> (keys u64, vals u32) in emission order."""
    vis = _c(vis, np.uint8); dbits = _c(dbits, np.uint32); rect = _c(rect, np.int32)
    V, N = vis.shape
    L = lib()
    cnt = L.or_tile_keys(V, N, _p(vis, C.c_uint8), _p(dbits, C.c_uint32), _p(rect, C.c_int32), ntx, nty,
                         None, None)
    keys = np.zeros(cnt, np.uint64); vals = np.zeros(cnt, np.uint32)
    L.or_tile_keys(V, N, _p(vis, C.c_uint8), _p(dbits, C.c_uint32), _p(rect, C.c_int32), ntx, nty,
                   _p(keys, C.c_uint64), _p(vals, C.c_uint32))
    return keys, vals


def stable_sort(keys, vals, insertion=False):
    k = _c(keys, np.uint64).copy(); v = _c(vals, np.uint32).copy()
    fn = lib().or_insertion_sort_u64 if insertion else lib().or_stable_sort_u64
    fn(_p(k, C.c_uint64), _p(v, C.c_uint32), k.size)
    return k, v


def tile_ranges(keys, n_views, n_tiles):
    k = _c(keys, np.uint64)
    r = np.zeros((n_views, n_tiles, 2), np.int64)
    lib().or_tile_ranges(_p(k, C.c_uint64), k.size, n_views, n_tiles, _p(r, C.c_int64))
    return r


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---------------------------------------------------------------------------
# learned candidate proposal (cnn_oracle.c)
# ---------------------------------------------------------------------------

CNN_IN = (47, 176, 2)


def cnn_param_count() -> int:
    return int(lib().orc_param_count())


def bf16_round(x: float) -> float:
    """Round to nearest even BF16 of the FP32 value of x (the oracle's rounding)."""
    return float(lib().orc_bf16_round(float(x)))


def cnn_forward(params, inputs, act_bf16=False) -> np.ndarray:
    """logits [B][64] of inputs [B][47][176][2] (FP64); act_bf16: every stored
    activation rounded to BF16 (the BF16 network's storage format)."""
    p = _c(params, np.float64)
    x = _c(inputs, np.float64)
    B = x.shape[0]
    out = np.zeros((B, 64))
    lib().orc_forward_ex(_p(p, C.c_double), _p(x, C.c_double), B, _p(out, C.c_double), 1 if act_bf16 else 0)
    return out


def cnn_loss_grad(params, inputs, labels, want_input_grad=False, act_bf16=False):
    """(mean softmax cross-entropy, gradient w.r.t. params [, w.r.t. inputs]);
    act_bf16: activations stored in BF16, the chain rule at those values."""
    p = _c(params, np.float64)
    x = _c(inputs, np.float64)
    y = _c(labels, np.int32)
    g = np.zeros(p.size)
    gi = np.zeros(x.shape) if want_input_grad else None
    loss = lib().orc_loss_grad_ex(_p(p, C.c_double), _p(x, C.c_double), _p(y, C.c_int32), x.shape[0],
                                  _p(g, C.c_double), _p(gi, C.c_double), 1 if act_bf16 else 0)
    return (float(loss), g, gi) if want_input_grad else (float(loss), g)


def adam(w, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    w = _c(w, np.float64).copy(); m = _c(m, np.float64).copy(); v = _c(v, np.float64).copy()
    gg = _c(g, np.float64)
    lib().orc_adam(_p(w, C.c_double), _p(m, C.c_double), _p(v, C.c_double), _p(gg, C.c_double), w.size, lr, b1, b2,
                   eps, t)
    return w, m, v


def downsample_gray(img, f) -> np.ndarray:
    a = _c(img, np.float32)
    _, H, W = a.shape
    out = np.zeros((H // f, W // f))
    lib().orc_downsample_gray(_p(a, C.c_float), H, W, f, _p(out, C.c_double))
    return out


def conv3x3s2(x, w, b):
    """One conv layer of the proposal (+ bias, ReLU): x [H][W][Ci], w [Co][3][3][Ci]."""
    xx = _c(x, np.float64); ww = _c(w, np.float64); bb = _c(b, np.float64)
    H, W, Ci = xx.shape
    Co = ww.shape[0]
    y = np.zeros(((H - 1) // 2 + 1, (W - 1) // 2 + 1, Co))
    lib().orc_conv3x3s2(_p(xx, C.c_double), H, W, Ci, _p(ww, C.c_double), _p(bb, C.c_double), Co, _p(y, C.c_double))
    return y


def cnn_offsets():
    """(w_offset, b_offset, w_shape) of the 7 parameter tensors in the flat layout."""
    cin, cout = [2, 32, 64, 64, 128], [32, 64, 64, 128, 128]
    out, o = [], 0
    for l in range(5):
        shape = (cout[l], 3, 3, cin[l])
        n = int(np.prod(shape))
        out.append((o, o + n, shape)); o += n + cout[l]
    for shape in [(1024, 1536), (64, 1024)]:
        n = shape[0] * shape[1]
        out.append((o, o + n, shape)); o += n + shape[0]
    return out
