"""Python binding of the C ABI in include/reloc.h (ctypes; marshalling only).

Every function here forwards to the CUDA library ``_lib/libreloc.so``.
There is no fallback: if the library is missing or fails to load, importing
this module raises.  Device buffers are passed as torch CUDA tensors (their
data pointers) and the stream as torch's current stream handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libreloc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOMAP, ENUMERIC, EOVERFLOW = range(8)
FP32, FP16, BF16 = 0, 1, 2
STAGES = ["cull", "project", "depth_sort", "tile_count", "tile_emit", "blend", "score"]


class RelocError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"reloc status {status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_plane", C.c_float),
                ("fov_clamp", C.c_float), ("eps2d", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("t_min", C.c_float), ("cut", C.c_float), ("det_fp64", C.c_float),
                ("block_size", C.c_double), ("inst_capacity", C.c_int64), ("blend_rpl", C.c_int32),
                ("ncc_gray", C.c_int32), ("reserved", C.c_int32 * 6)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]


class GaussiansHost(C.Structure):
    _fields_ = [("mean", C.POINTER(C.c_float)), ("scale", C.POINTER(C.c_float)),
                ("quat", C.POINTER(C.c_float)), ("opacity", C.POINTER(C.c_float)),
                ("sh", C.POINTER(C.c_float))]


class Range(C.Structure):
    _fields_ = [("begin", C.c_int64), ("end", C.c_int64)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nyaw", C.c_int32), ("step_xy", C.c_double),
                ("step_yaw_deg", C.c_double)]


class Query(C.Structure):
    _fields_ = [("query_dev", C.c_void_p), ("coarse_pose", C.c_double * 16), ("radius", C.c_double),
                ("grid", Grid)]


class BatchOptions(C.Structure):
    _fields_ = [("use_graph", C.c_int32), ("reserved0", C.c_int32), ("mem_budget", C.c_int64),
                ("reserved", C.c_int32 * 8)]


class TuneResult(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("blend_rpl", C.c_int32), ("from_table", C.c_int32),
                ("ms_per_query", C.c_double), ("n_tried", C.c_int32), ("reserved", C.c_int32 * 5)]


class Result(C.Structure):
    _fields_ = [("best_index", C.c_int32), ("n_candidates", C.c_int32), ("best_score", C.c_double),
                ("best_pose", C.c_double * 16), ("n_gauss", C.c_int64), ("n_blocks", C.c_int32),
                ("degenerate", C.c_int32), ("n_scored", C.c_int32), ("stopped_early", C.c_int32)]


class Search(C.Structure):
    _fields_ = [("fraction", C.c_double), ("ncc_stop", C.c_double), ("batch", C.c_int32), ("n_order", C.c_int32),
                ("seed", C.c_uint64), ("order", C.c_void_p), ("reserved", C.c_int32 * 4)]


class PnpOptions(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("reserved0", C.c_int32), ("huber_px", C.c_double),
                ("alpha_min", C.c_double), ("tol", C.c_double), ("reserved", C.c_int32 * 4)]


class PnpResult(C.Structure):
    _fields_ = [("pose", C.c_double * 16), ("rms_px", C.c_double), ("cost", C.c_double), ("n_used", C.c_int32),
                ("iters", C.c_int32), ("reserved", C.c_int32 * 2)]


class TrainOptions(C.Structure):
    _fields_ = [("lambda_dssim", C.c_double), ("w_photo", C.c_double), ("w_reproj", C.c_double),
                ("lr_mean", C.c_double), ("lr_scale", C.c_double), ("lr_quat", C.c_double),
                ("lr_opacity", C.c_double), ("lr_color", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("reproj_alpha_min", C.c_double), ("views_per_group", C.c_int32),
                ("reserved", C.c_int32 * 7)]


class Counts(C.Structure):
    _fields_ = [("n_views", C.c_int64), ("n_gauss", C.c_int64), ("n_visible", C.c_int64),
                ("n_instances", C.c_int64), ("inst_stride", C.c_int64), ("retries", C.c_int32),
                ("kernel_launches", C.c_int32)]


# exported symbols and their signatures (name -> (restype, argtypes))
_vp, _dp, _fp, _ip, _i64p, _u32p, _i32p = (C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float),
                                           C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_int32))
SIGNATURES = {
    "reloc_version": (C.c_char_p, []),
    "reloc_last_error": (C.c_char_p, []),
    "reloc_default_config": (None, [C.POINTER(Config)]),
    "reloc_create": (C.c_int, [C.POINTER(Config), C.c_int, C.POINTER(_vp)]),
    "reloc_destroy": (C.c_int, [_vp]),
    "reloc_load_map": (C.c_int, [_vp, C.POINTER(GaussiansHost), C.c_int64, C.c_int, C.c_int]),
    "reloc_map_order": (C.c_int, [_vp, _i64p]),
    "reloc_select_block": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.POINTER(Range), C.c_int, _ip,
                                     _i64p, _ip]),
    "reloc_render": (C.c_int, [_vp, C.POINTER(Range), C.c_int, _dp, C.c_int, C.POINTER(Camera), _vp, _vp, _vp,
                               _vp]),
    "reloc_score": (C.c_int, [_vp, C.POINTER(Range), C.c_int, _dp, C.c_int, C.POINTER(Camera), _vp, _dp, _ip,
                              _vp]),
    "reloc_score_grad": (C.c_int, [_vp, C.POINTER(Range), C.c_int, _dp, C.c_int, C.POINTER(Camera), _vp, _dp, _dp,
                                   _vp]),
    "reloc_localize": (C.c_int, [_vp, _vp, _dp, C.c_double, C.POINTER(Grid), C.POINTER(Camera), C.POINTER(Result),
                                 _dp, _vp, _vp, _vp, _vp]),
    "reloc_localize_random": (C.c_int, [_vp, _vp, _dp, C.c_double, C.POINTER(Grid), C.POINTER(Camera),
                                        C.POINTER(Search), C.POINTER(Result), _dp, _vp, _vp, _vp, _vp]),
    "reloc_localize_host": (C.c_int, [_vp, _vp, _dp, C.c_double, C.POINTER(Grid), C.POINTER(Camera),
                                      C.POINTER(Result), _vp, _vp, _vp]),
    "reloc_localize_batch": (C.c_int, [_vp, C.POINTER(Query), C.c_int, C.POINTER(Camera), C.POINTER(Result), _dp,
                                       _vp, _vp, _vp]),
    "reloc_set_batch_options": (C.c_int, [_vp, C.POINTER(BatchOptions)]),
    "reloc_autotune": (C.c_int, [_vp, C.POINTER(Query), C.c_int, C.POINTER(Camera), C.c_char_p, C.c_int,
                                 C.POINTER(TuneResult), _vp]),
    "reloc_proposal_init": (C.c_int, [_vp, C.c_uint64]),
    "reloc_proposal_get": (C.c_int, [_vp, C.c_int, _fp]),
    "reloc_proposal_set_params": (C.c_int, [_vp, _fp]),
    "reloc_proposal_make_input": (C.c_int, [_vp, _vp, _vp, C.POINTER(Camera), _vp, _vp]),
    "reloc_proposal_forward": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp]),
    "reloc_proposal_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_float, C.c_int, _fp, _vp]),
    "reloc_set_proposal": (C.c_int, [_vp, C.c_int, C.c_int, C.c_float]),
    "reloc_gemm_bf16": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp]),
    "reloc_last_counts": (C.c_int, [_vp, C.POINTER(Counts)]),
    "reloc_set_profiling": (C.c_int, [_vp, C.c_int]),
    "reloc_stage_times": (C.c_int, [_vp, _dp, _i64p]),
    "reloc_export_debug": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i64p, _vp, _vp]),
    "reloc_ncc_images_noalloc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
    "reloc_measure_peaks": (C.c_int, [C.c_int, _dp, _dp, _dp]),
    "reloc_default_pnp_options": (None, [C.POINTER(PnpOptions)]),
    "reloc_refine_pnp": (C.c_int, [_vp, _dp, _dp, C.POINTER(Camera), _vp, _vp, _vp, C.c_int, C.POINTER(PnpOptions),
                                   C.POINTER(PnpResult), _vp]),
    "reloc_default_train_options": (None, [C.POINTER(TrainOptions)]),
    "reloc_train_grad": (C.c_int, [_vp, C.POINTER(Range), C.c_int, _dp, C.c_int, C.POINTER(Camera), _vp,
                                   C.POINTER(TrainOptions), _dp, _vp, _vp]),
    "reloc_train_step": (C.c_int, [_vp, C.POINTER(Range), C.c_int, _dp, C.c_int, C.POINTER(Camera), _vp,
                                   C.POINTER(TrainOptions), _dp, _vp]),
    "reloc_train_reset": (C.c_int, [_vp]),
    "reloc_read_map": (C.c_int, [_vp, _fp, _fp, _fp, _fp, _fp]),
    "reloc_inject_faults": (C.c_int, [C.c_int, C.c_int]),
}
NOALLOC_MAX_VIEWS = 512
PROPOSAL_H, PROPOSAL_W, PROPOSAL_CLASSES, PROPOSAL_PARAMS = 47, 176, 64, 1916960


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libreloc.so not built ({LIB_PATH}); run paper_2403_11367_gb300/build.py "
                          "or __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status):
    if status != OK:
        raise RelocError(status, lib.reloc_last_error().decode())


_F32, _F64, _I32, _U16 = ("float32",), ("float64",), ("int32",), ("bfloat16", "int16", "uint16")


def _ptr(t, dtype=None, numel=None, shape=None, name="buffer"):
    """Device pointer of a torch CUDA tensor (or None), after checking what the
    C call will read or write through it: its dtype (one of the names in
    ``dtype``), its exact shape or at least ``numel`` elements, contiguity and
    placement on the current CUDA device.  A wrong buffer raises ValueError
    here, before any launch could read or write past it."""
    if t is None:
        return None
    if dtype is not None and str(t.dtype).replace("torch.", "") not in dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {' or '.join(dtype)}")
    if shape is not None and tuple(t.shape) != tuple(int(x) for x in shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(int(x) for x in shape)}")
    if numel is not None and t.numel() < int(numel):
        raise ValueError(f"{name}: {t.numel()} elements, at least {int(numel)} needed")
    if not t.is_contiguous():
        raise ValueError(f"{name}: device buffers must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name}: device buffers must be CUDA tensors")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")
    return C.c_void_p(t.data_ptr())


def _qptr(q, c, name="query"):
    """A [3][H][W] float32 image on the device for camera c."""
    return _ptr(q, _F32, shape=(3, c.height, c.width), name=name)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _poses(poses):
    p = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 16)
    return p, p.ctypes.data_as(_dp), p.shape[0]


def camera(cam) -> Camera:
    return Camera(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy))


def reloc_version() -> str:
    return lib.reloc_version().decode()


def reloc_ncc_images_noalloc(images, query, scores_out, degenerate_out=None, stream=None):
    """NCC of rendered images [V,3,H,W] against query [3,H,W] into scores_out
    [V] (float64) and degenerate_out [V] (int32), all CUDA tensors; the library
    allocates nothing for this call (see include/reloc.h)."""
    if images.dim() != 4 or images.shape[1] != 3:
        raise ValueError(f"images: shape {tuple(images.shape)}, expected (V, 3, H, W)")
    V, _, H, W = images.shape
    _check(lib.reloc_ncc_images_noalloc(_ptr(images, _F32, name="images"), V, H, W,
                                        _ptr(query, _F32, shape=(3, H, W), name="query"),
                                        _ptr(scores_out, _F64, numel=V, name="scores_out"),
                                        _ptr(degenerate_out, _I32, numel=V, name="degenerate_out"), _stream(stream)))


FAULT_GEMM_WAIT, FAULT_ALLOC = 1, 2


def reloc_inject_faults(kind: int, count: int = 1):
    """Test hook: make the next `count` GEMM launches' tensor-core waits run out
    (FAULT_GEMM_WAIT) or the next `count` device allocations fail (FAULT_ALLOC)."""
    _check(lib.reloc_inject_faults(kind, count))


def reloc_measure_peaks(device: int = 0) -> dict:
    """Measured FP32 FMA (scalar, packed f32x2) TFLOP/s and ex2 G/s of a device."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib.reloc_measure_peaks(device, C.byref(a), C.byref(b), C.byref(c)))
    return {"fp32_scalar_tflops": a.value, "fp32_packed_tflops": b.value, "ex2_gops": c.value}


def reloc_default_config(**over) -> Config:
    cfg = Config()
    lib.reloc_default_config(C.byref(cfg))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


class Context:
    """Owns one reloc_ctx.  Method names follow the C ABI without the prefix."""

    def __init__(self, cfg: Config | None = None, device: int = 0):
        self._h = _vp()
        _check(lib.reloc_create(C.byref(cfg) if cfg is not None else None, device, C.byref(self._h)))
        self.n = 0
        self._cfg = cfg if cfg is not None else reloc_default_config()
        self._cam = None                 # camera of the last rendering call (export_debug sizes)

    def close(self):
        if self._h:
            lib.reloc_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- map ------------------------------------------------------------------
    def load_map(self, g, precision: int = FP32):
        self._keep = [_f32(g.mean), _f32(g.scale), _f32(g.quat), _f32(g.opacity), _f32(g.sh)]
        m, s, q, o, sh = self._keep
        gh = GaussiansHost(*(a.ctypes.data_as(_fp) for a in (m, s, q, o, sh)))
        _check(lib.reloc_load_map(self._h, C.byref(gh), g.n, g.sh_degree, precision))
        self._keep = None
        self.n = g.n
        self.sh_degree = g.sh_degree

    def map_order(self) -> np.ndarray:
        out = np.zeros(self.n, np.int64)
        _check(lib.reloc_map_order(self._h, out.ctypes.data_as(_i64p)))
        return out

    def select_block(self, x, y, radius, max_ranges=4096):
        rng = (Range * max_ranges)()
        nr, ng, nb = C.c_int(0), C.c_int64(0), C.c_int(0)
        _check(lib.reloc_select_block(self._h, x, y, radius, rng, max_ranges, C.byref(nr), C.byref(ng),
                                      C.byref(nb)))
        return [(rng[i].begin, rng[i].end) for i in range(nr.value)], int(ng.value), int(nb.value)

    @staticmethod
    def _ranges(ranges):
        arr = (Range * max(1, len(ranges)))(*[Range(int(b), int(e)) for b, e in ranges])
        return arr, len(ranges)

    # -- hot path ---------------------------------------------------------------
    def render(self, ranges, poses, cam, rgb=None, depth=None, alpha=None, stream=None):
        ra, nr = self._ranges(ranges)
        p, pp, V = _poses(poses)
        c = camera(cam)
        hw = c.height * c.width
        self._cam = c
        _check(lib.reloc_render(self._h, ra, nr, pp, V, C.byref(c), _ptr(rgb, _F32, V * 3 * hw, name="rgb"),
                                _ptr(depth, _F32, V * hw, name="depth"), _ptr(alpha, _F32, V * hw, name="alpha"),
                                _stream(stream)))

    def score(self, ranges, poses, cam, query, stream=None):
        ra, nr = self._ranges(ranges)
        p, pp, V = _poses(poses)
        c = camera(cam)
        sc = np.zeros(V)
        dg = np.zeros(V, np.int32)
        self._cam = c
        _check(lib.reloc_score(self._h, ra, nr, pp, V, C.byref(c), _qptr(query, c), sc.ctypes.data_as(_dp),
                               dg.ctypes.data_as(_ip), _stream(stream)))
        return sc, dg

    def localize(self, query, coarse_pose, radius, grid, cam, best_rgb=None, best_depth=None, best_alpha=None,
                 stream=None, want_scores=True):
        cp = np.ascontiguousarray(coarse_pose, np.float64).reshape(16)
        g = Grid(*grid) if not isinstance(grid, Grid) else grid
        c = camera(cam)
        res = Result()
        V = g.nx * g.ny * g.nyaw
        sc = np.zeros(V) if want_scores else None
        hw = c.height * c.width
        self._cam = c
        _check(lib.reloc_localize(self._h, _qptr(query, c), cp.ctypes.data_as(_dp), radius, C.byref(g), C.byref(c),
                                  C.byref(res), sc.ctypes.data_as(_dp) if sc is not None else None,
                                  _ptr(best_rgb, _F32, 3 * hw, name="best_rgb"),
                                  _ptr(best_depth, _F32, hw, name="best_depth"),
                                  _ptr(best_alpha, _F32, hw, name="best_alpha"), _stream(stream)))
        return res, sc

    def localize_random(self, query, coarse_pose, radius, grid, cam, fraction=0.2, ncc_stop=float("inf"), batch=64,
                        seed=0, order=None, best_rgb=None, best_depth=None, best_alpha=None, stream=None,
                        want_scores=True):
        """Random search with early stop over the grid's cells (include/reloc.h).
        order: optional explicit visiting order (cell indices).  Returns
        (Result, scores per cell with NaN for unvisited cells, or None)."""
        cp = np.ascontiguousarray(coarse_pose, np.float64).reshape(16)
        g = Grid(*grid) if not isinstance(grid, Grid) else grid
        c = camera(cam)
        opt = Search()
        opt.fraction, opt.ncc_stop, opt.batch, opt.seed = float(fraction), float(ncc_stop), int(batch), int(seed)
        ordr = None
        if order is not None:
            ordr = np.ascontiguousarray(order, np.int32)
            opt.order, opt.n_order = ordr.ctypes.data, len(ordr)
        res = Result()
        n = g.nx * g.ny * g.nyaw
        sc = np.zeros(n) if want_scores else None
        hw = c.height * c.width
        self._cam = c
        _check(lib.reloc_localize_random(self._h, _qptr(query, c), cp.ctypes.data_as(_dp), radius, C.byref(g),
                                         C.byref(c), C.byref(opt), C.byref(res),
                                         sc.ctypes.data_as(_dp) if sc is not None else None,
                                         _ptr(best_rgb, _F32, 3 * hw, name="best_rgb"),
                                         _ptr(best_depth, _F32, hw, name="best_depth"),
                                         _ptr(best_alpha, _F32, hw, name="best_alpha"), _stream(stream)))
        return res, sc

    def score_grad(self, ranges, poses, cam, query, stream=None):
        """NCC of each view and its gradient w.r.t. the view's pose (rho, phi):
        returns (scores [V], grads [V, 6])."""
        ra, nr = self._ranges(ranges)
        p, pp, V = _poses(poses)
        c = camera(cam)
        sc = np.zeros(V)
        gr = np.zeros((V, 6))
        self._cam = c
        _check(lib.reloc_score_grad(self._h, ra, nr, pp, V, C.byref(c), _qptr(query, c), sc.ctypes.data_as(_dp),
                                    gr.ctypes.data_as(_dp), _stream(stream)))
        return sc, gr

    @staticmethod
    def train_options(**opts) -> TrainOptions:
        o = TrainOptions()
        lib.reloc_default_train_options(C.byref(o))
        for k, v in opts.items():
            if k not in dict(TrainOptions._fields_):
                raise TypeError(f"unknown training option {k}")
            setattr(o, k, v)
        return o

    def train_grad(self, ranges, poses, cam, targets, grad, stream=None, **opts):
        """Map-training loss (Sec. III-B.3) over the views at poses [V,4,4]
        against targets [V,3,H,W] (CUDA float32); its gradient is written to
        grad [14, n] (CUDA float32, block order).  Returns the loss."""
        ra, nr = self._ranges(ranges)
        p, pp, V = _poses(poses)
        c = camera(cam)
        o = self.train_options(**opts)
        loss = C.c_double(0)
        self._cam = c
        _check(lib.reloc_train_grad(self._h, ra, nr, pp, V, C.byref(c),
                                    _ptr(targets, _F32, shape=(V, 3, c.height, c.width), name="targets"),
                                    C.byref(o), C.byref(loss), _ptr(grad, _F32, 14 * self.n, name="grad"),
                                    _stream(stream)))
        return loss.value

    def train_step(self, ranges, poses, cam, targets, stream=None, **opts):
        """One Adam step of map training; returns the loss before the step."""
        ra, nr = self._ranges(ranges)
        p, pp, V = _poses(poses)
        c = camera(cam)
        o = self.train_options(**opts)
        loss = C.c_double(0)
        self._cam = c
        _check(lib.reloc_train_step(self._h, ra, nr, pp, V, C.byref(c),
                                    _ptr(targets, _F32, shape=(V, 3, c.height, c.width), name="targets"),
                                    C.byref(o), C.byref(loss), _stream(stream)))
        return loss.value

    def train_reset(self):
        _check(lib.reloc_train_reset(self._h))

    def read_map(self):
        """The device map in block order: (mean, scale, quat, opacity, sh)."""
        K = (self.sh_degree + 1) ** 2
        out = (np.zeros((self.n, 3), np.float32), np.zeros((self.n, 3), np.float32),
               np.zeros((self.n, 4), np.float32), np.zeros(self.n, np.float32),
               np.zeros((self.n, K, 3), np.float32))
        _check(lib.reloc_read_map(self._h, *(a.ctypes.data_as(_fp) for a in out)))
        return out

    def refine_pnp(self, pose_render, cam, depth, alpha, pairs, pose_init=None, stream=None, **opts):
        """PnP refinement (include/reloc.h): depth/alpha [H,W] and pairs [n,4]
        (u_r, v_r, u_q, v_q) are CUDA float32 tensors.  Returns PnpResult."""
        o = PnpOptions()
        lib.reloc_default_pnp_options(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        pr = np.ascontiguousarray(pose_render, np.float64).reshape(16)
        pi = pr if pose_init is None else np.ascontiguousarray(pose_init, np.float64).reshape(16)
        c = camera(cam)
        res = PnpResult()
        hw = c.height * c.width
        if pairs.dim() != 2 or pairs.shape[1] != 4:
            raise ValueError(f"pairs: shape {tuple(pairs.shape)}, expected (n, 4)")
        _check(lib.reloc_refine_pnp(self._h, pr.ctypes.data_as(_dp), pi.ctypes.data_as(_dp), C.byref(c),
                                    _ptr(depth, _F32, hw, name="depth"), _ptr(alpha, _F32, hw, name="alpha"),
                                    _ptr(pairs, _F32, name="pairs"), int(pairs.shape[0]), C.byref(o),
                                    C.byref(res), _stream(stream)))
        return res

    def localize_batch(self, queries, cam, best_rgb=None, best_depth=None, stream=None, want_scores=True):
        """queries: list of (query tensor [3,H,W] on the device, coarse_pose 4x4, radius, grid tuple).
        Returns (list of Result, scores per query as numpy arrays or None)."""
        n = len(queries)
        arr = (Query * n)()
        counts = []
        c = camera(cam)
        for i, (img, pose, radius, grid) in enumerate(queries):
            arr[i].query_dev = _qptr(img, c, name=f"queries[{i}]").value
            arr[i].coarse_pose = (C.c_double * 16)(*np.asarray(pose, np.float64).reshape(16))
            arr[i].radius = float(radius)
            arr[i].grid = Grid(*grid) if not isinstance(grid, Grid) else grid
            counts.append(arr[i].grid.nx * arr[i].grid.ny * arr[i].grid.nyaw)
        res = (Result * n)()
        sc = np.zeros(sum(counts)) if want_scores else None
        hw = c.height * c.width
        self._cam = c
        _check(lib.reloc_localize_batch(self._h, arr, n, C.byref(c), res,
                                        sc.ctypes.data_as(_dp) if sc is not None else None,
                                        _ptr(best_rgb, _F32, n * 3 * hw, name="best_rgb"),
                                        _ptr(best_depth, _F32, n * hw, name="best_depth"), _stream(stream)))
        split = None
        if sc is not None:
            split = np.split(sc, np.cumsum(counts)[:-1])
        return list(res), split

    @staticmethod
    def _queries(queries, c):
        arr = (Query * len(queries))()
        for i, (img, pose, radius, grid) in enumerate(queries):
            arr[i].query_dev = _qptr(img, c, name=f"queries[{i}]").value
            arr[i].coarse_pose = (C.c_double * 16)(*np.asarray(pose, np.float64).reshape(16))
            arr[i].radius = float(radius)
            arr[i].grid = Grid(*grid) if not isinstance(grid, Grid) else grid
        return arr

    def autotune(self, sample, cam, table_path=None, force=False, stream=None) -> TuneResult:
        out = TuneResult()
        c = camera(cam)
        _check(lib.reloc_autotune(self._h, self._queries(sample, c), len(sample), C.byref(c),
                                  table_path.encode() if table_path else None, 1 if force else 0, C.byref(out),
                                  _stream(stream)))
        return out

    def set_batch_options(self, use_graph=True, mem_budget=16 << 30):
        o = BatchOptions()
        o.use_graph = 1 if use_graph else 0
        o.mem_budget = int(mem_budget)
        _check(lib.reloc_set_batch_options(self._h, C.byref(o)))

    def localize_host(self, query_host, coarse_pose, radius, grid, cam, best_rgb_host=None, best_depth_host=None,
                      stream=None):
        """Host buffers: query_host / best_* are numpy float32 or pinned CPU torch tensors."""
        cp = np.ascontiguousarray(coarse_pose, np.float64).reshape(16)
        g = Grid(*grid) if not isinstance(grid, Grid) else grid
        c = camera(cam)
        res = Result()

        hw = c.height * c.width

        def hp(a, n, name):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float32":
                    raise ValueError(f"{name}: host buffers must be contiguous float32 CPU tensors")
                if a.numel() < n:
                    raise ValueError(f"{name}: {a.numel()} elements, at least {n} needed")
                return C.c_void_p(a.data_ptr())
            if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"{name}: host buffers must be contiguous float32")
            if a.size < n:
                raise ValueError(f"{name}: {a.size} elements, at least {n} needed")
            return C.c_void_p(a.ctypes.data)
        _check(lib.reloc_localize_host(self._h, hp(query_host, 3 * hw, "query_host"), cp.ctypes.data_as(_dp), radius,
                                       C.byref(g), C.byref(c), C.byref(res), hp(best_rgb_host, 3 * hw, "best_rgb_host"),
                                       hp(best_depth_host, hw, "best_depth_host"), _stream(stream)))
        return res

    # -- learned proposal ------------------------------------------------------------
    def proposal_init(self, seed=0):
        _check(lib.reloc_proposal_init(self._h, seed))

    def proposal_get(self, which=0) -> np.ndarray:
        out = np.zeros(PROPOSAL_PARAMS, np.float32)
        _check(lib.reloc_proposal_get(self._h, which, out.ctypes.data_as(_fp)))
        return out

    def proposal_set_params(self, flat):
        f = np.ascontiguousarray(flat, np.float32)
        assert f.size == PROPOSAL_PARAMS
        _check(lib.reloc_proposal_set_params(self._h, f.ctypes.data_as(_fp)))

    def proposal_make_input(self, query, coarse_rgb, cam, out, stream=None):
        c = camera(cam)
        _check(lib.reloc_proposal_make_input(self._h, _qptr(query, c), _qptr(coarse_rgb, c, name="coarse_rgb"),
                                             C.byref(c), _ptr(out, _U16, PROPOSAL_H * PROPOSAL_W * 2, name="out"),
                                             _stream(stream)))

    def proposal_forward(self, inputs, logits, stream=None):
        B = inputs.shape[0]
        _check(lib.reloc_proposal_forward(self._h, _ptr(inputs, _U16, shape=(B, PROPOSAL_H, PROPOSAL_W, 2), name="inputs"),
                                          B, _ptr(logits, _F32, B * PROPOSAL_CLASSES, name="logits"), _stream(stream)))

    def proposal_train_step(self, inputs, labels, lr, update=True, stream=None) -> float:
        loss = C.c_float(0)
        B = inputs.shape[0]
        _check(lib.reloc_proposal_train_step(self._h, _ptr(inputs, _U16, shape=(B, PROPOSAL_H, PROPOSAL_W, 2), name="inputs"),
                                             _ptr(labels, _I32, shape=(B,), name="labels"), B, lr,
                                             1 if update else 0, C.byref(loss), _stream(stream)))
        return float(loss.value)

    def gemm_bf16(self, A, B, C, bias=None, relu=False, split_k=1, stream=None):
        """C[M,N] (float32) = A[M,K] @ B[N,K]^T for bfloat16 CUDA tensors."""
        M, K = A.shape
        N = B.shape[0]
        _check(lib.reloc_gemm_bf16(self._h, _ptr(A, _U16, shape=(M, K), name="A"), _ptr(B, _U16, shape=(N, K), name="B"),
                                   _ptr(bias, _F32, N, name="bias"), _ptr(C, _F32, M * N, name="C"), M, N, K,
                                   1 if relu else 0, split_k, _stream(stream)))

    def set_proposal(self, enabled=True, top_k=8, margin=0.0):
        _check(lib.reloc_set_proposal(self._h, 1 if enabled else 0, top_k, margin))

    # -- introspection ------------------------------------------------------------
    def last_counts(self) -> Counts:
        c = Counts()
        _check(lib.reloc_last_counts(self._h, C.byref(c)))
        return c

    def set_profiling(self, enabled: bool):
        _check(lib.reloc_set_profiling(self._h, 1 if enabled else 0))

    def stage_times(self):
        ms = np.zeros(len(STAGES))
        calls = np.zeros(len(STAGES), np.int64)
        _check(lib.reloc_stage_times(self._h, ms.ctypes.data_as(_dp), calls.ctypes.data_as(_i64p)))
        return dict(zip(STAGES, ms)), dict(zip(STAGES, calls))

    def export_debug(self, records=None, rects=None, inst_tiles=None, inst_gauss=None, ranges=None, n_views=None,
                     stream=None):
        k = self.last_counts()
        V, S = k.n_views, k.n_gauss
        if n_views is not None and n_views != V:
            raise ValueError(f"n_views {n_views}, the last call rendered {V} views")
        cnt = np.zeros(max(1, V), np.int64)
        ntiles = 0
        if ranges is not None:
            if self._cam is None:
                raise ValueError("ranges: no rendering call yet")
            tw, th = self._cfg.tile_w, self._cfg.tile_h
            ntiles = ((self._cam.width + tw - 1) // tw) * ((self._cam.height + th - 1) // th)
        _check(lib.reloc_export_debug(self._h, _ptr(records, _F32, V * S * 12, name="records"),
                                      _ptr(rects, _I32, V * S * 4, name="rects"),
                                      _ptr(inst_tiles, _I32, V * k.inst_stride, name="inst_tiles"),
                                      _ptr(inst_gauss, _I32, V * k.inst_stride, name="inst_gauss"),
                                      cnt.ctypes.data_as(_i64p),
                                      _ptr(ranges, _I32, V * 2 * ntiles, name="ranges"), _stream(stream)))
        return cnt
