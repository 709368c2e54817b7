"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI,
run the oracle on the same seeded inputs, and compare.

Tolerances (FP32 path vs FP64 oracle):
  RGB, alpha   max |diff| <= 1e-4 on every pixel the oracle does not flag as
               threshold-adjacent (footprint edge, alpha-skip edge, stop edge,
               depth near-tie between consecutive contributors);
  depth        max |diff| <= 1e-4 * z_ref, z_ref = the largest camera depth of
               a visible Gaussian (depth is a weighted sum of z_i with the same
               weights as colour, colour values lie in [0, 1]);
  NCC          |diff| <= 2e-6 (derived from the pixel bound over n samples,
               measured margin in the test output);
  argmax       identical unless the oracle's top-two margin is below the NCC
               tolerance, in which case the GPU winner must be one of the tied.
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_RGB = 1e-4
TOL_DEPTH_REL = 1e-4
TOL_NCC = 2e-6


def torch_device():
    import torch
    return torch.device("cuda:0")


def z_ref(g, poses, cam):
    zs = []
    for W in poses[:4]:
        rec = oracle.project(g, W, cam)
        vis = rec[:, oracle.F["visible"]] == 1
        if vis.any():
            zs.append(rec[vis, oracle.F["depth"]].max())
    return max([1.0] + zs)


def compare_rgb(rgb, ref, tol_rgb=TOL_RGB):
    """compare_images for a colour-only render (V,3,H,W): unflagged pixels
    within the tolerance, flagged ones within it plus the oracle's bound."""
    mask = ref["flags"] == 0
    e_rgb = np.abs(rgb - ref["rgb"]).max(axis=1)
    stats = dict(flagged=float(1 - mask.mean()), rgb=float(e_rgb[mask].max(initial=0)),
                 rgb_flagged=float(e_rgb[~mask].max(initial=0)),
                 flagged_excess=float(np.max(e_rgb - ref["bound"], initial=0)))
    assert stats["rgb"] <= tol_rgb, stats
    assert np.all(e_rgb <= tol_rgb + ref["bound"]), stats
    return stats


def compare_images(rgb, depth, alpha, ref, zr, tol_rgb=TOL_RGB, tol_depth_rel=TOL_DEPTH_REL):
    """rgb (V,3,H,W), depth/alpha (V,H,W) numpy from the GPU; ref: oracle.render_views output.

    Every pixel is checked: unflagged ones against the tolerance, flagged ones
    against the tolerance plus the oracle's bound of what the flagged decisions
    can move (depth: that bound times z_ref)."""
    mask = ref["flags"] == 0
    bnd = ref["bound"]
    e_rgb = np.abs(rgb - ref["rgb"]).max(axis=1)
    e_d = np.abs(depth - ref["depth"])
    e_a = np.abs(alpha - ref["alpha"])
    tol_d = tol_depth_rel * zr
    stats = dict(flagged=float(1 - mask.mean()),
                 rgb=float(e_rgb[mask].max(initial=0)), depth=float(e_d[mask].max(initial=0)),
                 alpha=float(e_a[mask].max(initial=0)), depth_tol=tol_d,
                 rgb_flagged=float(e_rgb[~mask].max(initial=0)),
                 flagged_excess=float(np.max(e_rgb - bnd, initial=0)))
    assert stats["rgb"] <= tol_rgb, stats
    assert stats["alpha"] <= tol_rgb, stats
    assert stats["depth"] <= tol_d, stats
    assert np.all(e_rgb <= tol_rgb + bnd), stats
    assert np.all(e_a <= tol_rgb + bnd), stats
    assert np.all(e_d <= tol_d + bnd * zr), stats
    return stats


def replay_tile_lists(records, rects, inst_tiles, inst_gauss, inst_count, ranges, cam_w, cam_h, tile_w, tile_h):
    """Bit-exact check of the GPU's sorted tile lists against the oracle's
    integer replay (key build + stable sort + ranges) on the GPU's own
    visibility, float32 depth bits and tile rectangles."""
    V, S = rects.shape[:2]
    ntx = (cam_w + tile_w - 1) // tile_w
    nty = (cam_h + tile_h - 1) // tile_h
    nt = ntx * nty
    vis = (rects[..., 0] >= 0).astype(np.uint8)
    dbits = np.ascontiguousarray(records[..., 2]).view(np.uint32)
    keys, vals = oracle.tile_keys(vis, dbits, rects, ntx, nty)
    ks, vs = oracle.stable_sort(keys, vals)
    tb = oracle.tile_bits(nt)
    rg = oracle.tile_ranges(ks, V, nt)
    view = (ks >> np.uint64(32 + tb)).astype(np.int64)
    tile = ((ks >> np.uint64(32)) & np.uint64((1 << tb) - 1)).astype(np.uint32)
    starts = np.searchsorted(view, np.arange(V + 1))
    for v in range(V):
        a, b = starts[v], starts[v + 1]
        n = int(inst_count[v])
        assert n == b - a, (v, n, b - a)
        assert np.array_equal(inst_tiles[v, :n], tile[a:b]), v
        assert np.array_equal(inst_gauss[v, :n], vs[a:b]), v
        exp = rg[v] - a                               # oracle ranges are global
        nonempty = rg[v, :, 1] > rg[v, :, 0]
        got = ranges[v]
        assert np.array_equal(got[nonempty], exp[nonempty]), v
        assert np.all(got[~nonempty] == 0), v
    return int(len(ks))
