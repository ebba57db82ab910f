"""Shared helpers of the test suite: run a workload through libgs and through the oracle."""
from __future__ import annotations

import numpy as np

from paper_2605_10760_gb300 import scenes as S

TOL_IMAGE = 2e-4      # max abs error of rgb / depth / alpha / final_T
TOL_GRAD = 1e-3       # relative L2 error per gradient tensor


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def gpu_problem(wl: S.Workload, views=None, params=None, key_capacity=None, device="cuda"):
    from paper_2605_10760_gb300 import raster as R
    views = list(range(len(wl.cameras))) if views is None else list(views)
    sov = wl.scene_of_view[views]
    vb = wl.scene_offsets[sov]
    vc = wl.scene_offsets[sov + 1] - vb
    cams = R.cameras_tensor([wl.cameras[v] for v in views], device)
    pb = R.Problem(vb, vc, wl.scene.n, wl.width, wl.height, cams, params=params, key_capacity=key_capacity,
                   device=device)
    g = R.Gaussians.from_scene(wl.scene, device)
    return pb, g


def oracle_params_from(params):
    from oracle.oracle import Params
    if params is None:
        return Params()
    return Params(tile_w=params.tile_w, tile_h=params.tile_h, near_plane=params.near_plane,
                  dilation=params.dilation, radius_sigmas=params.radius_sigmas, alpha_max=params.alpha_max,
                  alpha_min=params.alpha_min, t_min=params.t_min, bg=tuple(params.bg))


def upstream(wl: S.Workload, V, seed=7, depth_w=0.1, alpha_w=0.0):
    """Seeded upstream gradients standing in for a loss: L1-like signs plus small noise."""
    rng = np.random.default_rng(seed)
    H, W = wl.height, wl.width
    d_rgb = (rng.choice([-1.0, 1.0], (V, 3, H, W)) / (3 * V * H * W)).astype(np.float32)
    d_depth = (depth_w * rng.choice([-1.0, 1.0], (V, H, W)) / (V * H * W)).astype(np.float32)
    d_alpha = (alpha_w * rng.normal(0, 1, (V, H, W)) / (V * H * W)).astype(np.float32)
    return d_rgb, d_depth, d_alpha
