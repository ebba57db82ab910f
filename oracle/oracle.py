"""Python wrapper of the C rasterizer oracle (gs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the benchmark's CPU-baseline
and reference legs.  The product path never imports this module.

The oracle takes two copies of every input: the FP32 copy drives the decision chain (culling,
binning, key order, skip/stop masks) and the FP64 copy drives the value chain.  Normally the FP64
copy is the FP32 one widened; finite-difference tests perturb only the FP64 copy so that all
decisions stay fixed while the differentiable values move.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.og_create.restype = C.c_void_p
        L.og_create.argtypes = [C.c_void_p]
        L.og_destroy.argtypes = [C.c_void_p]
        L.og_num_keys.restype = C.c_int64
        L.og_num_keys.argtypes = [C.c_void_p]
        L.og_num_pairs.restype = C.c_int64
        L.og_num_pairs.argtypes = [C.c_void_p]
        L.og_get_projection.argtypes = [C.c_void_p] + [C.c_void_p] * 9
        L.og_get_bins.argtypes = [C.c_void_p] * 4
        L.og_forward.restype = C.c_int64
        L.og_forward.argtypes = [C.c_void_p] * 6
        L.og_backward.argtypes = [C.c_void_p] * 11
        L.og_expf_batch.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        _LIB = L
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_views", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
        ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("pad0", C.c_int32),
        ("n_gauss", C.c_int64),
        ("view_begin", C.c_void_p), ("view_end", C.c_void_p),
        ("mu_f", C.c_void_p), ("ls_f", C.c_void_p), ("q_f", C.c_void_p), ("o_f", C.c_void_p),
        ("cam_f", C.c_void_p),
        ("mu_d", C.c_void_p), ("ls_d", C.c_void_p), ("q_d", C.c_void_p), ("o_d", C.c_void_p),
        ("c_d", C.c_void_p), ("cam_d", C.c_void_p),
        ("near_plane", C.c_float), ("dilation", C.c_float), ("radius_sigmas", C.c_float),
        ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("t_min", C.c_float),
        ("bg", C.c_float * 3), ("pad1", C.c_int32),
        ("tile_mask", C.c_void_p),
    ]


def expf(x: np.ndarray) -> np.ndarray:
    """The FP32 exponential of the decision chain, elementwise."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().og_expf_batch(x.ctypes.data, y.ctypes.data, x.size)
    return y


@dataclass
class Params:
    tile_w: int = 16
    tile_h: int = 16
    near_plane: float = 0.2
    dilation: float = 0.3
    radius_sigmas: float = 3.0
    alpha_max: float = 0.99
    alpha_min: float = float(np.float32(1.0) / np.float32(255.0))
    t_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)


def _p(a):
    return a.ctypes.data if a is not None else None


class Oracle:
    """One oracle evaluation of a (possibly batched) rendering problem.

    scene arrays are [n,...]; cams is [V,16] (R row-major, t, fx, fy, cx, cy); view v renders the
    Gaussian rows [view_begin[v], view_end[v]).  `values` optionally overrides the FP64 value
    inputs: dict with any of means, log_scales, quats, opacities, colors, cams (float64).
    """

    def __init__(self, means, log_scales, quats, opacities, colors, cams, view_begin, view_end,
                 width, height, params: Params | None = None, tile_mask=None, values: dict | None = None):
        self.params = params or Params()
        P = self.params
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.mu_f, self.ls_f, self.q_f, self.o_f = f32(means), f32(log_scales), f32(quats), f32(opacities)
        self.cam_f = f32(cams).reshape(-1, 16)
        values = values or {}
        self.mu_d = f64(values.get("means", self.mu_f))
        self.ls_d = f64(values.get("log_scales", self.ls_f))
        self.q_d = f64(values.get("quats", self.q_f))
        self.o_d = f64(values.get("opacities", self.o_f))
        self.c_d = f64(values.get("colors", f32(colors)))
        self.cam_d = f64(values.get("cams", self.cam_f)).reshape(-1, 16)
        self.vb = np.ascontiguousarray(view_begin, dtype=np.int64)
        self.ve = np.ascontiguousarray(view_end, dtype=np.int64)
        self.V = int(self.vb.shape[0])
        self.W, self.H = int(width), int(height)
        self.Tx = -(-self.W // P.tile_w)
        self.Ty = -(-self.H // P.tile_h)
        self.G = self.V * self.Tx * self.Ty
        self.n = int(self.mu_f.shape[0])
        self.tile_mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
        pr = _Problem()
        pr.n_views, pr.width, pr.height, pr.tile_w, pr.tile_h = self.V, self.W, self.H, P.tile_w, P.tile_h
        pr.n_gauss = self.n
        pr.view_begin, pr.view_end = _p(self.vb), _p(self.ve)
        pr.mu_f, pr.ls_f, pr.q_f, pr.o_f, pr.cam_f = (_p(self.mu_f), _p(self.ls_f), _p(self.q_f), _p(self.o_f),
                                                      _p(self.cam_f))
        pr.mu_d, pr.ls_d, pr.q_d, pr.o_d, pr.c_d, pr.cam_d = (_p(self.mu_d), _p(self.ls_d), _p(self.q_d),
                                                              _p(self.o_d), _p(self.c_d), _p(self.cam_d))
        pr.near_plane, pr.dilation, pr.radius_sigmas = P.near_plane, P.dilation, P.radius_sigmas
        pr.alpha_max, pr.alpha_min, pr.t_min = P.alpha_max, P.alpha_min, P.t_min
        for k in range(3):
            pr.bg[k] = P.bg[k]
        pr.tile_mask = _p(self.tile_mask)
        self._pr = pr
        self._ctx = lib().og_create(C.byref(pr))
        self.K = int(lib().og_num_keys(self._ctx))
        self.VN = int(lib().og_num_pairs(self._ctx))

    def __del__(self):
        if getattr(self, "_ctx", None):
            lib().og_destroy(self._ctx)
            self._ctx = None

    @classmethod
    def from_workload(cls, wl, params: Params | None = None, views=None, **kw):
        """Oracle of a scenes.Workload (optionally a subset of its views)."""
        views = list(range(len(wl.cameras))) if views is None else list(views)
        cams = np.stack([wl.cameras[v].as_row() for v in views])
        sov = wl.scene_of_view[views]
        vb = wl.scene_offsets[sov]
        ve = wl.scene_offsets[sov + 1]
        s = wl.scene
        return cls(s.means, s.log_scales, s.quats, s.opacities, s.colors, cams, vb, ve, wl.width, wl.height,
                   params, **kw)

    # ---------------------------------------------------------------------------------------
    def projection(self) -> dict:
        VN = self.VN
        out = dict(mean2d=np.empty((VN, 2), np.float32), conic=np.empty((VN, 3), np.float32),
                   depth=np.empty(VN, np.float32), radius=np.empty(VN, np.float32),
                   rect=np.empty((VN, 4), np.int32), touched=np.empty(VN, np.uint32),
                   mean2d_d=np.empty((VN, 2)), conic_d=np.empty((VN, 3)), depth_d=np.empty(VN))
        lib().og_get_projection(self._ctx, *[out[k].ctypes.data for k in
                                             ("mean2d", "conic", "depth", "radius", "rect", "touched",
                                              "mean2d_d", "conic_d", "depth_d")])
        return out

    def bins(self) -> dict:
        keys = np.empty(max(self.K, 1), np.uint64)
        vals = np.empty(max(self.K, 1), np.uint32)
        ranges = np.empty((self.G, 2), np.uint32)
        lib().og_get_bins(self._ctx, keys.ctypes.data, vals.ctypes.data, ranges.ctypes.data)
        return dict(keys=keys[:self.K], vals=vals[:self.K], ranges=ranges)

    def forward(self) -> dict:
        V, H, W = self.V, self.H, self.W
        out = dict(rgb=np.zeros((V, 3, H, W)), depth=np.zeros((V, H, W)), alpha=np.zeros((V, H, W)),
                   final_T=np.ones((V, H, W)), last=np.zeros((V, H, W), np.int32))
        out["pairs"] = int(lib().og_forward(self._ctx, *[out[k].ctypes.data for k in
                                                         ("rgb", "depth", "alpha", "final_T", "last")]))
        return out

    def backward(self, g_rgb=None, g_depth=None, g_alpha=None) -> dict:
        V, H, W, n = self.V, self.H, self.W, self.n
        c = lambda a, shp: None if a is None else np.ascontiguousarray(np.broadcast_to(a, shp), dtype=np.float64)
        gr, gd, ga = c(g_rgb, (V, 3, H, W)), c(g_depth, (V, H, W)), c(g_alpha, (V, H, W))
        out = dict(g2d=np.empty((self.VN, 10)), means=np.empty((n, 3)), log_scales=np.empty((n, 3)),
                   quats=np.empty((n, 4)), opacities=np.empty(n), colors=np.empty((n, 3)), pose=np.empty((V, 6)))
        lib().og_backward(self._ctx, _p(gr), _p(gd), _p(ga),
                          *[out[k].ctypes.data for k in ("g2d", "means", "log_scales", "quats", "opacities",
                                                         "colors", "pose")])
        return out


def exp_se3_left(cam_row: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Apply the left perturbation T <- Exp(xi) T to a [16] camera row (float64), xi = (rho, phi).

    Exp(xi) = [Exp(phi), Jl(phi) rho; 0, 1] with Exp(phi) by Rodrigues' formula and Jl the left
    Jacobian of SO(3)."""
    cam = np.array(cam_row, dtype=np.float64)
    R = cam[:9].reshape(3, 3)
    t = cam[9:12]
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        Rx = np.eye(3) + K
        Jl = np.eye(3) + 0.5 * K
    else:
        Rx = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
        Jl = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * K @ K
    out = cam.copy()
    out[:9] = (Rx @ R).reshape(9)
    out[9:12] = Rx @ t + Jl @ rho
    return out
