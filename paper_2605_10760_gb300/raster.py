"""Torch-facing binding of libgs: a problem object owning the workspace, one function per C-ABI
call, and a torch.autograd.Function.  Every computation runs in libgs; this module only passes
device pointers (torch tensors are used as device memory and for the current CUDA stream).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_params(**over) -> L.gs_params:
    p = L.gs_params()
    L.load().gs_default_params(C.byref(p))
    for k, v in over.items():
        if k == "bg":
            for i in range(3):
                p.bg[i] = float(v[i])
        else:
            setattr(p, k, v)
    return p


@dataclass
class Gaussians:
    """Device float32 tensors: means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z), opacities [N],
    colors [N,3]."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacities: torch.Tensor
    colors: torch.Tensor

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=torch.float32)
        return cls(t(scene.means), t(scene.log_scales), t(scene.quats), t(scene.opacities), t(scene.colors))

    def struct(self) -> L.gs_gaussians:
        s = L.gs_gaussians()
        s.means, s.log_scales, s.quats = self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr()
        s.opacities, s.colors = self.opacities.data_ptr(), self.colors.data_ptr()
        return s

    @property
    def n(self):
        return int(self.means.shape[0])


def zeros_like_grads(g: Gaussians) -> Gaussians:
    return Gaussians(*[torch.zeros_like(getattr(g, k)) for k in ("means", "log_scales", "quats", "opacities",
                                                                  "colors")])


def cameras_tensor(cameras, device="cuda") -> torch.Tensor:
    """[V,16] float32 device tensor (R row-major, t, fx, fy, cx, cy) from scenes.Camera objects."""
    rows = np.stack([c.as_row() for c in cameras]).astype(np.float32)
    return torch.from_numpy(rows).to(device)


class Problem:
    """V views of one or more scenes plus the libgs workspace that serves them.

    view_gauss_begin / view_gauss_count: first row and row count of each view's scene in the
    concatenated Gaussian arrays.  cameras: [V,16] device tensor.  The workspace is one device
    byte tensor; key_capacity bounds the number of duplicated (tile, depth) keys.
    """

    def __init__(self, view_gauss_begin, view_gauss_count, num_gaussians, width, height, cameras=None,
                 params: L.gs_params | None = None, key_capacity: int | None = None, device="cuda",
                 visible_capacity: int = 0):
        self.lib = L.load()
        self.device = torch.device(device)
        self.vb = np.ascontiguousarray(view_gauss_begin, dtype=np.int64)
        self.vc = np.ascontiguousarray(view_gauss_count, dtype=np.int64)
        self.V = int(self.vb.shape[0])
        self.W, self.H = int(width), int(height)
        self.N = int(num_gaussians)
        self.P = int(self.vc.sum())
        self.params = params if params is not None else default_params()
        if key_capacity is None:
            key_capacity = int(min((1 << 30) - 1, max(1 << 20, 4 * self.P)))
        self.cap = int(key_capacity)
        self.vcap = int(visible_capacity)          # 0: all pairs, always enough
        self.cameras = cameras
        self._pb = L.gs_problem()
        self._sync_struct()
        self._alloc()

    # -- struct / workspace ------------------------------------------------------------------
    def _sync_struct(self):
        pb = self._pb
        pb.num_views, pb.width, pb.height = self.V, self.W, self.H
        pb.num_gaussians = self.N
        pb.view_gauss_begin = self.vb.ctypes.data_as(C.POINTER(C.c_int64))
        pb.view_gauss_count = self.vc.ctypes.data_as(C.POINTER(C.c_int64))
        pb.cameras = None if self.cameras is None else self.cameras.data_ptr()
        pb.key_capacity = self.cap
        pb.visible_capacity = self.vcap
        pb.params = self.params

    @property
    def pb(self):
        self._sync_struct()
        return C.byref(self._pb)

    def _alloc(self):
        n = C.c_size_t()
        L.check(self.lib.gs_workspace_size(self.pb, C.byref(n)), "gs_workspace_size")
        self.ws_bytes = int(n.value)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        L.check(self.lib.gs_workspace_init(self.pb, _ptr(self.ws), _stream()), "gs_workspace_init")

    def set_capacity(self, cap: int, visible: int | None = None):
        """Re-size the workspace for `cap` keys (and `visible` visible pairs when given)."""
        self.cap = int(min((1 << 30) - 1, cap))
        if visible is not None:
            self.vcap = int(min((1 << 31) - 1, visible))
        self._alloc()

    def set_cameras(self, cameras: torch.Tensor):
        assert cameras.dtype == torch.float32 and cameras.is_contiguous() and cameras.shape == (self.V, 16)
        self.cameras = cameras

    @property
    def tiles(self):
        tw, th = self.params.tile_w, self.params.tile_h
        return -(-self.W // tw), -(-self.H // th)

    # -- inspection ----------------------------------------------------------------------------
    def workspace(self) -> dict:
        """Tensors viewing the workspace (proj, tiles_touched, sorted keys/vals, ranges, grad2d, K)."""
        v = L.gs_ws_view()
        L.check(self.lib.gs_workspace_view(self.pb, _ptr(self.ws), C.byref(v)), "gs_workspace_view")
        base = self.ws.data_ptr()

        def sl(ptr, count, dtype):
            off = ptr - base
            nbytes = count * torch.empty((), dtype=dtype).element_size()
            return self.ws[off:off + nbytes].view(dtype)

        P, G, VC = int(v.num_pairs), int(v.num_tiles), int(v.visible_capacity)
        slot = sl(v.pair_slot, P, torch.int32)
        proj_s = sl(v.proj, 12 * VC, torch.float32).view(VC, 12)
        g2d_s = sl(v.grad2d, 12 * VC, torch.float32).view(VC, 12)

        def by_pair(t):
            # inspection copy in pair order (zero rows for culled pairs): records live by slot
            out = torch.zeros(P, 12, dtype=t.dtype, device=t.device)
            s64 = slot.long() & 0xffffffff
            ok = s64 < VC
            out[ok] = t[s64[ok]]
            return out

        return dict(proj=by_pair(proj_s), grad2d=by_pair(g2d_s), proj_slots=proj_s, grad2d_slots=g2d_s,
                    pair_slot=slot, tiles_touched=sl(v.tiles_touched, P, torch.int32),
                    sorted_keys=sl(v.sorted_keys, self.cap, torch.int64),
                    sorted_vals=sl(v.sorted_vals, self.cap, torch.int32),
                    tile_ranges=sl(v.tile_ranges, 2 * G, torch.int32).view(G, 2),
                    num_keys=sl(v.num_keys, 2, torch.int32), passes=int(v.sort_passes), visible_capacity=VC,
                    claim_count=sl(v.claim_count, 32, torch.int32),
                    claim_list=sl(v.claim_list, 32 * G, torch.int32).view(32, G))

    def check_status(self):
        req = C.c_int64()
        rc = self.lib.gs_check_status(self.pb, _ptr(self.ws), _stream(), C.byref(req))
        return rc, int(req.value)

    def check_guards(self):
        """(status, index of the first overwritten workspace guard block or -1); synchronises."""
        bad = C.c_int32(-1)
        rc = self.lib.gs_check_guards(self.pb, _ptr(self.ws), _stream(), C.byref(bad))
        return rc, int(bad.value)

    def stats(self) -> dict:
        s = L.gs_stats()
        L.check(self.lib.gs_read_stats(self.pb, _ptr(self.ws), _stream(), C.byref(s)), "gs_read_stats")
        return dict(num_keys=int(s.num_keys), fwd_pairs=int(s.fwd_pairs), bwd_pairs=int(s.bwd_pairs),
                    num_visible=int(s.num_visible))

    # -- stages ----------------------------------------------------------------------------
    def project(self, g: Gaussians):
        gs_ = g.struct()
        L.check(self.lib.gs_project(self.pb, C.byref(gs_), _ptr(self.ws), _stream()), "gs_project")

    def bin_sort(self):
        L.check(self.lib.gs_bin_sort(self.pb, _ptr(self.ws), _stream()), "gs_bin_sort")

    def alloc_image(self) -> dict:
        V, H, W = self.V, self.H, self.W
        d = self.device
        return dict(rgb=torch.empty(V, 3, H, W, device=d), depth=torch.empty(V, H, W, device=d),
                    alpha=torch.empty(V, H, W, device=d), final_T=torch.empty(V, H, W, device=d),
                    last_idx=torch.empty(V, H, W, dtype=torch.int32, device=d))

    def render_fwd(self, img: dict | None = None) -> dict:
        img = img if img is not None else self.alloc_image()
        s = L.gs_image(_ptr(img.get("rgb")), _ptr(img.get("depth")), _ptr(img.get("alpha")),
                       _ptr(img["final_T"]), _ptr(img["last_idx"]))
        L.check(self.lib.gs_render_fwd(self.pb, _ptr(self.ws), C.byref(s), _stream()), "gs_render_fwd")
        return img

    def render_fwd_l1(self, img: dict, rgb_t, depth_t=None, w_rgb=1.0, w_depth=0.0, d_rgb=None, d_depth=None,
                      loss=None):
        """gs_render_fwd with the L1 loss terms fused into its epilogue.  Returns (img, loss, d_rgb,
        d_depth); img's rgb / depth may be absent (not written)."""
        V, H, W = self.V, self.H, self.W
        d_rgb = d_rgb if d_rgb is not None else torch.empty(V, 3, H, W, device=self.device)
        if w_depth != 0.0 and d_depth is None:
            d_depth = torch.empty(V, H, W, device=self.device)
        loss = loss if loss is not None else torch.zeros(1, dtype=torch.float64, device=self.device)
        s = L.gs_image(_ptr(img.get("rgb")), _ptr(img.get("depth")), _ptr(img.get("alpha")),
                       _ptr(img["final_T"]), _ptr(img["last_idx"]))
        t = L.gs_l1_target(_ptr(rgb_t), _ptr(depth_t) if w_depth != 0.0 else None, float(w_rgb), float(w_depth),
                           _ptr(d_rgb), _ptr(d_depth) if w_depth != 0.0 else None, _ptr(loss))
        L.check(self.lib.gs_render_fwd_l1(self.pb, _ptr(self.ws), C.byref(s), C.byref(t), _stream()),
                "gs_render_fwd_l1")
        return img, loss, d_rgb, d_depth

    def render_bwd(self, g: Gaussians, img: dict, d_rgb=None, d_depth=None, d_alpha=None,
                   grads: Gaussians | None = None) -> Gaussians:
        grads = grads if grads is not None else zeros_like_grads(g)
        gs_ = g.struct()
        fi = L.gs_image(None, None, None, _ptr(img["final_T"]), _ptr(img["last_idx"]))
        di = L.gs_image_grad(_ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha))
        go = L.gs_grads(*[getattr(grads, k).data_ptr() for k in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")])
        L.check(self.lib.gs_render_bwd(self.pb, C.byref(gs_), _ptr(self.ws), C.byref(fi), C.byref(di), C.byref(go),
                                       _stream()), "gs_render_bwd")
        return grads

    def render_bwd_composite(self, img: dict, d_rgb=None, d_depth=None, d_alpha=None):
        """The compositing adjoint alone (2-D gradients into the workspace)."""
        fi = L.gs_image(None, None, None, _ptr(img["final_T"]), _ptr(img["last_idx"]))
        di = L.gs_image_grad(_ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha))
        L.check(self.lib.gs_render_bwd_composite(self.pb, _ptr(self.ws), C.byref(fi), C.byref(di), _stream()),
                "gs_render_bwd_composite")

    def project_bwd(self, g: Gaussians, grads: Gaussians) -> Gaussians:
        """The projection adjoint alone, accumulated into grads (after render_bwd_composite)."""
        gs_ = g.struct()
        go = L.gs_grads(*[getattr(grads, k).data_ptr() for k in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")])
        L.check(self.lib.gs_project_bwd(self.pb, C.byref(gs_), _ptr(self.ws), C.byref(go), _stream()),
                "gs_project_bwd")
        return grads

    def pose_grad(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = out if out is not None else torch.empty(self.V, 6, device=self.device)
        L.check(self.lib.gs_pose_grad(self.pb, _ptr(self.ws), _ptr(out), _stream()), "gs_pose_grad")
        return out

    def forward_checked(self, g: Gaussians, img: dict | None = None, max_retries: int = 2) -> dict:
        """project + bin_sort + render_fwd, growing the key capacity when K exceeds it and the
        visible-pair capacity when the visible pairs exceed it (syncs)."""
        for _ in range(max_retries + 1):
            self.project(g)
            self.bin_sort()
            rc, req = self.check_status()
            if rc == L.GS_ERR_CAPACITY:
                nv = self.stats()["num_visible"]
                vis = int(nv * 1.25) + 1024 if self.vcap and nv > self.vcap else None
                self.set_capacity(max(self.cap, int(req * 1.25) + 1024) if req > self.cap else self.cap, vis)
                continue
            L.check(rc, "gs_bin_sort")
            return self.render_fwd(img)
        raise L.GsError(L.GS_ERR_CAPACITY, "forward_checked")


# ------------------------------------------------------------------------------------------
# losses and optimiser
# ------------------------------------------------------------------------------------------

def loss_l1(rgb, rgb_t, depth=None, depth_t=None, w_rgb=1.0, w_depth=0.0, d_rgb=None, d_depth=None, loss=None):
    """Returns (loss [1] float64 device, d_rgb, d_depth)."""
    V, _, H, W = rgb.shape
    d_rgb = d_rgb if d_rgb is not None else torch.empty_like(rgb)
    if w_depth != 0.0 and d_depth is None:
        d_depth = torch.empty_like(depth)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=rgb.device)
    L.check(L.load().gs_loss_l1(V, W, H, _ptr(rgb), _ptr(rgb_t), _ptr(depth), _ptr(depth_t), float(w_rgb),
                                float(w_depth), _ptr(d_rgb), _ptr(d_depth) if w_depth != 0.0 else None, _ptr(loss),
                                _stream()), "gs_loss_l1")
    return loss, d_rgb, d_depth


def loss_normal(depth, prior, cams, weight=1e-2, d_depth=None, loss=None):
    """Normal term of the mapping loss (Eq. 4, lambda_n = 1e-2): weight * mean over all pixels of
    |1 - N_hat . N_bar| for the depth-induced normal N_hat and the prior N_bar [V,3,H,W].  ADDS the
    loss to `loss` and dL/d depth to `d_depth` (zero tensors are created when None); returns both."""
    V, H, W = depth.shape
    if d_depth is None:
        d_depth = torch.zeros_like(depth)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=depth.device)
    L.check(L.load().gs_loss_normal(V, W, H, _ptr(depth), _ptr(prior), _ptr(cams), float(weight), _ptr(d_depth),
                                    _ptr(loss), _stream()), "gs_loss_normal")
    return loss, d_depth


def ssim_scratch(V, H, W, device="cuda") -> torch.Tensor:
    n = L.load().gs_ssim_scratch_size(V, W, H)
    return torch.empty(int(n), dtype=torch.uint8, device=device)


def loss_l1_ssim(rgb, rgb_t, w_l1=0.8, w_ssim=0.2, d_rgb=None, loss=None, scratch=None):
    V, _, H, W = rgb.shape
    d_rgb = d_rgb if d_rgb is not None else torch.empty_like(rgb)
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=rgb.device)
    scratch = scratch if scratch is not None else ssim_scratch(V, H, W, rgb.device)
    L.check(L.load().gs_loss_l1_ssim(V, W, H, _ptr(rgb), _ptr(rgb_t), float(w_l1), float(w_ssim), _ptr(d_rgb),
                                     _ptr(loss), _ptr(scratch), _stream()), "gs_loss_l1_ssim")
    return loss, d_rgb


class AdamState:
    """Adam moments and parameter views for the in-kernel optimiser step.  Opacity is optimised
    through its logit; `g.opacities` is rewritten as sigmoid(logit) by every step."""

    def __init__(self, g: Gaussians, lr=(1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3)):
        self.g = g
        o = g.opacities.clamp(1e-6, 1 - 1e-6)
        self.logits = torch.log(o / (1 - o)).contiguous()
        n = g.n
        self.m = torch.zeros(14 * n, device=g.means.device)   # group-major, the parameters' layout
        self.v = torch.zeros(14 * n, device=g.means.device)
        self.step = torch.zeros(1, dtype=torch.int32, device=g.means.device)
        self.lr = (C.c_float * 5)(*lr)

    def apply(self, grads: Gaussians, zero_grads=True, iso_weight=0.0, iso_loss=None):
        """One Adam step; iso_weight > 0 adds the isotropy regulariser lambda_s L_iso (Eq. 4)."""
        st = L.gs_adam_state(self.g.means.data_ptr(), self.g.log_scales.data_ptr(), self.g.quats.data_ptr(),
                             self.logits.data_ptr(), self.g.opacities.data_ptr(), self.g.colors.data_ptr(),
                             self.m.data_ptr(), self.v.data_ptr(), self.step.data_ptr())
        go = L.gs_grads(*[getattr(grads, k).data_ptr() for k in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")])
        L.check(L.load().gs_adam_step_reg(self.g.n, C.byref(st), C.byref(go), self.lr, float(iso_weight),
                                          int(bool(zero_grads)), _ptr(iso_loss), _stream()), "gs_adam_step_reg")


# ------------------------------------------------------------------------------------------
# checkpoint / resume
# ------------------------------------------------------------------------------------------

_GFIELDS = ("means", "log_scales", "quats", "opacities", "colors")


def save_checkpoint(path, g: Gaussians, adam: AdamState | None = None, extra: dict | None = None):
    """Write the Gaussian parameters (and, with `adam`, its logits, moments, step counter and
    learning rates) to `path` as a dict of CPU tensors."""
    state = {"gaussians": {k: getattr(g, k).detach().cpu() for k in _GFIELDS}}
    if adam is not None:
        state["adam"] = {"logits": adam.logits.detach().cpu(), "m": adam.m.detach().cpu(),
                         "v": adam.v.detach().cpu(), "step": adam.step.detach().cpu(), "lr": list(adam.lr)}
    if extra:
        state["extra"] = {k: (v.detach().cpu() if torch.is_tensor(v) else v) for k, v in extra.items()}
    torch.save(state, path)


def load_checkpoint(path, device="cuda"):
    """Read a checkpoint written by save_checkpoint: returns (Gaussians, AdamState or None, extra).
    The optimiser resumes exactly: same moments, step counter and learning rates."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    g = Gaussians(*[state["gaussians"][k].to(device).contiguous() for k in _GFIELDS])
    adam = None
    if "adam" in state:
        a = state["adam"]
        adam = AdamState(g, tuple(a["lr"]))
        adam.logits.copy_(a["logits"].to(device))
        adam.m.copy_(a["m"].to(device))
        adam.v.copy_(a["v"].to(device))
        adam.step.copy_(a["step"].to(device))
    return g, adam, state.get("extra", {})


# ------------------------------------------------------------------------------------------
# autograd
# ------------------------------------------------------------------------------------------

class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacities, colors, pose_delta, problem):
        g = Gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(), opacities.contiguous(),
                      colors.contiguous())
        img = problem.forward_checked(g)
        ctx.problem = problem
        ctx.g = g
        ctx.save_for_backward(img["final_T"], img["last_idx"])
        ctx.mark_non_differentiable(img["final_T"])
        return img["rgb"], img["depth"], img["alpha"]

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_alpha):
        final_T, last_idx = ctx.saved_tensors
        pb = ctx.problem
        img = dict(final_T=final_T, last_idx=last_idx)
        c = lambda t: None if t is None else t.contiguous()
        grads = pb.render_bwd(ctx.g, img, c(d_rgb), c(d_depth), c(d_alpha))
        pose = pb.pose_grad()
        return grads.means, grads.log_scales, grads.quats, grads.opacities, grads.colors, pose, None


def rasterize(means, log_scales, quats, opacities, colors, problem: Problem, pose_delta=None):
    """Render (rgb [V,3,H,W], depth [V,H,W], alpha [V,H,W]) of the problem's views.

    Differentiable w.r.t. the five Gaussian tensors and w.r.t. `pose_delta` [V,6]: a zero-valued
    leaf standing for the left perturbation Exp(xi) T of each world-to-camera pose (its gradient
    is dL/dxi at xi = 0; the forward renders at the problem's cameras)."""
    if pose_delta is None:
        pose_delta = torch.zeros(problem.V, 6, device=means.device, requires_grad=False)
    return _Rasterize.apply(means, log_scales, quats, opacities, colors, pose_delta, problem)


# ------------------------------------------------------------------------------------------
# joint refinement (exposure-compensated loss, pruning, per-view pose / exposure Adam)
# ------------------------------------------------------------------------------------------

def refine_scratch(V, H, W, device="cuda") -> torch.Tensor:
    n = L.load().gs_refine_scratch_size(V, W, H)
    return torch.empty(int(n), dtype=torch.uint8, device=device)


def loss_refine(rgb, rgb_t, expo, depth=None, depth_t=None, w_l1=1.75, w_ssim=0.2, w_depth=0.25,
                d_rgb=None, d_depth=None, d_expo=None, loss=None, scratch=None):
    """Eq. 23 on I~ = exp(a) I^ + b.  Returns (loss, d_rgb, d_depth, d_expo)."""
    V, _, H, W = rgb.shape
    dev = rgb.device
    d_rgb = d_rgb if d_rgb is not None else torch.empty_like(rgb)
    use_d = depth is not None and w_depth != 0.0
    if use_d and d_depth is None:
        d_depth = torch.empty_like(depth)
    d_expo = d_expo if d_expo is not None else torch.empty(V, 2, device=dev)
    loss = loss if loss is not None else torch.zeros(1, dtype=torch.float64, device=dev)
    scratch = scratch if scratch is not None else refine_scratch(V, H, W, dev)
    L.check(L.load().gs_loss_refine(V, W, H, _ptr(rgb), _ptr(rgb_t), _ptr(depth) if use_d else None,
                                    _ptr(depth_t) if use_d else None, _ptr(expo), float(w_l1), float(w_ssim),
                                    float(w_depth) if use_d else 0.0, _ptr(d_rgb), _ptr(d_depth) if use_d else None,
                                    _ptr(d_expo), _ptr(loss), _ptr(scratch), _stream()), "gs_loss_refine")
    return loss, d_rgb, d_depth, d_expo


def prune(g: Gaussians, threshold=0.005) -> Gaussians:
    """Gaussians with opacity >= threshold, in order (the refinement's pruning).  Syncs to read the count."""
    n = g.n
    out = Gaussians(*[torch.empty_like(getattr(g, k)) for k in ("means", "log_scales", "quats", "opacities",
                                                                 "colors")])
    kept = torch.zeros(1, dtype=torch.int64, device=g.means.device)
    scratch = torch.empty(int(L.load().gs_prune_scratch_size(n)), dtype=torch.uint8, device=g.means.device)
    gi = g.struct()
    go = L.gs_gaussian_arrays(*[getattr(out, k).data_ptr() for k in ("means", "log_scales", "quats", "opacities",
                                                                      "colors")])
    L.check(L.load().gs_prune(n, C.byref(gi), float(threshold), C.byref(go), _ptr(kept), _ptr(scratch), _stream()),
            "gs_prune")
    k = int(kept.item())
    return Gaussians(*[getattr(out, f)[:k].contiguous() for f in ("means", "log_scales", "quats", "opacities",
                                                                   "colors")])


class ViewAdamState:
    """Adam over each view's pose delta (applied to the problem's cameras as T <- Exp(delta) T) and
    exposure (a, b)."""

    def __init__(self, problem: Problem, lr_pose=1e-4, lr_expo=1e-3):
        dev = problem.device
        self.pb = problem
        self.expo = torch.zeros(problem.V, 2, device=dev)
        self.m = torch.zeros(problem.V, 8, device=dev)
        self.v = torch.zeros(problem.V, 8, device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.lr_pose, self.lr_expo = float(lr_pose), float(lr_expo)

    def apply(self, pose_grad: torch.Tensor, expo_grad: torch.Tensor):
        st = L.gs_view_adam_state(self.pb.cameras.data_ptr(), self.expo.data_ptr(), self.m.data_ptr(),
                                  self.v.data_ptr(), self.step.data_ptr())
        L.check(L.load().gs_view_adam_step(self.pb.V, C.byref(st), _ptr(pose_grad), _ptr(expo_grad), self.lr_pose,
                                           self.lr_expo, _stream()), "gs_view_adam_step")


# ------------------------------------------------------------------------------------------
# occupancy-aware fusion (Sim(3) action, voxel sets, deduplication)
# ------------------------------------------------------------------------------------------

def sim3_apply(g: Gaussians, q, t, s, out: Gaussians | None = None) -> Gaussians:
    """Eq. 19: the Sim(3) correction (rotation quaternion q (w,x,y,z), translation t, scale s)."""
    out = out if out is not None else Gaussians(*[torch.empty_like(getattr(g, k)) for k in
                                                  ("means", "log_scales", "quats", "opacities", "colors")])
    c = L.gs_sim3()
    for i in range(4):
        c.q[i] = float(q[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.s = float(s)
    gi = g.struct()
    go = L.gs_gaussian_arrays(*[getattr(out, k).data_ptr() for k in ("means", "log_scales", "quats", "opacities",
                                                                      "colors")])
    L.check(L.load().gs_sim3_apply(g.n, C.byref(gi), C.byref(c), C.byref(go), _stream()), "gs_sim3_apply")
    return out


class VoxSet:
    """A device hash set of packed voxel keys (Eqs. 20-22)."""

    def __init__(self, capacity: int, device="cuda"):
        cap = 1
        while cap < capacity:
            cap <<= 1
        self.capacity = max(cap, 2)
        self.mem = torch.empty(int(L.load().gs_voxset_bytes(self.capacity)), dtype=torch.uint8, device=device)
        self.clear()

    def clear(self):
        L.check(L.load().gs_voxset_clear(_ptr(self.mem), self.capacity, _stream()), "gs_voxset_clear")

    def add_boxes(self, means, log_scales, k, voxel):
        L.check(L.load().gs_voxset_add_boxes(_ptr(self.mem), self.capacity, int(means.shape[0]), _ptr(means),
                                             _ptr(log_scales), float(k), float(voxel), _stream()), "gs_voxset_add_boxes")

    def add_rays(self, cams, depth, stride, voxel):
        V, H, W = depth.shape
        L.check(L.load().gs_voxset_add_rays(_ptr(self.mem), self.capacity, V, W, H, _ptr(cams), _ptr(depth),
                                            int(stride), float(voxel), _stream()), "gs_voxset_add_rays")

    def status(self):
        """(recorded error code, number of stored keys); synchronises."""
        n = C.c_int64()
        rc = L.load().gs_voxset_status(_ptr(self.mem), _stream(), C.byref(n), self.capacity)
        return rc, int(n.value)

    def keys(self) -> set:
        k = self.mem[256:256 + 8 * self.capacity].view(torch.int64).cpu().numpy().view(np.uint64)
        return set(int(x) for x in k[k != np.uint64(0xFFFFFFFFFFFFFFFF)])


def dedup_keep(means, occ: VoxSet, free: VoxSet | None, voxel) -> torch.Tensor:
    """Eq. 22: uint8 keep flag per borrowed Gaussian."""
    n = int(means.shape[0])
    keep = torch.empty(n, dtype=torch.uint8, device=means.device)
    L.check(L.load().gs_voxset_keep(n, _ptr(means), _ptr(occ.mem), occ.capacity,
                                    None if free is None else _ptr(free.mem), 0 if free is None else free.capacity,
                                    float(voxel), _ptr(keep), _stream()), "gs_voxset_keep")
    return keep


# ------------------------------------------------------------------------------------------
# anchor-image photometric residuals of the submap pose graph (Eq. 12)
# ------------------------------------------------------------------------------------------

def pho_edges(edges, device="cuda") -> torch.Tensor:
    """Device array of gs_pho_edge from [(src_image, tgt_image, src_corr, tgt_corr, weight)]."""
    n = len(edges)
    raw = np.zeros((max(n, 1), 8), np.int32)
    for i, (a, b, ca, cb, w) in enumerate(edges):
        raw[i, :4] = (a, b, ca, cb)
        raw[i, 4] = np.array([w], np.float32).view(np.int32)[0]
    return torch.from_numpy(raw[:n].copy()).to(device)


def sim3_tensor(corrs, device="cuda") -> torch.Tensor:
    """[C, 8] float32 device array of gs_sim3 from [(q[4], t[3], s)]."""
    return torch.tensor(np.array([np.concatenate([np.asarray(q, np.float32), np.asarray(t, np.float32),
                                                  [np.float32(s)]]) for q, t, s in corrs], np.float32),
                        device=device)


class PhoResidual:
    """Eq. 12 photometric blocks of a batch of pose-graph edges (gs_pho_residual); the scratch is
    allocated once for `max_edges`."""

    def __init__(self, max_edges: int, device="cuda"):
        self.max_edges = max(1, int(max_edges))
        self.scratch = torch.empty(int(L.load().gs_pho_scratch_size(self.max_edges)), dtype=torch.uint8,
                                   device=device)

    def __call__(self, edges, images, depths, cams, corrs, stride=1, huber_delta=None, near_plane=None, out=None):
        """edges: device [E, 8] int32 (pho_edges); images [M, 3, H, W]; depths [M, H, W]; cams [M, 16];
        corrs [C, 8].  Returns dict(cost [E] f64, count [E] i64, H [E, 14, 14] f64, g [E, 14] f64)."""
        E = int(edges.shape[0])
        if E > self.max_edges:
            raise ValueError("more edges than the scratch was sized for")
        M, _, Hh, W = images.shape
        p = L.load().gs_default_pho_params()
        p.stride = int(stride)
        if huber_delta is not None:
            p.huber_delta = float(huber_delta)
        if near_plane is not None:
            p.near_plane = float(near_plane)
        dev = images.device
        o = out or dict(cost=torch.empty(E, dtype=torch.float64, device=dev),
                        count=torch.empty(E, dtype=torch.int64, device=dev),
                        H=torch.empty(E, 14, 14, dtype=torch.float64, device=dev),
                        g=torch.empty(E, 14, dtype=torch.float64, device=dev))
        L.check(L.load().gs_pho_residual(E, _ptr(edges), M, W, Hh, _ptr(images), _ptr(depths), _ptr(cams),
                                         int(corrs.shape[0]), _ptr(corrs), C.byref(p), _ptr(o["cost"]),
                                         _ptr(o["count"]), _ptr(o["H"]), _ptr(o["g"]), _ptr(self.scratch),
                                         self.scratch.numel(), _stream()), "gs_pho_residual")
        return o

