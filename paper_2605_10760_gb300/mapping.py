"""Graph-captured mapping loop and the tile/launch autotuner.

One mapping iteration (Sec. III-A: a submap optimised against its keyframe window by gradient
descent; Sec. III-C: the refinement loss of Eq. 23 with its SSIM term) is

    gs_project -> gs_bin_sort -> gs_render_fwd -> gs_loss_l1_ssim -> gs_render_bwd -> gs_pose_grad
    -> gs_adam_step (which also clears the gradients for the next iteration)

with no host synchronisation, so `iters` iterations are captured into one CUDA graph and replayed
with a single launch.  The number of duplicated keys K is data dependent; the workspace is sized
with headroom and every replay is followed (when checked) by gs_check_status, which reports
GS_ERR_CAPACITY with the K that was needed.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import raster as R

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


class MappingLoop:
    def __init__(self, problem: R.Problem, g: R.Gaussians, rgb_target: torch.Tensor,
                 lr=(1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3), w_l1=0.8, w_ssim=0.2, headroom=2.0, iso_weight=0.0):
        self.pb, self.g = problem, g
        self.iso_weight = float(iso_weight)      # lambda_s of Eq. 4's isotropy term (10 in the paper)
        self.rgb_t = rgb_target.contiguous()
        self.w_l1, self.w_ssim = float(w_l1), float(w_ssim)
        self.adam = R.AdamState(g, lr)
        self.grads = R.zeros_like_grads(g)
        self.img = problem.alloc_image()
        V, H, W = problem.V, problem.H, problem.W
        self.d_rgb = torch.empty_like(self.img["rgb"])
        self.loss = torch.zeros(1, dtype=torch.float64, device=g.means.device)
        self.pose = torch.zeros(V, 6, device=g.means.device)
        self.scratch = R.ssim_scratch(V, H, W, g.means.device)
        self.graph = None
        self.graph_iters = 0
        # size the key capacity from the first frame
        problem.forward_checked(g, self.img)
        torch.cuda.synchronize()
        k = problem.stats()["num_keys"]
        want = int(k * headroom) + 4096
        if want > problem.cap:
            problem.set_capacity(want)

    def iteration(self):
        pb = self.pb
        pb.project(self.g)
        pb.bin_sort()
        pb.render_fwd(self.img)
        R.loss_l1_ssim(self.img["rgb"], self.rgb_t, self.w_l1, self.w_ssim, self.d_rgb, self.loss, self.scratch)
        pb.render_bwd(self.g, self.img, self.d_rgb, None, None, self.grads)
        pb.pose_grad(self.pose)
        self.adam.apply(self.grads, zero_grads=True, iso_weight=self.iso_weight)

    def capture(self, iters: int = 100):
        """Capture `iters` iterations into one CUDA graph (after one eager warm-up iteration)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.iteration()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(iters):
                self.iteration()
        self.graph, self.graph_iters = g, iters
        return g

    def replay(self, check=False):
        self.graph.replay()
        if check:
            rc, req = self.pb.check_status()
            return rc, req
        return 0, 0


# (tile_w, tile_h, records per staged render batch) candidates of the autotuner
TUNE_CANDIDATES = ((16, 16, 256), (16, 16, 128), (16, 8, 128), (16, 8, 64), (32, 16, 256), (32, 16, 128))


def autotune(make_problem, g: R.Gaussians, rgb_target, candidates=TUNE_CANDIDATES, iters=5, reps=3,
             cache_key=None):
    """Time `iters` eager mapping iterations for each (tile shape, staged batch size) and return the
    fastest as (params kwargs, ms_per_iteration, table).  `make_problem(params)` builds a Problem.
    The choice is recorded in _build/autotune.json under cache_key."""
    table = []
    for tw, th, nb in candidates:
        params = R.default_params(tile_w=tw, tile_h=th, batch_records=nb)
        pb = make_problem(params)
        gg = R.Gaussians(*[getattr(g, k).clone() for k in ("means", "log_scales", "quats", "opacities", "colors")])
        loop = MappingLoop(pb, gg, rgb_target)
        loop.iteration()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(iters):
                loop.iteration()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b) / iters)
        rc, _ = pb.check_status()
        table.append({"tile": [tw, th], "batch_records": nb, "ms_per_iter": best, "status": rc})
        del loop, pb, gg
    ok = [t for t in table if t["status"] == 0]
    pick = min(ok, key=lambda t: t["ms_per_iter"])
    if cache_key:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        data = {}
        if os.path.exists(_CACHE):
            try:
                data = json.load(open(_CACHE))
            except Exception:  # noqa: BLE001
                data = {}
        data[cache_key] = {"pick": pick, "table": table, "when": time.time()}
        json.dump(data, open(_CACHE, "w"), indent=1)
    kw = dict(tile_w=pick["tile"][0], tile_h=pick["tile"][1], batch_records=pick["batch_records"])
    return kw, pick["ms_per_iter"], table


class RefineLoop:
    """Joint pose-Gaussian photometric refinement of a fused map (Sec. III-C): each iteration
    renders every keyframe, evaluates Eq. 23 on the exposure-compensated render
    (w_l1 = 1.75, w_ssim = 0.2, w_depth = 0.25), back-propagates to the Gaussians (Adam at half the
    per-agent learning rates) and to each keyframe's pose delta and exposure (per-view Adam, pose
    applied as T <- Exp(delta) T).  Iterations are graph-capturable like MappingLoop; pruning of
    Gaussians with opacity below 0.005 is a separate call (`prune`) that rebuilds the problem."""

    def __init__(self, problem: R.Problem, g: R.Gaussians, rgb_target, depth_target=None,
                 lr=(0.8e-4, 2.5e-3, 0.5e-3, 2.5e-2, 1.25e-3), lr_pose=1e-4, lr_expo=1e-3,
                 w_l1=1.75, w_ssim=0.2, w_depth=0.25, headroom=2.0):
        self.pb, self.g = problem, g
        self.rgb_t = rgb_target.contiguous()
        self.depth_t = None if depth_target is None else depth_target.contiguous()
        self.w = (float(w_l1), float(w_ssim), float(w_depth) if depth_target is not None else 0.0)
        self.adam = R.AdamState(g, lr)
        self.view = R.ViewAdamState(problem, lr_pose, lr_expo)
        self.grads = R.zeros_like_grads(g)
        self.img = problem.alloc_image()
        V, H, W = problem.V, problem.H, problem.W
        dev = g.means.device
        self.d_rgb = torch.empty_like(self.img["rgb"])
        self.d_depth = torch.empty_like(self.img["depth"]) if depth_target is not None else None
        self.d_expo = torch.zeros(V, 2, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.pose = torch.zeros(V, 6, device=dev)
        self.scratch = R.refine_scratch(V, H, W, dev)
        self.graph = None
        problem.forward_checked(g, self.img)
        torch.cuda.synchronize()
        want = int(problem.stats()["num_keys"] * headroom) + 4096
        if want > problem.cap:
            problem.set_capacity(want)

    def iteration(self):
        pb = self.pb
        pb.project(self.g)
        pb.bin_sort()
        pb.render_fwd(self.img)
        R.loss_refine(self.img["rgb"], self.rgb_t, self.view.expo, self.img["depth"], self.depth_t, *self.w,
                      d_rgb=self.d_rgb, d_depth=self.d_depth, d_expo=self.d_expo, loss=self.loss,
                      scratch=self.scratch)
        pb.render_bwd(self.g, self.img, self.d_rgb, self.d_depth, None, self.grads)
        pb.pose_grad(self.pose)
        self.adam.apply(self.grads, zero_grads=True)
        self.view.apply(self.pose, self.d_expo)

    capture = MappingLoop.capture
    replay = MappingLoop.replay
