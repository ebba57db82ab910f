#!/usr/bin/env python3
"""Benchmark: forward + backward views/s of the differentiable Gaussian rasterizer.

Workload (one step = one pass of the whole hot path over one view):
  500,000 Gaussians on the surfaces of a 6 x 5 x 3 m room with 12 furniture boxes, one 1200x680
  pinhole view (fx = fy = 600), seeded synthetic data; project -> bin + onesweep sort -> forward
  compositing with the L1(RGB) + 0.1 L1(depth) loss and its gradient fused into its epilogue ->
  backward compositing + projection adjoint -> SE(3) pose gradient.
Also measured in the same run: the batched multi-agent launch (8 submaps of 50k..400k Gaussians x 4
views = 32 views in one problem) against the same 32 views rendered one call at a time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank renders its own view of the room (weak scaling, no collective
on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

_WL_CACHE: dict = {}


def workload(S, name):
    """Seeded workload, generated once per process (the measurements below only read it)."""
    if name not in _WL_CACHE:
        _WL_CACHE[name] = S.workload(name)
    return _WL_CACHE[name]


METRIC = "fwd+bwd views/s @1200x680, 500k Gaussians; batched vs per-view speedup"
# algorithmic FP32 work per unit of the compositing kernels: per (pixel, list entry) pair visited by
# the forward (sigma, exp, alpha, transmittance, blend) and per pair walked by the backward
FLOP_FWD, FLOP_BWD = 25, 80
WORKLOAD = "room500k: 500k-Gaussian room, 1 view 1200x680 per step"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), src="measured", sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)))
    return dict(hbm_gbs=6800.0, src="fallback", sm_max_mhz=2070.0)


# ------------------------------------------------------------------------------------------
# clocks sampling during the timed region
# ------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampled every 20 ms in a background thread; summary() keeps the samples taken
    between mark_start() and mark_end() (the timed region), widened by 50 ms on each side."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index=0):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.time() + 5.0
            while not self.samples and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:  # noqa: BLE001
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.06)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        sel = [s for t, s in self.samples if self.t0 is not None and self.t0 - 0.05 <= t <= self.t1 + 0.05]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        num = lambda x: float(x) if x.replace(".", "", 1).isdigit() else None
        sm = [num(s[1]) for s in sel if len(s) > 2 and num(s[1]) is not None]
        mx = [num(s[2]) for s in sel if len(s) > 2 and num(s[2]) is not None]
        reasons = set()
        for s in sel:
            for i, n in enumerate(self.NAMES):
                if len(s) > 5 + i and s[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sel)}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
class Pipeline:
    """One fwd+bwd mapping step of a problem, every stage a libgs call."""

    def __init__(self, R, S, wl, views, target_seed=21, key_capacity=None, w_depth=0.1, uniform_target=False):
        import torch
        self.R, self.torch = R, torch
        self.w_depth = w_depth
        sov = wl.scene_of_view[views]
        vb = wl.scene_offsets[sov]
        vc = wl.scene_offsets[sov + 1] - vb
        cams = R.cameras_tensor([wl.cameras[v] for v in views])
        self.pb = R.Problem(vb, vc, wl.scene.n, wl.width, wl.height, cams, key_capacity=key_capacity)
        self.g = R.Gaussians.from_scene(wl.scene)
        V, H, W = len(views), wl.height, wl.width
        self.V = V
        tgt = np.stack([S.uniform_image(W, H, target_seed + v) if uniform_target else
                        S.smooth_image(W, H, target_seed + v) for v in range(V)])
        dtg = np.stack([S.smooth_image(W, H, target_seed + 100 + v, channels=1, lo=0.5, hi=5.0)[0] for v in range(V)])
        self.rgb_t = torch.from_numpy(tgt).cuda()
        self.depth_t = torch.from_numpy(dtg).cuda()
        self.img = self.pb.alloc_image()
        self.d_rgb = torch.empty_like(self.img["rgb"])
        self.d_depth = torch.empty_like(self.img["depth"])
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.grads = R.zeros_like_grads(self.g)
        self.pose = torch.zeros(V, 6, device="cuda")
        # size the key and visible-pair capacities once (outside any timing)
        self.pb.forward_checked(self.g, self.img)
        torch.cuda.synchronize()
        st = self.pb.stats()
        k, nv = st["num_keys"], st["num_visible"]
        if key_capacity is None and k * 1.3 + 4096 < self.pb.cap:
            self.pb.set_capacity(int(k * 1.3) + 4096, visible=int(nv * 1.3) + 4096)

    def zero_grads(self):
        import ctypes as C
        gg = self.R.L.gs_grads(*[getattr(self.grads, k).data_ptr() for k in ("means", "log_scales", "quats",
                                                                              "opacities", "colors")])
        self.R.L.check(self.R.L.load().gs_grads_zero(self.g.n, C.byref(gg), self.R._stream()), "gs_grads_zero")

    def stages(self, zero=True):
        pb = self.pb
        return [
            lambda: pb.project(self.g),
            lambda: pb.bin_sort(),
            # forward compositing with the L1 loss and its gradient in the same kernel's epilogue
            lambda: pb.render_fwd_l1(self.img, self.rgb_t, self.depth_t, 1.0, self.w_depth, self.d_rgb,
                                     self.d_depth, self.loss),
            lambda: pb.render_bwd_composite(self.img, self.d_rgb, self.d_depth, None),
            lambda: (zero and self.zero_grads(), pb.project_bwd(self.g, self.grads)),
            lambda: pb.pose_grad(self.pose),
        ]

    def step(self, ev=None):
        """Eager: every stage's libgs calls issued from the host."""
        for i, fn in enumerate(self.stages()):
            if ev:
                ev[i].record()
            fn()
        if ev:
            ev[len(STAGES)].record()

    def capture(self):
        """Capture each stage as its own CUDA graph (after one eager warm-up step), so a step is six
        graph launches with events between them."""
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graphs = []
        for fn in self.stages():
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr):
                fn()
            self.graphs.append(gr)
        # the whole step: the gradient zeroing runs on a branch of the graph forked after the
        # projection, concurrently with the sort (whose passes leave most SMs idle) and the
        # forward, and joined before the backward (a zeroing still running beside the persistent
        # compositing adjoint would wait for free SMs)
        self.whole = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.graph(self.whole):
            main = torch.cuda.current_stream()
            st = self.stages(zero=False)
            st[0]()
            side.wait_stream(main)
            with torch.cuda.stream(side):
                self.zero_grads()
            for fn in st[1:3]:
                fn()
            main.wait_stream(side)
            for fn in st[3:]:
                fn()
        torch.cuda.synchronize()

    def step_graph(self, ev=None):
        """Per-stage graphs with events between them (the stage breakdown)."""
        for i, gr in enumerate(self.graphs):
            if ev:
                ev[i].record()
            gr.replay()
        if ev:
            ev[len(STAGES)].record()

    def step_whole(self, ev=None):
        """The whole step as one graph launch (events only around it)."""
        if ev:
            ev[0].record()
        self.whole.replay()
        if ev:
            ev[len(STAGES)].record()


STAGES = ["project", "bin_sort", "render_fwd_l1", "render_bwd", "project_bwd", "pose_grad"]


# L2 flush buffer: 160 MB of int64 (GB300's L2 holds under 130 MB), written with 8-byte stores
FLUSH_WORDS = 20 << 20


def l2_flush(buf):
    buf.zero_()


def rank_views(S, wl, rank, world):
    """Weak scaling: with N ranks every rank renders its own camera of the room (N cameras drawn
    from one seed), so per-GPU work is fixed as N grows; a single process renders camera 0."""
    if world > 1:
        wl.cameras = S.room_cameras(wl.scene, world, seed=11)
        wl.scene_of_view = np.zeros(world, np.int32)
        return [rank]
    return [0]


def max_over_ranks(x, dist, device):
    """The slowest rank's value (timing only; no data-path collective)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(pipe, steps, warmup, flush_buf, torch, graphs=True, barrier=None, whole=False):
    run = (pipe.step_whole if whole else pipe.step_graph) if graphs else pipe.step
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    rc, _ = pipe.pb.check_status()
    if rc != 0:
        raise RuntimeError("device status %d during warm-up" % rc)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(steps)]
    with Clocks() as clk:
        if barrier:
            barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        for i in range(steps):
            l2_flush(flush_buf)
            run(evs[i])
        torch.cuda.synchronize()
        if barrier:
            barrier()
        clk.mark_end()
    step_ms = [e[0].elapsed_time(e[len(STAGES)]) for e in evs]
    stage_ms = None if whole and graphs else {
        s: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, s in enumerate(STAGES)}
    return step_ms, stage_ms, clk.summary()


def time_e2e(pipes, steps, torch, flush_buf):
    """Same step through host buffers, software-pipelined over two device copies of the problem:
    every step copies its Gaussians, camera and targets in from pinned host memory (copy stream),
    flushes L2 and runs the step (compute stream; the step's libgs calls replayed as one captured
    graph when the pipeline has one), and copies the loss, pose gradient and Gaussian
    gradients out to pinned host memory (second copy stream); step i's input copy overlaps step
    i-1's compute and step i-2's output copy.  The time runs from before the first input copy to
    after the last output copy; per step = total / steps."""
    host_in = {k: getattr(pipes[0].g, k).cpu().pin_memory() for k in ("means", "log_scales", "quats", "opacities",
                                                                      "colors")}
    host_cam = pipes[0].pb.cameras.cpu().pin_memory()
    host_t = pipes[0].rgb_t.cpu().pin_memory()
    host_dt = pipes[0].depth_t.cpu().pin_memory()
    outs = []
    for p in pipes:
        outs.append(dict(g={k: torch.empty_like(getattr(p.g, k), device="cpu").pin_memory() for k in host_in},
                         loss=torch.empty(1, dtype=torch.float64).pin_memory(),
                         pose=torch.empty(p.V, 6).pin_memory()))
    h2d = sum(t.numel() * t.element_size() for t in host_in.values()) + host_cam.numel() * 4 + \
        host_t.numel() * 4 + host_dt.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in outs[0]["g"].values()) + 8 + outs[0]["pose"].numel() * 4
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def run(n):
        ev_comp, ev_out = [None, None], [None, None]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(comp)
        s_in.wait_event(start)
        for i in range(n):
            b = i % 2
            p, o = pipes[b], outs[b]
            with torch.cuda.stream(s_in):
                if ev_comp[b] is not None:
                    s_in.wait_event(ev_comp[b])        # the last step on this copy has read its inputs
                for k, t in host_in.items():
                    getattr(p.g, k).copy_(t, non_blocking=True)
                p.pb.cameras.copy_(host_cam, non_blocking=True)
                p.rgb_t.copy_(host_t, non_blocking=True)
                p.depth_t.copy_(host_dt, non_blocking=True)
                e_in = s_in.record_event()
            comp.wait_event(e_in)
            if ev_out[b] is not None:
                comp.wait_event(ev_out[b])             # its previous results have been copied out
            l2_flush(flush_buf)
            if getattr(p, "whole", None) is not None:
                p.step_whole()                         # the step's libgs calls, captured as one graph
            else:
                p.step()
            ev_comp[b] = comp.record_event()
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_comp[b])
                o["loss"].copy_(p.loss, non_blocking=True)
                o["pose"].copy_(p.pose, non_blocking=True)
                for k, t in o["g"].items():
                    t.copy_(getattr(p.grads, k), non_blocking=True)
                ev_out[b] = s_out.record_event()
        end.record(s_out)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / n

    run(4)                                             # warm-up
    ms = run(steps)
    return ms, h2d, d2h


def cloud_bench(R, S, torch, flush_buf, steps=30, warmup=5):
    """Config 1 (cloud10k: 10k Gaussians, one 320x240 view, L1 against a U[0,1] target, pose
    gradient): the same step as the headline, replayed as one graph with L2 flushed before each."""
    wl = workload(S, "cloud10k")
    pipe = Pipeline(R, S, wl, [0], target_seed=2, w_depth=0.0, uniform_target=True)
    pipe.capture()
    step_ms, _, _ = time_steps(pipe, steps, warmup, flush_buf, torch, graphs=True, whole=True)
    rc, _ = pipe.pb.check_status()
    ms = statistics.median(step_ms)
    st = pipe.pb.stats()
    out = {"workload": "cloud10k: 10k Gaussians, 1 view 320x240, L1(rgb) vs a U[0,1] target + pose gradient",
           "ms_per_step": ms, "views_per_s": 1e3 / ms, "keys": st["num_keys"], "fwd_pairs": st["fwd_pairs"],
           "status": rc}
    del pipe
    return out


def batched_speedup(R, S, torch, flush_buf, reps=3):
    wl = workload(S, "agents8x4")
    V = len(wl.cameras)
    batched = Pipeline(R, S, wl, list(range(V)))
    singles = [Pipeline(R, S, wl, [v]) for v in range(V)]

    def run(pipes):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l2_flush(flush_buf)
        a.record()
        for p in pipes:
            p.step()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    for _ in range(2):
        run([batched])
        run(singles)
    tb = statistics.median([run([batched]) for _ in range(reps)])
    ts = statistics.median([run(singles) for _ in range(reps)])
    rc1, _ = batched.pb.check_status()
    # identical accuracy: the batched images equal the per-view images
    same = all(torch.equal(batched.img["last_idx"][v], singles[v].img["last_idx"][0]) and
               torch.equal(batched.img["rgb"][v], singles[v].img["rgb"][0]) for v in range(V))
    return {"workload": "agents8x4: 8 rooms (50k..400k Gaussians), 4 views each, 1200x680",
            "views": V, "batched_ms": tb, "per_view_ms": ts, "batched_views_per_s": V / tb * 1e3,
            "per_view_views_per_s": V / ts * 1e3, "speedup": ts / tb, "identical_images": bool(same),
            "status": rc1}


def mapping_graph(R, S, torch, iters=100, reps=2):
    """room1m: 1M-Gaussian room, 8 views; `iters` mapping iterations (project, bin + sort, forward,
    0.8 L1 + 0.2 (1 - SSIM), backward, pose gradient, Adam) captured in one CUDA graph; the tile
    shape and the staged batch size are picked first by the autotuner."""
    from paper_2605_10760_gb300 import mapping as M
    wl = workload(S, "room1m")
    V, H, W = len(wl.cameras), wl.height, wl.width
    cams = R.cameras_tensor(wl.cameras)
    tgt = torch.from_numpy(np.stack([S.smooth_image(W, H, 300 + v) for v in range(V)])).cuda()
    g0 = R.Gaussians.from_scene(wl.scene)

    def make(params):
        return R.Problem(np.zeros(V, np.int64), np.full(V, wl.scene.n, np.int64), wl.scene.n, W, H, cams,
                         params=params)

    kw, _, table = M.autotune(make, g0, tgt, iters=3, reps=2, cache_key="room1m_8views")
    tw, th = kw["tile_w"], kw["tile_h"]
    pb = make(R.default_params(**kw))
    loop = M.MappingLoop(pb, g0, tgt)
    loop.capture(iters)
    loop.replay()
    torch.cuda.synchronize()
    rc0, _ = pb.check_status()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        loop.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    rc, req = pb.check_status()
    ms_iter = statistics.median(times) / iters
    # the same loop with Eq. 4's isotropy regulariser (lambda_s = 10) fused into the Adam step
    pb_iso = make(R.default_params(**kw))
    loop_iso = M.MappingLoop(pb_iso, R.Gaussians.from_scene(wl.scene), tgt, iso_weight=10.0)
    loop_iso.capture(iters)
    loop_iso.replay()
    torch.cuda.synchronize()
    t_iso = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        loop_iso.replay()
        b.record()
        torch.cuda.synchronize()
        t_iso.append(a.elapsed_time(b))
    rc_iso, _ = pb_iso.check_status()
    return {"workload": "room1m: 1M-Gaussian room, 8 views 1200x680, 0.8 L1 + 0.2 (1-SSIM), Adam, "
                        "%d iterations per CUDA graph" % iters,
            "tile": [tw, th], "batch_records": kw["batch_records"], "autotune": table, "ms_per_iteration": ms_iter,
            "iterations_per_s": 1e3 / ms_iter, "views_per_s": V * 1e3 / ms_iter,
            "loss_after": float(loop.loss.item()), "status": rc or rc0, "required_keys": req,
            "with_isotropy": {"lambda_s": 10.0, "ms_per_iteration": statistics.median(t_iso) / iters,
                              "status": rc_iso}}


def refine_graph(R, S, torch, iters=100, reps=2):
    """room1m: joint pose / exposure / Gaussian refinement (Eq. 23 on the exposure-compensated
    render, 1.75 L1 + 0.2 (1 - SSIM) + 0.25 L1 depth, Adam on Gaussians at half the mapping rates,
    per-view Adam on pose deltas and exposures), 8 views, `iters` iterations per CUDA graph."""
    from paper_2605_10760_gb300 import mapping as M
    wl = workload(S, "room1m")
    V, H, W = len(wl.cameras), wl.height, wl.width
    cams = R.cameras_tensor(wl.cameras)
    tgt = torch.from_numpy(np.stack([S.smooth_image(W, H, 400 + v) for v in range(V)])).cuda()
    dtg = torch.from_numpy(np.stack([S.smooth_image(W, H, 500 + v, channels=1, lo=0.5, hi=5.0)[0]
                                     for v in range(V)])).cuda()
    pb = R.Problem(np.zeros(V, np.int64), np.full(V, wl.scene.n, np.int64), wl.scene.n, W, H, cams)
    loop = M.RefineLoop(pb, R.Gaussians.from_scene(wl.scene), tgt, dtg)
    loop.capture(iters)
    loop.replay()
    torch.cuda.synchronize()
    rc0, _ = pb.check_status()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        loop.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    rc, _ = pb.check_status()
    ms_iter = statistics.median(times) / iters
    return {"workload": "room1m: 1M-Gaussian room, 8 views, exposure-compensated refinement (Eq. 23), "
                        "%d iterations per CUDA graph" % iters,
            "ms_per_iteration": ms_iter, "iterations_per_s": 1e3 / ms_iter, "views_per_s": V * 1e3 / ms_iter,
            "status": rc or rc0}


# algorithmic FP32 work of one in-frame anchor pixel of the Eq. 12 kernel (FMA = 2): decision chain
# 94, bilinear sample + gradient + Huber + moments for 3 channels 81, A = d pi / d xi 53, the
# 2 x 2 fold 42, the 7-vector 28, the 28 upper-triangle entries 112
FLOP_PHO = 410
# HBM bytes per anchor pixel: source RGB + depth (16 B) and the target RGB once (12 B)
BYTES_PHO = 28


def normal_bench(R, S, torch, reps=20):
    """Normal term of Eq. 4 over 8 views at 1200x680: a smooth synthetic depth surface per view and a
    random camera-facing unit prior; inputs and gradient (~130 MB) exceed L2, and the L2 is flushed
    between timed calls."""
    V, H, W = 8, 680, 1200
    rng = np.random.default_rng(31)
    y, x = np.mgrid[0:H, 0:W].astype(np.float32)
    depth = np.stack([2.5 + 1.2 * x / W - 0.8 * y / H + 0.4 * np.sin(9.0 * x / W + v) * np.cos(7.0 * y / H)
                      for v in range(V)]).astype(np.float32)
    prior = rng.normal(size=(V, 3, H, W)).astype(np.float32)
    prior[:, 2] = -np.abs(prior[:, 2]) - 0.5
    prior /= np.linalg.norm(prior, axis=1, keepdims=True)
    cams = np.zeros((V, 16), np.float32)
    cams[:, 0] = cams[:, 4] = cams[:, 8] = 1.0
    cams[:, 12:16] = (600.0, 600.0, 600.0, 340.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d, p, c = t(depth), t(prior), t(cams)
    d_depth = torch.zeros_like(d)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(FLUSH_WORDS, dtype=torch.int64, device="cuda")
    for _ in range(3):
        R.loss_normal(d, p, c, 1e-2, d_depth, loss)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    n0 = R.L.load().gs_launch_count()
    for e0, e1 in evs:
        l2_flush(flush)
        e0.record(st)
        R.loss_normal(d, p, c, 1e-2, d_depth, loss)
        e1.record(st)
    torch.cuda.synchronize()
    ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)
    px = V * H * W
    # depth 4 B + prior 12 B read, d_depth 4 B read + 4 B written
    ach = 24.0 * px / (ms * 1e-3) / 1e9
    peaks = _peaks()
    return {"workload": "8 views 1200x680, smooth synthetic depth, random camera-facing prior, lambda_n 1e-2",
            "ms_per_call": ms, "pixels_per_s": px / (ms * 1e-3),
            "launches_per_call": (R.L.load().gs_launch_count() - n0) // reps,
            "loss_per_call": loss.item() / (reps + 3),
            "roofline": {"kernel": "k_normal", "bound": "hbm", "achieved": ach,
                         "unit": "GB/s", "peak": peaks["hbm_gbs"], "frac": ach / peaks["hbm_gbs"],
                         "bytes_per_pixel": 24}}


def pho_bench(R, S, torch, reps=20):
    """Eq. 12 photometric blocks of 16 pose-graph edges: 8 rooms of agents8x4 (50k..400k
    Gaussians), in each an anchor keyframe and a second one moved 8 cm / 2 deg, rendered at
    1200x680 (RGB + normalised depth); edges in both directions, a perturbed source correction."""
    from scipy.linalg import expm
    wl = workload(S, "agents8x4")
    cams, sov = [], []
    sk = lambda v: np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    for r in range(8):
        c = wl.cameras[4 * r]
        Rb = (expm(sk([0.01, -0.03, 0.02])) @ c.R.astype(np.float64)).astype(np.float32)
        tb = (c.t.astype(np.float64) + np.array([0.08, -0.02, 0.03])).astype(np.float32)
        cams += [c, S.Camera(Rb, tb, c.fx, c.fy, c.cx, c.cy, c.width, c.height)]
        sov += [r, r]
    sov = np.array(sov)
    vb = wl.scene_offsets[sov]
    vc = wl.scene_offsets[sov + 1] - vb
    pb = R.Problem(vb, vc, wl.scene.n, wl.width, wl.height, R.cameras_tensor(cams))
    img = pb.forward_checked(R.Gaussians.from_scene(wl.scene))
    a = img["alpha"]
    depth = torch.where(a > 0.5, img["depth"] / a.clamp_min(1e-6), torch.zeros_like(a)).contiguous()
    rgb = img["rgb"].contiguous()
    ident = ([1.0, 0, 0, 0], [0.0, 0, 0], 1.0)
    pert = ([0.99999, 0.002, -0.0015, 0.001], [0.005, -0.003, 0.003], 1.002)
    corrs = R.sim3_tensor([ident, pert])
    edges = R.pho_edges([e for r in range(8) for e in ((2 * r, 2 * r + 1, 1, 0, 1.0), (2 * r + 1, 2 * r, 0, 1, 1.0))])
    pr = R.PhoResidual(16)
    out = pr(edges, rgb, depth, pb.cameras, corrs)
    for _ in range(3):
        pr(edges, rgb, depth, pb.cameras, corrs, out=out)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = R.L.load().gs_launch_count()
    ev0.record(st)
    for _ in range(reps):
        pr(edges, rgb, depth, pb.cameras, corrs, out=out)
    ev1.record(st)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    count = out["count"].cpu().numpy()
    px = 16 * wl.width * wl.height
    inframe = int(count.sum())
    flops = FLOP_PHO * inframe + 94 * (px - inframe)
    ach = flops / (ms * 1e-3) / 1e12
    peak = 152 * 128 * 2 * _peaks()["sm_max_mhz"] * 1e6 / 1e12
    return {"workload": "agents8x4 anchor pairs: 16 edges, 1200x680 anchors, stride 1, Huber 9/255",
            "ms_per_call": ms, "edges_per_s": 16 / (ms * 1e-3), "anchor_pixels_per_s": px / (ms * 1e-3),
            "in_frame_fraction": inframe / px, "launches_per_call": (R.L.load().gs_launch_count() - n0) // reps,
            "roofline": {"kernel": "k_pho_edge + k_pho_finish", "bound": "alu", "achieved": ach, "unit": "TFLOP/s",
                         "peak": peak, "frac": ach / peak,
                         "hbm_gbs": BYTES_PHO * px / (ms * 1e-3) / 1e9}}


def fusion_bench(R, S, torch, voxel=0.05, k=3.0, stride=2, reps=3):
    """floor4m split into a target map (agents 0-7) and a borrowed map (agents 8-15, moved by a
    Sim(3) correction): Eq. 19 on the borrowed Gaussians, Eq. 20 occupied voxels of the target,
    Eq. 21 free voxels carved from 8 target keyframe depth maps (rendered, every 2nd pixel), Eq. 22
    keep flags of the borrowed Gaussians.  Times each stage with CUDA events."""
    wl = workload(S, "floor4m")
    ao = wl.meta["agent_offsets"]
    half = int(ao[8])
    g = R.Gaussians.from_scene(wl.scene)
    tgt = R.Gaussians(*[getattr(g, f)[:half].contiguous() for f in ("means", "log_scales", "quats", "opacities",
                                                                     "colors")])
    bor = R.Gaussians(*[getattr(g, f)[half:].contiguous() for f in ("means", "log_scales", "quats", "opacities",
                                                                     "colors")])
    views = list(range(8))
    cams = R.cameras_tensor([wl.cameras[v] for v in views])
    pb = R.Problem(np.zeros(8, np.int64), np.full(8, tgt.n, np.int64), tgt.n, wl.width, wl.height, cams)
    img = pb.forward_checked(tgt)
    a = img["alpha"]
    depth = torch.where(a > 0.5, img["depth"] / a.clamp_min(1e-6), torch.zeros_like(a)).contiguous()
    occ, fre = R.VoxSet(1 << 25), R.VoxSet(1 << 25)
    moved = R.sim3_apply(bor, [1.0, 0.0, 0.0, 0.02], [0.05, -0.03, 0.0], 1.01)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    t = {"sim3": [], "occupied": [], "free": [], "keep": []}
    for _ in range(reps):
        occ.clear()
        fre.clear()
        ev[0].record()
        R.sim3_apply(bor, [1.0, 0.0, 0.0, 0.02], [0.05, -0.03, 0.0], 1.01, out=moved)
        ev[1].record()
        occ.add_boxes(tgt.means, tgt.log_scales, k, voxel)
        ev[2].record()
        fre.add_rays(pb.cameras, depth, stride, voxel)
        ev[3].record()
        keep = R.dedup_keep(moved.means, occ, fre, voxel)
        ev[4].record()
        torch.cuda.synchronize()
        for i, key in enumerate(t):
            t[key].append(ev[i].elapsed_time(ev[i + 1]))
    rc_o, n_o = occ.status()
    rc_f, n_f = fre.status()
    kept = int(keep.sum().item())
    ms = {key: statistics.median(val) for key, val in t.items()}
    hbm = _peaks()["hbm_gbs"]
    # Sim(3) reads and writes 56 B per Gaussian.  The keep pass reads a mean (12 B) and writes a
    # flag (1 B) per Gaussian, and each distinct voxel of the borrowed means needs one 32-byte sector
    # of each voxel table (256 MB each, far larger than L2, so a first probe is a random DRAM
    # sector; Gaussians that share a voxel share its sectors)
    sim3_gbs = bor.n * 112 / (ms["sim3"] * 1e-3) / 1e9
    vk = np.floor(moved.means.cpu().numpy().astype(np.float64) / voxel).astype(np.int64)
    distinct = int(np.unique(vk[:, 0] * (1 << 42) + vk[:, 1] * (1 << 21) + vk[:, 2]).size)
    keep_bytes = bor.n * 13 + distinct * 64
    keep_gbs = keep_bytes / (ms["keep"] * 1e-3) / 1e9
    rays = 8 * ((wl.width + stride - 1) // stride) * ((wl.height + stride - 1) // stride)
    return {"workload": "floor4m halves: 2M target / 2M borrowed Gaussians, 8 keyframes 1200x680 (stride 2), "
                        "voxel %.2f m, k = %g" % (voxel, k),
            "ms": ms, "total_ms": sum(ms.values()), "borrowed": bor.n, "kept": kept,
            "occupied_voxels": n_o, "free_voxels": n_f, "status": [rc_o, rc_f], "rays": rays,
            "roofline": {"sim3": {"bound": "hbm", "achieved": sim3_gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": sim3_gbs / hbm},
                         "keep": {"bound": "hbm", "achieved": keep_gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": keep_gbs / hbm, "bytes": keep_bytes, "distinct_voxels": distinct,
                                  "note": "13 B per Gaussian + one 32-byte sector of each table per distinct "
                                          "voxel (random DRAM sectors)"},
                         "occupied_gaussians_per_s": tgt.n / (ms["occupied"] * 1e-3),
                         "free_rays_per_s": rays / (ms["free"] * 1e-3),
                         "note": "hash insertion (occupied, free) is bound by L2 compare-and-swap traffic"}}


def fused_map(R, S, torch, steps=3):
    """floor4m: 16 agents' submaps merged into 4M Gaussians (multi-room floor), 64 views in one
    batched problem, forward + backward with per-view pose gradients."""
    wl = workload(S, "floor4m")
    V = len(wl.cameras)
    pipe = Pipeline(R, S, wl, list(range(V)))
    pipe.step()
    torch.cuda.synchronize()
    times, stage = [], {k: [] for k in STAGES}
    for _ in range(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
        pipe.step(ev)
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[-1]))
        for i, k in enumerate(STAGES):
            stage[k].append(ev[i].elapsed_time(ev[i + 1]))
    rc, _ = pipe.pb.check_status()
    st = pipe.pb.stats()
    ms = statistics.median(times)
    wsv = pipe.pb.workspace()
    out = {"workload": "floor4m: 4M Gaussians (16 submaps), 64 views 1200x680", "views": V, "ms_per_step": ms,
           "views_per_s": V * 1e3 / ms, "stages_ms": {k: statistics.median(v) for k, v in stage.items()},
           "keys": st["num_keys"], "sort_passes": wsv["passes"],
           "fwd_pairs": st["fwd_pairs"], "bwd_pairs": st["bwd_pairs"], "status": rc,
           "workspace_gb": pipe.pb.ws_bytes / 1e9}
    del wsv
    del pipe
    torch.cuda.empty_cache()
    return out


# CPU-baseline samples: (workload, views, loss weight of depth, label).  The agents8x4 sample is
# the first camera of four of its rooms (50k, 120k, 200k and 330k Gaussians): a labelled subset.
CPU_SAMPLES = {
    "cloud10k": (None, 0.0, "cloud10k: 10k Gaussians, 1 view 320x240, L1(rgb)"),
    "room500k": (None, 0.1, "room500k: 500k-Gaussian room, 1 view 1200x680, L1(rgb) + 0.1 L1(depth)"),
    "agents8x4": ([0, 9, 18, 27], 0.1, "agents8x4 subset: views 0, 9, 18, 27 (rooms of 50k, 120k, 200k, 330k "
                                       "Gaussians) at 1200x680, L1(rgb) + 0.1 L1(depth)"),
}


def oracle_pass(S, wl, views, w_depth, seed=21):
    """One full oracle fwd + bwd pass over the given views: a closure to time."""
    from oracle import losses as OL
    from oracle.oracle import Oracle
    views = list(range(len(wl.cameras))) if views is None else list(views)
    W, H = wl.width, wl.height
    tgt = np.stack([S.smooth_image(W, H, seed + i) for i in range(len(views))])
    dtg = np.stack([S.smooth_image(W, H, seed + 100 + i, channels=1, lo=0.5, hi=5.0)[0] for i in range(len(views))])

    def one():
        orc = Oracle.from_workload(wl, views=views)
        fw = orc.forward()
        _, g_rgb, g_d = OL.mapping_l1_loss(fw["rgb"], tgt, fw["depth"], dtg, 1.0, w_depth)
        orc.backward(g_rgb, g_d)
    return one, len(views)


def cpu_sample(name, seconds):
    """Time the oracle as it stands on one CPU sample; the process's OMP_NUM_THREADS sets its threads."""
    from paper_2605_10760_gb300 import scenes as S
    views, w_depth, label = CPU_SAMPLES[name]
    wl = S.workload(name)
    one, nv = oracle_pass(S, wl, views, w_depth)
    n, t0 = 0, time.perf_counter()
    while True:
        one()
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * nv / el, "unit": "views/s", "cores": threads, "kind": "oracle",
            "sample": "%d fwd+bwd pass(es) of %s (FP64 values, FP32 decisions)" % (n, label)}


def cpu_baseline(seconds=4.0):
    """The FP64 oracle as it stands, timed on this host's cores: configs 1-3 on all cores and on one
    core, each sample in a child process whose OMP_NUM_THREADS is the core count (the oracle's
    OpenMP pool is sized once per process).  The headline figure is room500k on all cores."""
    allc = os.cpu_count() or 1
    out = {"all_cores": {}, "one_core": {}}
    for key, threads in (("all_cores", allc), ("one_core", 1)):
        for name in CPU_SAMPLES:
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", name,
                                "--cpu-seconds", str(seconds)], env=env, capture_output=True, text=True)
            try:
                out[key][name] = json.loads(r.stdout.strip().splitlines()[-1])
            except (IndexError, ValueError):
                out[key][name] = {"error": (r.stderr or r.stdout)[-300:]}
    head = out["all_cores"].get("room500k", {})
    return {"value": head.get("value"), "unit": "views/s", "cores": allc, "kind": "oracle",
            "sample": head.get("sample"), **out}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2605_10760_gb300 import scenes as S
    wl = S.workload("room500k")
    one, _ = oracle_pass(S, wl, None, 0.1)

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    el = time.perf_counter() - t0
    v = args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "views/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "views/s", "cores": cores, "kind": "oracle",
                             "sample": "each step one full fwd+bwd pass of the room500k view"},
            "e2e": {"value": v, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the graph-loop and 4M/64-view measurements")
    ap.add_argument("--cpu-sample", choices=sorted(CPU_SAMPLES), help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=4.0, help=argparse.SUPPRESS)
    ap.add_argument("--only", choices=["photometric", "normal", "fusion", "mapping", "refine", "fused", "batched"],
                    help="run one secondary measurement alone and print its JSON (not the headline line)")
    args = ap.parse_args()
    if args.cpu_sample:       # child process of cpu_baseline(): one oracle timing, no GPU
        print(json.dumps(cpu_sample(args.cpu_sample, args.cpu_seconds)))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.only:
        import torch
        from paper_2605_10760_gb300 import raster as R
        from paper_2605_10760_gb300 import scenes as S
        R.L.load()
        flush = torch.empty(FLUSH_WORDS, dtype=torch.int64, device="cuda")
        fn = {"photometric": pho_bench, "normal": normal_bench, "fusion": fusion_bench, "mapping": mapping_graph,
              "refine": refine_graph,
              "fused": fused_map, "batched": lambda R, S, torch: batched_speedup(R, S, torch, flush)}[args.only]
        print(json.dumps({"section": args.only, "result": fn(R, S, torch)}))
        return 0

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2605_10760_gb300 import raster as R
    from paper_2605_10760_gb300 import scenes as S
    R.L.load()
    wl = S.workload("room500k")
    pipe = Pipeline(R, S, wl, rank_views(S, wl, rank, world))
    flush = torch.empty(FLUSH_WORDS, dtype=torch.int64, device="cuda")
    launches0 = R.L.load().gs_launch_count()
    pipe.step()
    torch.cuda.synchronize()
    launches_per_step = R.L.load().gs_launch_count() - launches0
    stats = pipe.pb.stats()
    pipe.capture()
    eager_ms, eager_stage_ms, _ = time_steps(pipe, max(5, args.steps // 3), 2, flush, torch, graphs=False)
    barrier = dist.barrier if world > 1 else None
    _, stage_ms, _ = time_steps(pipe, args.steps, args.warmup, flush, torch, graphs=True)
    step_ms, _, clocks = time_steps(pipe, args.steps, args.warmup, flush, torch, graphs=True, barrier=barrier,
                                    whole=True)
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
    rc, _ = pipe.pb.check_status()
    ms = total_ms / args.steps
    value = world * pipe.V / (ms / 1e3)
    pipe2 = Pipeline(R, S, wl, rank_views(S, wl, rank, world))
    pipe2.capture()
    e2e_ms, h2d, d2h = time_e2e([pipe, pipe2], args.steps, torch, flush)
    del pipe2
    stats = pipe.pb.stats()
    if rank != 0:
        dist.barrier()
        return 0
    peaks = _peaks()
    # roofline of the dominant stage
    dom = max(stage_ms, key=stage_ms.get)
    P, K = pipe.pb.P, stats["num_keys"]
    wsv = pipe.pb.workspace()
    passes, G = wsv["passes"], wsv["tile_ranges"].shape[0]
    onesweep = pipe.pb.params.sort_mode == R.L.GS_SORT_ONESWEEP
    vis = int((wsv["tiles_touched"] != 0).sum().item()) if not onesweep else 0
    npx = pipe.V * pipe.pb.W * pipe.pb.H
    alg_bytes = {
        "project": P * 60 + 0,
        "bin_sort": (P * 8 + K * 12 + passes * K * 24 + K * 8 + G * 8) if onesweep else
                    (G * 8 + vis * 32 + K * 12 + K * 116),
        "render_fwd_l1": npx * 48,
        "project_bwd": P * 60,
        "pose_grad": 0,
    }
    fp32_peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12   # TFLOP/s at max SM clock
    # DRAM bytes (read + write) of one launch from an ncu capture of this workload's current
    # kernel code (profiles/*_room500k.md); a stage without such a capture reports None
    traffic = {"render_fwd_l1": 26_724_352, "render_bwd": 35_204_864}
    if dom in ("render_fwd_l1", "render_bwd"):
        flops = stats["fwd_pairs"] * FLOP_FWD if dom == "render_fwd_l1" else stats["bwd_pairs"] * FLOP_BWD
        ach = flops / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": traffic.get(dom),
                "peak_note": "FP32 FMA pipes: 152 SM x 128 lanes x 2 FLOP x max SM clock (derived)"}
    else:
        ach = alg_bytes[dom] / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic.get(dom), "peak_note": "of %s" % peaks["src"]}
    cloud = cloud_bench(R, S, torch, flush)
    batched = None if args.no_batched else batched_speedup(R, S, torch, flush)
    graph_loop = None if args.no_extra else mapping_graph(R, S, torch)
    refine = None if args.no_extra else refine_graph(R, S, torch)
    fusion = None if args.no_extra else fusion_bench(R, S, torch)
    pho = None if args.no_extra else pho_bench(R, S, torch)
    fused = None if args.no_extra else fused_map(R, S, torch)
    normal = None
    if not args.no_extra:      # the last device work of the run; an error is reported in the line
        try:
            normal = normal_bench(R, S, torch)
        except Exception as e:  # noqa: BLE001
            normal = {"error": repr(e)[:300]}
    cpu = None if args.no_cpu else cpu_baseline()
    line = {
        "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": pipe.g.n, "width": 1200, "height": 680,
                   "loss": "L1(rgb) + 0.1 L1(depth)", "l2": "flushed between timed steps (160 MB write; L2 under 130 MB)",
                   "keys": K, "sort_passes": passes,
                   "fwd_pairs": stats["fwd_pairs"], "bwd_pairs": stats["bwd_pairs"],
                   "status": rc},
        "stages_ms": stage_ms,
        "timing": "value: the whole step replayed as one CUDA graph, events around each step, L2 flushed "
                  "before each; stages_ms: each stage as its own graph with events between stages; eager "
                  "(host-issued) step for comparison in eager_ms_per_step",
        "eager_ms_per_step": statistics.mean(eager_ms), "eager_stages_ms": eager_stage_ms,
        "roofline": roof,
        "e2e": {"value": world * pipe.V / (e2e_ms / 1e3), "unit": "views/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "launches_per_step": launches_per_step,
        "cloud10k": cloud,
        "batched": batched,
        "mapping_graph": graph_loop,
        "refine_graph": refine,
        "fusion": fusion,
        "photometric": pho,
        "normal_loss": normal,
        "fused_map": fused,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
