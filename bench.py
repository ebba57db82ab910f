#!/usr/bin/env python3
"""Benchmark: forward + backward views/s of the differentiable Gaussian rasterizer.

Workload (one step = one pass of the whole hot path over one view):
  500,000 Gaussians on the surfaces of a 6 x 5 x 3 m room with 12 furniture boxes, one 1200x680
  pinhole view (fx = fy = 600), seeded synthetic data; project -> bin + onesweep sort -> forward
  compositing -> L1(RGB) + 0.1 L1(depth) loss and gradient -> backward compositing + projection
  adjoint -> SE(3) pose gradient.
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

METRIC = "fwd+bwd views/s @1200x680, 500k Gaussians; batched vs per-view speedup"
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

    def __init__(self, R, S, wl, views, target_seed=21, key_capacity=None):
        import torch
        self.R, self.torch = R, torch
        sov = wl.scene_of_view[views]
        vb = wl.scene_offsets[sov]
        vc = wl.scene_offsets[sov + 1] - vb
        cams = R.cameras_tensor([wl.cameras[v] for v in views])
        self.pb = R.Problem(vb, vc, wl.scene.n, wl.width, wl.height, cams, key_capacity=key_capacity)
        self.g = R.Gaussians.from_scene(wl.scene)
        V, H, W = len(views), wl.height, wl.width
        self.V = V
        tgt = np.stack([S.smooth_image(W, H, target_seed + v) for v in range(V)])
        dtg = np.stack([S.smooth_image(W, H, target_seed + 100 + v, channels=1, lo=0.5, hi=5.0)[0] for v in range(V)])
        self.rgb_t = torch.from_numpy(tgt).cuda()
        self.depth_t = torch.from_numpy(dtg).cuda()
        self.img = self.pb.alloc_image()
        self.d_rgb = torch.empty_like(self.img["rgb"])
        self.d_depth = torch.empty_like(self.img["depth"])
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.grads = R.zeros_like_grads(self.g)
        self.pose = torch.zeros(V, 6, device="cuda")
        # size the key capacity once (outside any timing)
        self.pb.forward_checked(self.g, self.img)
        torch.cuda.synchronize()
        k = self.pb.stats()["num_keys"]
        if key_capacity is None and k * 1.3 + 4096 < self.pb.cap:
            self.pb.set_capacity(int(k * 1.3) + 4096)

    def zero_grads(self):
        import ctypes as C
        gg = self.R.L.gs_grads(*[getattr(self.grads, k).data_ptr() for k in ("means", "log_scales", "quats",
                                                                              "opacities", "colors")])
        self.R.L.check(self.R.L.load().gs_grads_zero(self.g.n, C.byref(gg), self.R._stream()), "gs_grads_zero")

    def step(self, ev=None):
        R, pb = self.R, self.pb
        rec = (lambda i: ev[i].record()) if ev else (lambda i: None)
        rec(0)
        pb.project(self.g)
        rec(1)
        pb.bin_sort()
        rec(2)
        pb.render_fwd(self.img)
        rec(3)
        R.loss_l1(self.img["rgb"], self.rgb_t, self.img["depth"], self.depth_t, 1.0, 0.1, self.d_rgb, self.d_depth,
                  self.loss)
        rec(4)
        self.zero_grads()
        pb.render_bwd(self.g, self.img, self.d_rgb, self.d_depth, None, self.grads)
        rec(5)
        pb.pose_grad(self.pose)
        rec(6)


STAGES = ["project", "bin_sort", "render_fwd", "loss", "render_bwd", "pose_grad"]


def l2_flush(buf):
    buf.zero_()


def time_steps(pipe, steps, warmup, flush_buf, torch):
    for _ in range(warmup):
        pipe.step()
    torch.cuda.synchronize()
    rc, _ = pipe.pb.check_status()
    if rc != 0:
        raise RuntimeError("device status %d during warm-up" % rc)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
    with Clocks() as clk:
        torch.cuda.synchronize()
        clk.mark_start()
        for i in range(steps):
            l2_flush(flush_buf)
            pipe.step(evs[i])
        torch.cuda.synchronize()
        clk.mark_end()
    step_ms = [e[0].elapsed_time(e[6]) for e in evs]
    stage_ms = {s: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, s in enumerate(STAGES)}
    return step_ms, stage_ms, clk.summary()


def time_e2e(pipe, steps, torch, flush_buf):
    """Same step through host buffers: H2D of the Gaussians, camera and targets from pinned memory,
    D2H of the loss, pose gradient and Gaussian gradients, all inside the timed region."""
    g = pipe.g
    host_in = {k: getattr(g, k).cpu().pin_memory() for k in ("means", "log_scales", "quats", "opacities", "colors")}
    host_cam = pipe.pb.cameras.cpu().pin_memory()
    host_t = pipe.rgb_t.cpu().pin_memory()
    host_dt = pipe.depth_t.cpu().pin_memory()
    out_g = {k: torch.empty_like(getattr(g, k), device="cpu").pin_memory() for k in host_in}
    out_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    out_pose = torch.empty(pipe.V, 6).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host_in.values()) + host_cam.numel() * 4 + \
        host_t.numel() * 4 + host_dt.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in out_g.values()) + 8 + out_pose.numel() * 4
    times = []
    for i in range(steps + 2):
        l2_flush(flush_buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k, t in host_in.items():
            getattr(g, k).copy_(t, non_blocking=True)
        pipe.pb.cameras.copy_(host_cam, non_blocking=True)
        pipe.rgb_t.copy_(host_t, non_blocking=True)
        pipe.depth_t.copy_(host_dt, non_blocking=True)
        pipe.step()
        out_loss.copy_(pipe.loss, non_blocking=True)
        out_pose.copy_(pipe.pose, non_blocking=True)
        for k, t in out_g.items():
            t.copy_(getattr(pipe.grads, k), non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if i >= 2:
            times.append(a.elapsed_time(b))
    return statistics.mean(times), h2d, d2h


def batched_speedup(R, S, torch, flush_buf, reps=3):
    wl = S.workload("agents8x4")
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


def cpu_baseline(seconds=12.0):
    """The FP64 oracle as it stands, timed on this host's cores on the same workload."""
    from oracle import losses as OL
    from oracle.oracle import Oracle
    from paper_2605_10760_gb300 import scenes as S
    wl = S.workload("room500k")
    W, H = wl.width, wl.height
    tgt = S.smooth_image(W, H, 21)[None]
    dtg = S.smooth_image(W, H, 121, channels=1, lo=0.5, hi=5.0)
    n, t0 = 0, time.perf_counter()
    while True:
        orc = Oracle.from_workload(wl)
        fw = orc.forward()
        _, g_rgb, g_d = OL.mapping_l1_loss(fw["rgb"], tgt, fw["depth"], dtg, 1.0, 0.1)
        orc.backward(g_rgb, g_d)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n / el, "unit": "views/s", "cores": threads, "kind": "oracle",
            "sample": "%d full fwd+bwd passes of the room500k view (FP64 values, FP32 decisions)" % n}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import losses as OL
    from oracle.oracle import Oracle
    from paper_2605_10760_gb300 import scenes as S
    wl = S.workload("room500k")
    W, H = wl.width, wl.height
    tgt = S.smooth_image(W, H, 21)[None]
    dtg = S.smooth_image(W, H, 121, channels=1, lo=0.5, hi=5.0)

    def one():
        orc = Oracle.from_workload(wl)
        fw = orc.forward()
        _, g_rgb, g_d = OL.mapping_l1_loss(fw["rgb"], tgt, fw["depth"], dtg, 1.0, 0.1)
        orc.backward(g_rgb, g_d)

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
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

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
    if world > 1:   # each rank its own camera in the room (weak scaling)
        wl.cameras = S.room_cameras(wl.scene, world, seed=11)
    pipe = Pipeline(R, S, wl, [rank if world > 1 else 0])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    launches0 = R.L.load().gs_launch_count()
    pipe.step()
    torch.cuda.synchronize()
    launches_per_step = R.L.load().gs_launch_count() - launches0
    stats = pipe.pb.stats()
    if world > 1:
        dist.barrier()
    step_ms, stage_ms, clocks = time_steps(pipe, args.steps, args.warmup, flush, torch)
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    rc, _ = pipe.pb.check_status()
    ms = total_ms / args.steps
    value = world * pipe.V / (ms / 1e3)
    e2e_ms, h2d, d2h = time_e2e(pipe, max(3, args.steps // 3), torch, flush)
    stats = pipe.pb.stats()
    if rank != 0:
        dist.barrier()
        return 0
    peaks = _peaks()
    # roofline of the dominant stage
    dom = max(stage_ms, key=stage_ms.get)
    P, K = pipe.pb.P, stats["num_keys"]
    passes = pipe.pb.workspace()["passes"]
    npx = pipe.V * pipe.pb.W * pipe.pb.H
    alg_bytes = {
        "project": P * 60 + 0,
        "bin_sort": P * 8 + K * 12 + K * 8 + passes * K * 24 + K * 8 + pipe.pb.V * 3225 * 8,
        "loss": npx * 48,
        "pose_grad": 0,
    }
    fp32_peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12   # TFLOP/s at max SM clock
    if dom in ("render_fwd", "render_bwd"):
        flops = stats["fwd_pairs"] * 33 if dom == "render_fwd" else stats["bwd_pairs"] * 90
        ach = flops / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None,
                "peak_note": "FP32 FMA pipes: 152 SM x 128 lanes x 2 FLOP x max SM clock (derived)"}
    else:
        ach = alg_bytes[dom] / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_note": "of %s" % peaks["src"]}
    batched = None if args.no_batched else batched_speedup(R, S, torch, flush)
    cpu = None if args.no_cpu else cpu_baseline()
    line = {
        "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": pipe.g.n, "width": 1200, "height": 680,
                   "loss": "L1(rgb) + 0.1 L1(depth)", "l2": "flushed between timed steps (256 MB write)",
                   "keys": K, "fwd_pairs": stats["fwd_pairs"], "bwd_pairs": stats["bwd_pairs"],
                   "status": rc},
        "stages_ms": stage_ms,
        "roofline": roof,
        "e2e": {"value": world * pipe.V / (e2e_ms / 1e3), "unit": "views/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "launches_per_step": launches_per_step,
        "batched": batched,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
