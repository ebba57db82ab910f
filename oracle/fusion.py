"""Oracle of the occupancy-aware fusion steps (Sec. III-C, Eqs. 19-22).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU baseline).

* Eq. 19, the Sim(3) action of a submap correction C = (s, R, t) on a Gaussian:
  mu' = s R mu + t, Sigma' = s^2 R Sigma R^T (so rotation q' = q_R (x) q and per-axis scales
  s_i' = s s_i, i.e. log-scales + ln s), opacity and colour unchanged.  FP64.
* Voxel index kappa(x) = floor(x / v) per axis, packed into a 64-bit key (21 bits per axis, offset
  2^20).  The voxel decisions are taken in FP32 with a fixed operation order so that any FP32
  implementation following it produces the same voxel sets bit for bit:
    - Eq. 20, occupied voxels of the target map: every voxel of the box
      [kappa(mu - k s), kappa(mu + k s)] with s = exp(log-scales) (the decision-chain exp),
      k s and mu -/+ k s rounded once each;
    - Eq. 21, free voxels: for each (strided) pixel with depth d > 0 of each keyframe, the voxels
      crossed by the segment from the camera centre c (t = 0) to the back-projected point r (t = 1),
      t in [0, 1), found by a 3-D digital differential analyser (Amanatides-Woo traversal) whose
      steps are specified operation by operation (ties between axes go to the lowest axis);
    - Eq. 22, a borrowed Gaussian is kept iff kappa(mu) is in neither set.
Readings: the paper names neither k nor the voxel size v (parameters here, k = 3 by default);
the box of Eq. 20 uses the per-axis scale vector directly, as written.
"""
from __future__ import annotations

import ctypes
import ctypes.util

import numpy as np

from .oracle import expf

F = np.float32
KEY_BITS = 21
KEY_OFF = 1 << 20

_libm = ctypes.CDLL(ctypes.util.find_library("m"))
_libm.fmaf.restype = ctypes.c_float
_libm.fmaf.argtypes = [ctypes.c_float] * 3


def _fmaf(a, b, c):
    return F(_libm.fmaf(float(a), float(b), float(c)))


def quat_mul(a, b):
    """Hamilton product of (w, x, y, z) quaternions (FP64)."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], -1)


def quat_to_matrix(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def sim3_apply(means, log_scales, quats, s, q_rot, t):
    """Eq. 19 in FP64.  Returns (means', log_scales', quats')."""
    R = quat_to_matrix(np.asarray(q_rot, np.float64))
    mu = s * (np.asarray(means, np.float64) @ R.T) + np.asarray(t, np.float64)
    qn = np.asarray(q_rot, np.float64) / np.linalg.norm(q_rot)
    return mu, np.asarray(log_scales, np.float64) + np.log(s), quat_mul(qn, np.asarray(quats, np.float64))


# ------------------------------------------------------------------------------------------
# voxel keys and sets (FP32 decisions)
# ------------------------------------------------------------------------------------------

def _clamp_idx(i):
    return np.clip(i, -KEY_OFF, KEY_OFF - 1)


def pack(ix, iy, iz):
    ix, iy, iz = (np.asarray(_clamp_idx(a), np.int64) + KEY_OFF for a in (ix, iy, iz))
    return (ix << (2 * KEY_BITS)) | (iy << KEY_BITS) | iz


def voxel_index(x, v):
    """floor(fl(x / v)) of float32 coordinates, per element."""
    return np.floor(np.asarray(x, F) / F(v)).astype(np.int64)


def occupied_set(means, log_scales, k, v):
    """Eq. 20 (see module docstring).  Returns a Python set of packed keys."""
    mu = np.asarray(means, F)
    s = expf(np.asarray(log_scales, F))
    ks = (F(k) * s).astype(F)
    lo = voxel_index((mu - ks).astype(F), v)
    hi = voxel_index((mu + ks).astype(F), v)
    out = set()
    for i in range(mu.shape[0]):
        xs = np.arange(lo[i, 0], hi[i, 0] + 1)
        ys = np.arange(lo[i, 1], hi[i, 1] + 1)
        zs = np.arange(lo[i, 2], hi[i, 2] + 1)
        X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
        out.update(pack(X.ravel(), Y.ravel(), Z.ravel()).tolist())
    return out


def camera_center(cam):
    """c = -R^T t in FP32: c_a = -fma(R0a, t0, fma(R1a, t1, R2a * t2))."""
    R = np.asarray(cam[:9], F).reshape(3, 3)
    t = np.asarray(cam[9:12], F)
    return np.array([-_fmaf(R[0, a], t[0], _fmaf(R[1, a], t[1], F(R[2, a] * t[2]))) for a in range(3)], F)


def backproject(cam, x, y, d):
    """World point of pixel (x, y) (sampled at +0.5) at camera depth d, FP32 fixed order."""
    R = np.asarray(cam[:9], F).reshape(3, 3)
    t = np.asarray(cam[9:12], F)
    fx, fy, cx, cy = (F(c) for c in cam[12:16])
    d = F(d)
    xn = F(F(F(x) + F(0.5) - cx) / fx)
    yn = F(F(F(y) + F(0.5) - cy) / fy)
    pc = (F(xn * d) - t[0], F(yn * d) - t[1], F(d - t[2]))
    pc = tuple(F(p) for p in pc)
    return np.array([_fmaf(R[0, a], pc[0], _fmaf(R[1, a], pc[1], F(R[2, a] * pc[2]))) for a in range(3)], F)


def dda_voxels(c, r, v, max_steps=1 << 16):
    """Voxels crossed by the segment c + t (r - c), t in [0, 1) (FP32 traversal)."""
    v = F(v)
    cur = [int(np.floor(F(c[a] / v))) for a in range(3)]
    d = [F(F(r[a]) - F(c[a])) for a in range(3)]
    step, tmax, tdel = [0] * 3, [F(np.inf)] * 3, [F(np.inf)] * 3
    for a in range(3):
        if d[a] > 0:
            step[a] = 1
            tmax[a] = F(F(F(F(cur[a] + 1) * v) - F(c[a])) / d[a])
            tdel[a] = F(v / d[a])
        elif d[a] < 0:
            step[a] = -1
            tmax[a] = F(F(F(F(cur[a]) * v) - F(c[a])) / d[a])
            tdel[a] = F(-v / d[a])
    out = [tuple(cur)]
    for _ in range(max_steps):
        a = 0
        if tmax[1] < tmax[a]:
            a = 1
        if tmax[2] < tmax[a]:
            a = 2
        if not (tmax[a] < F(1.0)):
            break
        cur[a] += step[a]
        tmax[a] = F(tmax[a] + tdel[a])
        out.append(tuple(cur))
    return out


def free_set(cams, depth, v, stride=1):
    """Eq. 21: voxels carved by the rays of every stride-th pixel (row and column) with depth > 0."""
    out = set()
    V, H, W = depth.shape
    for k in range(V):
        c = camera_center(cams[k])
        for y in range(0, H, stride):
            for x in range(0, W, stride):
                d = depth[k, y, x]
                if not (d > 0) or not np.isfinite(d):
                    continue
                r = backproject(cams[k], x, y, d)
                vox = dda_voxels(c, r, v)
                out.update(int(pack(a, b, cc)) for a, b, cc in vox)
    return out


def dedup_keep(means, occ, free, v):
    """Eq. 22: keep iff kappa(mu) is in neither set."""
    idx = voxel_index(np.asarray(means, F), v)
    keys = pack(idx[:, 0], idx[:, 1], idx[:, 2])
    return np.array([(int(kk) not in occ) and (int(kk) not in free) for kk in keys], bool)
