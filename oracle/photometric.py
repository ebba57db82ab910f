"""Oracle of the anchor-image photometric residual of the submap pose graph (Sec. III-B, Eq. 12)
and its Jacobians w.r.t. the two submap corrections, reduced to robust Gauss-Newton blocks.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU baseline).

For an inter-agent edge e with a source anchor keyframe (image I_s, depth D_s, camera K_s, world-
to-camera pose (R_s, t_s) in its submap) and a target anchor keyframe (I_t, K_t, (R_a, t_a) in its
submap), and submap corrections C_src, C_tgt in Sim(3) (x -> s R(q) x + t, submap to global):

  p(u)  = R_s^T (d(u) K_s^-1 [u + 0.5, 1] - t_s)       back-projection of anchor pixel u
  w     = C_src p,  q = C_tgt^-1 w,  c = R_a q + t_a     (Eq. 12's C_tgt^-1 o C_src . p_src(u))
  r_ch(u) = I_s,ch(u) - I_t,ch(pi_t(c))                    one residual per colour channel
  pi_t(c) = (f_x c_x / c_z + c_x0, f_y c_y / c_z + c_y0), sampled bilinearly at pi_t - 0.5.

U_e (the in-frame, finite-depth anchor-pixel set) holds the anchor pixels (every `stride`-th row
and column) with 0 < d < inf, c_z > near, and both bilinear taps inside the target image.
Perturbations are left Sim(3) twists xi = (rho, phi, sigma) (translation, rotation, log-scale) of
the global frame: C <- Exp(xi) C, so dw/dxi_src = [I, -[w]x, w] and dq/dxi_tgt = -dq/dxi_src.
Robust norm: Huber per scalar residual with threshold delta (IRLS weight 1 or delta/|r|).
Per edge (n = |U_e|, w_e the edge weight):
  cost = (w_e / n) sum rho(r),  H = (w_e / n) sum omega J^T J,  g = (w_e / n) sum omega J^T r
with J = dr/d(xi_src, xi_tgt) (1 x 14); the cost gradient is 2 g.  Empty U_e gives zeros.

Readings (the paper gives none of these): the robust norm is Huber with delta = 9/255; pixel
centres at +0.5 (as in the rasterizer); near plane 0.2; the anchor depth is the keyframe's z-depth.
The membership of U_e and the bilinear cell are integer decisions: they are taken in FP32 with the
fixed operation sequence of `decision_chain` (IEEE-rounded multiply, add, subtract, divide and
square root, no fused multiply-add; divisions by f_x, f_y and s_tgt are multiplications by their
rounded reciprocals, and 1 / c_z is rounded once per pixel), values in FP64.
"""
from __future__ import annotations

import numpy as np

F = np.float32
HUBER_DELTA = 9.0 / 255.0
NEAR = 0.2


# ------------------------------------------------------------------------------------------
# FP32 decision chain (vectorised numpy float32: every operation rounds once)
# ------------------------------------------------------------------------------------------

def quat_matrix_f32(q):
    """Rotation matrix of a (w, x, y, z) quaternion, normalised first, in FP32."""
    w, x, y, z = (F(v) for v in q)
    n = F(np.sqrt(F(F(F(w * w) + F(x * x)) + F(y * y)) + F(z * z)))
    w, x, y, z = F(w / n), F(x / n), F(y / n), F(z / n)
    two, one = F(2.0), F(1.0)
    return np.array([
        [F(one - F(two * F(F(y * y) + F(z * z)))), F(two * F(F(x * y) - F(w * z))), F(two * F(F(x * z) + F(w * y)))],
        [F(two * F(F(x * y) + F(w * z))), F(one - F(two * F(F(x * x) + F(z * z)))), F(two * F(F(y * z) - F(w * x)))],
        [F(two * F(F(x * z) - F(w * y))), F(two * F(F(y * z) + F(w * x))), F(one - F(two * F(F(x * x) + F(y * y))))],
    ], F)


def _mv(M, v):
    """(M v)_i = (M_i0 v_0 + M_i1 v_1) + M_i2 v_2, each operation rounded to FP32."""
    return [F(F(F(M[i, 0] * v[0]) + F(M[i, 1] * v[1])) + F(M[i, 2] * v[2])) for i in range(3)]


def _mtv(M, v):
    """(M^T v)_i = (M_0i v_0 + M_1i v_1) + M_2i v_2, each operation rounded to FP32."""
    return [F(F(F(M[0, i] * v[0]) + F(M[1, i] * v[1])) + F(M[2, i] * v[2])) for i in range(3)]


def decision_chain(cam_s, cam_t, sim_s, sim_t, W, H, depth, stride=1, near=NEAR):
    """FP32 decisions for every strided anchor pixel: (valid mask, x0, y0, sx, sy, xs, ys).

    cam_*: 16 floats (R row-major, t, fx, fy, cx, cy); sim_*: (q[4], t[3], s)."""
    ys, xs = np.meshgrid(np.arange(0, H, stride), np.arange(0, W, stride), indexing="ij")
    ys, xs = ys.ravel(), xs.ravel()
    d = np.asarray(depth, F)[ys, xs]
    cs = np.asarray(cam_s, F)
    ct = np.asarray(cam_t, F)
    Rs, ts = cs[:9].reshape(3, 3), cs[9:12]
    Ra, ta = ct[:9].reshape(3, 3), ct[9:12]
    with np.errstate(all="ignore"):
        ifx, ify = F(F(1.0) / cs[12]), F(F(1.0) / cs[13])
        xn = (F(F(xs.astype(F) + F(0.5)) - cs[14]) * ifx).astype(F)
        yn = (F(F(ys.astype(F) + F(0.5)) - cs[15]) * ify).astype(F)
        pc = [(F(xn * d) - ts[0]).astype(F), (F(yn * d) - ts[1]).astype(F), (d - ts[2]).astype(F)]
        p = _mtv(Rs, pc)
        Q1 = quat_matrix_f32(sim_s[0])
        Q2 = quat_matrix_f32(sim_t[0])
        s1, s2 = F(sim_s[2]), F(sim_t[2])
        t1, t2 = np.asarray(sim_s[1], F), np.asarray(sim_t[1], F)
        rp = _mv(Q1, p)
        w = [(F(s1 * rp[i]) + t1[i]).astype(F) for i in range(3)]
        dw = [(w[i] - t2[i]).astype(F) for i in range(3)]
        rq = _mtv(Q2, dw)
        is2 = F(F(1.0) / s2)
        q = [(rq[i] * is2).astype(F) for i in range(3)]
        rc = _mv(Ra, q)
        c = [(rc[i] + ta[i]).astype(F) for i in range(3)]
        iz = (F(1.0) / c[2]).astype(F)
        px = (F(ct[12] * F(c[0] * iz)) + ct[14]).astype(F)
        py = (F(ct[13] * F(c[1] * iz)) + ct[15]).astype(F)
        sx, sy = (px - F(0.5)).astype(F), (py - F(0.5)).astype(F)
        valid = (d > 0) & (d < np.inf) & (c[2] > F(near))
        valid &= (sx >= 0) & (sx < F(W - 1)) & (sy >= 0) & (sy < F(H - 1))
        x0 = np.where(valid, np.floor(sx), 0).astype(np.int64)
        y0 = np.where(valid, np.floor(sy), 0).astype(np.int64)
    return valid, x0, y0, sx, sy, xs, ys


# ------------------------------------------------------------------------------------------
# FP64 values
# ------------------------------------------------------------------------------------------

def quat_matrix(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def huber(r, delta):
    """(rho(r), IRLS weight omega(r)) of the Huber norm on r^2."""
    a = np.abs(r)
    inl = a <= delta
    rho = np.where(inl, r * r, 2 * delta * a - delta * delta)
    om = np.where(inl, 1.0, delta / np.where(inl, 1.0, a))
    return rho, om


def sim3_matrix(sim):
    """(s R, t) of a correction (q, t, s), FP64."""
    return float(sim[2]) * quat_matrix(sim[0]), np.asarray(sim[1], np.float64)


def edge_terms(img_s, depth_s, img_t, cam_s, cam_t, sim_s, sim_t, weight=1.0, stride=1,
               delta=HUBER_DELTA, near=NEAR, decisions=None, per_pixel=False):
    """Eq. 12 residuals of one edge and their robust Gauss-Newton blocks (module docstring).

    Returns dict(cost, n, H [14, 14], g [14]) (+ r [n, 3], J [n, 3, 14] with per_pixel)."""
    _, Himg, Wimg = np.asarray(img_t).shape
    sim_s = (np.asarray(sim_s[0], F), np.asarray(sim_s[1], F), F(sim_s[2]))
    sim_t = (np.asarray(sim_t[0], F), np.asarray(sim_t[1], F), F(sim_t[2]))
    dec = decisions or decision_chain(cam_s, cam_t, sim_s, sim_t, Wimg, Himg, depth_s, stride, near)
    valid, x0, y0, _, _, xs, ys = dec
    xs, ys, x0, y0 = xs[valid], ys[valid], x0[valid], y0[valid]
    n = int(valid.sum())
    out = dict(cost=0.0, n=n, H=np.zeros((14, 14)), g=np.zeros(14))
    if n == 0:
        if per_pixel:
            out.update(r=np.zeros((0, 3)), J=np.zeros((0, 3, 14)))
        return out
    cs = np.asarray(cam_s, F).astype(np.float64)
    ct = np.asarray(cam_t, F).astype(np.float64)
    # values in FP64 from the FP32 inputs
    d = np.asarray(depth_s, np.float32)[ys, xs].astype(np.float64)
    Rs, ts = cs[:9].reshape(3, 3), cs[9:12]
    Ra, ta = ct[:9].reshape(3, 3), ct[9:12]
    fx, fy, cx, cy = cs[12:16]
    pc = np.stack([(xs + 0.5 - cx) / fx * d, (ys + 0.5 - cy) / fy * d, d], 1) - ts
    p = pc @ Rs                                         # rows: R_s^T (pc - t_s)
    As, bs = sim3_matrix(sim_s)
    At, bt = sim3_matrix(sim_t)
    w = p @ As.T + bs
    q = np.linalg.solve(At, (w - bt).T).T               # C_tgt^-1 w
    c = q @ Ra.T + ta
    fxa, fya, cxa, cya = ct[12:16]
    sx = fxa * c[:, 0] / c[:, 2] + cxa - 0.5
    sy = fya * c[:, 1] / c[:, 2] + cya - 0.5
    ax, ay = sx - x0, sy - y0                           # bilinear weights inside the FP32-chosen cell
    It = np.asarray(img_t, np.float32).astype(np.float64)
    i00, i01 = It[:, y0, x0].T, It[:, y0, x0 + 1].T          # [n, 3]
    i10, i11 = It[:, y0 + 1, x0].T, It[:, y0 + 1, x0 + 1].T
    axc, ayc = ax[:, None], ay[:, None]
    top = i00 + axc * (i01 - i00)
    bot = i10 + axc * (i11 - i10)
    val = top + ayc * (bot - top)
    gx = (i01 - i00) * (1 - ayc) + (i11 - i10) * ayc         # dI/dsx, [n, 3]
    gy = bot - top                                           # dI/dsy
    r = np.asarray(img_s, np.float32).astype(np.float64)[:, ys, xs].T - val
    # Jacobian of the projected point w.r.t. xi_src (2 x 7 per pixel)
    Minv = Ra @ np.linalg.inv(At)                            # dc/dw
    dpi = np.zeros((n, 2, 3))
    dpi[:, 0, 0] = fxa / c[:, 2]
    dpi[:, 0, 2] = -fxa * c[:, 0] / c[:, 2] ** 2
    dpi[:, 1, 1] = fya / c[:, 2]
    dpi[:, 1, 2] = -fya * c[:, 1] / c[:, 2] ** 2
    dw = np.zeros((n, 3, 7))
    dw[:, :, 0:3] = np.eye(3)
    dw[:, :, 3:6] = -np.stack([skew(v) for v in w])
    dw[:, :, 6] = w
    A = dpi @ Minv @ dw                                      # [n, 2, 7]
    grad = np.stack([gx, gy], 2)                             # [n, 3, 2]
    js = -(grad @ A)                                         # dr/dxi_src, [n, 3, 7]
    J = np.concatenate([js, -js], 2)                         # dr/dxi_tgt = -dr/dxi_src
    rho, om = huber(r, delta)
    scale = weight / n
    out["cost"] = scale * float(rho.sum())
    out["H"] = scale * np.einsum("nc,nci,ncj->ij", om, J, J)
    out["g"] = scale * np.einsum("nc,nci,nc->i", om, J, r)
    if per_pixel:
        out.update(r=r, J=J)
    return out


def photometric(edges, images, depths, cams, corrs, stride=1, delta=HUBER_DELTA, near=NEAR):
    """All edges: edges = [(src_image, tgt_image, src_corr, tgt_corr, weight)], images [M,3,H,W],
    depths [M,H,W], cams [M,16], corrs = [(q, t, s)].  Returns (cost [E], n [E], H [E,14,14], g [E,14])."""
    res = [edge_terms(images[a], depths[a], images[b], cams[a], cams[b], corrs[ca], corrs[cb], w, stride, delta,
                      near) for a, b, ca, cb, w in edges]
    return (np.array([x["cost"] for x in res]), np.array([x["n"] for x in res], np.int64),
            np.stack([x["H"] for x in res]) if res else np.zeros((0, 14, 14)),
            np.stack([x["g"] for x in res]) if res else np.zeros((0, 14)))
