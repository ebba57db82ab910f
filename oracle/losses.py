"""FP64 oracles of the losses and the optimiser step on the mapping hot path.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

* L1 terms of the mapping loss (Eq. 4: alpha L1(I_hat, I) + beta L1(D_hat, D)) as means over
  elements, with sign(0) = 0.
* SSIM term of the refinement loss (Eq. 23: lambda (1 - SSIM)), with an 11x11 Gaussian window of
  sigma 1.5 normalised to sum 1, zero padding of 5 pixels, C1 = 0.01^2, C2 = 0.03^2 (data range 1),
  averaged over views, channels and pixels.  The paper gives only the weight lambda = 0.2.
* Adam with bias correction, as the per-agent optimiser (Sec. III-A, "optimized ... by gradient
  descent"; Sec. III-C, refinement "at half the per-agent learning rate").
* The normal term of the mapping loss (Eq. 4: lambda_n L_normal, lambda_n = 1e-2): a cosine
  loss |1 - N_hat . N_bar| between the normal induced by the rendered depth and a given normal
  prior (the prior is an input; its monocular network is not part of this path).
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window_1d(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    k = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return g / g.sum()


def _conv(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Zero-padded 'same' correlation of [..., H, W] with the separable window outer(g, g)."""
    r = (len(g) - 1) // 2
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W + 2 * r))
    pad[..., r:r + H, r:r + W] = img
    tmp = np.zeros(img.shape[:-2] + (H + 2 * r, W))
    for k in range(len(g)):
        tmp += g[k] * pad[..., :, k:k + W]
    out = np.zeros(img.shape)
    for k in range(len(g)):
        out += g[k] * tmp[..., k:k + H, :]
    return out


def l1(x: np.ndarray, y: np.ndarray):
    """mean |x - y| and its gradient w.r.t. x."""
    x = np.asarray(x, np.float64)
    d = x - np.asarray(y, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def ssim(x: np.ndarray, y: np.ndarray, size: int = 11, sigma: float = 1.5):
    """SSIM(x, y) averaged over all leading dims and pixels, and dSSIM/dx.  x, y: [..., H, W]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    g = gaussian_window_1d(size, sigma)
    mx, my = _conv(x, g), _conv(y, g)
    exx, eyy, exy = _conv(x * x, g), _conv(y * y, g), _conv(x * y, g)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    S = (A1 * A2) / (B1 * B2)
    n = S.size
    dS_dmx = (2 * my * A2 - 2 * my * A1) / (B1 * B2) - S * (2 * mx / B1 - 2 * mx / B2)
    dS_dexx = -S / B2
    dS_dexy = 2 * A1 / (B1 * B2)
    grad = (_conv(dS_dmx, g) + 2 * x * _conv(dS_dexx, g) + y * _conv(dS_dexy, g)) / n
    return float(S.mean()), grad


def mapping_l1_loss(rgb, rgb_t, depth=None, depth_t=None, w_rgb=1.0, w_depth=0.1):
    """w_rgb mean|rgb - rgb_t| + w_depth mean|depth - depth_t|, with gradients."""
    L, g_rgb = l1(rgb, rgb_t)
    L *= w_rgb
    g_rgb = g_rgb * w_rgb
    g_d = None
    if depth is not None and w_depth != 0.0:
        Ld, g_d = l1(depth, depth_t)
        L += w_depth * Ld
        g_d = g_d * w_depth
    return L, g_rgb, g_d


def l1_ssim_loss(rgb, rgb_t, w_l1=0.8, w_ssim=0.2):
    """w_l1 L1 + w_ssim (1 - SSIM) over [V,3,H,W] images, with the gradient w.r.t. rgb."""
    L1, g1 = l1(rgb, rgb_t)
    S, gs = ssim(rgb, rgb_t)
    return w_l1 * L1 + w_ssim * (1.0 - S), w_l1 * g1 - w_ssim * gs


def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One bias-corrected Adam update (step counts from 1).  Returns new (param, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def refine_loss(rgb, rgb_t, depth, depth_t, a, b, w_l1=1.75, w_ssim=0.2, w_depth=0.25, fp32_sign=False):
    """Refinement loss of Eq. 23 on the exposure-compensated render (the normal term needs a
    monocular normal prior and is not included):

        I~_v = exp(a_v) I^_v + b_v      (per keyframe log-gain a_v and bias b_v, every channel)
        L = w_l1 L1(I~, I) + w_ssim (1 - SSIM(I~, I)) + w_depth L1(D^, D-)

    with w_l1 = alpha' = 1.75, w_ssim = lambda = 0.2, w_depth = beta = 0.25 (Eq. 4's beta).
    rgb, rgb_t: [V,3,H,W]; depth, depth_t: [V,H,W] (or None); a, b: [V].
    fp32_sign: take the sign of the L1 term (a decision) on I~ formed in FP32 as fl(fl(e^a I^) + b)
    with the decision-chain exponential, the way an FP32 implementation forms it; values stay FP64.
    Returns (L, dL/drgb, dL/ddepth or None, dL/da [V], dL/db [V])."""
    rgb = np.asarray(rgb, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ea = np.exp(a)[:, None, None, None]
    It = ea * rgb + b[:, None, None, None]
    L1v, g1 = l1(It, rgb_t)
    if fp32_sign:
        from .oracle import expf
        ea32 = expf(a.astype(np.float32))[:, None, None, None]
        It32 = (ea32 * np.asarray(rgb, np.float32)).astype(np.float32) + b.astype(np.float32)[:, None, None, None]
        g1 = np.sign(It32.astype(np.float64) - np.asarray(rgb_t, np.float32)) / It.size
    S, gs = ssim(It, rgb_t)
    g_It = w_l1 * g1 - w_ssim * gs
    L = w_l1 * L1v + w_ssim * (1.0 - S)
    g_d = None
    if depth is not None and w_depth != 0.0:
        Ld, g_d = l1(depth, depth_t)
        L += w_depth * Ld
        g_d = g_d * w_depth
    g_rgb = ea * g_It
    g_a = (g_It * ea * rgb).sum(axis=(1, 2, 3))
    g_b = g_It.sum(axis=(1, 2, 3))
    return L, g_rgb, g_d, g_a, g_b


def prune_keep(opacities, threshold=0.005):
    """Gaussians kept by the refinement's pruning (opacity below 0.005 removed, Sec. III-C), in
    their original order: the indices i with o_i >= threshold."""
    o = np.asarray(opacities, np.float32)
    return np.nonzero(o >= np.float32(threshold))[0]


def view_adam_step(cam_row, expo, pose_grad, expo_grad, m, v, step, lr_pose, lr_expo, beta1=0.9, beta2=0.999,
                   eps=1e-15):
    """One Adam step on a keyframe's pose delta and exposure (Sec. III-C joint refinement of pose
    deltas and log-gain / bias): the 8 gradients (rho, phi, a, b) update bias-corrected moments;
    the pose part of the step, delta, is applied as the left perturbation T <- Exp(delta) T of the
    world-to-camera pose; the exposure part is added.  Returns (cam_row, expo, m, v)."""
    from .oracle import exp_se3_left
    g = np.concatenate([np.asarray(pose_grad, np.float64), np.asarray(expo_grad, np.float64)])
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    lr = np.array([lr_pose] * 6 + [lr_expo] * 2)
    d = -lr * (m / (1 - beta1 ** step)) / (np.sqrt(v / (1 - beta2 ** step)) + eps)
    return exp_se3_left(cam_row, d[:6]), np.asarray(expo, np.float64) + d[6:], m, v


def iso_loss(log_scales, weight=10.0):
    """Isotropy regulariser of the mapping loss (Eq. 4: lambda_s L_iso, lambda_s = 10) with
    L_iso = sum_i sum_axes |s_i - mean(s_i)|, s_i = exp(log-scales) the Gaussian's per-axis scales:
    it pulls each Gaussian's scales toward their mean.  Returns (weight * L_iso, d/d log_scales)."""
    ls = np.asarray(log_scales, np.float64)
    s = np.exp(ls)
    sbar = s.mean(axis=1, keepdims=True)
    d = s - sbar
    sg = np.sign(d)
    # d|s_a - sbar| / d s_b = sg_a (delta_ab - 1/3); chain through s_b = exp(l_b)
    g_s = sg - sg.sum(axis=1, keepdims=True) / 3.0
    return weight * np.abs(d).sum(), weight * g_s * s


def pixel_rays(W, H, fx, fy, cx, cy):
    """Ray of every pixel in the camera frame, r = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1)
    (pixel centres at +0.5, camera x right, y down, z forward): [3, H, W]."""
    X, Y = np.meshgrid((np.arange(W) + 0.5 - cx) / fx, (np.arange(H) + 0.5 - cy) / fy)
    return np.stack([X, Y, np.ones_like(X)])


def depth_normals(depth, fx, fy, cx, cy):
    """Normal induced by one view's depth map (the N_hat of Eq. 4's normal term).  The pixel's
    point is P = D r; t_x = P(x+1, y) - P(x-1, y), t_y = P(x, y+1) - P(x, y-1) (central
    differences); u = t_y x t_x and N_hat = u / |u|, which faces the camera for a surface seen from
    the front (-z for a fronto-parallel plane).  A pixel is valid when it is not on the image
    border, its depth and its four neighbours' depths are positive and finite, and |u| > 0.
    Returns (N_hat [3,H,W] (zero where invalid), valid [H,W], t_x, t_y, |u|)."""
    D = np.asarray(depth, np.float64)
    H, W = D.shape
    P = D[None] * pixel_rays(W, H, fx, fy, cx, cy)
    ok = (D > 0) & np.isfinite(D)
    valid = np.zeros((H, W), bool)
    valid[1:-1, 1:-1] = ok[1:-1, 1:-1] & ok[1:-1, 2:] & ok[1:-1, :-2] & ok[2:, 1:-1] & ok[:-2, 1:-1]
    tx, ty = np.zeros((3, H, W)), np.zeros((3, H, W))
    tx[:, 1:-1, 1:-1] = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
    ty[:, 1:-1, 1:-1] = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
    tx[:, ~valid] = 0.0
    ty[:, ~valid] = 0.0
    u = np.cross(ty, tx, axis=0)
    nu = np.sqrt((u * u).sum(0))
    valid &= nu > 0
    safe = np.where(valid, nu, 1.0)
    n = np.where(valid[None], u / safe[None], 0.0)
    return n, valid, tx, ty, safe


def normal_loss(depth, prior, intr, weight=1e-2):
    """Normal term of the mapping loss (Eq. 4, lambda_n L_normal with lambda_n = 1e-2):
    L_normal = |1 - N_hat . N_bar| per valid pixel (depth_normals), averaged over all V*H*W pixels
    (invalid ones add 0), with N_bar the given normal prior [V,3,H,W] in the camera frame and
    intr [V,4] = (fx, fy, cx, cy).  sign(0) = 0.  Returns (weight * L_normal, d/d depth [V,H,W]).

    Adjoint: g_n = dL/dN_hat = -scale sign(c) N_bar (c = 1 - N_hat . N_bar, scale = weight / VHW);
    g_u = (g_n - N_hat (N_hat . g_n)) / |u|; for u = t_y x t_x, dL/dt_y = t_x x g_u and
    dL/dt_x = g_u x t_y; P(q) enters t_x at q -+ 1 and t_y at q -+ W, so
    dL/dP(q) = G_x(q-x) - G_x(q+x) + G_y(q-y) - G_y(q+y) and dL/dD(q) = r(q) . dL/dP(q)."""
    depth = np.asarray(depth, np.float64)
    prior = np.asarray(prior, np.float64)
    V, H, W = depth.shape
    scale = weight / (V * H * W)
    total = 0.0
    grad = np.zeros_like(depth)
    for v in range(V):
        fx, fy, cx, cy = (float(t) for t in intr[v])
        n, valid, tx, ty, nu = depth_normals(depth[v], fx, fy, cx, cy)
        c = 1.0 - (n * prior[v]).sum(0)
        total += scale * np.abs(c)[valid].sum()
        sg = np.where(valid, np.sign(c), 0.0)
        g_n = -scale * sg[None] * prior[v]
        g_u = (g_n - n * (n * g_n).sum(0)[None]) / nu[None]
        gx = np.cross(g_u, ty, axis=0) * valid[None]
        gy = np.cross(tx, g_u, axis=0) * valid[None]
        dP = np.zeros((3, H, W))
        dP[:, :, 1:] += gx[:, :, :-1]
        dP[:, :, :-1] -= gx[:, :, 1:]
        dP[:, 1:, :] += gy[:, :-1, :]
        dP[:, :-1, :] -= gy[:, 1:, :]
        grad[v] = (pixel_rays(W, H, fx, fy, cx, cy) * dP).sum(0)
    return total, grad
