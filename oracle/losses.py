"""FP64 oracles of the losses and the optimiser step on the mapping hot path.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

* L1 terms of the mapping loss (Eq. 4: alpha L1(I_hat, I) + beta L1(D_hat, D)) as means over
  elements, with sign(0) = 0.
* SSIM term of the refinement loss (Eq. 23: lambda (1 - SSIM)), with an 11x11 Gaussian window of
  sigma 1.5 normalised to sum 1, zero padding of 5 pixels, C1 = 0.01^2, C2 = 0.03^2 (data range 1),
  averaged over views, channels and pixels.  The paper gives only the weight lambda = 0.2.
* Adam with bias correction, as the per-agent optimiser (Sec. III-A, "optimized ... by gradient
  descent"; Sec. III-C, refinement "at half the per-agent learning rate").
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
