"""Pins of the FP64 loss and optimiser oracles.

* L1 and SSIM gradients against torch.autograd in float64 (an automatic differentiation of the
  forward definition, independent of the oracle's hand-derived adjoint);
* SSIM closed forms: SSIM(x, x) = 1; for constant images a, b the interior value is
  (2ab + C1) / (a^2 + b^2 + C1); a constant shift leaves the structure term at 1;
* Adam against torch.optim.Adam in float64;
* the normal term of Eq. 4: closed forms on planes, invariance under scaling the depth (with
  Euler's relation sum D dL/dD = 0 for the gradient), autograd and finite differences, holes.
"""
import numpy as np
import pytest
import torch

from oracle import losses as L


def _torch_ssim(x, y):
    g = torch.tensor(L.gaussian_window_1d(), dtype=torch.float64)
    w = (g[:, None] * g[None, :])[None, None]
    c = x.shape[1]
    xs, ys = x.reshape(-1, 1, *x.shape[-2:]), y.reshape(-1, 1, *y.shape[-2:])
    conv = lambda a: torch.nn.functional.conv2d(a, w, padding=5)
    mx, my = conv(xs), conv(ys)
    vx, vy, cxy = conv(xs * xs) - mx * mx, conv(ys * ys) - my * my, conv(xs * ys) - mx * my
    S = ((2 * mx * my + L.C1) * (2 * cxy + L.C2)) / ((mx * mx + my * my + L.C1) * (vx + vy + L.C2))
    return S.mean()


def test_l1_gradient_vs_autograd():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, (2, 3, 9, 13)), rng.uniform(0, 1, (2, 3, 9, 13))
    val, grad = L.l1(x, y)
    xt = torch.tensor(x, requires_grad=True)
    lt = (xt - torch.tensor(y)).abs().mean()
    lt.backward()
    assert abs(val - lt.item()) < 1e-14
    np.testing.assert_allclose(grad, xt.grad.numpy(), rtol=1e-13, atol=1e-16)


def test_ssim_gradient_vs_autograd():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (2, 3, 20, 27)), rng.uniform(0, 1, (2, 3, 20, 27))
    val, grad = L.ssim(x, y)
    xt = torch.tensor(x, requires_grad=True)
    st = _torch_ssim(xt, torch.tensor(y))
    st.backward()
    assert abs(val - st.item()) < 1e-12
    np.testing.assert_allclose(grad, xt.grad.numpy(), rtol=1e-9, atol=1e-14)


def test_ssim_closed_forms():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (1, 3, 24, 24))
    assert abs(L.ssim(x, x)[0] - 1.0) < 1e-12
    a, b = 0.3, 0.7
    H = W = 30
    xa, yb = np.full((1, 1, H, W), a), np.full((1, 1, H, W), b)
    # interior pixels (>= 5 px from the border) see no padding
    g = L.gaussian_window_1d()
    conv = lambda im: L._conv(im, g)
    mx, my = conv(xa), conv(yb)
    inner = (slice(None), slice(None), slice(5, H - 5), slice(5, W - 5))
    np.testing.assert_allclose(mx[inner], a, rtol=1e-14)
    S_cf = (2 * a * b + L.C1) / (a * a + b * b + L.C1)
    # whole-image SSIM of constants: recompute the map from its definition on interior pixels only
    vx = conv(xa * xa) - mx * mx
    assert np.abs(vx[inner]).max() < 1e-14
    S_map_inner = ((2 * mx * my + L.C1) * (2 * (conv(xa * yb) - mx * my) + L.C2)) / (
        (mx * mx + my * my + L.C1) * (vx + conv(yb * yb) - my * my + L.C2))
    np.testing.assert_allclose(S_map_inner[inner], S_cf, rtol=1e-12)
    # a shift by a constant keeps the contrast-structure term at one on the interior
    y = x + 0.1
    val, _ = L.ssim(x[..., 5:-5, 5:-5] * 0 + x[..., 5:-5, 5:-5], x[..., 5:-5, 5:-5])
    assert abs(val - 1.0) < 1e-12
    assert L.ssim(x, y)[0] < 1.0


def test_window_is_normalised_gaussian():
    g = L.gaussian_window_1d()
    assert g.shape == (11,) and abs(g.sum() - 1) < 1e-15
    assert abs(g[6] / g[5] - np.exp(-1 / (2 * 1.5 ** 2))) < 1e-15


@pytest.mark.parametrize("steps", [1, 5])
def test_adam_vs_torch(steps):
    rng = np.random.default_rng(3)
    p = rng.normal(0, 1, 50)
    grads = [rng.normal(0, 1, 50) for _ in range(steps)]
    pt = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=5e-3, betas=(0.9, 0.999), eps=1e-15)
    m, v = np.zeros(50), np.zeros(50)
    for s, g in enumerate(grads, 1):
        p, m, v = L.adam_step(p, g, m, v, s, 5e-3)
        pt.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_refine_loss_gradients_vs_autograd():
    """Exposure-compensated refinement loss (Eq. 23): every gradient against torch.autograd."""
    rng = np.random.default_rng(4)
    V, H, W = 2, 18, 23
    rgb, tgt = rng.uniform(0, 1, (V, 3, H, W)), rng.uniform(0, 1, (V, 3, H, W))
    d, dt = rng.uniform(1, 4, (V, H, W)), rng.uniform(1, 4, (V, H, W))
    a, b = rng.normal(0, 0.2, V), rng.normal(0, 0.05, V)
    Lv, g_rgb, g_d, g_a, g_b = L.refine_loss(rgb, tgt, d, dt, a, b)
    t = lambda x: torch.tensor(x, requires_grad=True)
    rt, dtt, at, bt = t(rgb), t(d), t(a), t(b)
    It = torch.exp(at)[:, None, None, None] * rt + bt[:, None, None, None]
    yt = torch.tensor(tgt)
    Lt = (1.75 * (It - yt).abs().mean() + 0.2 * (1 - _torch_ssim(It, yt))
          + 0.25 * (dtt - torch.tensor(dt)).abs().mean())
    Lt.backward()
    assert abs(Lv - Lt.item()) < 1e-12
    np.testing.assert_allclose(g_rgb, rt.grad.numpy(), rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(g_d, dtt.grad.numpy(), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(g_a, at.grad.numpy(), rtol=1e-9)
    np.testing.assert_allclose(g_b, bt.grad.numpy(), rtol=1e-9)
    # zero exposure reduces to the plain loss terms
    L0, g0, _, _, _ = L.refine_loss(rgb, tgt, None, None, np.zeros(V), np.zeros(V), 1.75, 0.2, 0.0)
    Lp, gp = L.l1_ssim_loss(rgb, tgt, 1.75, 0.2)
    assert abs(L0 - Lp) < 1e-14
    np.testing.assert_allclose(g0, gp, rtol=1e-14)


def test_prune_keep_threshold():
    o = np.array([0.5, 0.004, 0.005, 0.0049999, 1.0, 0.0], np.float32)
    assert list(L.prune_keep(o)) == [0, 2, 4]


def test_iso_loss_vs_autograd_and_isotropic_minimum():
    rng = np.random.default_rng(6)
    ls = rng.normal(-3, 0.5, (40, 3))
    val, g = L.iso_loss(ls, 10.0)
    lt = torch.tensor(ls, requires_grad=True)
    st = torch.exp(lt)
    (10.0 * (st - st.mean(1, keepdim=True)).abs().sum()).backward()
    assert abs(val - 10.0 * np.abs(np.exp(ls) - np.exp(ls).mean(1, keepdims=True)).sum()) < 1e-12
    np.testing.assert_allclose(g, lt.grad.numpy(), rtol=1e-12, atol=1e-15)
    iso = np.full((5, 3), -2.0)
    v0, g0 = L.iso_loss(iso)
    assert v0 == 0.0 and np.all(g0 == 0.0)


# ---- normal term of Eq. 4 ------------------------------------------------------------------------
_INTR = np.array([[22.0, 20.0, 6.5, 5.0], [18.0, 24.0, 5.0, 6.0]])


def _unit(a, axis):
    return a / np.linalg.norm(a, axis=axis, keepdims=True)


def _plane_depth(m, d0, H, W, intr):
    """Depth of the plane {P : m . P = d0} along every pixel's ray."""
    r = L.pixel_rays(W, H, *intr)
    return d0 / np.tensordot(m, r, axes=(0, 0))


def test_normal_loss_plane_closed_form():
    # every interior pixel of a plane seen from the front has N_hat = -m (facing the camera); a prior
    # of -m costs 0, of +m costs 2 and of any perpendicular unit vector 1 per valid pixel
    H, W = 12, 15
    m = _unit(np.array([0.3, -0.2, 1.0]), 0)
    depth = _plane_depth(m, 2.5, H, W, _INTR[0])[None]
    n, valid, *_ = L.depth_normals(depth[0], *_INTR[0])
    assert valid.sum() == (H - 2) * (W - 2)
    assert np.allclose(n[:, valid].T, -m, atol=1e-12)
    perp = _unit(np.cross(m, [1.0, 0.0, 0.0]), 0)
    for prior_dir, per_px in ((-m, 0.0), (m, 2.0), (perp, 1.0)):
        prior = np.broadcast_to(prior_dir[None, :, None, None], (1, 3, H, W))
        loss, _ = L.normal_loss(depth, prior, _INTR[:1], weight=1.0)
        assert loss == pytest.approx(per_px * (H - 2) * (W - 2) / (H * W), abs=1e-12)


def _smooth_depth(rng, V, H, W):
    y, x = np.mgrid[0:H, 0:W]
    d = np.empty((V, H, W))
    for v in range(V):
        a, b, c = rng.uniform(-0.05, 0.05, 3)
        d[v] = 2.0 + a * x + b * y + 0.3 * np.sin(0.4 * x + c) * np.cos(0.3 * y)
    return d


def _random_prior(rng, V, H, W):
    p = rng.normal(size=(V, 3, H, W))
    p[:, 2] = -np.abs(p[:, 2]) - 0.5          # facing the camera
    return _unit(p, 1)


def test_normal_loss_is_scale_invariant():
    # N_hat does not change when all depths are scaled, so L(k D) = L(D) and sum_q D(q) dL/dD(q) = 0
    # (Euler's relation for a function homogeneous of degree 0): a dropped or mis-signed adjoint
    # term breaks the second identity
    rng = np.random.default_rng(3)
    depth, prior = _smooth_depth(rng, 2, 10, 13), _random_prior(rng, 2, 10, 13)
    l1, g = L.normal_loss(depth, prior, _INTR)
    l2, _ = L.normal_loss(2.7 * depth, prior, _INTR)
    assert l2 == pytest.approx(l1, rel=1e-12)
    assert abs((depth * g).sum()) <= 1e-12 * np.abs(depth * g).sum()


def test_normal_loss_gradient_vs_autograd():
    rng = np.random.default_rng(4)
    V, H, W = 2, 9, 11
    depth, prior = _smooth_depth(rng, V, H, W), _random_prior(rng, V, H, W)
    depth[0, 4, 5] = 0.0                      # a hole: its neighbours' normals are invalid
    loss, g = L.normal_loss(depth, prior, _INTR, weight=0.5)
    D = torch.tensor(depth, requires_grad=True)
    total = 0.0
    for v in range(V):
        r = torch.tensor(L.pixel_rays(W, H, *_INTR[v]))
        P = D[v][None] * r
        ok = (D[v] > 0).detach()
        valid = ok[1:-1, 1:-1] & ok[1:-1, 2:] & ok[1:-1, :-2] & ok[2:, 1:-1] & ok[:-2, 1:-1]
        tx = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
        ty = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
        u = torch.linalg.cross(ty, tx, dim=0)
        n = u / torch.linalg.vector_norm(u, dim=0, keepdim=True)
        c = 1.0 - (n * torch.tensor(prior[v][:, 1:-1, 1:-1])).sum(0)
        total = total + torch.where(valid, c.abs(), torch.zeros_like(c)).sum()
    total = 0.5 * total / (V * H * W)
    total.backward()
    assert loss == pytest.approx(total.item(), rel=1e-12)
    np.testing.assert_allclose(g, D.grad.numpy(), rtol=1e-9, atol=1e-15)


def test_normal_loss_finite_differences():
    rng = np.random.default_rng(5)
    depth, prior = _smooth_depth(rng, 1, 8, 10), _random_prior(rng, 1, 8, 10)
    _, g = L.normal_loss(depth, prior, _INTR[:1])
    h = 1e-6
    for (y, x) in ((1, 1), (3, 4), (6, 8), (0, 5), (4, 9)):
        dp, dm = depth.copy(), depth.copy()
        dp[0, y, x] += h
        dm[0, y, x] -= h
        fd = (L.normal_loss(dp, prior, _INTR[:1])[0] - L.normal_loss(dm, prior, _INTR[:1])[0]) / (2 * h)
        assert fd == pytest.approx(g[0, y, x], rel=1e-6, abs=1e-13)


def test_normal_loss_holes_and_borders():
    rng = np.random.default_rng(6)
    H, W = 9, 12
    depth, prior = _smooth_depth(rng, 1, H, W), _random_prior(rng, 1, H, W)
    depth[0, 4, 6] = 0.0
    n, valid, *_ = L.depth_normals(depth[0], *_INTR[0])
    assert not valid[0].any() and not valid[-1].any() and not valid[:, 0].any() and not valid[:, -1].any()
    for (y, x) in ((4, 6), (3, 6), (5, 6), (4, 5), (4, 7)):   # the hole and the pixels that use it
        assert not valid[y, x]
    assert valid.sum() == (H - 2) * (W - 2) - 5
    _, g = L.normal_loss(depth, prior, _INTR[:1])
    assert g[0, 4, 6] == 0.0                  # no valid normal uses the hole's depth
