"""Graph-captured mapping loop and the full-size batched workloads.

* graph replay equals eager execution of the same iterations (same kernels, same order);
* the loop lowers the loss (0.8 L1 + 0.2 (1 - SSIM)) on a target rendered from perturbed params;
* floor4m at full size (4M Gaussians, 64 views in one batched problem, the benchmark's launch
  configuration): tile lists, images and gradients compared with the oracle on sampled tiles of two
  views.  Upstream gradients are zero outside the sampled tiles, so the oracle's tile-restricted
  backward is the exact expected value of every Gaussian and pose gradient.
"""
import numpy as np
import pytest

from helpers import TOL_GRAD, TOL_IMAGE, gpu_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def _loop(R, wl, seed=5):
    from paper_2605_10760_gb300 import mapping as M
    V = len(wl.cameras)
    pb, g = gpu_problem(wl)
    tgt = torch.from_numpy(np.stack([S.smooth_image(wl.width, wl.height, seed + v) for v in range(V)])).cuda()
    return M.MappingLoop(pb, g, tgt), g


def test_graph_replay_equals_eager(R):
    wl = S.workload("room1m", scale=0.02)
    wl.cameras = wl.cameras[:2]
    wl.scene_of_view = wl.scene_of_view[:2]
    eager, ge = _loop(R, wl)
    graph, gg = _loop(R, wl)
    graph.capture(3)                      # capture runs one eager warm-up iteration first
    eager.iteration()
    for _ in range(3):
        eager.iteration()
    graph.replay()
    torch.cuda.synchronize()
    assert eager.pb.check_status()[0] == 0 and graph.pb.check_status()[0] == 0
    lrs = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "colors": 2.5e-3}
    for k, lr in lrs.items():
        a, b = getattr(ge, k).cpu().numpy(), getattr(gg, k).cpu().numpy()
        # identical up to gradient summation order: Adam steps are bounded by lr per iteration
        assert np.abs(a - b).max() <= 8 * lr, k
        assert np.mean(np.abs(a - b) > 1e-6 * lr) < 0.02, k
    assert int(eager.adam.step.item()) == int(graph.adam.step.item()) == 4
    assert abs(eager.loss.item() - graph.loss.item()) <= 1e-4 * abs(eager.loss.item())


def test_mapping_loop_reduces_loss(R):
    from paper_2605_10760_gb300 import mapping as M
    wl = S.workload("room500k", scale=0.05)
    pb, g = gpu_problem(wl)
    img = pb.forward_checked(g)
    target = img["rgb"].clone()
    # perturb the colours and opacities, then optimise back towards the rendered target
    rng = np.random.default_rng(0)
    g.colors.copy_(torch.from_numpy(np.clip(wl.scene.colors + rng.normal(0, 0.15, wl.scene.colors.shape), 0, 1)
                                    .astype(np.float32)).cuda())
    loop = M.MappingLoop(pb, g, target, lr=(1.6e-4, 5e-3, 1e-3, 5e-2, 1e-2))
    loop.iteration()
    l0 = loop.loss.item()
    loop.capture(20)
    for _ in range(3):
        loop.replay()
    torch.cuda.synchronize()
    assert pb.check_status()[0] == 0
    assert loop.loss.item() < 0.7 * l0


def test_floor4m_full_size_sampled_tiles(R):
    wl = S.workload("floor4m")
    V = len(wl.cameras)
    pb, g = gpu_problem(wl)
    img = pb.forward_checked(g)
    ws = pb.workspace()
    Tx, Ty = pb.tiles
    tpv = Tx * Ty
    rng = np.random.default_rng(1)
    views = [3, 40]
    sampled = {v: rng.choice(tpv, 24, replace=False) for v in views}
    # upstream gradients only on the sampled tiles of the two views
    H, W = wl.height, wl.width
    d_rgb = np.zeros((V, 3, H, W), np.float32)
    d_depth = np.zeros((V, H, W), np.float32)
    for v in views:
        for t in sampled[v]:
            ty, tx = divmod(int(t), Tx)
            sl = (slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16)))
            d_rgb[v][(slice(None),) + sl] = rng.choice([-1.0, 1.0], (3,) + d_rgb[v][(0,) + sl].shape) * 1e-6
            d_depth[v][sl] = rng.choice([-1.0, 1.0], d_depth[v][sl].shape) * 1e-7
    grads = pb.render_bwd(g, img, torch.from_numpy(d_rgb).cuda(), torch.from_numpy(d_depth).cuda(), None)
    pose = pb.pose_grad().cpu().numpy()
    torch.cuda.synchronize()
    assert pb.check_status()[0] == 0
    ranges = ws["tile_ranges"].cpu().numpy().view(np.uint32)
    vals = ws["sorted_vals"].cpu().numpy().view(np.uint32)
    N = wl.scene.n
    # oracle on the two views only, restricted to their sampled tiles
    mask = np.zeros(len(views) * tpv, np.uint8)
    for j, v in enumerate(views):
        mask[j * tpv + sampled[v]] = 1
    orc = Oracle.from_workload(wl, views=views, tile_mask=mask)
    ob = orc.bins()
    fw = orc.forward()
    bw = orc.backward(d_rgb[views].astype(np.float64), d_depth[views].astype(np.float64))
    for j, v in enumerate(views):
        for t in sampled[v]:
            gs_, ge_ = (int(u) for u in ranges[v * tpv + t])
            os_, oe_ = (int(u) for u in ob["ranges"][j * tpv + t])
            # GPU values are pair indices v*N + i; the oracle's are j*N + i
            np.testing.assert_array_equal(vals[gs_:ge_].astype(np.int64) - v * N,
                                          ob["vals"][os_:oe_].astype(np.int64) - j * N)
            ty, tx = divmod(int(t), Tx)
            sl = (slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16)))
            np.testing.assert_array_equal(img["last_idx"][v].cpu().numpy()[sl], fw["last"][j][sl])
            err = np.abs(img["rgb"][v].cpu().numpy()[(slice(None),) + sl] - fw["rgb"][j][(slice(None),) + sl]).max()
            assert err <= TOL_IMAGE
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        assert rel_l2(getattr(grads, k).cpu().numpy(), bw[k]) <= TOL_GRAD, k
    for j, v in enumerate(views):
        assert rel_l2(pose[v], bw["pose"][j]) <= TOL_GRAD
    others = [v for v in range(V) if v not in views]
    assert np.abs(pose[others]).max() == 0.0


def test_room1m_full_size_iteration_sampled_tiles(R):
    """The graph-captured mapping workload at full size (1M-Gaussian room, 8 views at 1200x680 in one
    batched problem) for one iteration: tile lists, images, every Gaussian and pose gradient and the
    in-kernel Adam step (config-4 learning rates, opacity through its logit) against the oracle on
    24 sampled tiles of two views.  The upstream gradient is seeded and non-zero only on the sampled
    tiles, so the oracle's tile-restricted backward is the exact expected gradient of every Gaussian
    and pose.  The L1 + SSIM loss of the loop is checked at the same full size on seeded images of
    the same shape (its inputs do not come from the GPU render)."""
    from oracle import losses as OL
    wl = S.workload("room1m")
    V = len(wl.cameras)
    H, W = wl.height, wl.width
    # (a) the mapping loss at full size: 0.8 L1 + 0.2 (1 - SSIM) over [8, 3, 680, 1200]
    rng = np.random.default_rng(4)
    y = np.stack([S.uniform_image(W, H, 40 + v) for v in range(V)])
    x = np.clip(y + rng.normal(0, 0.05, y.shape), 0, 1).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, d_loss = R.loss_l1_ssim(t(x), t(y), 0.8, 0.2)
    Lr, gr = OL.l1_ssim_loss(x, y, 0.8, 0.2)
    assert abs(loss.item() - Lr) <= 1e-5 * abs(Lr)
    assert rel_l2(d_loss.cpu().numpy(), gr) <= 1e-4
    del d_loss
    # (b) forward, backward, pose gradients and one Adam step of the 8-view problem
    pb, g = gpu_problem(wl)
    img = pb.forward_checked(g)
    ws = pb.workspace()
    Tx, Ty = pb.tiles
    tpv = Tx * Ty
    views = [1, 6]
    sampled = {v: rng.choice(tpv, 24, replace=False) for v in views}
    d_rgb = np.zeros((V, 3, H, W), np.float32)
    d_depth = np.zeros((V, H, W), np.float32)
    for v in views:
        for tt in sampled[v]:
            ty, tx = divmod(int(tt), Tx)
            sl = (slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16)))
            d_rgb[v][(slice(None),) + sl] = rng.choice([-1.0, 1.0], (3,) + d_rgb[v][(0,) + sl].shape) * 1e-6
            d_depth[v][sl] = rng.choice([-1.0, 1.0], d_depth[v][sl].shape) * 1e-7
    grads = pb.render_bwd(g, img, t(d_rgb), t(d_depth), None)
    pose = pb.pose_grad().cpu().numpy()
    gpu_grads = {k: getattr(grads, k).cpu().numpy() for k in ("means", "log_scales", "quats", "opacities", "colors")}
    lrs = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "logit": 5e-2, "colors": 2.5e-3}
    before = {k: getattr(g, k).cpu().numpy().astype(np.float64) for k in ("means", "log_scales", "quats", "colors")}
    o0 = g.opacities.cpu().numpy().astype(np.float64)
    adam = R.AdamState(g, lr=(lrs["means"], lrs["log_scales"], lrs["quats"], lrs["logit"], lrs["colors"]))
    logit0 = adam.logits.cpu().numpy().astype(np.float64)
    adam.apply(grads, zero_grads=True)
    torch.cuda.synchronize()
    assert pb.check_status()[0] == 0
    ranges = ws["tile_ranges"].cpu().numpy().view(np.uint32)
    vals = ws["sorted_vals"].cpu().numpy().view(np.uint32)
    N = wl.scene.n
    mask = np.zeros(len(views) * tpv, np.uint8)
    for j, v in enumerate(views):
        mask[j * tpv + sampled[v]] = 1
    orc = Oracle.from_workload(wl, views=views, tile_mask=mask)
    ob, fw = orc.bins(), orc.forward()
    bw = orc.backward(d_rgb[views].astype(np.float64), d_depth[views].astype(np.float64))
    last = img["last_idx"].cpu().numpy()
    rgb = img["rgb"].cpu().numpy()
    for j, v in enumerate(views):
        for tt in sampled[v]:
            gs_, ge_ = (int(u) for u in ranges[v * tpv + tt])
            os_, oe_ = (int(u) for u in ob["ranges"][j * tpv + tt])
            np.testing.assert_array_equal(vals[gs_:ge_].astype(np.int64) - v * N,
                                          ob["vals"][os_:oe_].astype(np.int64) - j * N)
            ty, tx = divmod(int(tt), Tx)
            sl = (slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16)))
            np.testing.assert_array_equal(last[v][sl], fw["last"][j][sl])
            assert np.abs(rgb[v][(slice(None),) + sl] - fw["rgb"][j][(slice(None),) + sl]).max() <= TOL_IMAGE
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        assert rel_l2(gpu_grads[k], bw[k]) <= TOL_GRAD, k
    for j, v in enumerate(views):
        assert rel_l2(pose[v], bw["pose"][j]) <= TOL_GRAD
    assert np.abs(pose[[v for v in range(V) if v not in views]]).max() == 0.0
    # Adam, first step from zero moments: m = 0.1 g, v = 0.001 g^2, theta -= lr g / (|g| + eps)
    go = dict(bw)
    go["logit"] = bw["opacities"] * o0 * (1 - o0)
    after = {k: getattr(g, k).cpu().numpy().astype(np.float64) for k in ("means", "log_scales", "quats", "colors")}
    after["logit"] = adam.logits.cpu().numpy().astype(np.float64)
    before["logit"] = logit0
    m_gpu = adam.m.cpu().numpy().astype(np.float64)
    off = {"means": 0, "log_scales": 3 * N, "quats": 6 * N, "logit": 10 * N, "colors": 11 * N}
    for k in ("means", "log_scales", "quats", "logit", "colors"):
        gk = go[k].reshape(N, -1)
        ref, m_ref, _ = OL.adam_step(before[k].reshape(N, -1), gk, 0.0, 0.0, 1, lrs[k])
        mk = m_gpu[off[k]:off[k] + gk.size].reshape(gk.shape)
        assert rel_l2(mk, m_ref) <= TOL_GRAD, k
        # where the gradient is well above its FP32 noise its sign is certain and the update exact;
        # everywhere else the step is bounded by the learning rate, and zero where nothing touched
        sure = np.abs(gk) > 1e-3 * np.abs(gk).max()
        a_k = after[k].reshape(N, -1)
        assert sure.sum() > 1000, k
        np.testing.assert_allclose(a_k[sure], ref[sure], rtol=1e-6, atol=1e-7 * lrs[k] / 1e-4)
        assert np.all(np.abs(a_k - before[k].reshape(N, -1)) <= lrs[k] * (1 + 1e-5) + 1e-6 * np.abs(a_k))
        untouched = np.all(gk == 0.0, axis=1)
        np.testing.assert_array_equal(a_k[untouched], before[k].reshape(N, -1)[untouched].astype(np.float32))
