"""GPU parity of the loss kernels and the in-kernel Adam step against the FP64 oracles."""
import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import losses as OL  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


# weights: the benchmark step's (1.0, 0.1) and Eq. 4's alpha = 0.95, beta = 0.25
@pytest.mark.parametrize("w_rgb,w_depth", [(1.0, 0.1), (0.95, 0.25)])
@pytest.mark.parametrize("V,H,W", [(1, 37, 53), (2, 68, 120), (1, 680, 1200)])
def test_l1_rgb_depth(R, V, H, W, w_rgb, w_depth):
    rng = np.random.default_rng(V * H)
    x = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    y = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    d = rng.uniform(0, 5, (V, H, W)).astype(np.float32)
    dt = rng.uniform(0, 5, (V, H, W)).astype(np.float32)
    x[0, 0, 0, :5] = y[0, 0, 0, :5]              # sign(0) = 0
    t = lambda a: torch.from_numpy(a).cuda()
    loss, d_rgb, d_d = R.loss_l1(t(x), t(y), t(d), t(dt), w_rgb, w_depth)
    L, gr, gd = OL.mapping_l1_loss(x, y, d, dt, w_rgb, w_depth)
    assert abs(loss.item() - L) <= 1e-6 * abs(L)
    np.testing.assert_allclose(d_rgb.cpu().numpy(), gr, rtol=1e-6, atol=0)
    np.testing.assert_allclose(d_d.cpu().numpy(), gd, rtol=1e-6, atol=0)


@pytest.mark.parametrize("V,H,W", [(1, 40, 45), (2, 70, 97), (1, 680, 1200)])
def test_l1_ssim(R, V, H, W):
    rng = np.random.default_rng(H + W)
    y = S.smooth_image(W, H, seed=3)[None].repeat(V, 0)
    x = np.clip(y + rng.normal(0, 0.05, y.shape), 0, 1).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, d_rgb = R.loss_l1_ssim(t(x), t(y), 0.8, 0.2)
    L, g = OL.l1_ssim_loss(x, y, 0.8, 0.2)
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    assert rel_l2(d_rgb.cpu().numpy(), g) <= 1e-4


def test_adam_step_matches_oracle(R):
    rng = np.random.default_rng(5)
    n = 3000
    sc = S.random_cloud(n, seed=9)
    g = R.Gaussians.from_scene(sc)
    st = R.AdamState(g, lr=(1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3))
    ref = {k: getattr(sc, k).astype(np.float64) for k in ("means", "log_scales", "quats", "colors")}
    o = sc.opacities.astype(np.float64)
    ref["logit"] = np.log(o / (1 - o))
    mom = {k: (np.zeros_like(v), np.zeros_like(v)) for k, v in ref.items()}
    lrs = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "logit": 5e-2, "colors": 2.5e-3}
    for step in range(1, 4):
        grads = {k: rng.normal(0, 1, getattr(sc, k).shape).astype(np.float32)
                 for k in ("means", "log_scales", "quats", "opacities", "colors")}
        gg = R.Gaussians(*[torch.from_numpy(grads[k]).cuda() for k in ("means", "log_scales", "quats", "opacities",
                                                                          "colors")])
        o_now = 1 / (1 + np.exp(-ref["logit"]))
        st.apply(gg, zero_grads=True)
        assert float(gg.means.abs().sum()) == 0.0
        for k in ("means", "log_scales", "quats", "colors", "logit"):
            gk = grads["opacities"].astype(np.float64) * o_now * (1 - o_now) if k == "logit" else grads[k]
            ref[k], m, v = OL.adam_step(ref[k], gk.astype(np.float64), *mom[k], step, lrs[k])
            mom[k] = (m, v)
    for k in ("means", "log_scales", "quats", "colors"):
        np.testing.assert_allclose(getattr(g, k).cpu().numpy(), ref[k], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(st.logits.cpu().numpy(), ref["logit"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(g.opacities.cpu().numpy(), 1 / (1 + np.exp(-ref["logit"])), rtol=1e-5, atol=1e-6)
    assert int(st.step.item()) == 3


def test_adam_with_isotropy_regulariser_matches_oracle(R):
    """Adam with lambda_s L_iso (Eq. 4) fused into the log-scale update."""
    rng = np.random.default_rng(8)
    sc = S.random_cloud(2000, seed=12)
    g = R.Gaussians.from_scene(sc)
    st = R.AdamState(g, lr=(1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3))
    ls = sc.log_scales.astype(np.float64)
    m, v = np.zeros_like(ls), np.zeros_like(ls)
    iso = torch.zeros(1, dtype=torch.float64, device="cuda")
    for step in range(1, 3):
        gls = rng.normal(0, 1, ls.shape).astype(np.float32)
        grads = R.zeros_like_grads(g)
        grads.log_scales.copy_(torch.from_numpy(gls).cuda())
        val, giso = OL.iso_loss(ls, 10.0)
        st.apply(grads, zero_grads=True, iso_weight=10.0, iso_loss=iso)
        torch.cuda.synchronize()
        assert abs(iso.item() - val) <= 1e-5 * val
        ls, m, v = OL.adam_step(ls, gls + giso, m, v, step, 5e-3)
    np.testing.assert_allclose(g.log_scales.cpu().numpy(), ls, rtol=1e-5, atol=2e-6)


def test_render_fwd_with_fused_l1_matches_separate_calls(R):
    """gs_render_fwd_l1 = gs_render_fwd followed by gs_loss_l1 on its outputs."""
    from helpers import gpu_problem
    wl = S.workload("room500k", scale=0.1)
    pb, g = gpu_problem(wl)
    img = pb.forward_checked(g)
    H, W = wl.height, wl.width
    tgt = torch.from_numpy(S.smooth_image(W, H, 41)[None]).cuda()
    dtg = torch.from_numpy(S.smooth_image(W, H, 42, channels=1, lo=0.5, hi=5.0)).cuda()
    loss_a, d_rgb_a, d_d_a = R.loss_l1(img["rgb"], tgt, img["depth"], dtg, 1.0, 0.1)
    img2 = pb.alloc_image()
    img2, loss_b, d_rgb_b, d_d_b = pb.render_fwd_l1(img2, tgt, dtg, 1.0, 0.1)
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "alpha", "final_T", "last_idx"):
        assert torch.equal(img[k], img2[k]), k
    assert torch.equal(d_rgb_a, d_rgb_b) and torch.equal(d_d_a, d_d_b)
    assert abs(loss_a.item() - loss_b.item()) <= 1e-6 * abs(loss_a.item())
    # rgb-only loss, images not requested
    img3 = {"final_T": torch.empty_like(img["final_T"]), "last_idx": torch.empty_like(img["last_idx"])}
    _, loss_c, d_rgb_c, _ = pb.render_fwd_l1(img3, tgt, None, 1.0, 0.0)
    loss_r, d_rgb_r, _ = R.loss_l1(img["rgb"], tgt, None, None, 1.0, 0.0)
    torch.cuda.synchronize()
    assert torch.equal(d_rgb_c, d_rgb_r) and abs(loss_c.item() - loss_r.item()) <= 1e-6 * abs(loss_r.item())


def test_resume_from_checkpoint_continues_adam_exactly(R, tmp_path):
    """Two Adam steps, checkpoint, two more steps == reload, two more steps (bit for bit)."""
    sc = S.random_cloud(1000, seed=13)
    rng = np.random.default_rng(13)
    grads = [R.Gaussians(*[torch.from_numpy(rng.normal(0, 1, getattr(sc, k).shape).astype(np.float32)).cuda()
                           for k in ("means", "log_scales", "quats", "opacities", "colors")]) for _ in range(4)]
    g = R.Gaussians.from_scene(sc)
    st = R.AdamState(g)
    for i in range(2):
        st.apply(R.Gaussians(*[t.clone() for t in (grads[i].means, grads[i].log_scales, grads[i].quats,
                                                   grads[i].opacities, grads[i].colors)]), zero_grads=True)
    R.save_checkpoint(tmp_path / "c.pt", g, st)
    g2, st2, _ = R.load_checkpoint(tmp_path / "c.pt")
    for gg, ss in ((g, st), (g2, st2)):
        for i in range(2, 4):
            ss.apply(R.Gaussians(*[t.clone() for t in (grads[i].means, grads[i].log_scales, grads[i].quats,
                                                       grads[i].opacities, grads[i].colors)]), zero_grads=True)
    torch.cuda.synchronize()
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        assert torch.equal(getattr(g, k), getattr(g2, k)), k
    assert int(st.step.item()) == int(st2.step.item()) == 4

