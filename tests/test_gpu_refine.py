"""Joint pose-Gaussian refinement (Sec. III-C): exposure-compensated loss of Eq. 23, pruning and
the per-view pose / exposure Adam, against the FP64 oracles; and a refinement loop that recovers a
perturbed keyframe pose and exposure."""
import numpy as np
import pytest

from helpers import gpu_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import losses as OL  # noqa: E402
from oracle.oracle import exp_se3_left  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


@pytest.mark.parametrize("V,H,W", [(2, 70, 97), (1, 680, 1200)])
def test_refine_loss_matches_oracle(R, V, H, W):
    rng = np.random.default_rng(V + H)
    y = np.stack([S.smooth_image(W, H, 5 + v) for v in range(V)])
    x = np.clip(y * 0.9 + rng.normal(0, 0.05, y.shape), 0, 1).astype(np.float32)
    d = rng.uniform(1, 4, (V, H, W)).astype(np.float32)
    dt = (d + rng.normal(0, 0.1, d.shape)).astype(np.float32)
    expo = np.stack([rng.normal(0, 0.1, V), rng.normal(0, 0.02, V)], 1).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, g_rgb, g_d, g_e = R.loss_refine(t(x), t(y), t(expo), t(d), t(dt))
    Lr, gr, gd, ga, gb = OL.refine_loss(x, y, d, dt, expo[:, 0], expo[:, 1], fp32_sign=True)
    assert abs(loss.item() - Lr) <= 1e-5 * abs(Lr)
    assert rel_l2(g_rgb.cpu().numpy(), gr) <= 1e-4
    assert rel_l2(g_d.cpu().numpy(), gd) <= 1e-6
    ge = g_e.cpu().numpy()
    assert rel_l2(ge[:, 0], ga) <= 1e-4 and rel_l2(ge[:, 1], gb) <= 1e-4


def test_prune_matches_oracle(R):
    sc = S.random_cloud(50_000, seed=4)
    rng = np.random.default_rng(4)
    sc.opacities[rng.choice(sc.n, 7000, replace=False)] = rng.uniform(0, 0.0049, 7000).astype(np.float32)
    sc.opacities[:3] = np.float32(0.005)                        # exactly at the threshold: kept
    g = R.Gaussians.from_scene(sc)
    out = R.prune(g, 0.005)
    keep = OL.prune_keep(sc.opacities, 0.005)
    assert out.n == len(keep)
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), getattr(sc, k)[keep])


def test_view_adam_matches_oracle(R):
    wl = S.workload("agents8x4", scale=0.01)
    pb, g = gpu_problem(wl, views=[0, 5, 9])
    st = R.ViewAdamState(pb, lr_pose=1e-2, lr_expo=5e-2)
    rng = np.random.default_rng(2)
    cams = [pb.cameras[v].cpu().numpy().astype(np.float64) for v in range(3)]
    expo = [np.zeros(2) for _ in range(3)]
    mom = [(np.zeros(8), np.zeros(8)) for _ in range(3)]
    for step in range(1, 4):
        pg = rng.normal(0, 1, (3, 6)).astype(np.float32)
        eg = rng.normal(0, 1, (3, 2)).astype(np.float32)
        st.apply(torch.from_numpy(pg).cuda(), torch.from_numpy(eg).cuda())
        for v in range(3):
            cams[v], expo[v], m, vv = OL.view_adam_step(cams[v], expo[v], pg[v], eg[v], *mom[v], step, 1e-2, 5e-2)
            mom[v] = (m, vv)
    torch.cuda.synchronize()
    got = pb.cameras.cpu().numpy()
    for v in range(3):
        np.testing.assert_allclose(got[v], cams[v], atol=2e-5, rtol=1e-5)
        np.testing.assert_allclose(st.expo[v].cpu().numpy(), expo[v], atol=1e-5)
    assert int(st.step.item()) == 3


def test_refine_loop_recovers_pose_and_exposure(R):
    from paper_2605_10760_gb300 import mapping as M
    wl = S.workload("room500k", scale=0.1)
    wl.cameras = S.room_cameras(wl.scene, 2, seed=31, width=400, height=240, fx=200, fy=200, cx=200, cy=120)
    wl.scene_of_view = np.zeros(2, np.int32)
    wl.width, wl.height = 400, 240
    pb, g = gpu_problem(wl)
    true_cams = pb.cameras.clone()
    img = pb.forward_checked(g)
    a_true, b_true = 0.15, 0.03
    target = (np.exp(a_true) * img["rgb"] + b_true).contiguous()
    depth_t = img["depth"].clone()
    # perturb the poses (left perturbation) and start from zero exposure
    rng = np.random.default_rng(3)
    pert = pb.cameras.cpu().numpy().astype(np.float64)
    for v in range(2):
        pert[v] = exp_se3_left(pert[v], np.concatenate([rng.normal(0, 0.01, 3), rng.normal(0, 0.004, 3)]))
    pb.cameras.copy_(torch.from_numpy(pert.astype(np.float32)).cuda())
    err0 = (pb.cameras - true_cams)[:, :12].abs().max().item()
    loop = M.RefineLoop(pb, g, target, depth_t, lr=(0.0, 0.0, 0.0, 0.0, 0.0), lr_pose=2e-4, lr_expo=5e-3)
    loop.iteration()
    l0 = loop.loss.item()
    loop.capture(50)
    for _ in range(4):
        loop.replay()
    torch.cuda.synchronize()
    assert pb.check_status()[0] == 0
    err1 = (pb.cameras - true_cams)[:, :12].abs().max().item()
    expo = loop.view.expo.cpu().numpy()
    assert loop.loss.item() < 0.5 * l0
    assert err1 < 0.5 * err0
    assert np.abs(expo[:, 0] - a_true).max() < 0.05 and np.abs(expo[:, 1] - b_true).max() < 0.03
