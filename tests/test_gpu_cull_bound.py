"""The projection pre-tests every (view, Gaussian) pair before the decision chain and runs the chain
only on the pairs that pass: those in front of the near plane whose footprint, with a radius bounded
from above (the trace of the 2-D covariance), can reach a tile of the image.  The pre-test must
never reject a pair the chain finds visible.  The adversarial case: footprints centred just
outside the image, with radii within a factor 0.5..1.5 of the distance to the image edge, strongly
anisotropic scales, random orientations, depths down to the near plane, centres far off the side
where the Jacobian's clamp applies, and rotated cameras.  The bar: tiles_touched and every
projection record bit-exact against the oracle, the same keys, last_idx and visited pairs.
"""
import numpy as np
import pytest

from helpers import gpu_problem, oracle_params_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402

W, H = 640, 360
FX = FY = 420.0


def _cameras():
    cams = [S.identity_camera(W, H, FX, FY, W / 2, H / 2)]
    cams.append(S.look_at([0.3, -0.2, 0.1], [2.0, 3.0, 1.5], W, H, FX, FY, W / 2, H / 2))
    cams.append(S.look_at([-1.0, 0.5, 2.0], [1.0, -2.0, -0.5], W, H, FX, FY, W / 2 + 13.0, H / 2 - 7.0))
    return cams


def border_scene(cam, n, seed, zmax=30.0):
    """Gaussians whose projected centre lies d px outside the image (d in [-20, 300]; negative:
    just inside) and whose 3-sigma radius is about d times U[0.5, 1.5]; a tenth far off the side
    (|x / z| beyond the clamp limit), a tenth right behind / in front of the near plane; depths up
    to zmax."""
    rng = np.random.default_rng(seed)
    z = np.exp(rng.uniform(np.log(0.25), np.log(zmax), n))
    z[: n // 10] = rng.uniform(0.15, 0.3, n // 10)                 # around the near plane 0.2
    side = rng.integers(0, 4, n)
    d = rng.uniform(-20.0, 300.0, n)
    along = rng.uniform(0.0, 1.0, n)
    u = np.where(side == 0, -d, np.where(side == 1, W + d, along * W))
    v = np.where(side == 2, -d, np.where(side == 3, H + d, along * H))
    far = slice(n // 10, n // 5)                                   # centres far off the side
    u[far] = np.where(rng.random(n // 10) < 0.5, -1.0, 1.0) * rng.uniform(2.0, 6.0, n // 10) * W + W / 2
    pc = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1)
    pw = (pc - cam.t.astype(np.float64)) @ cam.R.astype(np.float64)          # R^T (p_c - t)
    r_px = np.maximum(np.abs(d), 2.0) * rng.uniform(0.5, 1.5, n)
    smax = r_px * z / (3.0 * cam.fx)
    aniso = np.exp(rng.uniform(-4.0, 0.0, (n, 2)))
    ls = np.log(np.stack([smax, smax * aniso[:, 0], smax * aniso[:, 1]], 1))
    perm = rng.permuted(np.tile(np.arange(3), (n, 1)), axis=1)
    ls = np.take_along_axis(ls, perm, 1)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = rng.uniform(0.2, 0.99, n)
    col = rng.uniform(0, 1, (n, 3))
    return S.Scene(pw.astype(np.float32), ls.astype(np.float32), q.astype(np.float32), o.astype(np.float32),
                   col.astype(np.float32))


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


@pytest.mark.parametrize("view", [0, 1, 2])
def test_border_footprints_keep_visibility_exact(R, view):
    cam = _cameras()[view]
    n = 20000
    sc = border_scene(cam, n, seed=31 + view)
    wl = S.Workload("border", sc, np.array([0, n], np.int64), [cam], np.zeros(1, np.int32), W, H)
    p = R.default_params()
    orc = Oracle.from_workload(wl, oracle_params_from(p))
    op = orc.projection()
    vis = op["touched"] > 0
    # adversarial: many visible pairs centred outside the image, many culled only by their extent
    mx, my = op["mean2d"][:, 0].astype(np.float64), op["mean2d"][:, 1].astype(np.float64)
    outside = (mx < 0) | (mx > W) | (my < 0) | (my > H)
    front = op["depth"] > p.near_plane
    assert (vis & outside).sum() > 0.15 * n, (vis & outside).sum()
    assert (front & outside & ~vis).sum() > 0.15 * n, (front & outside & ~vis).sum()
    pb, g = gpu_problem(wl, params=p, key_capacity=1 << 21)
    pb.project(g)
    ws = pb.workspace()
    touched = ws["tiles_touched"].clone().cpu().numpy().view(np.uint32)
    proj = ws["proj"].clone().cpu().numpy()
    np.testing.assert_array_equal(touched, op["touched"])
    np.testing.assert_array_equal(proj[vis, 0:2].view(np.uint32), op["mean2d"][vis].view(np.uint32))
    np.testing.assert_array_equal(proj[vis, 2:5].view(np.uint32), op["conic"][vis].view(np.uint32))
    np.testing.assert_array_equal(proj[vis, 7], op["radius"][vis])
    # every visible pair holds a slot; the slots taken also count the pre-test's candidates that
    # the decision chain culled (holes), never fewer than the visible pairs
    slots = ws["pair_slot"].clone().cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(slots != 0xFFFFFFFF, vis)
    assert pb.stats()["num_visible"] >= int(vis.sum())
    pb.bin_sort()
    img = pb.render_fwd()
    torch.cuda.synchronize()
    rc, _ = pb.check_status()
    assert rc == 0
    ws = pb.workspace()
    K = int(ws["num_keys"][0].item()) & 0xffffffff
    assert K == orc.K
    np.testing.assert_array_equal(ws["sorted_keys"][:K].cpu().numpy().view(np.uint64), orc.bins()["keys"])
    fw = orc.forward()
    np.testing.assert_array_equal(img["last_idx"].cpu().numpy(), fw["last"])
    assert pb.stats()["fwd_pairs"] == fw["pairs"]


def test_holes_skipped_by_the_projection_adjoint(R):
    """The border scene's pre-test keeps candidates that the decision chain then culls: their slots
    stay holes, which the projection adjoint must skip.  With holes present, every gradient (and
    the pose gradient) still matches the oracle.  Depths up to 6 m, as in the other parity scenes
    (the 2e-4 image tolerance is an absolute one, and the rendered depth grows with z)."""
    from test_gpu_parity import compare_all, run_gpu, run_oracle
    cam = _cameras()[1]
    n = 4000
    sc = border_scene(cam, n, seed=57, zmax=6.0)
    wl = S.Workload("border", sc, np.array([0, n], np.int64), [cam], np.zeros(1, np.int32), W, H)
    p = R.default_params()
    gpu = run_gpu(R, wl, params=p, key_capacity=1 << 21)
    assert gpu["rc"] == 0 and gpu["rc_end"] == 0
    visible = int((gpu["touched"] > 0).sum())
    assert gpu["stats"]["num_visible"] > visible > 0, (gpu["stats"]["num_visible"], visible)
    orc = run_oracle(wl, params=p, up=gpu["up"])
    compare_all(gpu, orc)
