"""Occupancy-aware fusion on the GPU (Eqs. 19-22) against the fusion oracle: the Sim(3) action,
the occupied and free-space voxel sets (bit-exact sets), the deduplication flags; the render of a
Sim(3)-transformed map equals the original render from the correspondingly moved camera, with depth
scaled by s; a full table reports GS_ERR_CAPACITY instead of looping."""
import numpy as np
import pytest

from helpers import gpu_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fusion as FU  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def test_sim3_matches_oracle(R):
    sc = S.random_cloud(20_000, seed=5)
    g = R.Gaussians.from_scene(sc)
    q, t, s = np.array([0.9, 0.1, -0.3, 0.2]), np.array([0.4, -1.2, 2.0]), 1.37
    out = R.sim3_apply(g, q, t, s)
    mu, ls, qq = FU.sim3_apply(sc.means, sc.log_scales, sc.quats, s, q, t)
    np.testing.assert_allclose(out.means.cpu().numpy(), mu, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(out.log_scales.cpu().numpy(), ls, atol=1e-5)
    np.testing.assert_allclose(out.quats.cpu().numpy(), qq, atol=1e-5)
    np.testing.assert_array_equal(out.opacities.cpu().numpy(), sc.opacities)
    np.testing.assert_array_equal(out.colors.cpu().numpy(), sc.colors)


def test_render_invariant_under_sim3(R):
    """Moving the map by C and the world-to-camera pose by T' = [R_c R^T, s t_c - R_c R^T t] gives
    p_c' = s p_c: the same image, depth times s (Eq. 19's scale block)."""
    wl = S.workload("room500k", scale=0.1)
    pb, g = gpu_problem(wl)
    img0 = {k: v.clone() for k, v in pb.forward_checked(g).items()}
    q, t, s = np.array([0.95, 0.05, 0.2, -0.1]), np.array([1.5, -0.5, 0.25]), 1.8
    g2 = R.sim3_apply(g, q, t, s)
    Rm = FU.quat_to_matrix(q)
    cam = pb.cameras[0].cpu().numpy().astype(np.float64)
    Rc, tc = cam[:9].reshape(3, 3), cam[9:12]
    cam2 = cam.copy()
    cam2[:9] = (Rc @ Rm.T).ravel()
    cam2[9:12] = s * tc - Rc @ Rm.T @ t
    pb.cameras.copy_(torch.from_numpy(cam2[None].astype(np.float32)).cuda())
    img1 = pb.forward_checked(g2)
    rgb0, rgb1 = img0["rgb"].cpu().numpy(), img1["rgb"].cpu().numpy()
    diff = np.abs(rgb0 - rgb1)
    assert diff.mean() < 1e-4 and np.mean(diff > 1e-2) < 2e-3
    d0, d1 = img0["depth"].cpu().numpy(), img1["depth"].cpu().numpy()
    m = img0["alpha"].cpu().numpy() > 0.5
    assert np.median(np.abs(d1[m] - s * d0[m]) / (s * d0[m])) < 1e-4


def _small_maps():
    wl = S.workload("room500k", scale=0.01)              # 5k-Gaussian room
    cams = [S.room_cameras(wl.scene, 2, seed=77, width=64, height=48, fx=32, fy=32, cx=32, cy=24)[i]
            for i in range(2)]
    return wl, cams


def test_voxel_sets_and_dedup_match_oracle(R):
    wl, cams = _small_maps()
    sc = wl.scene
    v, k = 0.05, 3.0
    g = R.Gaussians.from_scene(sc)
    occ = R.VoxSet(1 << 18)
    occ.add_boxes(g.means, g.log_scales, k, v)
    rc, n_occ = occ.status()
    ref_occ = FU.occupied_set(sc.means, sc.log_scales, k, v)
    assert rc == 0 and n_occ == len(ref_occ)
    assert occ.keys() == ref_occ
    # depth maps: rendered expected depth normalised by alpha where the surface is opaque
    wl2 = S.Workload("small", sc, np.array([0, sc.n], np.int64), cams, np.zeros(2, np.int32), 64, 48)
    pb, _ = gpu_problem(wl2)
    img = pb.forward_checked(g)
    a = img["alpha"]
    depth = torch.where(a > 0.5, img["depth"] / a.clamp_min(1e-6), torch.zeros_like(a)).contiguous()
    fre = R.VoxSet(1 << 18)
    fre.add_rays(pb.cameras, depth, 3, v)
    rc, n_free = fre.status()
    ref_free = FU.free_set(pb.cameras.cpu().numpy(), depth.cpu().numpy(), v, stride=3)
    assert rc == 0 and n_free == len(ref_free)
    assert fre.keys() == ref_free
    # borrowed map: another room moved by a Sim(3) into the same frame
    other = S.room_scene(6000, seed=91)
    gb = R.sim3_apply(R.Gaussians.from_scene(other), [1, 0, 0, 0.1], [0.3, 0.2, 0.0], 0.9)
    keep = R.dedup_keep(gb.means, occ, fre, v).cpu().numpy().astype(bool)
    ref_keep = FU.dedup_keep(gb.means.cpu().numpy(), ref_occ, ref_free, v)
    np.testing.assert_array_equal(keep, ref_keep)
    assert 0 < keep.sum() < len(keep)


def test_full_table_reports_capacity(R):
    sc = S.random_cloud(500, seed=3)
    g = R.Gaussians.from_scene(sc)
    small = R.VoxSet(64)
    small.add_boxes(g.means, g.log_scales, 3.0, 0.05)     # boxes of at most 17 voxels per axis
    rc, n = small.status()
    assert rc == R.L.GS_ERR_CAPACITY and n == 64


def test_box_beyond_supported_extent_is_flagged(R):
    sc = S.random_cloud(16, seed=4)
    sc.log_scales[5] = 0.0                                # 3 s = 3 m = 300 voxels of 1 cm per axis
    g = R.Gaussians.from_scene(sc)
    vs = R.VoxSet(1 << 20)
    vs.add_boxes(g.means, g.log_scales, 3.0, 0.01)
    rc, _ = vs.status()
    assert rc == R.L.GS_ERR_INVALID_ARG
