"""Eq. 12 anchor-image photometric residual blocks (gs_pho_residual) against the FP64 oracle:
synthetic and rendered anchors, ragged sizes, strides, empty and invalid edges, the full
1200x680 size, determinism, and a Gauss-Newton loop that recovers a perturbed submap correction."""
import numpy as np
import pytest
from scipy.linalg import expm

from helpers import gpu_problem, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import photometric as PH  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def _quat(Rm):
    w = np.sqrt(max(1e-12, 1 + np.trace(Rm))) / 2
    return np.array([w, (Rm[2, 1] - Rm[1, 2]) / (4 * w), (Rm[0, 2] - Rm[2, 0]) / (4 * w), (Rm[1, 0] - Rm[0, 1]) / (4 * w)])


def _retract(sim, xi):
    q, t, s = sim
    Rp = expm(_skew(xi[3:6]))
    Rm = Rp @ PH.quat_matrix(q)
    es = np.exp(xi[6])
    return (_quat(Rm).astype(np.float32), (es * Rp @ np.asarray(t, np.float64) + xi[:3]).astype(np.float32),
            np.float32(es * s))


IDENT = (np.array([1, 0, 0, 0], np.float32), np.zeros(3, np.float32), np.float32(1.0))


def _f32sim(q, t, s):
    return (np.asarray(q, np.float32), np.asarray(t, np.float32), np.float32(s))


def _compare(R, edges, images, depths, cams, corrs, stride=1, tol_h=1e-4, tol_g=1e-3):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pr = R.PhoResidual(len(edges))
    out = pr(R.pho_edges(edges), t(images), t(depths), t(cams), R.sim3_tensor(corrs), stride=stride)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    M = images.shape[0]
    for e, (a, b, ca, cb, w) in enumerate(edges):
        if not (0 <= a < M and 0 <= b < M and 0 <= ca < len(corrs) and 0 <= cb < len(corrs)):
            assert got["count"][e] == -1 and got["cost"][e] == 0 and not got["H"][e].any() and not got["g"][e].any()
            continue
        ref = PH.edge_terms(images[a], depths[a], images[b], cams[a], cams[b], corrs[ca], corrs[cb], w, stride)
        assert got["count"][e] == ref["n"], (e, got["count"][e], ref["n"])
        if ref["n"] == 0:
            assert got["cost"][e] == 0 and not got["H"][e].any() and not got["g"][e].any()
            continue
        assert abs(got["cost"][e] - ref["cost"]) <= 1e-5 * ref["cost"] + 1e-12, e
        assert rel_l2(got["H"][e], ref["H"]) <= tol_h, (e, rel_l2(got["H"][e], ref["H"]))
        assert rel_l2(got["g"][e], ref["g"]) <= tol_g, (e, rel_l2(got["g"][e], ref["g"]))
    return out


def _synthetic(W, H, seed):
    rng = np.random.default_rng(seed)
    imgs = np.stack([S.smooth_image(W, H, seed + k) for k in range(3)])
    deps = np.stack([S.smooth_image(W, H, seed + 10 + k, channels=1, lo=1.0, hi=4.0)[0] for k in range(3)])
    deps[2, :, :] = 0.0                                  # keyframe 2 has no valid depth
    cams = []
    for k in range(3):
        Rm = expm(_skew(rng.normal(0, 0.05, 3)))
        cams.append(np.concatenate([Rm.ravel(), rng.normal(0, 0.05, 3), [0.8 * W, 0.8 * W, W / 2, H / 2]]))
    corrs = [_f32sim(rng.normal(0, 1, 4) * [1, 0.02, 0.02, 0.02] + [2, 0, 0, 0], rng.normal(0, 0.05, 3), 1 + 0.05 * k)
             for k in range(4)]
    return imgs.astype(np.float32), deps.astype(np.float32), np.array(cams, np.float32), corrs


@pytest.mark.parametrize("W,H,stride", [(97, 70, 1), (97, 70, 3), (256, 64, 2)])
def test_synthetic_edges_match_oracle(R, W, H, stride):
    imgs, deps, cams, corrs = _synthetic(W, H, W + H + stride)
    edges = [(0, 1, 0, 1, 1.0), (1, 0, 1, 0, 0.5), (0, 1, 2, 3, 2.0), (1, 2, 0, 0, 1.0),
             (2, 0, 1, 2, 1.0),                         # empty U_e: keyframe 2 has no depth
             (0, 5, 0, 1, 1.0), (0, 1, 0, 9, 1.0)]      # out-of-range indices
    _compare(R, edges, imgs, deps, cams, corrs, stride=stride)


def _rendered(R, W, H, seed=31):
    wl = S.workload("room500k", scale=0.1)
    cam = S.room_cameras(wl.scene, 1, seed=seed, width=W, height=H, fx=W / 2, fy=W / 2, cx=W / 2, cy=H / 2)[0]
    Rb = expm(_skew([0.01, -0.03, 0.02])) @ cam.R.astype(np.float64)
    tb = cam.t.astype(np.float64) + np.array([0.08, -0.02, 0.03])
    camb = S.Camera(Rb.astype(np.float32), tb.astype(np.float32), cam.fx, cam.fy, cam.cx, cam.cy, W, H)
    wl.cameras = [cam, camb]
    wl.scene_of_view = np.zeros(2, np.int32)
    wl.width, wl.height = W, H
    pb, g = gpu_problem(wl)
    img = pb.forward_checked(g)
    a = img["alpha"]
    dep = torch.where(a > 0.5, img["depth"] / a.clamp_min(1e-6), torch.zeros_like(a))
    return (img["rgb"].cpu().numpy(), dep.cpu().numpy().astype(np.float32), pb.cameras.cpu().numpy())


def test_rendered_anchor_pair_matches_oracle(R):
    imgs, deps, cams = _rendered(R, 320, 200)
    corrs = [IDENT, _retract(IDENT, np.array([0.02, -0.01, 0.01, 0.004, -0.003, 0.002, 0.01])),
             _retract(IDENT, np.array([0.3, 0.1, -0.2, 0.5, 0.2, -0.1, 0.2]))]
    edges = [(0, 1, 0, 0, 1.0), (0, 1, 1, 0, 1.0), (1, 0, 0, 1, 3.0), (0, 1, 2, 2, 1.0)]
    _compare(R, edges, imgs, deps, cams, corrs)


def test_full_size_edge_and_determinism(R):
    imgs, deps, cams = _rendered(R, 1200, 680, seed=32)
    corrs = [IDENT, _retract(IDENT, np.array([0.02, -0.01, 0.01, 0.004, -0.003, 0.002, 0.01]))]
    edges = [(0, 1, 1, 0, 1.0), (1, 0, 0, 1, 1.0)]
    out1 = _compare(R, edges, imgs, deps, cams, corrs)
    o1 = {k: v.clone() for k, v in out1.items()}
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out2 = R.PhoResidual(2)(R.pho_edges(edges), t(imgs), t(deps), t(cams), R.sim3_tensor(corrs))
    for k in o1:
        assert torch.equal(o1[k], out2[k]), k


def test_gauss_newton_recovers_source_correction(R):
    """The rendered pair is consistent under identity corrections; starting C_src from a Sim(3)
    perturbed by about a pixel, damped Gauss-Newton steps on xi_src built from the GPU blocks reach
    the cost of the identity correction (the textured images give a basin of about a pixel)."""
    imgs, deps, cams = _rendered(R, 320, 200, seed=33)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ti, td, tc = t(imgs), t(deps), t(cams)
    edges = R.pho_edges([(0, 1, 0, 1, 1.0), (1, 0, 1, 0, 1.0)])
    pr = R.PhoResidual(2)
    c_ident = float(pr(edges, ti, td, tc, R.sim3_tensor([IDENT, IDENT]))["cost"].sum())
    cur = _retract(IDENT, np.array([0.005, -0.003, 0.003, 0.001, -0.0008, 0.0005, 0.002]))
    costs = []
    for _ in range(12):
        o = pr(edges, ti, td, tc, R.sim3_tensor([cur, IDENT]))
        costs.append(float(o["cost"].sum()))
        # edge 0 holds the perturbed correction in its source slot, edge 1 in its target slot
        Hx = o["H"][0, :7, :7].cpu().numpy() + o["H"][1, 7:, 7:].cpu().numpy()
        gx = o["g"][0, :7].cpu().numpy() + o["g"][1, 7:].cpu().numpy()
        step = -np.linalg.solve(Hx + 1e-6 * np.diag(np.diag(Hx)) + 1e-9 * np.eye(7), gx)
        cur = _retract(cur, step)
    assert costs[-1] < 0.5 * costs[0] and costs[-1] <= 1.02 * c_ident, (costs, c_ident)
    assert all(b <= a * 1.001 for a, b in zip(costs, costs[1:])), costs
