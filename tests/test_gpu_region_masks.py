"""The compositing kernels' per-warp region masks skip a list entry for a whole 8x8 pixel block
when sigma exceeds the entry's cut-off everywhere in the block.  That skip must never change a
decision of the FP32 chain, also for footprints where FP32 rounding of sigma is largest: very thin
Gaussians (conic entries of 1e4 to 1e6, |B| close to sqrt(AC)) whose sigma at a block corner lies
within 1e-2 of the cut-off.  The bar is the decision bar of the path: projection decisions, keys
and last_idx bit-exact against the oracle, and the same number of visited pairs.

(Colour values are not compared at these footprints: sigma's FP32 rounding error grows with the
conic entries, so FP32 values legitimately differ from the oracle's FP64 values there.)
"""
import numpy as np
import pytest

from helpers import gpu_problem, oracle_params_from

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.oracle import Oracle  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402

W = H = 512
F_PX = 400.0
Z = 3.0
DIL = 1e-6
AMIN = 1.0 / 255.0


def _design(n, seed, o_p=None, proj=None, corners=None, normals=None, dirs=None, targets=None):
    """Thin line-like Gaussians, each passing just outside the top-left pixel centre of an 8x8 block
    (the block's nearest point to the line), at the distance where the quadratic at that corner
    equals cut + eps, eps ~ U[-0.02, 0.02].  Second call: re-solve the distance from the conic of a
    first projection."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(np.deg2rad(-80), np.deg2rad(-10), n)
    u = np.stack([np.cos(th), np.sin(th)], 1)              # long axis in the image
    nout = np.stack([u[:, 1], -u[:, 0]], 1)                # normal pointing away from the block
    bx = rng.integers(2, W // 8 - 2, n)
    by = rng.integers(2, H // 8 - 2, n)
    corner = np.stack([bx * 8 + 0.5, by * 8 + 0.5], 1)
    o = rng.uniform(0.3, 0.99, n).astype(np.float32)
    thin = rng.uniform(-11.5, -8.5, n)
    ls = np.stack([np.full(n, -2.9), thin, thin - 0.5], 1).astype(np.float32)
    eps = rng.uniform(-0.02, 0.02, n)
    cut = np.log(o.astype(np.float64) / AMIN) + 1e-3
    target = cut + eps
    if proj is None:
        q_perp = np.full(n, 1.0 / (2 * (F_PX / Z * np.exp(thin)) ** 2 + DIL))
    else:
        A, B, C = proj["conic"][:, 0].astype(np.float64), proj["conic"][:, 1].astype(np.float64), \
            proj["conic"][:, 2].astype(np.float64)
        q_perp = 0.5 * (A * nout[:, 0] ** 2 + 2 * B * nout[:, 0] * nout[:, 1] + C * nout[:, 1] ** 2)
    delta = np.sqrt(target / q_perp)
    mean2d = corner + delta[:, None] * nout
    means = np.stack([(mean2d[:, 0] - W / 2) * Z / F_PX, (mean2d[:, 1] - H / 2) * Z / F_PX, np.full(n, Z)], 1)
    quats = np.stack([np.cos(th / 2), np.zeros(n), np.zeros(n), np.sin(th / 2)], 1)
    cols = rng.uniform(0, 1, (n, 3))
    sc = S.Scene(means.astype(np.float32), ls, quats.astype(np.float32), o, cols.astype(np.float32))
    return sc, corner, cut


def thin_workload(n=2500, seed=5):
    cam = S.identity_camera(W, H, F_PX, F_PX, W / 2, H / 2)
    sc0, _, _ = _design(n, seed)
    wl0 = S.Workload("thin", sc0, np.array([0, n], np.int64), [cam], np.zeros(1, np.int32), W, H)
    from oracle.oracle import Params
    pr0 = Oracle.from_workload(wl0, Params(dilation=DIL)).projection()
    sc, corner, cut = _design(n, seed, proj=pr0)
    return S.Workload("thin", sc, np.array([0, n], np.int64), [cam], np.zeros(1, np.int32), W, H), corner, cut


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def test_thin_footprints_near_the_cut_keep_decisions_exact(R):
    wl, corner, cut = thin_workload()
    p = R.default_params(dilation=DIL)
    orc = Oracle.from_workload(wl, oracle_params_from(p))
    op = orc.projection()
    # the workload is adversarial: thin footprints, corner sigma within 1e-2 of the cut
    A, B, C = (op["conic"][:, k].astype(np.float64) for k in range(3))
    vis = op["touched"] > 0
    d = corner - op["mean2d"].astype(np.float64)
    sig = 0.5 * (A * d[:, 0] ** 2 + C * d[:, 1] ** 2) + B * d[:, 0] * d[:, 1]
    near = vis & (np.abs(sig - cut) < 1e-2)
    assert near.sum() >= 0.3 * len(cut), near.sum()
    assert np.median(np.maximum(A, C)[vis]) > 1e4 and np.max(np.maximum(A, C)[vis]) > 5e5
    assert np.median((np.abs(B) / np.sqrt(A * C))[vis]) > 0.99
    fw = orc.forward()
    for mode in (1, 0):
        pm = R.default_params(dilation=DIL, sort_mode=mode)
        pb, g = gpu_problem(wl, params=pm)
        pb.project(g)
        proj = pb.workspace()["proj"].clone().cpu().numpy()
        pb.bin_sort()
        img = pb.render_fwd()
        torch.cuda.synchronize()
        rc, _ = pb.check_status()
        assert rc == 0
        np.testing.assert_array_equal(proj[vis, 0:2].view(np.uint32), op["mean2d"][vis].view(np.uint32))
        np.testing.assert_array_equal(proj[vis, 2:5].view(np.uint32), op["conic"][vis].view(np.uint32))
        ws = pb.workspace()
        K = int(ws["num_keys"][0].item()) & 0xffffffff
        assert K == orc.K
        np.testing.assert_array_equal(ws["sorted_vals"][:K].cpu().numpy().view(np.uint32), orc.bins()["vals"])
        last = img["last_idx"].cpu().numpy()
        bad = np.argwhere(last != fw["last"])
        assert bad.size == 0, ("last_idx differs at", bad[:10], last[tuple(bad[0])], fw["last"][tuple(bad[0])])
        assert pb.stats()["fwd_pairs"] == fw["pairs"]
