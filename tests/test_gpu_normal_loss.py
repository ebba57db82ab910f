"""GPU parity of the normal term of Eq. 4 (gs_loss_normal) against the FP64 oracle, on images that
span several of the kernel's 60-column x 16-row items in both directions or less than one, with
ragged last items, of even width (pixel pairs loaded as 8-byte pairs) and odd width, down to
images with no interior pixel."""
import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import losses as OL  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_10760_gb300 import raster
    raster.L.load()
    return raster


def _normal_case(rng, V, H, W):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    depth = np.empty((V, H, W))
    for v in range(V):
        a, b = rng.uniform(-1.5, 1.5, 2)
        ph = rng.uniform(0, 6.3)
        depth[v] = 2.5 + a * x / W + b * y / H + 0.4 * np.sin(9.0 * x / W + ph) * np.cos(7.0 * y / H)
    depth[0, H // 2, W // 3] = 0.0                       # holes: the normals that use them are invalid
    depth[-1, H // 3, W // 2] = np.nan
    prior = rng.normal(size=(V, 3, H, W))
    prior[:, 2] = -np.abs(prior[:, 2]) - 0.5             # facing the camera
    prior /= np.linalg.norm(prior, axis=1, keepdims=True)
    intr = np.array([[rng.uniform(0.4, 0.6) * W, rng.uniform(0.4, 0.6) * W, rng.uniform(0.45, 0.55) * W,
                      rng.uniform(0.45, 0.55) * H] for _ in range(V)])
    cams = np.zeros((V, 16), np.float32)
    cams[:, 0] = cams[:, 4] = cams[:, 8] = 1.0
    cams[:, 12:16] = intr
    return depth.astype(np.float32), prior.astype(np.float32), intr.astype(np.float32).astype(np.float64), cams


@pytest.mark.parametrize("V,H,W", [(2, 37, 53), (2, 21, 122), (3, 9, 33), (1, 2, 3), (1, 680, 1200)])
def test_normal_loss_matches_oracle(R, V, H, W):
    rng = np.random.default_rng(V * H + W)
    depth, prior, intr, cams = _normal_case(rng, V, H, W)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    off = 2.0 ** -10                                     # the call adds to d_depth and loss
    d_depth = torch.full((V, H, W), off, dtype=torch.float32, device="cuda")
    loss = torch.full((1,), 0.75, dtype=torch.float64, device="cuda")
    R.loss_normal(t(depth), t(prior), t(cams), 0.5, d_depth, loss)
    torch.cuda.synchronize()
    ref_l, ref_g = OL.normal_loss(depth, prior, intr, weight=0.5)
    assert abs((loss.item() - 0.75) - ref_l) <= 1e-4 * abs(ref_l)
    g = d_depth.cpu().numpy().astype(np.float64) - off
    assert rel_l2(g, ref_g) <= 1e-3
    assert np.all(g[ref_g == 0.0] == 0.0)                # no gradient where no valid normal reads the depth
