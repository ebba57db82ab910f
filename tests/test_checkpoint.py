"""Checkpoint / resume of Gaussian parameters and Adam state (host logic, CPU tensors)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_10760_gb300 import raster as R  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


def test_checkpoint_round_trip(tmp_path):
    sc = S.random_cloud(257, seed=5)
    g = R.Gaussians.from_scene(sc, device="cpu")
    adam = R.AdamState(g, lr=(1e-4, 2e-3, 3e-3, 4e-2, 5e-3))
    gen = torch.Generator().manual_seed(0)
    adam.m.copy_(torch.randn(adam.m.shape, generator=gen))
    adam.v.copy_(torch.rand(adam.v.shape, generator=gen))
    adam.step.fill_(17)
    path = tmp_path / "ckpt.pt"
    R.save_checkpoint(path, g, adam, extra={"pose": torch.arange(12.0).view(2, 6), "iteration": 17})
    g2, adam2, extra = R.load_checkpoint(path, device="cpu")
    for k in ("means", "log_scales", "quats", "opacities", "colors"):
        assert torch.equal(getattr(g, k), getattr(g2, k))
    for k in ("logits", "m", "v", "step"):
        assert torch.equal(getattr(adam, k), getattr(adam2, k))
    np.testing.assert_allclose(list(adam2.lr), list(adam.lr))
    assert adam2.g is g2 and extra["iteration"] == 17 and torch.equal(extra["pose"], torch.arange(12.0).view(2, 6))


def test_checkpoint_without_optimizer(tmp_path):
    g = R.Gaussians.from_scene(S.random_cloud(10, seed=6), device="cpu")
    path = tmp_path / "g.pt"
    R.save_checkpoint(path, g)
    g2, adam2, extra = R.load_checkpoint(path, device="cpu")
    assert adam2 is None and extra == {} and torch.equal(g.means, g2.means)
