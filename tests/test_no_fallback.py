"""The product path has no CPU fallback: without libgs, or without a CUDA device, its calls raise
instead of computing anything on the host."""
import numpy as np
import pytest
import torch

from paper_2605_10760_gb300 import _lib as L


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "lib_path", lambda: str(tmp_path / "absent" / "libgs.so"))
    with pytest.raises(ImportError):
        L.load(build_if_missing=False)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_problem_without_cuda_device_raises():
    from paper_2605_10760_gb300 import raster as R
    with pytest.raises((RuntimeError, AssertionError), match="(?i)nvidia|cuda"):
        R.Problem(np.array([0]), np.array([16]), 16, 32, 32)
