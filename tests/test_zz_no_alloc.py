"""gs_loss_l1_ssim_noalloc: the fused L1 + SSIM loss for callers that cannot allocate device memory
(a front-end with a fixed device-memory budget, or a host program whose allocator belongs to
another component).  It keeps its scratch in a static device array inside libgs instead of a
buffer the caller allocates.

Checked here through the C ABI against gs_loss_l1_ssim (which takes a caller-allocated scratch
buffer) on two calls in a row with different inputs and sizes, so that whatever the first call
leaves in the shared static area cannot leak into the second.  Kept in a file of its own that
pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_10760_gb300 import _lib as L  # noqa: E402
from paper_2605_10760_gb300 import scenes as S  # noqa: E402


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _inputs(V, H, W, seed):
    rng = np.random.default_rng(seed)
    y = np.stack([S.smooth_image(W, H, seed + v) for v in range(V)])
    x = np.clip(y + rng.normal(0, 0.05, y.shape), 0, 1).astype(np.float32)
    return torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()


def _with_scratch(lib, x, y):
    V, _, H, W = x.shape
    scratch = torch.empty(int(lib.gs_ssim_scratch_size(V, W, H)), dtype=torch.uint8, device="cuda")
    d = torch.empty_like(x)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.gs_loss_l1_ssim(V, W, H, _p(x), _p(y), 0.8, 0.2, _p(d), _p(loss), _p(scratch), _stream()) == 0
    return loss, d


def _noalloc(lib, x, y):
    V, _, H, W = x.shape
    d = torch.empty_like(x)
    loss = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")   # overwritten by the call
    assert lib.gs_loss_l1_ssim_noalloc(V, W, H, _p(x), _p(y), 0.8, 0.2, _p(d), _p(loss), _stream()) == 0
    return loss, d


def test_noalloc_ssim_matches_scratch_version_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = L.load()
    cases = [(2, 70, 97, 11), (1, 680, 1200, 12)]
    results = []
    for V, H, W, seed in cases:                     # two calls in a row, different inputs and sizes
        x, y = _inputs(V, H, W, seed)
        results.append((_with_scratch(lib, x, y), _noalloc(lib, x, y)))
    torch.cuda.synchronize()
    for (ref_loss, ref_d), (loss, d) in results:
        assert abs(loss.item() - ref_loss.item()) <= 1e-5 * abs(ref_loss.item())
        assert rel_l2(d.cpu().numpy(), ref_d.cpu().numpy()) <= 1e-4


def test_noalloc_ssim_rejects_planes_beyond_the_static_limit():
    lib = L.load()
    big = L.GS_SSIM_NOALLOC_MAX_PLANE + 1
    dummy = C.c_void_p(256)
    assert lib.gs_loss_l1_ssim_noalloc(1, big, 1, dummy, dummy, 0.8, 0.2, dummy, dummy, None) == L.GS_ERR_TOO_LARGE
    assert lib.gs_loss_l1_ssim_noalloc(1, 2048, 1024, dummy, dummy, 0.8, 0.2, dummy, dummy, None) == \
        L.GS_ERR_TOO_LARGE
