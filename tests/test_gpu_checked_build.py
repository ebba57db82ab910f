"""The bounds-checked build of the library (libgs_checked.so: every index a kernel takes from data is
compared with its buffer's length first, and a violation is recorded as GS_ERR_DEVICE_FAULT instead
of being followed).  The parity suite's projection, binning, compositing, backward and edge-case
tests run against it in a child process; any recorded violation fails them through their status
checks, and every run also checks the workspace guard blocks."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(900)
def test_parity_suite_on_the_bounds_checked_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, GS_LIBGS_VARIANT="checked")
    sel = "variant or single_view or batched or other_tiles or background or capacity or edge_cases or longer"
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_parity.py"), "-m", "gpu",
                        "-q", "-x", "-p", "no:cacheprovider", "-k", sel], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=850)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and " failed" not in r.stdout
