"""The bounds-checked build (the same sources with SPGEMM_CHECK: the kernels check the indices
of their result writes and shared-memory scatters, record a site code in a device status word
and skip the access, with no trap).  Every kernel path runs on small cases in a process of its
own that loads that build; each C must equal the oracle's and no check may have fired."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_every_path_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, SPGEMM_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all clean" in r.stdout

