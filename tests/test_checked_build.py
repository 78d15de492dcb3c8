"""The bounds-checked debug build (-DFRW_CHECKS; compute-sanitizer is not
available): the GPU parity, MicroWalk-E, serving and batched tests run against
libfrw_checked.so, whose kernels test every lattice coordinate, queue, list and
table index and record / batch / sum offset before use and report a failed test
as an error status.  They must pass unchanged (needs a GB300)."""
import os
import subprocess
import sys

import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


def test_gpu_suites_pass_on_the_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_mwe.py", "tests/test_serving.py", "tests/test_batched.py",
             "tests/test_gpu_ws.py"]
    env = dict(os.environ, FRW_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
