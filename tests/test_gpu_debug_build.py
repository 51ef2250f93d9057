"""GPU: the debug build of the library (compiled with -DQSLAB_DEBUG: the
sort, gather, chunk-table, k-space, k = 0 and combine kernels check their
indices against the arrays and set a status bit instead of accessing out of
range). The small and ragged cases of tests/debug_build_cases.py run through
it in a child process: no check may fire, and the FP64 results equal the
oracle's."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_small_cases():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01521_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, QSLAB_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "DEBUG-CASES OK" in r.stdout
