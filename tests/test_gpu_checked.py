"""The checked build (kernels check every index they compute against the sizes of their
buffers and record the first failure instead of touching memory; the entry points return
BANG_E_BOUNDS) stands in for compute-sanitizer, which is not available here: the whole GPU
suite runs against it and must pass, i.e. no kernel index left its buffer in any tested
configuration.  The recording path itself is exercised by a device-side check that fails
without any access."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checked_env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import build as b
    b.build(checked=True)
    return dict(os.environ, BANG_CHECKED="1")


def run_py(code, env):
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_selftest_records_and_clears(checked_env):
    code = (
        "from paper_2205_06819_gb300 import _lib\n"
        "L = _lib.lib()\n"
        "assert L.bang_checked_build() == 1\n"
        "assert L.bang_check_selftest(0, 2, 3) == 0\n"
        "assert L.bang_check_selftest(0, 3, 3) == 6, L.bang_last_error()\n"
        "msg = L.bang_last_error().decode()\n"
        "assert 'selftest' in msg and 'index 3' in msg and '[0, 3)' in msg, msg\n"
        "assert L.bang_check_selftest(0, -1, 3) == 6\n"
        "assert L.bang_check_selftest(0, 0, 3) == 0   # the record was cleared\n"
        "print('ok')\n")
    r = run_py(code, checked_env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_normal_build_has_no_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import _lib
    L = _lib.lib()
    assert L.bang_checked_build() == 0
    assert L.bang_check_selftest(0, 3, 3) == 4   # BANG_E_UNSUPPORTED


def test_gpu_suite_passes_under_the_checked_build(checked_env):
    files = sorted(os.path.join(HERE, f) for f in os.listdir(HERE)
                   if f.startswith("test_") and f.endswith(".py") and f != os.path.basename(__file__))
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=checked_env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
