"""The bounds-checked build (PFAC_CHECKED) over the small-case suites.

compute-sanitizer is not available here, so the library has a second build
in which the compressed-layout kernels range-check every table, shared-
memory, queue and input index (an index out of range is replaced by 0 and
the call reports PFAC_EDEVICE).  This test builds it (libpfac_checked.so),
then runs the small-case parity suites in a child process that loads it
instead of the regular library: every call must give the oracle's keys and
report no out-of-range index."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_suites_under_the_checked_build():
    sys.path.insert(0, os.path.join(ROOT, "paper_1704_02272_gb300"))
    import build as pfac_build  # the build script, not the package
    lib = pfac_build.build(checked=True)
    assert lib.endswith("libpfac_checked.so") and os.path.exists(lib)
    env = dict(os.environ, PFAC_LIB=lib)
    probe = subprocess.run(
        [sys.executable, "-c", "import paper_1704_02272_gb300 as p; print(p.binding.LIB_PATH)"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert probe.returncode == 0 and probe.stdout.strip() == lib, probe.stdout + probe.stderr
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
         "tests/test_gpu_small.py", "tests/test_gpu_register.py", "tests/test_gpu_prefix.py",
         "tests/test_gpu_suffix_merge.py", "tests/test_gpu_records.py",
         "-k", "not full_size"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout, r.stdout[-2000:]
