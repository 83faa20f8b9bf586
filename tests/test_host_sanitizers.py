"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

- The set-up code (`csrc/usr_setup.cpp`: series terms, the pair kernel's fit, periodised kernels, tile tables,
  the multilevel split) is built with g++ -fsanitize=address,undefined,float-cast-overflow beside a small driver
  that plans 8,640 parameter sets (valid and invalid) and 1,920 sets of extreme and out-of-range values, and the
  driver must finish without a report.  For every valid plan of the first sweep the driver also checks, exactly in
  single precision, that the spreading stencil of every wrapped coordinate fits the shared-memory tile of its
  block of cells (the spreading kernel's tile-base check then never fires).
- The oracle's C code is rebuilt with the same sanitizers (ORACLE_SANITIZE=1) and its pins run against it in a
  child process with the sanitizer runtimes preloaded.
Skipped where the compiler has no sanitizer runtimes.
"""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_01377_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g", "-O1"]
# float-to-int conversions out of range are not part of -fsanitize=undefined in GCC: the set-up code gets them too
SAN_SETUP = SAN + ["-fsanitize=float-cast-overflow", "-fno-sanitize-recover=float-cast-overflow"]


def _runtime(name):
    if shutil.which("g++") is None:
        return None
    p = subprocess.run(["g++", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


needs_san = pytest.mark.skipif(_runtime("libasan.so") is None or not os.path.isdir(CUDA_INC),
                               reason="no sanitizer runtimes or CUDA headers")


@needs_san
def test_setup_code_under_sanitizers():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "plan_driver")
        cmd = ["g++", "-std=c++17", "-ffp-contract=off"] + SAN_SETUP + ["-I", CUDA_INC, "-I", CSRC,
                                             os.path.join(ROOT, "tests", "host_sanitize", "plan_driver.cpp"),
                                             os.path.join(CSRC, "usr_setup.cpp"), "-o", exe]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600,
                           env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1"))
        assert r.returncode == 0, r.stderr[-4000:]
        assert "plans ok" in r.stdout and "tile violations 0" in r.stdout and "runtime error" not in r.stderr


@needs_san
def test_oracle_pins_under_sanitizers():
    pre = " ".join(p for p in (_runtime("libasan.so"), _runtime("libubsan.so")) if p)
    env = dict(os.environ, ORACLE_SANITIZE="1", ASAN_OPTIONS="detect_leaks=0", LD_PRELOAD=pre)
    tests = sorted(f for f in os.listdir(os.path.join(ROOT, "tests")) if f.startswith("test_oracle_"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"]
                       + [os.path.join("tests", f) for f in tests],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr
