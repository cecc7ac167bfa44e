"""Host checks of the index arithmetic behind the box-mesh kernels (multiply-shift division,
E-vector layouts): `tests/host/index_math.cpp` built with the host compiler against the
library's internal header and run.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    return None


def test_index_math(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("host compiler or CUDA headers not found")
    exe = str(tmp_path / "index_math")
    src = os.path.join(HERE, "host", "index_math.cpp")
    r = subprocess.run([cxx, "-O2", "-std=c++17", f"-I{ROOT}/paper_1910_03032_b300/csrc", f"-I{ROOT}/include",
                        f"-I{inc}", src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-4000:]
