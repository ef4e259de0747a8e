"""The device memory cache's policy (csrc/devmem.h), checked on the host with
a fake backend: reuse of released blocks of about the requested size, best
fit, the byte limit with least-recently-released eviction, the retry after a
failed allocation, foreign pointers, and concurrent use (tests/devmem_check.cpp).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_cache_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "devmem_check"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-pthread", "-Wall", "-Werror",
                           "-I", os.path.join(ROOT, "paper_2004_11040_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "devmem_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 30
