"""Host symbolic pass of the CUDA library (C++), checked on the CPU.

Compiles tests/host/symbolic_check.cpp against csrc/symbolic.cpp: every
position the kernels dereference (frontal lists, merge maps, face / edge row
maps) must point at the DOF it claims, and the front counts must match the
closed forms of §2.1 (c^3 cells, 3(c-1)c^2 faces, 3(c-1)^2 c edges).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("sym") / "symcheck")
    src = os.path.join(ROOT, "paper_1607_00346_gb300", "csrc")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", src,
                    os.path.join(ROOT, "tests", "host", "symbolic_check.cpp"),
                    os.path.join(src, "symbolic.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("n,m", [(8, 4), (16, 4), (12, 3), (20, 5), (24, 3), (32, 4), (64, 4)])
def test_symbolic_consistent(checker, n, m):
    p = subprocess.run([checker, str(n), str(m)], stdout=subprocess.PIPE, text=True)
    assert p.returncode == 0, p.stdout
    assert p.stdout.strip().endswith("OK")
    root = [l for l in p.stdout.splitlines() if "root" in l][0]
    assert int(root.split(":")[1].split()[0]) == n ** 3 - (n - 1) ** 3


@pytest.mark.parametrize("n,m", [(8, 4), (16, 4), (12, 3), (20, 5), (32, 4)])
def test_symbolic_consistent_periodic(checker, n, m):
    # periodic grid: wrapping closures, c^3 / 3c^3 / 3c^3 fronts per level, and
    # at eps = 0 the root keeps the last level's separator planes, 0 and n/2
    p = subprocess.run([checker, str(n), str(m), "p"], stdout=subprocess.PIPE, text=True)
    assert p.returncode == 0, p.stdout
    assert p.stdout.strip().endswith("OK")
    root = [l for l in p.stdout.splitlines() if "root" in l][0]
    assert int(root.split(":")[1].split()[0]) == n ** 3 - (n - 2) ** 3
