"""Host check of the tcgen05 kernel's pair walk (csrc/walk.h), no GPU.

walk_check.cpp compiles the walk for the host and checks, for slice counts
1..64, 191 and 239, accumulator limits of 1 to 2^20 pairs and work items of
1 to 7 pair-range chunks, that both orders visit every pair of the triangle
t + u <= s + 1 (Sec. 3, Algorithm 1) exactly once and form valid groups
(one diagonal, at most ppd pairs, one accumulator, closed within the item),
and that in the snake consecutive pairs share an operand slice and no
accumulator is reused before one pair of the other has run.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pair_walk_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "walk_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-Wall", "-Werror", "-o", exe, os.path.join(HERE, "walk_check.cpp")],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok "), r.stdout
    assert int(r.stdout.split()[1]) > 30000
