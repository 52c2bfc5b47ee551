"""The hyperplane enumeration of the 3D kernels for n >= 3 layers
(paper_1706_03791_gb300/csrc/hyper_box.h), checked on the host over 729
shapes by tests/native/hyper_box_test.cpp: every point visited exactly once,
boxes inside the field, no empty hyperplane."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_hyperplane_boxes(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "hyper_box_test")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-o", exe,
                        os.path.join(HERE, "native", "hyper_box_test.cpp")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "failures 0" in r.stdout, r.stdout + r.stderr
