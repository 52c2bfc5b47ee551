"""The hyperplane kernels' device code (3D n = 3, 4 and 4D n = 1..4), run
thread by thread on the host by tests/native/hyper_emulate.cpp, against the
oracle: codes, recorded values, reconstruction and the 4D adaptive m, bit for
bit.  No GPU needed; the GPU parity cases are in test_zy_gpu_hyper.py."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_hyperplane_kernels_emulated(tmp_path):
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if gcc is None or gxx is None:
        pytest.skip("no host compiler")
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math"]
    obj, exe = str(tmp_path / "szo.o"), str(tmp_path / "hyper_emulate")
    for cmd in ([gcc, "-std=c11", *flags, "-c", os.path.join(ROOT, "oracle", "szo.c"), "-o", obj],
                [gxx, "-std=c++17", *flags, "-Wno-unknown-pragmas", "-o", exe,
                 os.path.join(HERE, "native", "hyper_emulate.cpp"), obj, "-lm"]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "failures 0" in r.stdout, r.stdout + r.stderr
