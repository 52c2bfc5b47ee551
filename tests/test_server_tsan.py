"""The serving loop's host concurrency under ThreadSanitizer (no GPU needed):
the server source is built instrumented and linked with the library's other
objects into tests/native/server_tsan.cpp, which submits, waits, polls and
races two takers for one result from several threads while another reads
the statistics, then destroys the server with requests still queued."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_server_threads_under_tsan(tmp_path):
    from paper_1706_03791_gb300 import build as B
    B.build()
    objs = [os.path.join(B.BUILD, os.path.splitext(s)[0] + ".o") for s in B.SOURCES if s != "szgb_server.cu"]
    if not all(os.path.exists(o) for o in objs):
        B.build(force=True)
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(B.nvcc())), "lib64")
    srv_o, drv_o, exe = (str(tmp_path / n) for n in ("server_tsan.o", "driver_tsan.o", "server_tsan"))
    steps = [
        [B.nvcc(), *B.ARCH, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-fsanitize=thread",
         "-c", os.path.join(B.CSRC, "szgb_server.cu"), "-o", srv_o],
        [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-c", os.path.join(HERE, "native", "server_tsan.cpp"),
         "-o", drv_o],
        [gxx, "-fsanitize=thread", "-o", exe, drv_o, srv_o, *objs, "-L" + cuda_lib, "-lcudart", "-lpthread"],
    ]
    for cmd in steps:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            if "tsan" in r.stderr or "sanitize" in r.stderr:
                pytest.skip("ThreadSanitizer unavailable: " + r.stderr.strip().splitlines()[-1])
            raise RuntimeError(r.stderr)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1:exitcode=66")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "failures 0" in r.stdout
