"""The Python binding's ctypes structs mirror include/szgb.h exactly: size
and offset of every field, as a C compiler lays them out
(tests/native/abi_layout.c)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_struct_layouts_match(tmp_path):
    from paper_1706_03791_gb300 import build
    build.build()
    from paper_1706_03791_gb300 import szgb
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "abi_layout")
    r = subprocess.run([gcc, "-std=c11", "-o", exe, os.path.join(HERE, "native", "abi_layout.c")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([exe], capture_output=True, text=True).stdout.splitlines())
    py = {"szgb_params": szgb.Params, "szgb_stats": szgb.Stats, "szgb_quality": szgb.Quality,
          "szgb_request": szgb.Request}
    names = {"in": "in_"}
    for key, val in got.items():
        s, f = key.split(".")
        cls = py[s]
        if f == "sizeof":
            assert C.sizeof(cls) == int(val), key
        else:
            assert getattr(cls, names.get(f, f)).offset == int(val), key
