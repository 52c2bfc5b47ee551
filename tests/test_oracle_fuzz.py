"""Robustness of the oracle's stream reader under AddressSanitizer and
UndefinedBehaviorSanitizer: corrupted and truncated streams of the exact
method (1D..4D) and of the lattice variant either decode within the declared
shape or return an error code, with no invalid access and no undefined
behaviour (the driver is tests/native/oracle_fuzz.c)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def fuzz_bin(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    out = str(tmp_path_factory.mktemp("fuzz") / "oracle_fuzz")
    cmd = [gcc, "-std=c11", "-O1", "-g", "-ffp-contract=off", "-fno-fast-math",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-o", out, os.path.join(ROOT, "oracle", "szo.c"), os.path.join(HERE, "native", "oracle_fuzz.c"), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "sanitize" in (r.stderr or "") or "asan" in (r.stderr or ""):
            pytest.skip("sanitizer runtime unavailable: " + r.stderr.strip().splitlines()[-1])
        raise RuntimeError(r.stderr)
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_corrupt_streams_are_safe(fuzz_bin, seed):
    r = subprocess.run([fuzz_bin, str(seed), "120"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "decoded" in r.stdout
