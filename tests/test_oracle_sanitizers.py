"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a driver
(tests/sanitize_oracle_main.c) calls every oracle entry point on small, ragged, empty and
full grids and on points and spheres outside the grid; any invalid access, leak or
undefined operation aborts it, and an EDT that differs from the brute-force definition
makes it fail."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "sanitized_oracle")
    cmd = [gcc, "-O1", "-g", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-o", exe,
           os.path.join(HERE, "sanitize_oracle_main.c"), os.path.join(ROOT, "oracle", "edt_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "sanitized oracle run ok" in r.stdout
