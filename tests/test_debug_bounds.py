"""The bounds-checked debug build (libvedt_debug.so, -DVEDT_DEBUG_BOUNDS): the EDT parity,
batched-EDT, incremental and band-junction tests run again in a child process that loads it.  Every index
the EDT passes compute is checked against its buffer there; an out-of-range one would set
the error word, which every test reads through vedt_check, so the run passing shows that
no pass computed a bad index on these inputs (and the fields still match the oracle)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_parity_suites_pass_on_the_index_checked_build():
    from paper_2407_02363_b300 import build
    build.build(debug=True)
    env = dict(os.environ, VEDT_DEBUG_BOUNDS="1")
    probe = subprocess.run([sys.executable, "-c", "from paper_2407_02363_b300 import vedt; print(vedt.version())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr
    assert "index checks" in probe.stdout
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_parity_edt.py"), os.path.join(HERE, "test_batch.py"),
                        os.path.join(HERE, "test_incremental.py"), os.path.join(HERE, "test_junctions.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
