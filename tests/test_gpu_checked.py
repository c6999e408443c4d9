"""The bounds-check build (AR_CHECKED): every variant of every loop and one
executor batch run with every index check compiled in; no check may fire and
every result must still match the oracle.  The checks only observe: a
failing one records itself and skips its access, nothing faults."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_checked_build_runs_every_variant_without_a_failed_check():
    sys.path.insert(0, os.path.join(ROOT, "paper_2303_08873_b300"))
    import build

    build.build(checked=True)
    env = dict(os.environ, AR_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["enabled"] is True
    assert res["failures"] == 0, f"check at source {res['first_failure'] >> 16} line {res['first_failure'] & 0xffff}"
    assert res["bad"] == []
