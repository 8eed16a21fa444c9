"""The bounds-check build (libpacksell_checks.so, -DPACKSELL_CHECKS): run in
a child process with PACKSELL_CHECKS=1 (the library a process loads is fixed
at its first call). Valid matrices give the regular products and no skips;
a word rewritten to decode one past the end of x is skipped and reported as
PACKSELL_ERR_CHECK by every checked product (tests/_checks_run.py)."""
import os
import subprocess
import sys

import pytest

from _gpu import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checks_build_skips_and_reports_out_of_range_columns():
    need_gpu()
    env = dict(os.environ, PACKSELL_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checks_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checks ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]


def test_regular_build_is_not_the_checks_build():
    need_gpu()
    from paper_2604_13433_gb300 import packsell as ps
    if os.environ.get("PACKSELL_CHECKS") == "1":
        pytest.skip("this process runs the checks build")
    assert ps.lib().packsell_checks_build() == 0
