"""The checked build: the library compiled with -DHWENO_CHECKS=1, whose
kernels check their shared-memory and global indices (a failed check sets a
status bit, HWENO_EBOUNDS, with no trap) and whose stage scratch starts as
NaN, stands in for a memory checker. Every kernel family runs on tiny and
ragged grids (N = 4, 5, 31, 123-125, 248, 249; 2D grids of 13-40 points)
through it, in a subprocess that loads that build; the results must match
the oracle and no check may fail. A self-test confirms the checks are live."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_tiny_grids_under_the_checked_build():
    from paper_2207_05258_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, HWENO_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
