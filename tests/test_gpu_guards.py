"""Guard words and the checked build.

Every hot-path family (single pulse, ragged batch, the bank on each
spectrum-apply form, exact sinc on tensor cores) runs with canary values
around its device outputs: nothing is written outside the output, and the
results match the FP64 oracle.  The same calls then run against the checked
build of the library (compiled with DC_CHECKED, loaded with DC_CHECKED=1 in a
subprocess), whose kernels check their shared-memory and scratch indices and
report a failed check through dc_check: it must run clean.
"""

import os
import subprocess
import sys

import pytest

from tests import _guarded_calls as gc

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dcg():
    import paper_2508_04951_gb300 as m
    m.build.build()
    m.load()
    return m


def test_guard_words_intact_and_results_match(dcg):
    res = gc.run_all(dcg)
    for name, e, tol in res:
        assert e <= tol, (name, e, tol)


def test_checked_build_runs_clean():
    env = dict(os.environ, DC_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "tests._guarded_calls"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "CHECKED OK" in r.stdout
