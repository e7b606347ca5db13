"""The parity cases of tests/debug_build_cases.py against the debug build of
the library (device index checks in every kernel, in place of a memory
checker), in a process of their own."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_index_checks_hold_on_parity_cases():
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")],
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "all cases match" in r.stdout
