"""The bounds-checking build (libfrkc2_debug.so, -DFRKC2_DEBUG_BOUNDS): every global index of
the main pass kernels -- the 2D streaming pass, the wavefront pass's row copies and stores,
the register regions, the shared-memory tiles, the 3D z-streaming pass and the 1D cluster
kernel -- is checked against its array before the access.  On ragged grids of both boundary
kinds, and on grids of one or two cells along an axis, no check fires (no EBOUNDS latched) and
every result still matches the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checking_build_parity():
    from paper_1702_03818_gb300 import build as B

    lib = os.path.join(ROOT, "paper_1702_03818_gb300", "_lib", "libfrkc2_debug.so")
    if not os.path.exists(lib):
        B.build(debug=True)
    env = dict(os.environ, FRKC2_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    cases = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(cases) == 12 + 7 * 2 * 2 + 2
    for c in cases:
        assert c["status"] == 0, c  # 9 would be FRKC2_EBOUNDS
        assert c["err"] < c["tol"], c
