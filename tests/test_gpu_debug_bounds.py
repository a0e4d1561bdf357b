"""The bounds-checked build of the library (-DCQR_DEBUG_BOUNDS; needs a GB300): the stand-in
for a memory checker.  Every kernel of the hot path checks that the indices it is about to
use lie inside the extents it was given, records CQR_EBOUNDS with a site number when one does
not, and returns without the access (it never traps).  On small odd shapes through every path
no check may fire and the factors must match the oracle; the self-test's guarded write past a
four-element array must be caught (site 199) and its record cleared by the read."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_index_checks_hold_and_the_planted_one_fires():
    from paper_2311_11943_gb300 import binding as B
    from paper_2311_11943_gb300 import build
    build.build(debug_bounds=True)
    # a child process, so that the binding loads the bounds-checked library
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_bounds_child.py")],
                       capture_output=True, text=True, timeout=900, cwd=ROOT,
                       env=dict(os.environ, CQR_LIBRARY="debug"))
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    for c in out["cases"]:
        assert c["status"] == 0 and c["bounds"] == 0 and c["site"] == 0, c
        assert c["err"] < c["tol"], c
    assert out["selftest"] == [B.CQR_EBOUNDS, 199]
    assert out["after"] == [0, 0]
    # the normal build has no checks and says so
    assert B.debug_bounds() == (B.CQR_ENOTSUP, 0)
