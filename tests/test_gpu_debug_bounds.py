"""The bounds-checked build (libcrsolve_debug.so, CRSOLVE_DEBUG_BOUNDS): the
stated substitute for a memory checker, which this GPU pool does not offer.
Every global-memory index of the level kernels is checked against the
extents that the level sizes imply; an out-of-range index is recorded in the
plan's (or batch's) debug word and skipped.  The parity suite's small cases
(plain, breakdown, keep-levels, host buffers, mixed precision, Algorithm 1,
batched, the tensor-core residual) run on that build in a child process
(the library is chosen when it is loaded) and must match the oracle with
every record empty."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_small_cases_on_the_bounds_checked_build(cuda_ok):
    from paper_1807_00370_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, CRSOLVE_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "cases ok" in r.stdout, r.stdout[-2000:]
