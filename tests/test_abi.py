"""The C-ABI library loads and exports every entry point that include/*.h
declares; host-side argument checks run without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_1807_00370_gb300 import _native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|const char \*|void)\s*\*?\s*(crsolve_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["crsolve_factor", "crsolve_solve", "crsolve_backward", "crsolve_info_get",
              "crsolve_plan_create", "crsolve_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = nat.load()
    for n in sorted(_declared()):
        assert hasattr(lib, n), n
        assert n in nat.SIGNATURES, f"binding lacks {n}"


def test_library_is_built_for_sm_103a_only():
    from paper_1807_00370_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _create(N, m, k, prec=0, flags=0):
    h = ctypes.c_void_p()
    rc = nat.load().crsolve_plan_create(N, m, k, prec, flags, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("N,m,k,prec,flags,code", [
    (0, 4, 1, 0, 0, nat.CRSOLVE_EINVAL),
    (8, 0, 1, 0, 0, nat.CRSOLVE_EINVAL),
    (8, 4, 0, 0, 0, nat.CRSOLVE_EINVAL),
    (8, 65, 1, 0, 0, nat.CRSOLVE_EUNSUPPORTED),
    (8, 4, 5000, 0, 0, nat.CRSOLVE_EUNSUPPORTED),
    (8, 4, 1, 7, 0, nat.CRSOLVE_EUNSUPPORTED),
    (8, 4, 1, 0, 8, nat.CRSOLVE_EINVAL),
    # Algorithm 1 needs N a power of two and FP64
    (6, 4, 1, 0, nat.CRSOLVE_PLAN_ALG1, nat.CRSOLVE_EUNSUPPORTED),
    (8, 4, 1, nat.CRSOLVE_MIXED, nat.CRSOLVE_PLAN_ALG1, nat.CRSOLVE_EUNSUPPORTED),
])
def test_plan_argument_errors_are_host_side(N, m, k, prec, flags, code):
    rc, h = _create(N, m, k, prec, flags)
    assert rc == code
    assert not h.value


def test_null_plan_is_rejected():
    lib = nat.load()
    assert lib.crsolve_factor(None, None, None, None) == nat.CRSOLVE_EINVAL
    assert lib.crsolve_solve(None, 1, None, None, None) == nat.CRSOLVE_EINVAL
    assert lib.crsolve_backward(None, 1, None, None, None, None, None, None) == nat.CRSOLVE_EINVAL
    assert lib.crsolve_info_get(None, None, None) == nat.CRSOLVE_EINVAL
    assert lib.crsolve_workspace_bytes(None, None) == nat.CRSOLVE_EINVAL
    assert nat.strerror(nat.CRSOLVE_NOT_PD).startswith("matrix is not positive definite")


def test_peak_probe_rejects_bad_arguments_without_a_gpu():
    lib = nat.load()
    v = ctypes.c_double()
    assert lib.crsolve_peak_probe(7, ctypes.byref(v), None, None, None) == nat.CRSOLVE_EINVAL
    assert lib.crsolve_peak_probe(nat.CRSOLVE_PROBE_FP64_FMA, None, None, None, None) == nat.CRSOLVE_EINVAL
