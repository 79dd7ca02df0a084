"""A plain C program (tests/c_client/crsolve_c_client.c) linked against
libcrsolve.so drives the C ABI without Python or torch: caller-allocated
workspace, factor, solve, error codes, the host-buffer solve (bit-identical
to the device path) and breakdown reporting.  Its own check is the residual
of the block-tridiagonal system, computed on the host."""
import os
import subprocess

import pytest

from paper_1807_00370_gb300 import build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def client(tmp_path_factory, cuda_ok):
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("c_client") / "crsolve_c_client")
    libdir = os.path.dirname(lib)
    subprocess.run([build._nvcc(), "-O2", "-I", build.INCLUDE, os.path.join(HERE, "c_client", "crsolve_c_client.c"),
                    "-o", exe, "-L", libdir, "-lcrsolve", "-Xlinker", f"-rpath={libdir}"], check=True)
    return exe


@pytest.mark.parametrize("N,m,k", [(1000, 8, 3), (2, 5, 1), (4097, 16, 2)])
def test_c_client(client, N, m, k):
    out = subprocess.run([client, str(N), str(m), str(k)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "ok" in out.stdout
