"""GPU: the C ABI from a plain C program (tests/c_abi_ring.c), compiled against
include/gbx.h and linked with libgbx.so: a ring exchange in both forms and its backward give
the expected values, a start on an active request is refused, and every handle frees."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller_ring_exchange():
    import __graft_entry__
    __graft_entry__.build()
    libdir = os.path.join(ROOT, "paper_2309_07337_gb300")
    exe = os.path.join(ROOT, "_build", "c_abi_ring")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    from paper_2309_07337_gb300 import build
    subprocess.run([build.nvcc(), "-O2", "-o", exe, os.path.join(ROOT, "tests", "c_abi_ring.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lgbx", "-Xlinker", "-rpath=" + libdir],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "c_abi_ring ok" in r.stdout
