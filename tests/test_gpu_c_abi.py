"""The C ABI from a plain C caller on the GPU: tests/c/abi_example.c builds
a 20-qubit GHZ state (H, then a CNOT chain) and reads its norm, <Z0 Z1 + X0>
and four samples, all of which have closed forms (1, 1, and 0 for u < 1/2,
2^20 - 1 for u > 1/2)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller_ghz(tmp_path):
    import paper_2203_16044_gb300 as qs
    cc = shutil.which("gcc") or shutil.which("cc")
    assert cc, "a C compiler is needed"
    libdir = os.path.dirname(qs.LIB_PATH)
    exe = tmp_path / "abi_example"
    r = subprocess.run([cc, "-std=c99", os.path.join(ROOT, "tests", "c", "abi_example.c"), "-I", ROOT, "-L", libdir,
                        "-lqs", "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    f = r.stdout.split()
    assert f[0] == "status" and f[1] == "0"
    assert abs(float(f[3]) - 1.0) < 1e-12
    assert abs(float(f[5]) - 1.0) < 1e-12
    assert [int(v) for v in f[7:11]] == [0, 0, (1 << 20) - 1, (1 << 20) - 1]
