"""The C-ABI library loads and exports every entry point include/qs.h
declares; host-side argument validation and plan building (no GPU calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*(qs_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_16044_gb300 as qs
    return qs


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["qs_alloc", "qs_apply_1q", "qs_apply_diag", "qs_apply_controlled", "qs_apply_fused",
                 "qs_permute_qubits", "qs_expect_pauli", "qs_run_plan"]:
        assert must in names


def test_library_exports_every_declared_symbol(qs):
    lib = ctypes.CDLL(qs.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", qs.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (qs_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported
    # the binding wraps every declared entry point
    assert set(declared_functions()) <= set(qs.EXPORTED)


def test_null_and_range_checks_without_gpu(qs):
    L = qs.lib()
    U = (ctypes.c_double * 8)(1, 0, 0, 0, 0, 0, 1, 0)
    assert L.qs_apply_1q(None, 0, U) == qs.QS_EINVAL
    assert "NULL" in L.qs_last_error().decode()
    h = ctypes.c_void_p()
    assert L.qs_alloc(0, qs.C128, ctypes.byref(h)) == qs.QS_EINVAL
    assert L.qs_alloc(35, qs.C128, ctypes.byref(h)) == qs.QS_EINVAL
    assert L.qs_alloc(10, 7, ctypes.byref(h)) == qs.QS_EINVAL
    assert L.qs_wrap(10, qs.C128, ctypes.c_void_p(8), ctypes.byref(h)) == qs.QS_EINVAL  # misaligned
    assert L.qs_free(None) == qs.QS_OK
    # measurement entry points check their arguments before touching a device
    qv = (ctypes.c_int * 1)(0)
    out = (ctypes.c_double * 2)()
    o = ctypes.c_int()
    assert L.qs_probabilities(None, qv, 1, out) == qs.QS_EINVAL
    assert L.qs_measure(None, 0, 0.5, ctypes.byref(o), out) == qs.QS_EINVAL
    uu = (ctypes.c_double * 1)(0.5)
    res = (ctypes.c_uint64 * 1)()
    assert L.qs_sample(None, 1, uu, res) == qs.QS_EINVAL
    assert L.qs_plan_step_qubits(None, 0, qv, 1, ctypes.byref(o)) == qs.QS_EINVAL


def test_circuit_and_plan_host_logic(qs):
    import workloads as W
    c = qs.Circuit(W.brick(12, 20, 1))
    assert len(c) == 350
    p = qs.Plan(c, 12, "c128", mode=qs.PLAN_UNFUSED)
    s = p.stats()
    assert s["gates"] == 350 and s["passes"] == 350
    N, S = 1 << 12, 16
    assert s["metric_bytes"] == 2 * N * S * 350
    # U3: full pass; CNOT: half the amplitudes (one control)
    assert s["hbm_bytes"] == 240 * 2 * N * S + 110 * N * S
    # QFT: H full, CP touches a quarter, SWAP moves half
    q = qs.Plan(qs.Circuit(W.qft(12)), 12, "c64", mode=qs.PLAN_UNFUSED).stats()
    assert q["hbm_bytes"] == 12 * 2 * N * 8 + 66 * 2 * N * 8 / 4 + 6 * N * 8
    with pytest.raises(qs.QSError):
        qs.Plan(c, 11, "c128", mode=qs.PLAN_UNFUSED)  # gate on qubit 11 >= n
    with pytest.raises(qs.QSError):
        c.add("CNOT", [3, 3])
    with pytest.raises(qs.QSError):
        c.add("U3", [1], [0.1, 0.2, 0.3], param_index=0)  # only RX/RY/RZ trainable


def test_circuit_add_many_matches_single_adds(qs):
    # host-only: the bulk call and the per-gate call build the same circuit,
    # and a bad gate is rejected with its index, the gates before it kept
    import ctypes
    L = qs.lib()
    gates = W.brick(6, 3, 2) + W.qft(6)
    a, b = qs.Circuit(), qs.Circuit()
    for g in gates:
        a.add(g.name, g.qubits, g.params)
    b.add_many(gates)
    assert len(a) == len(b) == len(gates)
    kinds = np.array([qs.GATE_KIND["H"], qs.GATE_KIND["CNOT"], qs.GATE_KIND["RX"]], dtype=np.int32)
    qubits = np.array([[0, 0], [1, 1], [2, 0]], dtype=np.int32)  # the CNOT's qubits coincide
    params = np.zeros((3, 3))
    c = qs.Circuit()
    st = L.qs_circuit_add_many(c.handle, 3, kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               qubits.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               params.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert st == qs.QS_EINVAL
    assert b"gate 1" in L.qs_last_error()
    assert len(c) == 1


def test_plan_step_qubits(qs):
    # host-only: an unfused plan's steps are the circuit's gates in order
    # (controls first); a fused plan's blocks cover at most 6 distinct qubits
    # in range, and together with its gate steps every qubit the circuit uses
    gates = W.brick(5, 3, 1) + W.qft(4)
    p = qs.Plan(qs.Circuit(gates), 5, "c128", mode=qs.PLAN_UNFUSED)
    assert p.stats()["passes"] == len(gates)
    for i, g in enumerate(gates):
        assert p.step_qubits(i) == list(g.qubits)
    n = 14
    p = qs.Plan(qs.Circuit(W.brick(n, 12, 3)), n, "c64", mode=qs.PLAN_FUSED, fuse_qubits=6)
    seen = set()
    for i, (kind, _) in enumerate(p.step_info()):
        q = p.step_qubits(i)
        assert len(set(q)) == len(q) and all(0 <= x < n for x in q)
        if kind == "block":
            assert 1 <= len(q) <= 6
        seen.update(q)
    assert seen == set(range(n))
    with pytest.raises(qs.QSError):
        p.step_qubits(p.stats()["passes"])


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 (no torch or
    # C++ types) and as C++
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "include/qs.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-c", str(src), "-I", ROOT, "-o",
                        str(tmp_path / "h.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx:
        src2 = tmp_path / "h.cpp"
        src2.write_text('#include "include/qs.h"\nint main() { return 0; }\n')
        r = subprocess.run([cxx, "-std=c++11", "-Wall", "-Werror", "-c", str(src2), "-I", ROOT, "-o",
                            str(tmp_path / "h2.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_c_program_links_against_the_library(qs, tmp_path):
    # a plain C caller (tests/c/abi_example.c) compiles against the header and
    # links against libqs.so; running it needs a GPU
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(qs.LIB_PATH)
    exe = tmp_path / "abi_example"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", os.path.join(ROOT, "tests", "c", "abi_example.c"),
                        "-I", ROOT, "-L", libdir, "-lqs", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert exe.exists()
