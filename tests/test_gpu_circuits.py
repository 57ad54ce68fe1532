"""GPU parity of whole circuits against the FP64 oracle.

 * 12-qubit brick random circuit (U3 layer + nearest-neighbour CNOT layer,
   the QSB shape of §IV-F), depth 20 and 40, and a 12-qubit QFT on a seeded
   basis state: complex128 element-wise max error <= 1e-12; complex64
   infidelity 1 - |<psi64|psi128>|^2 <= 1e-5 against the oracle's state, in
   both the stated and the normalised form, norm within 1e-6.
 * The paper's own synthetic circuits (QSB structure §IV-F, Hadamard
   benchmark §IV-D, the QV-shaped random two-qubit blocks of §IV-E) at
   small n.
 * Every plan mode gives the same state.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from fidelity import check_c64

pytestmark = pytest.mark.gpu

C128_TOL = 1e-12


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs
    return qs


def run_gpu(qs, n, circ, dtype, mode, x0=0):
    s = qs.State(n, dtype)
    s.set_basis(x0)
    stats = qs.run_circuit(s, circ, mode=mode)
    return s.to_numpy(), stats


def oracle_state(n, circ, x0=0):
    psi = oracle.zero_state(n, x0)
    oracle.run_circuit(psi, circ)
    return psi


CASES = [
    ("brick12_d20", 12, lambda: W.brick(12, 20, 1), 0),
    ("brick12_d40", 12, lambda: W.brick(12, 40, 1), 0),
    ("qft12", 12, lambda: W.qft(12), W.basis_index(12, 2)),
    ("brick9_d40", 9, lambda: W.brick(9, 40, 21), 0),
    ("qsb10", 10, lambda: W.qsb(10, 22), 0),
    ("hadamard11x7", 7, lambda: W.hadamard_bench(7), 5),
    ("qv13_d10", 13, lambda: W.qv_like(13, 10, 13), 0),
    ("qv14_d10", 14, lambda: W.qv_like(14, 10, 17), 0),
    ("ghz16", 16, lambda: W.ghz(16), 0),
    ("brick3", 3, lambda: W.brick(3, 10, 23), 0),
    ("brick1", 1, lambda: W.brick(1, 5, 24), 0),
]


@pytest.mark.parametrize("name,n,make,x0", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode,fuse", [(0, 0), (1, 0), (2, 4), (2, 5), (2, 6), (2, 3)],
                         ids=["unfused", "tiled", "fused4", "fused5", "fused6", "fused3"])
def test_circuit_matches_oracle(qs, name, n, make, x0, dtype, mode, fuse):
    circ = make()
    want = oracle_state(n, circ, x0)
    s = qs.State(n, dtype)
    s.set_basis(x0)
    p = qs.Plan(qs.Circuit(circ), n, dtype, mode=mode, fuse_qubits=fuse)
    s.run(p)
    got, stats = s.to_numpy(), p.stats()
    assert stats["gates"] == len(circ)
    if dtype == "c128":
        err = np.max(np.abs(got - want))
        assert err <= C128_TOL, err
    else:
        check_c64(got, want, gates=len(circ))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", [0, 1], ids=["unfused", "tiled"])
def test_qft_closed_form_gpu(qs, dtype, mode):
    n = 14
    x0 = W.basis_index(n, 9)
    got, _ = run_gpu(qs, n, W.qft(n), dtype, mode, x0)
    delta = np.zeros(1 << n, dtype=complex)
    delta[x0] = 1
    want = np.fft.ifft(delta) * math.sqrt(1 << n)
    tol = C128_TOL if dtype == "c128" else 2e-6
    assert np.max(np.abs(got - want)) <= tol


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["unfused", "tiled", "fused"])
def test_c64_vs_oracle_depth40_16q(qs, mode):
    # the complex64 tolerance at depth 40 on a size the oracle runs in seconds
    n = 16
    circ = W.brick(n, 40, 8)
    want = oracle_state(n, circ)
    got, _ = run_gpu(qs, n, circ, "c64", mode)
    check_c64(got, want, gates=len(circ))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("slots,gpt,dense", [(3, 1, 0), (3, 2, 0), (3, 1, -1), (3, 2, -1), (4, 1, 0), (4, 2, 0)])
@pytest.mark.parametrize("tile,low", [(0, 0), (6, 2), (9, 1)])
def test_tile_variants_match_oracle(qs, dtype, slots, gpt, dense, tile, low):
    # every tile-kernel instantiation and a few tile shapes (many tiles per
    # pass, ragged stage counts) against the oracle
    n = 13
    circ = W.brick(n, 12, 31) + W.qft(n) + W.qsb(n, 32, sets=2)
    want = oracle_state(n, circ)
    s = qs.State(n, dtype)
    c = qs.Circuit(circ)
    p = qs.Plan(c, n, dtype, mode=qs.PLAN_TILED, tile_qubits=tile, low_qubits=low, slot_qubits=slots,
                groups_per_thread=gpt, dense=dense)
    s.run(p)
    got = s.to_numpy()
    if dtype == "c128":
        assert np.max(np.abs(got - want)) <= C128_TOL
    else:
        check_c64(got, want, gates=len(circ))


@pytest.mark.parametrize("k", [4, 5, 6])
def test_c64_tensor_core_blocks_vs_oracle_22q(qs, k):
    # complex64 dense blocks on the tensor cores over a depth-40 circuit on a
    # state larger than one tile row set (2^22 amplitudes): infidelity
    # against the FP64 oracle and the norm, which the unbiased per-group
    # restore keeps at 1 without any end-of-plan renormalisation
    n = 22
    circ = W.brick(n, 40, 12)
    want = oracle_state(n, circ)
    s = qs.State(n, "c64")
    p = qs.Plan(qs.Circuit(circ), n, "c64", mode=2, fuse_qubits=k)
    s.run(p)
    got = s.to_numpy()
    check_c64(got, want)


ROUTED = [
    ("qsb14", 14, lambda: W.qsb(14, 41, sets=2), 0),
    ("brick15_d12", 15, lambda: W.brick(15, 12, 42), 0),
    ("qv13_d6", 13, lambda: W.qv_like(13, 6, 43), 0),
    ("hadamard11x12", 12, lambda: W.hadamard_bench(12), 9),
    ("qft13", 13, lambda: W.qft(13), W.basis_index(13, 44)),
    ("ghz16", 16, lambda: W.ghz(16), 0),
]


@pytest.mark.parametrize("name,n,make,x0", ROUTED, ids=[r[0] for r in ROUTED])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", [3, 4], ids=["swap", "permute"])
@pytest.mark.parametrize("m", [6, 9])
def test_routed_plans_match_oracle(qs, name, n, make, x0, dtype, mode, m):
    # swap insertion and fused-permutation insertion (§III-D): tile passes
    # over the m lowest physical qubits, bit-pair exchange passes bringing
    # the other targets in, the state back in logical order at the end
    circ = make()
    want = oracle_state(n, circ, x0)
    s = qs.State(n, dtype)
    s.set_basis(x0)
    p = qs.Plan(qs.Circuit(circ), n, dtype, mode=mode, tile_qubits=m)
    s.run(p)
    got = s.to_numpy()
    assert any(k == "swap" for k, _ in p.step_info())
    if dtype == "c128":
        assert np.max(np.abs(got - want)) <= C128_TOL
    else:
        check_c64(got, want, gates=len(circ))
