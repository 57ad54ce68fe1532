"""The fusion planner's host arithmetic, without a GPU.

A QS_PLAN_FUSED plan replayed block by block with the oracle (apply_dense of
each block's matrix on its qubits, qs_plan_step_matrix / qs_plan_step_qubits)
must equal the circuit run gate by gate by the oracle.  This pins the
planner's block products (each absorbed gate multiplied onto the rows of the
running product, CNOT / SWAP / CZ / CP as row moves and scalings), the
widening of complex64 blocks with idle qubits, and the gate order across
blocks, independently of the kernels that later apply the blocks.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def qs():
    import paper_2203_16044_gb300 as qs
    return qs


def every_kind(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(60):
        name = ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P", "U3", "CNOT", "CZ", "CP", "SWAP"][i % 15]
        prm = tuple(float(v) for v in rng.uniform(-3, 3, W.N_PARAMS.get(name, 0)))
        nq = 1 if name in W.ONE_QUBIT else 2
        out.append(W.Gate(name, tuple(int(v) for v in rng.permutation(n)[:nq]), prm))
    return out


CIRCUITS = [
    ("brick", 9, lambda: W.brick(9, 10, 1)),
    ("qft", 8, lambda: W.qft(8)),
    ("qsb", 8, lambda: W.qsb(8, 3, sets=3)),
    ("qv", 9, lambda: W.qv_like(9, 4, 2)),
    ("hea", 8, lambda: W.hea(8, 3, 4)[0]),
    ("every_kind", 7, lambda: every_kind(7, 5)),
]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("name,n,make", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_fused_plan_replays_circuit(qs, dtype, k, name, n, make):
    circ = make()
    p = qs.Plan(qs.Circuit(circ), n, dtype, mode=qs.PLAN_FUSED, fuse_qubits=k)
    psi = W.random_state(n, 100 + n + k)
    got = psi.copy()
    for i, (kind, _) in enumerate(p.step_info()):
        assert kind == "block", kind
        q = p.step_qubits(i)
        M = p.step_matrix(i)
        assert M.shape == (1 << len(q), 1 << len(q)) and len(q) <= k + (3 if dtype == "c64" else 0)
        oracle.apply_dense(got, q, M)
    want = psi.copy()
    oracle.run_circuit(want, circ)
    assert np.max(np.abs(got - want)) < 1e-12


def test_step_matrix_errors(qs):
    p = qs.Plan(qs.Circuit(W.brick(6, 2, 1)), 6, "c64", mode=qs.PLAN_UNFUSED)
    with pytest.raises(qs.QSError):
        p.step_matrix(0)  # a gate step, not a block
    p = qs.Plan(qs.Circuit(W.brick(6, 2, 1)), 6, "c64", mode=qs.PLAN_FUSED, fuse_qubits=4)
    with pytest.raises(qs.QSError):
        p.step_matrix(p.stats()["passes"])
