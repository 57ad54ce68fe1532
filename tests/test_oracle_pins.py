"""Pins for the FP64 oracle, each independent of the oracle's own code.

Every operation the oracle implements is checked against something other
than itself: full 2^n x 2^n operators built with numpy Kronecker products
(n <= 7), scipy's matrix exponential for the rotation gates, numpy's FFT for
the quantum Fourier transform, closed-form states (GHZ, basis states),
unitarity, the inverse circuit, and the worked traffic example of §III-D.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def op_on(n, factors):
    """Kronecker product over qubits n-1 .. 0 (qubit 0 = least significant
    index bit) of the 2x2 factors given as {qubit: matrix}."""
    out = np.ones((1, 1), dtype=complex)
    for q in range(n - 1, -1, -1):
        out = np.kron(out, factors.get(q, I2))
    return out


def ket_bra(r, c):
    m = np.zeros((2, 2), dtype=complex)
    m[r, c] = 1
    return m


def dense_full(n, qubits, M):
    """sum_{r,c} M[r,c] (x)_i |r_i><c_i| on qubits[i], identity elsewhere."""
    k = len(qubits)
    D = 1 << k
    full = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(D):
        for c in range(D):
            if M[r, c] == 0:
                continue
            f = {qubits[i]: ket_bra((r >> i) & 1, (c >> i) & 1) for i in range(k)}
            full += M[r, c] * op_on(n, f)
    return full


def swap_full(n, i, j):
    return dense_full(n, [i, j], np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex))


# ---------------------------------------------------------------------------
# Gate application against brute-force operators
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 3, 6])
def test_apply_1q_kron(n):
    for q in range(n):
        psi = W.random_state(n, 100 + q)
        U = W.random_matrix(2, 200 + q)
        want = op_on(n, {q: U}) @ psi
        got = psi.copy()
        oracle.apply_1q(got, q, U)
        assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("n,nc", [(3, 1), (5, 1), (5, 2), (6, 3)])
def test_apply_controlled_kron(n, nc):
    for seed in range(4):
        qs = W.random_qubits(n, nc + 1, 300 + seed)
        ctrl, t = qs[:nc], qs[nc]
        U = W.random_matrix(2, 400 + seed)
        proj = op_on(n, {c: P1 for c in ctrl})
        want_op = np.eye(1 << n) - proj + proj @ op_on(n, {t: U})
        psi = W.random_state(n, 500 + seed)
        got = psi.copy()
        oracle.apply_controlled(got, ctrl, t, U)
        assert np.max(np.abs(got - want_op @ psi)) < 1e-14


@pytest.mark.parametrize("n,k", [(2, 1), (4, 2), (6, 3), (7, 4)])
def test_apply_diag_kron(n, k):
    qs = W.random_qubits(n, k, 600 + k)
    d = W.random_diag(1 << k, 700 + k, unit=False)
    full = dense_full(n, qs, np.diag(d))
    psi = W.random_state(n, 800 + k)
    got = psi.copy()
    oracle.apply_diag(got, qs, d)
    assert np.max(np.abs(got - full @ psi)) < 1e-13


@pytest.mark.parametrize("n,k", [(2, 2), (4, 2), (5, 3), (6, 4)])
def test_apply_dense_kron(n, k):
    qs = W.random_qubits(n, k, 900 + k)
    M = W.random_matrix(1 << k, 1000 + k)
    full = dense_full(n, qs, M)
    psi = W.random_state(n, 1100 + k)
    got = psi.copy()
    oracle.apply_dense(got, qs, M)
    assert np.max(np.abs(got - full @ psi)) < 1e-13


def test_dense_k1_equals_1q_and_matches_order():
    # A 2-qubit dense gate given with qubits (a, b) equals the same matrix with
    # the index bits exchanged given with qubits (b, a).
    n = 5
    M = W.random_matrix(4, 5)
    Pm = np.zeros((4, 4))
    for r in range(4):
        Pm[((r & 1) << 1) | (r >> 1), r] = 1
    Msw = Pm @ M @ Pm.T
    psi = W.random_state(n, 6)
    a, b = psi.copy(), psi.copy()
    oracle.apply_dense(a, [1, 3], M)
    oracle.apply_dense(b, [3, 1], Msw)
    assert np.max(np.abs(a - b)) < 1e-14


def test_swap_kron():
    n = 5
    psi = W.random_state(n, 7)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            got = psi.copy()
            oracle.swap(got, i, j)
            assert np.max(np.abs(got - swap_full(n, i, j) @ psi)) < 1e-15


def test_fused_swap_is_listing1_sequence():
    # fused_swap(p, q, s) behaves as swap(p+i, q+i) for i < s (Listing 1).
    n = 7
    for (p, q, s) in [(0, 4, 3), (4, 0, 3), (1, 3, 2), (0, 6, 1), (2, 5, 2)]:
        psi = W.random_state(n, 11 + p + q + s)
        op = np.eye(1 << n, dtype=complex)
        for i in range(s):
            op = swap_full(n, p + i, q + i) @ op
        got = psi.copy()
        moved = oracle.fused_swap(got, p, q, s)
        assert np.max(np.abs(got - op @ psi)) < 1e-15
        # amplitudes whose index changes: those whose two s-bit fields differ
        assert moved == (1 << n) - (1 << (n - s))
        assert moved == int(np.count_nonzero(np.abs(np.diag(op)) < 0.5))


def test_fused_swap_rejects_overlap():
    psi = W.random_state(4, 1)
    with pytest.raises(ValueError):
        oracle.fused_swap(psi, 0, 1, 2)
    with pytest.raises(ValueError):
        oracle.fused_swap(psi, 2, 3, 2)


def test_permute_matches_swap_products():
    # A general permutation decomposed into transpositions of qubit labels.
    n = 6
    for seed in range(6):
        perm = W.random_perm(n, 40 + seed)
        psi = W.random_state(n, 50 + seed)
        got = oracle.permute(psi, perm)
        # Build pi as a product of bit swaps: selection-sort the label map.
        pos = list(range(n))          # pos[j] = where bit j currently sits
        where = list(range(n))        # where[b] = which original bit sits at b
        op = np.eye(1 << n, dtype=complex)
        for j in range(n):
            cur = pos[j]
            tgt = perm[j]
            if cur != tgt:
                op = swap_full(n, cur, tgt) @ op
                other = where[tgt]
                where[cur], where[tgt] = other, j
                pos[other], pos[j] = cur, tgt
        assert np.max(np.abs(got - op @ psi)) < 1e-15
        inv = [0] * n
        for j, p in enumerate(perm):
            inv[p] = j
        back = oracle.permute(got, inv)
        assert np.max(np.abs(back - psi)) == 0.0


def test_permute_rejects_non_permutation():
    with pytest.raises(ValueError):
        oracle.permute(W.random_state(3, 1), [0, 0, 1])


# ---------------------------------------------------------------------------
# Gate matrices: identities and matrix exponentials
# ---------------------------------------------------------------------------

def test_gate_matrix_identities():
    H = oracle.gate_matrix("H")
    assert np.allclose(H @ H, I2, atol=1e-15)
    assert np.allclose(H @ X @ H, Z, atol=1e-15)
    assert np.allclose(oracle.gate_matrix("X"), X)
    assert np.allclose(oracle.gate_matrix("Y"), Y)
    assert np.allclose(oracle.gate_matrix("Z"), Z)
    S, T = oracle.gate_matrix("S"), oracle.gate_matrix("T")
    assert np.allclose(S @ S, Z, atol=1e-15)
    assert np.allclose(T @ T, S, atol=1e-15)
    for th in [0.0, 0.3, -1.7, 2 * math.pi - 0.1]:
        assert np.allclose(oracle.gate_matrix("RX", [th]), scipy.linalg.expm(-0.5j * th * X), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("RY", [th]), scipy.linalg.expm(-0.5j * th * Y), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("RZ", [th]), scipy.linalg.expm(-0.5j * th * Z), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("P", [th]), np.diag([1, np.exp(1j * th)]), atol=1e-15)
        # U3 special cases (OpenQASM): U3(t,-pi/2,pi/2) = RX(t), U3(t,0,0) = RY(t),
        # U3(0,0,l) = P(l).
        assert np.allclose(oracle.gate_matrix("U3", [th, -math.pi / 2, math.pi / 2]), oracle.gate_matrix("RX", [th]), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("U3", [th, 0, 0]), oracle.gate_matrix("RY", [th]), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("U3", [0, 0, th]), oracle.gate_matrix("P", [th]), atol=1e-14)
    # U3 = e^{i(p+l)/2} RZ(p) RY(t) RZ(l)
    t, p, l = 0.7, 1.9, -2.3
    want = np.exp(0.5j * (p + l)) * (scipy.linalg.expm(-0.5j * p * Z) @ scipy.linalg.expm(-0.5j * t * Y) @ scipy.linalg.expm(-0.5j * l * Z))
    assert np.allclose(oracle.gate_matrix("U3", [t, p, l]), want, atol=1e-14)
    for name, prm in [("U3", [1.1, 0.2, -0.4]), ("RX", [0.3]), ("H", [])]:
        U = oracle.gate_matrix(name, prm)
        assert np.allclose(U.conj().T @ U, I2, atol=1e-15)


def test_two_qubit_matrices():
    # bit 0 of the 4x4 index = qubits[0] (control for CNOT)
    cnot = oracle.gate_matrix("CNOT")
    want = np.kron(I2, P0) + np.kron(X, P1)  # target = bit 1, control = bit 0
    assert np.allclose(cnot, want)
    assert np.allclose(oracle.gate_matrix("CZ"), np.diag([1, 1, 1, -1]))
    assert np.allclose(oracle.gate_matrix("CP", [0.4]), np.diag([1, 1, 1, np.exp(0.4j)]))
    sw = oracle.gate_matrix("SWAP")
    # SWAP = CNOT(a,b) CNOT(b,a) CNOT(a,b)
    cnot_ba = np.kron(P0, I2) + np.kron(P1, X)
    assert np.allclose(sw, cnot @ cnot_ba @ cnot)


def test_swap_equals_three_cnots_on_states():
    n = 5
    psi = W.random_state(n, 77)
    a = psi.copy()
    oracle.run_circuit(a, [W.Gate("SWAP", (1, 4))])
    b = psi.copy()
    oracle.run_circuit(b, [W.Gate("CNOT", (1, 4)), W.Gate("CNOT", (4, 1)), W.Gate("CNOT", (1, 4))])
    assert np.max(np.abs(a - b)) < 1e-15


def test_run_circuit_matches_kron_product():
    # A short random circuit with every gate kind, against the product of
    # its brute-force operators.
    n = 4
    rng = np.random.Generator(np.random.PCG64(3))
    circ = []
    for i in range(30):
        name = ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P", "U3", "CNOT", "CZ", "CP", "SWAP"][i % 15]
        nparams = W.N_PARAMS.get(name, 0)
        prm = tuple(float(v) for v in rng.uniform(-3, 3, nparams))
        nq = 1 if name in W.ONE_QUBIT else 2
        qs = tuple(int(v) for v in rng.permutation(n)[:nq])
        circ.append(W.Gate(name, qs, prm))
    W.validate(circ, n)
    op = np.eye(1 << n, dtype=complex)
    for g in circ:
        m = oracle.gate_matrix(g.name, g.params)
        op = dense_full(n, list(g.qubits), m) @ op
    psi = W.random_state(n, 9)
    got = psi.copy()
    oracle.run_circuit(got, circ)
    assert np.max(np.abs(got - op @ psi)) < 1e-13


# ---------------------------------------------------------------------------
# Closed-form states and invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_ghz(n):
    psi = oracle.zero_state(n)
    oracle.run_circuit(psi, W.ghz(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 7, 12])
def test_qft_closed_form(n):
    N = 1 << n
    for x0 in {0, 1, N - 1, W.basis_index(n, 2), W.basis_index(n, 5)}:
        psi = oracle.zero_state(n, x0)
        oracle.run_circuit(psi, W.qft(n))
        delta = np.zeros(N, dtype=complex)
        delta[x0] = 1
        want = np.fft.ifft(delta) * math.sqrt(N)  # e^{+2 pi i x0 y / N} / sqrt(N)
        assert np.max(np.abs(psi - want)) < 1e-13


def test_brick_norm_and_inverse():
    n = 12
    circ = W.brick(n, 40, 1)
    assert len(circ) == 40 * n + 20 * 6 + 20 * 5
    psi = oracle.zero_state(n)
    oracle.run_circuit(psi, circ)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-13
    oracle.run_circuit(psi, W.inverse(circ))
    want = oracle.zero_state(n)
    assert np.max(np.abs(psi - want)) < 1e-12


def test_brick_gate_counts_match_config():
    # 12 qubits, depth 20: 240 U3 + 110 CNOT (6 on even layers, 5 on odd)
    c = W.brick(12, 20, 1)
    assert sum(g.name == "U3" for g in c) == 240
    assert sum(g.name == "CNOT" for g in c) == 110
    c = W.brick(28, 40, 3)
    assert sum(g.name == "U3" for g in c) == 1120 and sum(g.name == "CNOT" for g in c) == 540
    c = W.brick(30, 40, 6)
    assert sum(g.name == "U3" for g in c) == 1200 and sum(g.name == "CNOT" for g in c) == 580
    q = W.qft(28)
    assert (sum(g.name == "H" for g in q), sum(g.name == "CP" for g in q), sum(g.name == "SWAP" for g in q)) == (28, 378, 14)


def test_qsb_inverse():
    n = 8
    circ = W.qsb(n, 4)
    psi = W.random_state(n, 10)
    got = psi.copy()
    oracle.run_circuit(got, circ)
    oracle.run_circuit(got, W.inverse(circ))
    assert np.max(np.abs(got - psi)) < 1e-13


@pytest.mark.parametrize("n", [5, 8])
def test_qv_like_structure_and_inverse(n):
    # the QV-shaped workload (§IV-E): per layer a permutation pairs the
    # qubits, every pair gets 10 named gates, each qubit in at most one pair;
    # the pairings change between layers; the circuit is unitary (norm and
    # round trip through its inverse)
    depth = 6
    circ = W.qv_like(n, depth, 13)
    W.validate(circ, n)
    per_layer = 10 * (n // 2)
    assert len(circ) == depth * per_layer
    pairings = []
    for layer in range(depth):
        gates = circ[layer * per_layer:(layer + 1) * per_layer]
        pairs = [tuple(gates[i + 2].qubits) for i in range(0, per_layer, 10)]  # the first CNOT (a, b)
        used = [q for pr in pairs for q in pr]
        assert len(set(used)) == len(used) == 2 * (n // 2)
        for i in range(0, per_layer, 10):
            a, b = gates[i + 2].qubits
            assert [g.name for g in gates[i:i + 10]] == ["U3", "U3", "CNOT", "RZ", "RY", "CNOT", "RY", "CNOT", "U3", "U3"]
            assert [g.qubits for g in gates[i:i + 10]] == [(a,), (b,), (a, b), (a,), (b,), (b, a), (b,), (a, b), (a,), (b,)]
        pairings.append(frozenset(frozenset(pr) for pr in pairs))
    assert len(set(pairings)) > 1
    psi = W.random_state(n, 14)
    got = psi.copy()
    oracle.run_circuit(got, circ)
    assert abs(np.vdot(got, got).real - 1.0) < 1e-13
    oracle.run_circuit(got, W.inverse(circ))
    assert np.max(np.abs(got - psi)) < 1e-13


def test_qv_like_matches_kron_product():
    n = 4
    circ = W.qv_like(n, 3, 15)
    op = np.eye(1 << n, dtype=complex)
    for g in circ:
        op = dense_full(n, list(g.qubits), oracle.gate_matrix(g.name, g.params)) @ op
    psi = W.random_state(n, 16)
    got = psi.copy()
    oracle.run_circuit(got, circ)
    assert np.max(np.abs(got - op @ psi)) < 1e-13


# ---------------------------------------------------------------------------
# Reductions
# ---------------------------------------------------------------------------

def test_inner_matches_vdot():
    for n in [1, 5, 13]:
        a, b = W.random_state(n, 1, False), W.random_state(n, 2, False)
        assert abs(oracle.inner(a, b) - np.vdot(a, b)) < 1e-12 * (1 << n)


def pauli_full(n, t):
    f = {}
    for q in range(n):
        x, z = (t.xmask >> q) & 1, (t.zmask >> q) & 1
        if x and z:
            f[q] = Y
        elif x:
            f[q] = X
        elif z:
            f[q] = Z
    return op_on(n, f)


def test_expect_pauli_brute_force():
    n = 6
    terms = W.random_paulis(n, 25, 3)
    psi = W.random_state(n, 4)
    H = sum(t.coeff * pauli_full(n, t) for t in terms)
    want = np.vdot(psi, H @ psi).real
    assert abs(oracle.expect_pauli(psi, terms) - want) < 1e-13
    got = oracle.apply_pauli_sum(psi, terms)
    assert np.max(np.abs(got - H @ psi)) < 1e-13


@pytest.mark.parametrize("n", [2, 5, 10])
def test_tfim_closed_forms(n):
    H = W.tfim(n)
    # |0...0>: every ZZ = +1, every X = 0  ->  n - 1
    assert abs(oracle.expect_pauli(oracle.zero_state(n), H) - (n - 1)) < 1e-13
    # |+...+>: every X = +1, every ZZ = 0  ->  n
    psi = oracle.zero_state(n)
    oracle.run_circuit(psi, [W.Gate("H", (q,)) for q in range(n)])
    assert abs(oracle.expect_pauli(psi, H) - n) < 1e-12
    # Z_q on basis states = (-1)^{bit q}
    for x in [0, 1, (1 << n) - 1, W.basis_index(n, 9)]:
        for q in range(n):
            e = oracle.expect_pauli(oracle.zero_state(n, x), [W.PauliTerm(1.0, 0, 1 << q)])
            assert e == (-1.0) ** ((x >> q) & 1)


# ---------------------------------------------------------------------------
# Gradient: adjoint sweep vs parameter shift vs central differences
# ---------------------------------------------------------------------------

def test_adjoint_vs_parameter_shift_and_fd():
    n, layers = 4, 2
    circ, theta = W.hea(n, layers, 12)
    terms = W.tfim(n)
    psi0 = oracle.zero_state(n)
    e, g = oracle.adjoint_grad(psi0, circ, len(theta), terms)
    assert abs(e - oracle.expectation_of_circuit(n, circ, terms)) < 1e-13
    ps = np.zeros_like(theta)
    fd = np.zeros_like(theta)
    h = 1e-5
    for j in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += math.pi / 2
        tm[j] -= math.pi / 2
        ps[j] = 0.5 * (oracle.expectation_of_circuit(n, W.with_params(circ, tp), terms)
                       - oracle.expectation_of_circuit(n, W.with_params(circ, tm), terms))
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (oracle.expectation_of_circuit(n, W.with_params(circ, tp), terms)
                 - oracle.expectation_of_circuit(n, W.with_params(circ, tm), terms)) / (2 * h)
    assert np.max(np.abs(g - ps)) < 1e-12
    assert np.max(np.abs(g - fd)) < 1e-8


# ---------------------------------------------------------------------------
# The paper's traffic accounting (§III-B, §III-D, Eq. 5)
# ---------------------------------------------------------------------------

def test_fused_swap_traffic_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "fused_swap_traffic.json")))
    n, S = g["n"], g["bytes_per_amplitude"]
    m = n - len(g["global_qubits"])  # local qubits 0..m-1
    N = 1 << n
    # (1) A gate on a global qubit exchanges every amplitude: the partner of
    # each index lies in another slice of 2^m amplitudes.
    cross = sum(1 for x in range(N) for q in g["global_qubits"][:1] if (x >> m) != ((x ^ (1 << q)) >> m))
    assert cross * S * g["global_gate_count"] == g["bytes_original_circuit"]
    # (2) swap(local, global) moves half the vector.
    psi = W.random_state(n, 1)
    moved_swap = oracle.fused_swap(psi, 0, 2, 1)
    assert moved_swap * S * g["swap_count"] == g["bytes_swapped_circuit"]
    # (3) fused_swap(0, 2, 2) moves N (1 - 2^-s) amplitudes.
    moved_fused = oracle.fused_swap(psi, 0, 2, g["fused_swap_s"])
    assert moved_fused * S * g["fused_swap_count"] == g["bytes_fused_swap_circuit"]


def test_state_memory_accounting():
    g = json.load(open(os.path.join(GOLDEN, "state_memory.json")))
    for ex in g["examples"]:
        n = ex["n"]
        assert np.dtype(np.complex128).itemsize * (1 << n) == ex["state_bytes"]
        if "gate_traffic_bytes" in ex:
            assert 2 * ex["state_bytes"] == ex["gate_traffic_bytes"]


# ---------------------------------------------------------------------------
# Measurement, sampling, collapse (§II-A: circuits include measurements)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("qubits", [[0], [3], [6, 1], [2, 5, 0], [0, 1, 2, 3, 4, 5, 6]])
def test_probabilities_brute_force(qubits):
    # numpy: |psi|^2 reshaped by bits, summed over the other axes
    n = 7
    psi = W.random_state(n, 40)
    p = (np.abs(psi) ** 2).reshape([2] * n)  # axis j = bit n - 1 - j
    keep = [n - 1 - q for q in qubits]
    other = tuple(ax for ax in range(n) if ax not in keep)
    marg = p.sum(axis=other)
    # marg axes follow `keep` in increasing axis order; reorder to qubits[0] as bit 0
    order = sorted(keep)
    want = np.zeros(1 << len(qubits))
    for r in range(1 << len(qubits)):
        idx = [0] * len(order)
        for i, q in enumerate(qubits):
            idx[order.index(n - 1 - q)] = (r >> i) & 1
        want[r] = marg[tuple(idx)]
    got = oracle.probabilities(psi, qubits)
    assert np.max(np.abs(got - want)) < 1e-14
    assert abs(got.sum() - 1.0) < 1e-13


def test_probabilities_and_collapse_closed_forms():
    n = 5
    ghz = oracle.zero_state(n)
    oracle.run_circuit(ghz, W.ghz(n))
    assert np.allclose(oracle.probabilities(ghz, [0]), [0.5, 0.5], atol=1e-15)
    assert np.allclose(oracle.probabilities(ghz, [0, 4]), [0.5, 0, 0, 0.5], atol=1e-15)
    x0 = 0b10110
    basis = oracle.zero_state(n, x0)
    assert np.array_equal(oracle.probabilities(basis, [1, 2, 4]), [0, 0, 0, 0, 0, 0, 0, 1.0])
    # measuring a GHZ qubit leaves the matching basis state
    for outcome in (0, 1):
        s = ghz.copy()
        oracle.collapse(s, 2, outcome, 0.5)
        want = np.zeros(1 << n, complex)
        want[0 if outcome == 0 else (1 << n) - 1] = 1.0
        assert np.max(np.abs(s - want)) < 1e-15
    # collapse of a random state: the kept half renormalised, the other zero
    psi = W.random_state(6, 41)
    p1 = oracle.probabilities(psi, [3])[1]
    s = psi.copy()
    oracle.collapse(s, 3, 1, p1)
    idx = np.arange(1 << 6)
    assert np.all(s[(idx >> 3) & 1 == 0] == 0)
    assert np.max(np.abs(s[(idx >> 3) & 1 == 1] - psi[(idx >> 3) & 1 == 1] / math.sqrt(p1))) < 1e-15
    assert abs(np.vdot(s, s).real - 1.0) < 1e-14


@pytest.mark.parametrize("n", [4, 10, 12])
def test_sample_uniform_dyadic_is_floor(n):
    # every p_x = 2^-n exactly (amplitudes 2^(-n/2) set directly), so every
    # running sum is exact, F[x] = (x + 1) 2^-n: sample(u) = floor(u 2^n)
    # (a search for F[x] >= t instead of F[x] > t fails at u = 0.5)
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=complex)
    u = np.concatenate([[0.0, 0.5, 1 - 2.0 ** -53], np.random.default_rng(42).random(500)])
    got = oracle.sample(psi, u)
    assert np.array_equal(got, np.floor(u * (1 << n)).astype(np.uint64))


def test_sample_basis_ghz_and_monotone():
    n = 11
    x0 = 1234
    u = np.random.default_rng(43).random(300)
    assert np.all(oracle.sample(oracle.zero_state(n, x0), u) == x0)
    ghz = oracle.zero_state(n)
    oracle.run_circuit(ghz, W.ghz(n))
    g = oracle.sample(ghz, u)
    assert np.all(g[u < 0.49] == 0) and np.all(g[u > 0.51] == (1 << n) - 1)
    # the inverse CDF is monotone in u, and lands only where p_x > 0
    psi = W.random_state(12, 44)
    psi[::3] = 0
    uu = np.sort(np.random.default_rng(45).random(2000))
    x = oracle.sample(psi, uu)
    assert np.all(np.diff(x.astype(np.int64)) >= 0)
    assert np.all(np.abs(psi[x.astype(np.int64)]) > 0)


def test_sample_frequencies():
    # 200k samples of an 8-qubit state: every outcome's frequency within 5
    # standard deviations of its probability
    n = 8
    psi = W.random_state(n, 46)
    p = np.abs(psi) ** 2
    u = np.random.default_rng(47).random(200000)
    counts = np.bincount(oracle.sample(psi, u).astype(np.int64), minlength=1 << n)
    sd = np.sqrt(p * (1 - p) * u.size)
    assert np.all(np.abs(counts - p * u.size) <= 5 * sd + 1)


@pytest.mark.parametrize("n", [1, 7, 14])
def test_cdf_against_exactly_rounded_prefix(n):
    # F[x] against math.fsum (the exactly rounded sum of the same squares):
    # a sequential FP64 sum of x + 1 nonnegative terms is within
    # (x + 1) 2^-53 F[x] of it; a dropped or repeated term is not
    psi = W.random_state(n, 48 + n)
    psi[1::5] = 0
    p = psi.real ** 2 + psi.imag ** 2
    F = oracle.cdf(psi)
    idx = np.unique(np.concatenate([[0, p.size - 1], np.random.default_rng(n).integers(0, p.size, 50)]))
    for x in idx:
        exact = math.fsum(p[: x + 1])
        assert abs(F[x] - exact) <= (x + 1) * 2.0 ** -53 * exact + 1e-300
    assert np.all(np.diff(F) >= 0)


def test_sample_is_inverse_cdf_by_exact_rationals():
    # 3 qubits: the probabilities as exact rationals, the CDF summed exactly;
    # every sample x has Fexact(x - 1) <= u T < Fexact(x) up to the rounding
    # of 8 terms, and where u T is clear of every boundary it is the only x
    from fractions import Fraction
    n = 3
    psi = W.random_state(n, 49)
    psi[5] = 0
    p = [Fraction(float(v.real)) ** 2 + Fraction(float(v.imag)) ** 2 for v in psi]
    Fx = [sum(p[: x + 1], Fraction(0)) for x in range(8)]
    T = Fx[-1]
    u = np.concatenate([[0.0, 1 - 2.0 ** -53], np.random.default_rng(50).random(3000)])
    got = oracle.sample(psi, u)
    eps = Fraction(16, 2 ** 53) * T
    for ui, x in zip(u, got):
        x = int(x)
        ut = Fraction(float(ui)) * T
        lo = Fx[x - 1] if x > 0 else Fraction(0)
        assert p[x] > 0
        assert lo - eps <= ut < Fx[x] + eps
        if lo + eps < ut < Fx[x] - eps:
            continue
        # within eps of a boundary: x is one of the two neighbours of it
        assert any(abs(ut - b) <= eps for b in [Fraction(0)] + Fx)
