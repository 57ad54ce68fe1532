"""Adjoint gradients on the GPU against the oracle.

Hardware-efficient ansatz (RY, RZ on every qubit, CZ ladder) and the
transverse-field Ising observable; the oracle gives the adjoint reference
(pinned to parameter shift and finite differences in test_oracle_pins.py).
Tolerances: complex128 relative error <= 1e-6 (measured far below), complex64
<= 1e-3, relative to max |g_ref|.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs
    return qs


def rel(g, ref):
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-3)])
@pytest.mark.parametrize("n,layers", [(2, 1), (5, 2), (8, 3), (11, 2)])
def test_adjoint_matches_oracle(qs, dtype, tol, n, layers):
    circ, theta = W.hea(n, layers, 40 + n)
    terms = W.tfim(n)
    e_ref, g_ref = oracle.adjoint_grad(oracle.zero_state(n), circ, len(theta), terms)
    s = qs.State(n, dtype)
    e, g = qs.adjoint_grad(s, qs.Circuit(circ), theta, terms)
    assert abs(e - e_ref) <= (1e-10 if dtype == "c128" else 1e-4) * max(1.0, abs(e_ref))
    assert rel(g, g_ref) <= tol


def test_adjoint_batch_and_parameter_shift(qs):
    n, layers, batch = 6, 2, 3
    circ, theta0 = W.hea(n, layers, 77)
    terms = W.tfim(n) + W.random_paulis(n, 5, 78)
    rng = np.random.Generator(np.random.PCG64(79))
    thetas = np.stack([theta0] + [rng.uniform(-math.pi, math.pi, len(theta0)) for _ in range(batch - 1)])
    s = qs.State(n, "c128")
    e, g = qs.adjoint_grad(s, qs.Circuit(circ), thetas, terms)
    for b in range(batch):
        cb = W.with_params(circ, thetas[b])
        assert abs(e[b] - oracle.expectation_of_circuit(n, cb, terms)) <= 1e-11
        # parameter shift on a few parameters, from the oracle
        for j in (0, len(theta0) // 2, len(theta0) - 1):
            tp, tm = thetas[b].copy(), thetas[b].copy()
            tp[j] += math.pi / 2
            tm[j] -= math.pi / 2
            ps = 0.5 * (oracle.expectation_of_circuit(n, W.with_params(circ, tp), terms)
                        - oracle.expectation_of_circuit(n, W.with_params(circ, tm), terms))
            assert abs(g[b, j] - ps) <= 1e-10


def test_adjoint_with_other_gates(qs):
    # fixed one- and two-qubit gates of every kind between trainable ones
    n = 7
    circ = []
    rng = np.random.Generator(np.random.PCG64(5))
    pi = 0
    for layer in range(3):
        for q in range(n):
            circ.append(W.Gate(["RX", "RY", "RZ"][(q + layer) % 3], (q,), (float(rng.uniform(-3, 3)),), pi))
            pi += 1
        circ += [W.Gate("H", (0,)), W.Gate("CNOT", (1, 4)), W.Gate("CP", (2, 5), (0.7,)), W.Gate("SWAP", (3, 6)),
                 W.Gate("U3", (5,), (0.3, 0.2, 0.1)), W.Gate("CZ", (0, 6)), W.Gate("S", (2,)), W.Gate("T", (4,))]
    theta = np.array([g.params[0] for g in circ if g.param_index >= 0])
    terms = W.random_paulis(n, 12, 9)
    e_ref, g_ref = oracle.adjoint_grad(oracle.zero_state(n), circ, len(theta), terms)
    for dtype, tol in (("c128", 1e-9), ("c64", 1e-3)):
        e, g = qs.adjoint_grad(qs.State(n, dtype), qs.Circuit(circ), theta, terms)
        assert rel(g, g_ref) <= tol, dtype


def test_autograd_function(qs):
    import torch
    n, layers = 5, 2
    circ, theta0 = W.hea(n, layers, 91)
    terms = W.tfim(n)
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    fn = qs.expectation_fn()
    E = fn.apply(theta, qs.State(n, "c128"), qs.Circuit(circ), terms)
    (2.0 * E).backward()
    e_ref, g_ref = oracle.adjoint_grad(oracle.zero_state(n), circ, len(theta0), terms)
    assert abs(E.item() - e_ref) <= 1e-11
    assert np.max(np.abs(theta.grad.numpy() - 2.0 * g_ref)) <= 1e-10


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-3)])
@pytest.mark.parametrize("n,batch", [(7, 5), (12, 9)])
def test_adjoint_batched_sets(qs, dtype, tol, n, batch):
    # several parameter sets share one buffer (psi and lambda of every set);
    # an odd batch leaves a short last chunk.  Each set must match both the
    # oracle and the one-set call, with fixed gates of every kind in between.
    rng = np.random.Generator(np.random.PCG64(300 + n))
    circ, pi = [], 0
    for layer in range(2):
        for q in range(n):
            circ.append(W.Gate(["RX", "RY", "RZ"][(q + layer) % 3], (q,), (0.0,), pi))
            pi += 1
        circ += [W.Gate("H", (1,)), W.Gate("CNOT", (n - 1, 2)), W.Gate("CP", (0, n - 2), (0.4,)),
                 W.Gate("SWAP", (1, n - 3)), W.Gate("U3", (3,), (0.3, 1.2, -0.5)), W.Gate("CZ", (2, n - 1))]
    thetas = rng.uniform(-math.pi, math.pi, (batch, pi))
    terms = W.tfim(n) + W.random_paulis(n, 6, 301 + n)
    c = qs.Circuit(circ)
    e, g = qs.adjoint_grad(qs.State(n, dtype), c, thetas, terms)
    assert e.shape == (batch,) and g.shape == (batch, pi)
    for b in (0, batch // 2, batch - 1):
        cb = W.with_params(circ, thetas[b])
        e_ref, g_ref = oracle.adjoint_grad(oracle.zero_state(n), cb, pi, terms)
        assert abs(e[b] - e_ref) <= (1e-10 if dtype == "c128" else 1e-4) * max(1.0, abs(e_ref))
        assert rel(g[b], g_ref) <= tol
        e1, g1 = qs.adjoint_grad(qs.State(n, dtype), c, thetas[b:b + 1], terms)
        assert abs(e1[0] - e[b]) <= (1e-12 if dtype == "c128" else 1e-5) * max(1.0, abs(e_ref))
        assert rel(g1[0], g[b]) <= (1e-10 if dtype == "c128" else 1e-4)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-3)])
def test_adjoint_hea_tfim_sets_vs_oracle(qs, dtype, tol):
    # the differentiation workload's shape (RY and RZ layers, CZ ladder,
    # transverse-field Ising H, several parameter sets in one call) at a size
    # the oracle runs in seconds; diagonal runs (CZ ladder + RZ layer) and
    # one-qubit layers (RY) both take the fused sweep steps here
    n, layers, batch = 16, 4, 6
    circ, _ = W.hea(n, layers, 51)
    thetas = np.stack([W.hea(n, layers, 51 + b)[1] for b in range(batch)])
    terms = W.tfim(n)
    e, g = qs.adjoint_grad(qs.State(n, dtype), qs.Circuit(circ), thetas, terms)
    for b in (0, batch - 1):
        cb = W.with_params(circ, thetas[b])
        e_ref, g_ref = oracle.adjoint_grad(oracle.zero_state(n), cb, thetas.shape[1], terms)
        assert abs(e[b] - e_ref) <= (1e-10 if dtype == "c128" else 1e-4) * max(1.0, abs(e_ref))
        assert rel(g[b], g_ref) <= tol
    # parameter shift on two parameters of the last set (oracle energies)
    cb = W.with_params(circ, thetas[-1])
    for j in (3, thetas.shape[1] - 2):
        tp, tm = thetas[-1].copy(), thetas[-1].copy()
        tp[j] += math.pi / 2
        tm[j] -= math.pi / 2
        ps = 0.5 * (oracle.expectation_of_circuit(n, W.with_params(circ, tp), terms)
                    - oracle.expectation_of_circuit(n, W.with_params(circ, tm), terms))
        assert abs(g[-1, j] - ps) <= (1e-9 if dtype == "c128" else 1e-3 * max(1.0, abs(ps)))
