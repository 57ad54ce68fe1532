"""GPU parity at the configured sizes of the batching and differentiation
workloads, in the launch configuration the benchmark times.

* Differentiation: 20 qubits, hardware-efficient ansatz of 10 layers (RY then
  RZ on every qubit, CZ ladder; 400 parameters), transverse-field Ising open
  chain, 64 parameter sets in one qs_adjoint_grad call, complex128 and
  complex64.  Eight of the 64 sets against the oracle's adjoint gradient:
  relative error <= 1e-6 (complex128) and <= 1e-3 (complex64), as max |g -
  g_ref| / max |g_ref| and as ||g - g_ref||_2 / ||g_ref||_2.  Parameter shift
  with oracle energies on three parameters of one set, and central finite
  differences (h = 1e-5) through the GPU's own complex128 energies on three
  more.
* Batching: the 512 seeded circuits of 10 to 20 qubits (8 HEA layers,
  complex64) in one autotuned persistent launch, every circuit against the
  oracle: stated and normalised infidelity <= 1e-5, norm within the FP32
  per-gate bound (tests/fidelity.py).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from fidelity import check_c64

pytestmark = pytest.mark.gpu

N_ADJ, LAYERS_ADJ, SETS = 20, 10, 64
CHECKED_SETS = (0, 9, 18, 27, 36, 45, 54, 63)
TOL = {"c128": 1e-6, "c64": 1e-3}


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs
    return qs


@pytest.fixture(scope="module")
def diff_workload():
    circ, _ = W.hea(N_ADJ, LAYERS_ADJ, 11)
    thetas = np.stack([W.hea(N_ADJ, LAYERS_ADJ, 11 + b)[1] for b in range(SETS)])
    terms = W.tfim(N_ADJ)
    ref = {}
    for b in CHECKED_SETS:
        cb = W.with_params(circ, thetas[b])
        ref[b] = oracle.adjoint_grad(oracle.zero_state(N_ADJ), cb, thetas.shape[1], terms)
    return circ, thetas, terms, ref


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_20q_400p_64_sets_vs_oracle(qs, diff_workload, dtype):
    circ, thetas, terms, ref = diff_workload
    assert thetas.shape == (SETS, 400)
    e, g = qs.adjoint_grad(qs.State(N_ADJ, dtype), qs.Circuit(circ), thetas, terms)
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(e))
    for b in CHECKED_SETS:
        e_ref, g_ref = ref[b]
        assert abs(e[b] - e_ref) <= (1e-10 if dtype == "c128" else 1e-4) * max(1.0, abs(e_ref))
        rel_max = np.max(np.abs(g[b] - g_ref)) / np.max(np.abs(g_ref))
        rel_l2 = np.linalg.norm(g[b] - g_ref) / np.linalg.norm(g_ref)
        assert rel_max <= TOL[dtype], (b, rel_max)
        assert rel_l2 <= TOL[dtype], (b, rel_l2)


def test_adjoint_20q_parameter_shift_and_finite_differences(qs, diff_workload):
    circ, thetas, terms, ref = diff_workload
    b = 27
    _, g_ref = ref[b]
    scale = np.max(np.abs(g_ref))
    e, g = qs.adjoint_grad(qs.State(N_ADJ, "c128"), qs.Circuit(circ), thetas[b:b + 2], terms)
    # parameter shift, exact for exp(-i t P / 2), with oracle energies
    for j in (0, 201, 399):
        tp, tm = thetas[b].copy(), thetas[b].copy()
        tp[j] += math.pi / 2
        tm[j] -= math.pi / 2
        ps = 0.5 * (oracle.expectation_of_circuit(N_ADJ, W.with_params(circ, tp), terms)
                    - oracle.expectation_of_circuit(N_ADJ, W.with_params(circ, tm), terms))
        assert abs(g[0, j] - ps) <= 1e-6 * scale, (j, g[0, j], ps)
    # central differences through the GPU's complex128 energy: truncation
    # h^2 |E'''| / 6 ~ 1e-11 and rounding ~1e-15 / h ~ 1e-10, far inside 1e-6
    h = 1e-5
    s = qs.State(N_ADJ, "c128")

    def energy(theta):
        s.set_basis(0)
        s.run(qs.Plan(qs.Circuit(W.with_params(circ, theta)), N_ADJ, "c128", mode=qs.PLAN_UNFUSED))
        return s.expect_pauli(terms)

    for j in (5, 150, 333):
        tp, tm = thetas[b].copy(), thetas[b].copy()
        tp[j] += h
        tm[j] -= h
        fd = (energy(tp) - energy(tm)) / (2 * h)
        assert abs(g[0, j] - fd) <= 1e-6 * scale, (j, g[0, j], fd)


def test_batch_512_hea_every_circuit_vs_oracle(qs):
    sizes = W.batch_sizes(512, 10, 20, 9)
    circs = [W.hea(n, 8, 10 + i)[0] for i, n in enumerate(sizes)]
    b = qs.Batch(sizes, circs, dtype="c64", autotune=True)
    b.run(True)
    b.sync()
    st = b.stats()
    assert st["circuits"] == 512
    for i, (n, c) in enumerate(zip(sizes, circs)):
        want = oracle.zero_state(n)
        oracle.run_circuit(want, c)
        check_c64(b.state(i).cpu().numpy(), want, gates=len(c))
