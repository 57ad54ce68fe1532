"""GPU parity at the benchmark's full sizes.

* 28 qubits, complex128, plain per-gate kernels (the per-gate-class
  configuration) and tensor-core block plans (k = 5, 4): the brick circuit
  (depth 40) and the QFT of a seeded basis state, compared with the FP64
  oracle in full, max |error| <= 1e-12.
* 26 qubits, complex64 fused into 4-, 5- and 6-qubit tensor-core blocks, depth
  40: infidelity against the FP64 oracle <= 1e-5 (stated and normalised
  forms), norm within 1e-6.
* 30 qubits, the benchmark's own launch configuration (complex64,
  QS_PLAN_FUSED, 6-qubit blocks): infidelity against the complex128 GPU path
  (tiled plan, itself oracle-exact at every size above) <= 1e-5; the circuit
  followed by its inverse returns |0...0>; sampled amplitudes of the QFT of a
  basis state against the closed form e^(2 pi i x0 k / N) / sqrt(N), for both
  dtypes in the benchmark's plans; the Ising energy (plus Y terms) of a
  30-qubit product state against its closed form, for both dtypes.
The oracle runs on the host cores (OpenMP); the 28-qubit comparison takes
about a minute there.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from fidelity import check_c64_torch, C64_INFIDELITY, C64_NORM

pytestmark = pytest.mark.gpu

C128_TOL = 1e-12


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs
    return qs


def max_abs_diff(a, b, chunk=1 << 24):
    m = 0.0
    for i in range(0, a.size, chunk):
        m = max(m, float(np.max(np.abs(a[i:i + chunk].astype(np.complex128) - b[i:i + chunk]))))
    return m


def gpu_run(qs, n, circ, dtype, mode, fuse=0, x0=0):
    s = qs.State(n, dtype)
    s.set_basis(x0)
    s.run(qs.Plan(qs.Circuit(circ), n, dtype, mode=mode, fuse_qubits=fuse))
    return s


def test_c128_brick_and_qft_28q_vs_oracle_in_full(qs):
    # the plain per-gate kernels and the complex128 tensor-core block plans
    # (5- and 4-qubit blocks, FP64 operands split into integer digits)
    n = 28
    for circ, x0 in ((W.brick(n, 40, 3), 0), (W.qft(n), W.basis_index(n, 4))):
        want = oracle.zero_state(n, x0)
        oracle.run_circuit(want, circ)
        for mode, fuse in ((qs.PLAN_UNFUSED, 0), (qs.PLAN_FUSED, 5), (qs.PLAN_FUSED, 4)):
            s = gpu_run(qs, n, circ, "c128", mode, fuse=fuse, x0=x0)
            got = s.to_numpy()
            del s
            err = max_abs_diff(got, want)
            assert err <= C128_TOL, (mode, fuse, err)
            del got
        del want


@pytest.mark.parametrize("k", [4, 5, 6])
def test_c64_fused_26q_vs_oracle(qs, k):
    n = 26
    circ = W.brick(n, 40, 8)
    if not hasattr(test_c64_fused_26q_vs_oracle, "want"):
        want = oracle.zero_state(n)
        oracle.run_circuit(want, circ)
        test_c64_fused_26q_vs_oracle.want = want
    want = test_c64_fused_26q_vs_oracle.want
    got = gpu_run(qs, n, circ, "c64", qs.PLAN_FUSED, fuse=k).to_numpy().astype(np.complex128)
    ov = abs(oracle.inner(got, want)) ** 2
    na, nb = oracle.inner(got, got).real, oracle.inner(want, want).real
    assert 1.0 - ov <= C64_INFIDELITY
    assert 1.0 - ov / (na * nb) <= C64_INFIDELITY
    assert abs(na - nb) <= C64_NORM


def test_c64_fused_30q_vs_c128(qs):
    import torch
    n = 30
    circ = W.brick(n, 40, 6)
    s64 = gpu_run(qs, n, circ, "c64", qs.PLAN_FUSED, fuse=6)
    s128 = gpu_run(qs, n, circ, "c128", qs.PLAN_TILED)
    check_c64_torch(s64.tensor, s128.tensor)
    assert abs(s64.norm2() - 1.0) <= C64_NORM
    del s64, s128
    torch.cuda.empty_cache()


def test_c64_fused_30q_round_trip(qs):
    # the circuit and then its inverse (named gates with negated / permuted
    # angles): the identity, whatever blocks the planner forms
    n = 30
    circ = W.brick(n, 40, 6)
    s = gpu_run(qs, n, circ + W.inverse(circ), "c64", qs.PLAN_FUSED, fuse=6)
    a0 = complex(s.tensor[0].item())
    assert abs(a0) ** 2 >= 1.0 - C64_INFIDELITY
    assert abs(s.norm2() - 1.0) <= 1e-6


@pytest.mark.parametrize("dtype,mode,fuse", [("c64", 2, 6), ("c128", 1, 0)], ids=["c64_fused6", "c128_tiled"])
def test_qft_30q_sampled_closed_form(qs, dtype, mode, fuse):
    import torch
    n = 30
    N = 1 << n
    x0 = W.basis_index(n, 11)
    s = gpu_run(qs, n, W.qft(n), dtype, mode, fuse=fuse, x0=x0)
    rng = np.random.default_rng(5)
    ks = np.concatenate([np.arange(64), N - 1 - np.arange(64), rng.integers(0, N, 4096)]).astype(np.int64)
    got = s.tensor[torch.as_tensor(ks, device=s.tensor.device)].cpu().numpy().astype(np.complex128)
    # exact phase: (x0 k) mod N in integers, then one FP64 exponential
    ph = (ks.astype(np.uint64) * np.uint64(x0)) % np.uint64(N)
    want = np.exp(2j * math.pi * ph.astype(np.float64) / N) / math.sqrt(N)
    err = np.max(np.abs(got - want))
    tol = C128_TOL if dtype == "c128" else 1e-5 / math.sqrt(N)
    assert err <= tol, err


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_30q_product_state_closed_form(qs, dtype):
    # the benchmark's TFIM observable plus a Y term on every qubit, at the
    # full 30-qubit size (three complex64 tile passes, four complex128 ones,
    # CTAs running hundreds of tiles each), on the product state
    # prod_i U3(t_i, p_i, 0)|0>: <Z_i> = cos t_i, <X_i> = sin t_i cos p_i,
    # <Y_i> = sin t_i sin p_i, and Z_i Z_j factorises, so
    # E = sum_i cos t_i cos t_i+1 + sum_i sin t_i cos p_i + sum_i g_i sin t_i sin p_i.
    # Complex128 within 1e-12 of sum |coeff|; complex64 within 1e-5: its
    # amplitudes are products of 30 FP32-rounded factors (~30 * 2^-24
    # relative each) and its sums are FP32 per tile (~2^-20)
    n = 30
    rng = np.random.default_rng(30)
    t = rng.uniform(0.0, math.pi, n)
    p = rng.uniform(-math.pi, math.pi, n)
    g = rng.uniform(-1.0, 1.0, n)
    terms = W.tfim(n) + [W.PauliTerm(float(g[i]), 1 << i, 1 << i) for i in range(n)]
    s = qs.State(n, dtype)
    for i in range(n):
        c, sn = math.cos(t[i] / 2), math.sin(t[i] / 2)
        U = np.array([[c, -sn], [np.exp(1j * p[i]) * sn, np.exp(1j * p[i]) * c]], dtype=np.complex128)
        s.apply_1q(i, U)
    want = (sum(math.cos(t[i]) * math.cos(t[i + 1]) for i in range(n - 1))
            + sum(math.sin(t[i]) * math.cos(p[i]) for i in range(n))
            + sum(g[i] * math.sin(t[i]) * math.sin(p[i]) for i in range(n)))
    got = s.expect_pauli(terms)
    tol = (1e-12 if dtype == "c128" else 1e-5) * sum(abs(x.coeff) for x in terms)
    assert abs(got - want) <= tol, (got, want)
    del s
