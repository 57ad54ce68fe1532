"""Plain FP64 CPU oracle for state-vector gate application.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg -- never by the product path.  It shares
no code with the CUDA library; the only common input is the ``workloads``
generator module (gate names, qubit indices, angles; no arithmetic).

The arithmetic lives in oracle.cpp (compiled on first use); this wrapper only
marshals numpy complex128 arrays and gate records.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import build as _build

_KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5, "RX": 6, "RY": 7, "RZ": 8,
         "P": 9, "U3": 10, "CNOT": 16, "CZ": 17, "CP": 18, "SWAP": 19}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_uint64)
        c_int, c_ll, c_d = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        L.or_apply_1q.argtypes = [dp, c_int, c_int, dp]
        L.or_apply_controlled.argtypes = [dp, c_int, ip, c_int, c_int, dp]
        L.or_apply_diag.argtypes = [dp, c_int, ip, c_int, dp]
        L.or_apply_dense.argtypes = [dp, c_int, ip, c_int, dp]
        L.or_swap.argtypes = [dp, c_int, c_int, c_int]
        L.or_fused_swap.argtypes = [dp, c_int, c_int, c_int, c_int]
        L.or_fused_swap.restype = c_ll
        L.or_permute.argtypes = [dp, dp, c_int, ip]
        L.or_permute.restype = c_int
        L.or_gate_matrix.argtypes = [c_int, dp, dp]
        L.or_gate_matrix.restype = c_int
        L.or_run_circuit.argtypes = [dp, c_int, c_int, ip, ip, dp]
        L.or_run_circuit.restype = c_int
        L.or_inner.argtypes = [dp, dp, c_int, dp]
        L.or_expect_pauli.argtypes = [dp, c_int, c_int, up, up, dp]
        L.or_expect_pauli.restype = c_d
        L.or_apply_pauli_sum.argtypes = [dp, dp, c_int, c_int, up, up, dp]
        L.or_adjoint_grad.argtypes = [dp, c_int, c_int, ip, ip, dp, ip, c_int, c_int, up, up, dp, dp]
        L.or_adjoint_grad.restype = c_d
        L.or_probabilities.argtypes = [dp, c_int, ip, c_int, dp]
        L.or_collapse.argtypes = [dp, c_int, c_int, c_int, c_d]
        L.or_sample.argtypes = [dp, c_int, c_int, dp, up]
        L.or_cdf.argtypes = [dp, c_int, dp]
        L.or_sample.restype = c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _state(psi: np.ndarray) -> np.ndarray:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("oracle states are C-contiguous complex128 arrays")
    return psi


def _nq(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.size != (1 << n):
        raise ValueError("state length must be a power of two")
    return n


def _mat(m, dim) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(dim, dim))
    return m


def zero_state(n: int, x0: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x0] = 1.0
    return psi


def apply_1q(psi, q: int, U) -> None:
    psi = _state(psi)
    u = _mat(U, 2)
    lib().or_apply_1q(_dp(psi), _nq(psi), q, _dp(u))


def apply_controlled(psi, controls: Sequence[int], target: int, U) -> None:
    psi = _state(psi)
    c = np.ascontiguousarray(controls, dtype=np.int32)
    u = _mat(U, 2)
    lib().or_apply_controlled(_dp(psi), _nq(psi), _ip(c), len(c), target, _dp(u))


def apply_diag(psi, qubits: Sequence[int], d) -> None:
    psi = _state(psi)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    dd = np.ascontiguousarray(np.asarray(d, dtype=np.complex128).reshape(1 << len(q)))
    lib().or_apply_diag(_dp(psi), _nq(psi), _ip(q), len(q), _dp(dd))


def apply_dense(psi, qubits: Sequence[int], M) -> None:
    psi = _state(psi)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    m = _mat(M, 1 << len(q))
    lib().or_apply_dense(_dp(psi), _nq(psi), _ip(q), len(q), _dp(m))


def swap(psi, i: int, j: int) -> None:
    psi = _state(psi)
    lib().or_swap(_dp(psi), _nq(psi), i, j)


def fused_swap(psi, p: int, q: int, s: int) -> int:
    psi = _state(psi)
    r = lib().or_fused_swap(_dp(psi), _nq(psi), p, q, s)
    if r < 0:
        raise ValueError("fused_swap: ranges out of bounds or overlapping")
    return int(r)


def permute(psi, perm: Sequence[int]) -> np.ndarray:
    psi = _state(psi)
    p = np.ascontiguousarray(perm, dtype=np.int32)
    out = np.empty_like(psi)
    if lib().or_permute(_dp(psi), _dp(out), _nq(psi), _ip(p)) != 0:
        raise ValueError("not a permutation")
    return out


def gate_matrix(name: str, params: Sequence[float] = ()) -> np.ndarray:
    prm = np.zeros(3, dtype=np.float64)
    prm[: len(params)] = params
    out = np.zeros(32, dtype=np.float64)
    nq = lib().or_gate_matrix(_KIND[name], _dp(prm), _dp(out))
    if nq < 0:
        raise ValueError(name)
    d = 1 << nq
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


def _pack(circuit):
    g = len(circuit)
    kinds = np.zeros(max(g, 1), dtype=np.int32)
    qubits = np.zeros(2 * max(g, 1), dtype=np.int32)
    params = np.zeros(3 * max(g, 1), dtype=np.float64)
    pidx = np.full(max(g, 1), -1, dtype=np.int32)
    for i, gate in enumerate(circuit):
        kinds[i] = _KIND[gate.name]
        qubits[2 * i: 2 * i + len(gate.qubits)] = gate.qubits
        params[3 * i: 3 * i + len(gate.params)] = gate.params
        pidx[i] = gate.param_index
    return kinds, qubits, params, pidx


def run_circuit(psi, circuit) -> None:
    psi = _state(psi)
    kinds, qubits, params, _ = _pack(circuit)
    if lib().or_run_circuit(_dp(psi), _nq(psi), len(circuit), _ip(kinds), _ip(qubits), _dp(params)) != 0:
        raise ValueError("unknown gate kind")


def inner(a, b) -> complex:
    a, b = _state(a), _state(b)
    out = np.zeros(2)
    lib().or_inner(_dp(a), _dp(b), _nq(a), _dp(out))
    return complex(out[0], out[1])


def _terms(terms):
    xm = np.ascontiguousarray([t.xmask for t in terms], dtype=np.uint64)
    zm = np.ascontiguousarray([t.zmask for t in terms], dtype=np.uint64)
    cf = np.ascontiguousarray([t.coeff for t in terms], dtype=np.float64)
    return xm, zm, cf


def expect_pauli(psi, terms) -> float:
    psi = _state(psi)
    xm, zm, cf = _terms(terms)
    return float(lib().or_expect_pauli(_dp(psi), _nq(psi), len(terms), _up(xm), _up(zm), _dp(cf)))


def apply_pauli_sum(psi, terms) -> np.ndarray:
    psi = _state(psi)
    xm, zm, cf = _terms(terms)
    out = np.empty_like(psi)
    lib().or_apply_pauli_sum(_dp(psi), _dp(out), _nq(psi), len(terms), _up(xm), _up(zm), _dp(cf))
    return out


def adjoint_grad(psi0, circuit, nparam: int, terms):
    """Energy and gradient of <psi|H|psi> by the adjoint reverse sweep."""
    psi0 = _state(psi0)
    kinds, qubits, params, pidx = _pack(circuit)
    xm, zm, cf = _terms(terms)
    grad = np.zeros(max(nparam, 1), dtype=np.float64)
    e = lib().or_adjoint_grad(_dp(psi0), _nq(psi0), len(circuit), _ip(kinds), _ip(qubits), _dp(params),
                              _ip(pidx), nparam, len(terms), _up(xm), _up(zm), _dp(cf), _dp(grad))
    if np.isnan(e):
        raise ValueError("adjoint_grad: unsupported parameterised gate")
    return float(e), grad[:nparam]


def expectation_of_circuit(n: int, circuit, terms, x0: int = 0) -> float:
    psi = zero_state(n, x0)
    run_circuit(psi, circuit)
    return expect_pauli(psi, terms)


def probabilities(psi, qubits) -> np.ndarray:
    """Marginal Born-rule probabilities of the given qubits (bit i of the
    outcome index = qubits[i]), FP64 summed in index order."""
    psi = _state(psi)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    out = np.zeros(1 << len(q), dtype=np.float64)
    lib().or_probabilities(_dp(psi), _nq(psi), _ip(q), len(q), _dp(out))
    return out


def collapse(psi, q: int, outcome: int, p: float) -> None:
    """In place: the state after measuring qubit q with this outcome of
    probability p (other branch zeroed, kept one scaled by 1/sqrt(p))."""
    psi = _state(psi)
    lib().or_collapse(_dp(psi), _nq(psi), int(q), int(outcome), float(p))


def cdf(psi) -> np.ndarray:
    """Cumulative distribution in index order, F[x] = p_0 + ... + p_x, one
    running FP64 sum (oracle.cpp or_cdf)."""
    psi = _state(psi)
    out = np.empty(psi.size, dtype=np.float64)
    lib().or_cdf(_dp(psi), _nq(psi), _dp(out))
    return out


def sample(psi, u) -> np.ndarray:
    """Basis-state samples for the uniforms u: the smallest x with
    F[x] > u T (F = cdf(psi), T = F[-1]), or the largest x with p_x > 0 when
    rounding leaves none (oracle.cpp or_sample)."""
    psi = _state(psi)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(uu.size, dtype=np.uint64)
    r = lib().or_sample(_dp(psi), _nq(psi), uu.size, _dp(uu), _up(out))
    if r != 0:
        raise ValueError("sampling a state of zero norm")
    return out
