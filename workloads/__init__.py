"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module holds no gate arithmetic: it only draws random numbers and lays
out circuits as lists of ``Gate(name, qubits, params)`` records.  Building a
gate's matrix from its name and angles, and applying it, is done separately
(and independently) by ``oracle/`` and by the CUDA library.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit counter advanced by
the golden-ratio increment and passed through the published 64-bit finaliser.
A uniform double in [0, 1) is taken from the top 53 bits.

Workload shapes follow the paper's synthetic benchmark circuits: the
Quantum Software Benchmark structure of §IV-F (a rotation layer on every
qubit followed by a nearest-neighbour CNOT layer), the RX-per-qubit sweep of
§IV-C and the Hadamard benchmark of §IV-D (eleven H gates on every qubit).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Iterator, List, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream.  ``next_u64`` returns the finalised counter."""

    GOLDEN = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass(frozen=True)
class Gate:
    """One circuit operation.

    ``name`` is one of: H X Y Z S T RX RY RZ P U3 CNOT CZ CP SWAP.
    ``qubits`` lists the qubits the gate acts on: for CNOT (control, target),
    for CZ/CP/SWAP the two qubits.  ``params`` are the angles in radians
    (RX/RY/RZ/P: one; U3: theta, phi, lambda; CP: phi).
    ``param_index`` names the trainable parameter this gate's single angle
    comes from (-1 for a fixed gate); used by the differentiation workloads.
    """

    name: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    param_index: int = -1


ONE_QUBIT = {"H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P", "U3"}
TWO_QUBIT = {"CNOT", "CZ", "CP", "SWAP"}
N_PARAMS = {"RX": 1, "RY": 1, "RZ": 1, "P": 1, "U3": 3, "CP": 1}


def validate(circuit: Sequence[Gate], n: int) -> None:
    for g in circuit:
        want = 1 if g.name in ONE_QUBIT else 2 if g.name in TWO_QUBIT else None
        if want is None:
            raise ValueError(f"unknown gate {g.name}")
        if len(g.qubits) != want or len(set(g.qubits)) != want:
            raise ValueError(f"bad qubits for {g}")
        if any(q < 0 or q >= n for q in g.qubits):
            raise ValueError(f"qubit out of range in {g}")
        if len(g.params) != N_PARAMS.get(g.name, 0):
            raise ValueError(f"bad params for {g}")


# ---------------------------------------------------------------------------
# Circuits
# ---------------------------------------------------------------------------

def brick(n: int, depth: int, seed: int) -> List[Gate]:
    """Brick random circuit: per layer l, U3 on every qubit (angles i.i.d.
    uniform in [0, 2*pi), drawn qubit 0..n-1, theta then phi then lambda),
    then CNOT(control i, target i+1) for i = l mod 2, l mod 2 + 2, ...
    while i + 1 <= n - 1.  Rotation layer + nearest-neighbour CNOT layer is
    the structure of the paper's QSB circuit (§IV-F)."""
    rng = SplitMix64(seed)
    out: List[Gate] = []
    two_pi = 2.0 * math.pi
    for layer in range(depth):
        for q in range(n):
            th = two_pi * rng.uniform()
            ph = two_pi * rng.uniform()
            la = two_pi * rng.uniform()
            out.append(Gate("U3", (q,), (th, ph, la)))
        i = layer % 2
        while i + 1 <= n - 1:
            out.append(Gate("CNOT", (i, i + 1)))
            i += 2
    return out


def qft(n: int) -> List[Gate]:
    """Quantum Fourier transform on n qubits, qubit n-1 the most significant:
    for j = n-1 .. 0: H(j), then CP(pi / 2**(j-k)) on (k, j) for
    k = j-1 .. 0; finally SWAP(i, n-1-i) for i < n/2."""
    out: List[Gate] = []
    for j in range(n - 1, -1, -1):
        out.append(Gate("H", (j,)))
        for k in range(j - 1, -1, -1):
            out.append(Gate("CP", (k, j), (math.pi / float(1 << (j - k)),)))
    for i in range(n // 2):
        out.append(Gate("SWAP", (i, n - 1 - i)))
    return out


def qsb(n: int, seed: int, sets: int = 10) -> List[Gate]:
    """Quantum Software Benchmark structure of §IV-F: ``sets`` repetitions of
    a rotation layer (RZ, RX, RZ with random angles on every qubit) and a CNOT
    layer (target i, control (i+1) mod n for 0 <= i < n), followed by one more
    rotation layer.  Angles uniform in [0, 2*pi)."""
    rng = SplitMix64(seed)
    two_pi = 2.0 * math.pi
    out: List[Gate] = []

    def rot():
        for q in range(n):
            out.append(Gate("RZ", (q,), (two_pi * rng.uniform(),)))
            out.append(Gate("RX", (q,), (two_pi * rng.uniform(),)))
            out.append(Gate("RZ", (q,), (two_pi * rng.uniform(),)))

    for _ in range(sets):
        rot()
        for i in range(n):
            out.append(Gate("CNOT", ((i + 1) % n, i)))
    rot()
    return out


def qv_like(n: int, depth: int, seed: int) -> List[Gate]:
    """Random two-qubit blocks on random pairs, shaped like the Quantum Volume
    model circuit of §IV-E: per layer a seeded random permutation p of the
    qubit labels (Fisher-Yates, j drawn as next_u64 mod (i + 1) for i from
    n - 1 down to 1) pairs them as (p[0], p[1]), (p[2], p[3]), ...; every
    pair (a, b) gets a generic two-qubit block written with named gates:
    U3 on a, U3 on b, CNOT(a, b), RZ on a, RY on b, CNOT(b, a), RY on b,
    CNOT(a, b), U3 on a, U3 on b (17 angles uniform in [0, 2*pi), in that
    gate order).  With odd n the last qubit of p idles."""
    rng = SplitMix64(seed)
    two_pi = 2.0 * math.pi
    out: List[Gate] = []

    def u3(q):
        out.append(Gate("U3", (q,), (two_pi * rng.uniform(), two_pi * rng.uniform(), two_pi * rng.uniform())))

    for _ in range(depth):
        p = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.next_u64() % (i + 1)
            p[i], p[j] = p[j], p[i]
        for i in range(0, n - 1, 2):
            a, b = p[i], p[i + 1]
            u3(a)
            u3(b)
            out.append(Gate("CNOT", (a, b)))
            out.append(Gate("RZ", (a,), (two_pi * rng.uniform(),)))
            out.append(Gate("RY", (b,), (two_pi * rng.uniform(),)))
            out.append(Gate("CNOT", (b, a)))
            out.append(Gate("RY", (b,), (two_pi * rng.uniform(),)))
            out.append(Gate("CNOT", (a, b)))
            u3(a)
            u3(b)
    return out


def hadamard_bench(n: int, reps: int = 11) -> List[Gate]:
    """Hadamard benchmark of §IV-D: ``reps`` H gates on every qubit."""
    return [Gate("H", (q,)) for _ in range(reps) for q in range(n)]


def ghz(n: int) -> List[Gate]:
    """H(0) then CNOT(i, i+1) for i = 0..n-2."""
    return [Gate("H", (0,))] + [Gate("CNOT", (i, i + 1)) for i in range(n - 1)]


def hea(n: int, layers: int, seed: int, first_param: int = 0) -> Tuple[List[Gate], np.ndarray]:
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, then
    RZ(theta) on every qubit, then CZ(i, i+1) for i = 0..n-2.  Angles uniform
    in [-pi, pi).  Returns the circuit and its parameter vector; each rotation
    carries its parameter index."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    theta: List[float] = []
    for _ in range(layers):
        for name in ("RY", "RZ"):
            for q in range(n):
                t = -math.pi + 2.0 * math.pi * rng.uniform()
                gates.append(Gate(name, (q,), (t,), first_param + len(theta)))
                theta.append(t)
        for i in range(n - 1):
            gates.append(Gate("CZ", (i, i + 1)))
    return gates, np.array(theta, dtype=np.float64)


def with_params(circuit: Sequence[Gate], theta: np.ndarray) -> List[Gate]:
    """Replace the angle of every parameterised gate by theta[param_index]."""
    out = []
    for g in circuit:
        if g.param_index >= 0:
            out.append(Gate(g.name, g.qubits, (float(theta[g.param_index]),), g.param_index))
        else:
            out.append(g)
    return out


def microbench(n: int, gate_class: str, target: int, seed: int, reps: int = 10) -> List[Gate]:
    """Per-gate-class microbenchmark on one target (the RX-per-qubit sweep of
    §IV-C, widened to four classes): ``reps`` copies of
    U3 (random angles) / RZ (random angle) / CNOT(control (t+1) mod n, target t)
    / CZ(t, (t+1) mod n)."""
    rng = SplitMix64(seed)
    two_pi = 2.0 * math.pi
    other = (target + 1) % n
    out = []
    for _ in range(reps):
        if gate_class == "U3":
            out.append(Gate("U3", (target,), (two_pi * rng.uniform(), two_pi * rng.uniform(), two_pi * rng.uniform())))
        elif gate_class == "RZ":
            out.append(Gate("RZ", (target,), (two_pi * rng.uniform(),)))
        elif gate_class == "CNOT":
            out.append(Gate("CNOT", (other, target)))
        elif gate_class == "CZ":
            out.append(Gate("CZ", (target, other)))
        else:
            raise ValueError(gate_class)
    return out


def inverse(circuit: Sequence[Gate]) -> List[Gate]:
    """The inverse circuit, expressed with named gates only (no arithmetic on
    matrices): reverse order and negate or permute angles per the standard
    identities U3(t,p,l)^-1 = U3(-t,-l,-p), R(t)^-1 = R(-t), P(t)^-1 = P(-t),
    S^-1 = P(-pi/2), T^-1 = P(-pi/4); H, X, Y, Z, CNOT, CZ, SWAP are
    self-inverse."""
    out = []
    for g in reversed(circuit):
        if g.name in ("H", "X", "Y", "Z", "CNOT", "CZ", "SWAP"):
            out.append(g)
        elif g.name in ("RX", "RY", "RZ", "P", "CP"):
            out.append(Gate(g.name, g.qubits, (-g.params[0],)))
        elif g.name == "U3":
            t, p, l = g.params
            out.append(Gate("U3", g.qubits, (-t, -l, -p)))
        elif g.name == "S":
            out.append(Gate("P", g.qubits, (-math.pi / 2,)))
        elif g.name == "T":
            out.append(Gate("P", g.qubits, (-math.pi / 4,)))
        else:
            raise ValueError(g.name)
    return out


# ---------------------------------------------------------------------------
# Observables
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class PauliTerm:
    """coeff * prod_q P_q with P_q = X where only xmask has bit q, Z where
    only zmask has bit q, Y where both have it, identity elsewhere."""

    coeff: float
    xmask: int
    zmask: int


def tfim(n: int, hx: float = 1.0) -> List[PauliTerm]:
    """Transverse-field Ising chain, open boundary:
    H = sum_{i=0}^{n-2} Z_i Z_{i+1} + hx * sum_{i=0}^{n-1} X_i."""
    terms = [PauliTerm(1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    terms += [PauliTerm(hx, 1 << i, 0) for i in range(n)]
    return terms


def random_paulis(n: int, count: int, seed: int) -> List[PauliTerm]:
    """Random Pauli strings with random coefficients in [-1, 1)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        x = rng.next_u64() & ((1 << n) - 1)
        z = rng.next_u64() & ((1 << n) - 1)
        out.append(PauliTerm(2.0 * rng.uniform() - 1.0, x, z))
    return out


# ---------------------------------------------------------------------------
# Random states and matrices for kernel-level parity
# ---------------------------------------------------------------------------

def random_state(n: int, seed: int, normalise: bool = True) -> np.ndarray:
    """Complex128 vector of 2**n entries, real and imaginary parts standard
    normal (numpy PCG64 seeded with ``seed``), optionally normalised."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    if normalise:
        v /= np.sqrt(np.vdot(v, v).real)
    return v.astype(np.complex128)


def random_matrix(dim: int, seed: int) -> np.ndarray:
    """dim x dim complex matrix with standard-normal entries (not unitary)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2 * dim)


def random_unitary(dim: int, seed: int) -> np.ndarray:
    """Haar-random unitary via QR of a complex Gaussian matrix with the
    phases of R's diagonal divided out (Mezzadri, Notices AMS 54, 2007)."""
    z = random_matrix(dim, seed) * np.sqrt(2 * dim)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_diag(dim: int, seed: int, unit: bool = True) -> np.ndarray:
    """Random diagonal: unit-modulus phases (default) or Gaussian entries."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if unit:
        return np.exp(1j * 2 * np.pi * rng.random(dim))
    return rng.standard_normal(dim) + 1j * rng.standard_normal(dim)


def random_qubits(n: int, k: int, seed: int) -> List[int]:
    """k distinct qubits out of n, in random order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(x) for x in rng.permutation(n)[:k]]


def random_perm(n: int, seed: int) -> List[int]:
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(x) for x in rng.permutation(n)]


def basis_index(n: int, seed: int) -> int:
    """A seeded basis-state index in [0, 2**n)."""
    return SplitMix64(seed).next_u64() % (1 << n)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> List[int]:
    """``count`` qubit counts uniform in [lo, hi]."""
    rng = SplitMix64(seed)
    return [lo + rng.next_u64() % (hi - lo + 1) for _ in range(count)]
