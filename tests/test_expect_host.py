"""The Pauli expectation's pass planning, without a GPU.

qs_expect_pauli_passes returns how many reads of the whole state an
expectation makes: one per tile pass (groups of terms sharing an X/Y mask,
first fit into tiles of the 4 lowest qubits plus up to 9 higher ones, 8 for
complex128) plus one per group whose X/Y bits above qubit 3 exceed a tile.
The counts below follow from that rule by hand.
"""
import ctypes

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_16044_gb300 as qs
    return qs


def xs(qubits):
    return [W.PauliTerm(1.0, 1 << q, 0) for q in qubits]


def test_tfim_passes(qs):
    # Z-Z group plus single X on 30 qubits: complex64 tiles cover 13 qubits
    # (0..12, then 13..21, then 22..29 above the low four), complex128 12
    tf = W.tfim(30)
    assert qs.expect_pauli_passes(30, "c64", tf) == 3
    assert qs.expect_pauli_passes(30, "c128", tf) == 4


def test_tile_capacity_and_own_passes(qs):
    assert qs.expect_pauli_passes(13, "c64", xs(range(13))) == 1
    assert qs.expect_pauli_passes(13, "c128", xs(range(13))) == 2
    wide = [W.PauliTerm(0.5, ((1 << 10) - 1) << 4, 0)]  # X on 10 qubits above qubit 3
    assert qs.expect_pauli_passes(14, "c64", wide) == 1
    assert qs.expect_pauli_passes(14, "c64", wide + xs(range(4))) == 2
    # a state of 4 qubits holds no tile: every group reads the state itself
    assert qs.expect_pauli_passes(4, "c64", xs(range(4))) == 4


def test_argument_checks(qs):
    L = qs.lib()
    x = np.zeros(1, dtype=np.uint64)
    z = np.zeros(1, dtype=np.uint64)
    up = ctypes.POINTER(ctypes.c_uint64)
    out = ctypes.c_int()
    xp, zp = x.ctypes.data_as(up), z.ctypes.data_as(up)
    assert L.qs_expect_pauli_passes(0, qs.C64, 1, xp, zp, ctypes.byref(out)) == qs.QS_EINVAL
    assert L.qs_expect_pauli_passes(35, qs.C64, 1, xp, zp, ctypes.byref(out)) == qs.QS_EINVAL
    assert L.qs_expect_pauli_passes(10, 7, 1, xp, zp, ctypes.byref(out)) == qs.QS_EINVAL
    assert L.qs_expect_pauli_passes(10, qs.C64, 0, xp, zp, ctypes.byref(out)) == qs.QS_EINVAL
    assert L.qs_expect_pauli_passes(10, qs.C64, 1, xp, zp, None) == qs.QS_EINVAL
    x[0] = 1 << 10
    assert L.qs_expect_pauli_passes(10, qs.C64, 1, xp, zp, ctypes.byref(out)) == qs.QS_EINVAL
    assert "qubit >= n" in L.qs_last_error().decode()
    x[0] = 1 << 9
    assert L.qs_expect_pauli_passes(10, qs.C64, 1, xp, zp, ctypes.byref(out)) == qs.QS_OK
    assert out.value == 1


def test_small_states_and_mixed_groups(qs):
    # n = 5, 6: one tile covers the whole state (4 low qubits plus the rest),
    # so every group fitting it shares one pass, for both dtypes
    for n in (5, 6):
        terms = xs(range(n)) + [W.PauliTerm(1.0, 0, 3), W.PauliTerm(0.5, 0b11, 0b10)]
        assert qs.expect_pauli_passes(n, "c64", terms) == 1
        assert qs.expect_pauli_passes(n, "c128", terms) == 1
    # strings on a low and a high qubit share the tile of their high qubits;
    # high qubits 10..18 (9 of them) fill a complex64 tile, a tenth opens a
    # second pass, complex128 tiles hold 8
    terms = [W.PauliTerm(1.0, (1 << q) | 1, 0) for q in range(10, 19)]
    assert qs.expect_pauli_passes(24, "c64", terms) == 1
    assert qs.expect_pauli_passes(24, "c64", terms + [W.PauliTerm(1.0, 1 << 20, 0)]) == 2
    assert qs.expect_pauli_passes(24, "c128", terms) == 2
