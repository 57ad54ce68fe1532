"""GPU parity of every gate / reduction entry point against the FP64 oracle.

Same seeded inputs on both sides (workloads module).  Tolerances:
  complex128: max |a_gpu - a_oracle| <= 1e-12 (absolute, unit-norm states).
  complex64:  FP32 arithmetic; a 2x2 (or 2^k x 2^k) complex mat-vec with
              FMA contraction rounds each output with relative error about
              (k + 2) * 2^-24 of the sum of |terms|, and the inputs (state and
              matrix) are themselves rounded to FP32: tolerance
              C64_TOL * max|a| with C64_TOL = 4e-6 for single gates.
Sizes run from 1 qubit (less than one CTA of work) to 16 qubits (many CTAs
and grid-stride iterations), so tails and multi-tile cases are covered.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

C128_TOL = 1e-12
C64_TOL = 4e-6


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2203_16044_gb300 as qs
    return qs


def gpu_state(qs, psi, dtype):
    n = int(psi.size).bit_length() - 1
    s = qs.State(n, dtype)
    s.from_numpy(psi.astype(np.complex64 if dtype == "c64" else np.complex128))
    return s


def check(got, want, dtype, scale=None):
    err = np.max(np.abs(got.astype(np.complex128) - want))
    if dtype == "c128":
        assert err <= C128_TOL, err
    else:
        ref = scale if scale is not None else max(np.max(np.abs(want)), 1e-30)
        assert err <= C64_TOL * ref, (err, ref)


def start(psi, dtype):
    """The oracle's input: for c64 the same FP32-rounded values the GPU gets."""
    if dtype == "c64":
        return psi.astype(np.complex64).astype(np.complex128)
    return psi.copy()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 6, 11, 16])
def test_apply_1q_every_target(qs, dtype, n):
    psi = W.random_state(n, 1000 + n)
    for q in range(n):
        U = W.random_unitary(2, 2000 + 17 * n + q)
        s = gpu_state(qs, psi, dtype)
        s.apply_1q(q, U)
        want = start(psi, dtype)
        oracle.apply_1q(want, q, U)
        check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,nc", [(2, 1), (5, 1), (9, 2), (12, 3), (14, 1)])
def test_apply_controlled(qs, dtype, n, nc):
    psi = W.random_state(n, 3000 + n)
    for seed in range(6):
        qsel = W.random_qubits(n, nc + 1, 3100 + 31 * n + seed)
        ctrl, t = qsel[:nc], qsel[nc]
        U = W.random_matrix(2, 3200 + seed)
        s = gpu_state(qs, psi, dtype)
        s.apply_controlled(ctrl, t, U)
        want = start(psi, dtype)
        oracle.apply_controlled(want, ctrl, t, U)
        check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_cnot_every_pair(qs, dtype):
    n = 7
    X = np.array([[0, 1], [1, 0]])
    psi = W.random_state(n, 4000)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            s = gpu_state(qs, psi, dtype)
            s.apply_controlled([c], t, X)
            want = start(psi, dtype)
            oracle.apply_controlled(want, [c], t, X)
            check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", [(1, 1), (4, 1), (6, 2), (10, 3), (13, 5), (15, 8)])
def test_apply_diag_general(qs, dtype, n, k):
    psi = W.random_state(n, 5000 + n)
    for seed in range(3):
        qsel = W.random_qubits(n, k, 5100 + 7 * n + seed)
        d = W.random_diag(1 << k, 5200 + seed, unit=(seed != 2))
        s = gpu_state(qs, psi, dtype)
        s.apply_diag(qsel, d)
        want = start(psi, dtype)
        oracle.apply_diag(want, qsel, d)
        check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", [(1, 1), (3, 2), (8, 2), (12, 3), (16, 1)])
def test_apply_diag_phase_on_ones(qs, dtype, n, k):
    # CZ / CP / Z-type: every entry 1 but the last (the sparse kernel)
    psi = W.random_state(n, 6000 + n)
    for seed in range(4):
        qsel = W.random_qubits(n, k, 6100 + 5 * n + seed)
        d = np.ones(1 << k, dtype=complex)
        d[-1] = np.exp(1j * (0.3 + seed))
        s = gpu_state(qs, psi, dtype)
        s.apply_diag(qsel, d)
        want = start(psi, dtype)
        oracle.apply_diag(want, qsel, d)
        check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", [(2, 2), (5, 3), (9, 4), (12, 5), (13, 6), (11, 1), (4, 4), (6, 6), (16, 4), (15, 6),
                                 (20, 5)])
def test_apply_fused(qs, dtype, n, k):
    # complex64 with k >= 4 runs on the tensor cores (3xTF32 split products):
    # ~2^-21 relative per product, inside C64_TOL for 2^k-term sums
    psi = W.random_state(n, 7000 + n)
    for seed in range(2):
        qsel = W.random_qubits(n, k, 7100 + n + seed)
        M = W.random_unitary(1 << k, 7200 + seed)
        s = gpu_state(qs, psi, dtype)
        s.apply_fused(qsel, M)
        want = start(psi, dtype)
        oracle.apply_dense(want, qsel, M)
        check(s.to_numpy(), want, dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [2, 4, 7, 12, 15])
def test_fused_swap(qs, dtype, n):
    psi = W.random_state(n, 8000 + n)
    cases = [(0, n // 2, n // 2), (n // 2, 0, n // 2), (0, 1, 1), (n - 2, 0, 1), (1, n - 1, 1)]
    for (p, q, sw) in cases:
        if sw < 1 or p + sw > n or q + sw > n or not (p + sw <= q or q + sw <= p):
            continue
        s = gpu_state(qs, psi, dtype)
        s.fused_swap(p, q, sw)
        want = start(psi, dtype)
        oracle.fused_swap(want, p, q, sw)
        # a permutation moves values exactly
        assert np.array_equal(s.to_numpy().astype(np.complex128), want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 3, 6, 10, 14])
def test_permute_qubits(qs, dtype, n):
    psi = W.random_state(n, 9000 + n)
    for seed in range(4):
        perm = W.random_perm(n, 9100 + seed)
        s = gpu_state(qs, psi, dtype)
        s.permute_qubits(perm)
        want = oracle.permute(start(psi, dtype), perm)
        assert np.array_equal(s.to_numpy().astype(np.complex128), want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 5, 12, 17])
def test_norm_and_inner(qs, dtype, n):
    a = W.random_state(n, 10000 + n, normalise=False)
    b = W.random_state(n, 10100 + n, normalise=False)
    sa, sb = gpu_state(qs, a, dtype), gpu_state(qs, b, dtype)
    a0, b0 = start(a, dtype), start(b, dtype)
    want_n = oracle.inner(a0, a0).real
    want_i = oracle.inner(a0, b0)
    # FP64 accumulation of the same (FP32-exact for c64) inputs
    assert abs(sa.norm2() - want_n) <= 1e-12 * want_n
    assert abs(sa.inner(sb) - want_i) <= 1e-12 * (1 << n)
    # a state with itself: the norm, exactly
    assert sa.inner(sa) == complex(sa.norm2(), 0.0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [2, 6, 11])
def test_expect_pauli(qs, dtype, n):
    psi = W.random_state(n, 11000 + n)
    terms = W.random_paulis(n, 40, 11100 + n) + W.tfim(n)
    s = gpu_state(qs, psi, dtype)
    want = oracle.expect_pauli(start(psi, dtype), terms)
    got = s.expect_pauli(terms)
    assert abs(got - want) <= EXPECT_TOL[dtype] * sum(abs(t.coeff) for t in terms), (got, want)


# qs_expect_pauli: complex128 exact products summed in FP64; complex64
# single-term and Z-class groups with FP32 products and per-tile FP32 sums
# (bound ~10 roundings of 2^-24 per pair sum, times 2 sum |a_x||a_y| <= 2
# for a unit-norm state), the other complex64 groups exact
EXPECT_TOL = {"c128": 1e-12, "c64": 4e-6}


def test_set_basis_and_alloc_via_abi(qs):
    import ctypes
    L = qs.lib()
    h = ctypes.c_void_p()
    assert L.qs_alloc(9, qs.C128, ctypes.byref(h)) == qs.QS_OK
    buf = np.zeros(1 << 9, dtype=np.complex128)
    assert L.qs_copy_to_host(h, buf.ctypes.data_as(ctypes.c_void_p)) == qs.QS_OK
    assert buf[0] == 1 and np.count_nonzero(buf) == 1
    assert L.qs_set_basis(h, 300) == qs.QS_OK
    assert L.qs_copy_to_host(h, buf.ctypes.data_as(ctypes.c_void_p)) == qs.QS_OK
    assert buf[300] == 1 and np.count_nonzero(buf) == 1
    assert L.qs_set_basis(h, 512) == qs.QS_EINVAL
    assert L.qs_free(h) == qs.QS_OK


def test_invalid_arguments_leave_state_unchanged(qs):
    psi = W.random_state(5, 12000)
    s = gpu_state(qs, psi, "c128")
    with pytest.raises(qs.QSError):
        s.apply_1q(5, np.eye(2))
    with pytest.raises(qs.QSError):
        s.apply_controlled([2], 2, np.eye(2))
    with pytest.raises(qs.QSError):
        s.apply_diag([1, 1], np.ones(4))
    with pytest.raises(qs.QSError):
        s.fused_swap(0, 1, 2)
    with pytest.raises(qs.QSError):
        s.permute_qubits([0, 0, 1, 2, 3])
    assert np.array_equal(s.to_numpy(), psi)


@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("n,qubits", [
    (9, None),            # fewer than 128 groups: 8-byte accesses
    (14, "with0"),        # qubit 0 in the block: 16-byte amplitude pairs
    (14, "without0"),     # qubit 0 outside: lane pairs exchange halves
    (16, "high"),         # the block on the highest qubits
    (13, "high"),         # ... with k = 6 exactly one 128-group tile
    (15, "low"),          # the block is qubits 0 .. k-1: staged row transposes
    (8, "low"),           # ... with fewer than 128 groups (16-byte pairs)
    (14, "window2"),      # a window of consecutive qubits from 2 (TMA boxes of 32 x 4 rows)
    (13, "window2"),      # ... one tile at k = 6
    (14, "window3"),      # ... from 3 (16 x 8 rows)
    (14, "window5"),      # ... from 5 (4 x 32 rows)
    (15, "window6"),      # ... from 6 (2 x 64 rows)
    (17, "window8"),      # ... from 8 (one run of 128 rows)
    (14, "window1"),      # ... from 1 (the tile's qubit 0, then the block, then the rest)
    (15, "tworuns"),      # two runs of block qubits: a 5-D box
    (16, "tworunsup"),    # ... the upper run ending at the top qubit (4 runs)
    (15, "zero1"),        # qubit 0 in the block alone: gathered
    (16, "zero2"),        # qubits 0, 1 in the block: the innermost box dimension, 16-byte pairs
    (16, "lowrun"),       # qubits 0..3 plus high ones: 128-byte swizzled pieces per line
])
def test_apply_fused_tensor_core_access_modes(qs, k, n, qubits):
    # complex64 k = 4, 5, 6 blocks run on tcgen05; each way a group's
    # amplitudes are gathered and scattered, against the oracle
    if qubits == "lowrun":
        qsel = [12, 0, 2, 1, 3, 13][:k]
    elif qubits == "zero1":
        qsel = [6, 0, 5, 7, 8, 9][:k]
    elif qubits == "zero2":
        qsel = [10, 1, 0, 9, 11, 12][:k]
    elif qubits == "tworuns":
        qsel = [9, 1, 10, 2, 11, 3][:k]
    elif qubits == "tworunsup":
        qsel = [15, 2, 14, 3, 13, 4][:k]
    elif qubits is None:
        qsel = [1, 3, 4, 6, 8, 2][:k]
    elif qubits == "with0":
        qsel = [7, 0, 3, 11, 5, 9][:k]
    elif qubits == "without0":
        qsel = [2, 9, 5, 12, 1, 7][:k]
    elif qubits == "low":
        qsel = [q for q in [2, 0, 3, 1, 5, 4] if q < k]
    elif qubits.startswith("window"):
        s0 = int(qubits[6:])
        qsel = [s0 + i for i in [3, 0, 5, 1, 4, 2] if i < k]
    else:
        qsel = list(range(n - 1, n - 1 - k, -1))
    psi = W.random_state(n, 7500 + n + k)
    M = W.random_unitary(1 << k, 7600 + k)
    s = gpu_state(qs, psi, "c64")
    s.apply_fused(qsel, M)
    want = start(psi, "c64")
    oracle.apply_dense(want, qsel, M)
    check(s.to_numpy(), want, "c64")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_apply_fused_random_sets(qs, dtype):
    # random qubit sets of 4..6 (complex128: 4, 5) qubits on 11..16 qubits:
    # every way a tile can move (rows, low-run pieces, windows, run boxes,
    # boxes with qubits 0 and 1, gathers) picked by the set's shape, against
    # the oracle; the sets are drawn so that each shape class occurs
    import bench
    rng = np.random.default_rng(424242)
    seen = set()

    class _P:  # step_kernel's view of a one-block plan
        def __init__(self, n, q):
            self.n, self.dtype, self._q = n, dtype, q

        def step_qubits(self, i):
            return self._q

    for trial in range(36):
        n = int(rng.integers(11, 17))
        k = int(rng.choice([4, 5, 6] if dtype == "c64" else [4, 5]))
        shape = trial % 6
        if shape == 0:    # low run plus high qubits
            a = int(rng.integers(3, k + 1))
            q = list(range(a)) + sorted(rng.choice(np.arange(a + 1, n), size=k - a, replace=False).tolist())
        elif shape == 1:  # a window
            s0 = int(rng.integers(0, n - k + 1))
            q = list(range(s0, s0 + k))
        elif shape == 2:  # qubits 0, 1 and others
            q = [0, 1] + sorted(rng.choice(np.arange(3, n), size=k - 2, replace=False).tolist())
        elif shape == 3:  # two runs
            s1 = int(rng.integers(1, n - k))
            a = int(rng.integers(1, k))
            s2 = int(rng.integers(s1 + a + 1, n - (k - a) + 1)) if s1 + a + 1 <= n - (k - a) else None
            q = list(range(s1, s1 + a)) + (list(range(s2, s2 + k - a)) if s2 is not None else
                                           sorted(rng.choice(np.arange(s1 + a + 1, n), size=k - a, replace=False).tolist()))
        else:             # scattered
            q = sorted(rng.choice(np.arange(n), size=k, replace=False).tolist())
        lab = bench.step_kernel(_P(n, sorted(q)), 0, "block")
        seen.add(lab.split("<")[0] + "," + (lab.split(",")[1] if "," in lab else "gather>"))
        psi = W.random_state(n, 9100 + trial)
        M = W.random_unitary(1 << k, 9200 + trial)
        perm = rng.permutation(k)
        qsel = [q[i] for i in perm]
        s = gpu_state(qs, psi, dtype)
        s.apply_fused(qsel, M)
        want = start(psi, dtype)
        oracle.apply_dense(want, qsel, M)
        check(s.to_numpy(), want, dtype)
    name = "k_fused_c128" if dtype == "c128" else "k_fused_umma_tma"
    assert {name + ",rows>", name + ",lowrun>", name + ",window>", name + ",box>"} <= seen, seen


def _block_sets(k, mode):
    # one qubit set per tensor-core access path: a window of consecutive
    # qubits (TMA boxes), qubits 0..k-1 (TMA rows), a gathered set
    return {"window": [4 + i for i in [2, 0, 3, 1, 5, 4] if i < k],
            "rows": [q for q in [2, 0, 3, 1, 5, 4] if q < k],
            "gathered": [1, 9, 4, 12, 6, 2][:k]}[mode]


def _group_norms(psi, qsel):
    # ||v_g|| of every group (the 2^k amplitudes sharing the bits outside
    # qsel), broadcast back to the amplitudes
    mask = 0
    for q in qsel:
        mask |= 1 << q
    gid = np.arange(psi.size, dtype=np.int64) & ~mask
    sums = np.bincount(gid, weights=np.abs(psi) ** 2, minlength=psi.size)
    return np.sqrt(sums[gid])


@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("mode", ["window", "rows", "gathered"])
def test_apply_fused_c64_non_unitary(qs, k, mode):
    # a non-unitary block takes no group-norm restore: every output against
    # the oracle, relative to its own sum of term magnitudes (|M| |v|)_i,
    # plus the split's absolute floor of 2^-20 of the group norm times max |M|
    n = 14
    qsel = _block_sets(k, mode)
    psi = W.random_state(n, 7700 + k)
    M = W.random_matrix(1 << k, 7710 + k) * 1.7  # entries ~ N(0, 1.7^2 / 2^(k+1)) (re, im)
    s = gpu_state(qs, psi, "c64")
    s.apply_fused(qsel, M)
    v = start(psi, "c64")
    want = v.copy()
    oracle.apply_dense(want, qsel, M)
    mag = np.abs(v).astype(np.complex128)
    oracle.apply_dense(mag, qsel, np.abs(M).astype(np.complex128))
    bound = 4e-6 * mag.real + 2.0 ** -20 * _group_norms(v, qsel) * np.max(np.abs(M))
    err = np.abs(s.to_numpy().astype(np.complex128) - want)
    assert np.all(err <= bound), float(np.max(err / bound))
    # the norm is not restored: it changes as M dictates
    assert abs(np.vdot(want, want).real - 1.0) > 1e-3


@pytest.mark.parametrize("k", [4, 5, 6])
@pytest.mark.parametrize("mode", ["window", "rows", "gathered"])
def test_apply_fused_c64_dynamic_range(qs, k, mode):
    # groups whose amplitudes span 2^-20 of dynamic range (and whose norms
    # span 2^-30 across the state): the power-of-two row scaling keeps every
    # output within 2^-20 of its group's norm (unitary M: the group norm is
    # kept), compared element by element
    n = 14
    qsel = _block_sets(k, mode)
    psi = W.random_state(n, 7800 + k)
    x = np.arange(psi.size, dtype=np.int64)
    r = np.zeros(psi.size, dtype=np.int64)
    for i, q in enumerate(qsel):
        r |= ((x >> q) & 1) << i
    grp = x & ~sum(1 << q for q in qsel)
    psi = psi * 2.0 ** (-20.0 * r / ((1 << k) - 1)) * 2.0 ** (-(grp % 31).astype(np.float64))
    M = W.random_unitary(1 << k, 7810 + k)
    s = gpu_state(qs, psi, "c64")
    s.apply_fused(qsel, M)
    v = start(psi, "c64")
    want = v.copy()
    oracle.apply_dense(want, qsel, M)
    err = np.abs(s.to_numpy().astype(np.complex128) - want)
    gn = _group_norms(v, qsel)
    assert np.all(err <= 2.0 ** -20 * gn), float(np.max(err / gn))


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("n,qubits", [
    (9, None),            # fewer than 128 groups: gathered, a partial tile
    (14, "gathered"),     # a set spanning more than k qubits: per-thread gathers
    (15, "low"),          # qubits 0 .. k-1: 2-D TMA boxes in, TMA stores out
    (11, "low"),          # ... exactly one or a few tiles
    (14, "window1"),      # a window from qubit 1: one 3-D TMA box per tile
    (14, "window2"),
    (14, "window3"),
    (15, "window6"),
    (17, "window8"),      # ... from 8 (runs of 128 rows)
    (16, "high"),         # the block on the highest qubits
    (15, "tworuns"),      # two runs of block qubits: a 5-D box
    (15, "zero1"),        # qubit 0 in the block alone: gathered
    (16, "zero2"),        # qubits 0, 1 in the block: the innermost box dimension
    (15, "lowrun"),       # qubits 0..2 plus high ones: 128-byte swizzled pieces per line
])
def test_apply_fused_c128_tensor_core_access_modes(qs, k, n, qubits):
    # complex128 k = 4, 5 blocks run on tcgen05 with FP64 operands split into
    # 9-bit integer digits: every output against the oracle within 1e-12 and
    # within 2^-36 of its group's norm
    if qubits == "tworuns":
        qsel = [9, 1, 10, 2, 11][:k]
    elif qubits == "lowrun":
        qsel = [11, 0, 2, 1, 12][:k]
    elif qubits == "zero1":
        qsel = [6, 0, 5, 7, 8][:k]
    elif qubits == "zero2":
        qsel = [10, 1, 0, 9, 11][:k]
    elif qubits is None:
        qsel = [1, 3, 4, 6, 8][:k]
    elif qubits == "gathered":
        qsel = [2, 9, 5, 12, 1][:k]
    elif qubits == "low":
        qsel = [q for q in [2, 0, 3, 1, 4] if q < k]
    elif qubits.startswith("window"):
        s0 = int(qubits[6:])
        qsel = [s0 + i for i in [3, 0, 1, 4, 2] if i < k]
    else:
        qsel = list(range(n - 1, n - 1 - k, -1))
    psi = W.random_state(n, 7900 + n + k)
    M = W.random_unitary(1 << k, 7910 + k)
    s = gpu_state(qs, psi, "c128")
    s.apply_fused(qsel, M)
    want = psi.copy()
    oracle.apply_dense(want, qsel, M)
    err = np.abs(s.to_numpy() - want)
    assert np.max(err) <= C128_TOL, float(np.max(err))
    gn = _group_norms(psi, qsel)
    assert np.all(err <= 2.0 ** -36 * gn), float(np.max(err / gn))


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("mode", ["window", "rows", "gathered"])
def test_apply_fused_c128_dynamic_range_and_non_unitary(qs, k, mode):
    # groups spanning 2^-40 inside and 2^-60 across the state, some groups
    # entirely zero, and a non-unitary matrix with entries up to ~4: the
    # per-group fixed-point grid keeps every output within 2^-36 of its
    # group's norm times max |M|
    n = 14
    qsel = _block_sets(k, mode)
    psi = W.random_state(n, 7950 + k)
    x = np.arange(psi.size, dtype=np.int64)
    r = np.zeros(psi.size, dtype=np.int64)
    for i, q in enumerate(qsel):
        r |= ((x >> q) & 1) << i
    grp = x & ~sum(1 << q for q in qsel)
    psi = psi * 2.0 ** (-40.0 * r / ((1 << k) - 1)) * 2.0 ** (-((grp * 7) % 61).astype(np.float64))
    psi[(grp % 13) == 0] = 0
    M = W.random_matrix(1 << k, 7960 + k) * 4.0
    s = gpu_state(qs, psi, "c128")
    s.apply_fused(qsel, M)
    want = psi.copy()
    oracle.apply_dense(want, qsel, M)
    err = np.abs(s.to_numpy() - want)
    gn = _group_norms(psi, qsel)
    assert np.all(err <= 2.0 ** -36 * gn * np.max(np.abs(M))), float(np.max(err / np.maximum(gn, 1e-300)))
    assert np.all(s.to_numpy()[gn == 0] == 0)


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("mode", ["window", "rows", "gathered"])
def test_c128_plan_blocks_in_double_float_storage(qs, k, mode):
    # inside a complex128 plan the tensor-core blocks read and write the
    # double-float storage the plan switches to (digits formed by FP32
    # rounding, outputs left as float pairs): one block of gates on the
    # set, on a state whose groups span 2^-20 inside and down to 2^-89
    # across (rows below 2^-85 take the two-factor scaling), some groups
    # zero.  Every output within 2^-36 of its group's norm where the group's
    # values stay above 2^-80; below that the storage itself holds values to
    # float precision (the low float's last bit would leave FP32's normal
    # range), so there within 2^-22; zero groups stay zero
    n = 14
    qsel = sorted(_block_sets(k, mode))
    circ = []
    for layer in range(3):
        for q in qsel:
            circ.append(W.Gate("U3", (q,), tuple(0.3 + 0.7 * i + 0.11 * q + layer for i in range(3))))
        for a, b in zip(qsel[layer % 2::2], qsel[layer % 2 + 1::2]):
            circ.append(W.Gate("CNOT", (a, b)))
    p = qs.Plan(qs.Circuit(circ), n, "c128", mode=qs.PLAN_FUSED, fuse_qubits=k)
    assert [kind for kind, _ in p.step_info()] == ["block"] and sorted(p.step_qubits(0)) == qsel
    psi = W.random_state(n, 7970 + k)
    x = np.arange(psi.size, dtype=np.int64)
    r = np.zeros(psi.size, dtype=np.int64)
    for i, q in enumerate(qsel):
        r |= ((x >> q) & 1) << i
    grp = x & ~sum(1 << q for q in qsel)
    psi = psi * 2.0 ** (-20.0 * r / ((1 << k) - 1)) * 2.0 ** (-((grp * 7) % 90).astype(np.float64))
    psi[(grp % 13) == 0] = 0
    s = gpu_state(qs, psi, "c128")
    s.run(p)
    s.sync()
    want = psi.copy()
    oracle.run_circuit(want, circ)
    got = s.to_numpy()
    err = np.abs(got - want)
    gn = _group_norms(psi, qsel)
    tol = np.where(gn >= 2.0 ** -59, 2.0 ** -36, 2.0 ** -22) * gn
    assert np.all(err <= tol), float(np.max(err / np.maximum(tol, 1e-300)))
    assert np.any((gn > 0) & (gn < 2.0 ** -85))  # the two-factor scaling ran
    assert np.all(got[gn == 0] == 0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [5, 9, 14, 21])
def test_expect_pauli_tile_passes(qs, dtype, n):
    # groups whose X/Y bits fit a tile (the 4 lowest qubits plus up to 9, or
    # 8 for complex128, higher ones) share tile-resident passes: the
    # transverse-field Ising chain (one Z-only group, n single-X groups),
    # strings with X on a low and a high qubit, many Z-only and Y terms in
    # one group, and strings spanning too many high qubits for any tile
    psi = W.random_state(n, 11500 + n)
    terms = list(W.tfim(n))
    rng = np.random.default_rng(n)
    for _ in range(12):
        q = rng.choice(n, size=min(2, n), replace=False)
        x = int(sum(1 << int(v) for v in q))
        z = x if rng.random() < 0.5 else int(rng.integers(0, 1 << n))
        terms.append(W.PauliTerm(float(rng.normal()), x, z))
    for _ in range(20):  # one big diagonal group
        terms.append(W.PauliTerm(float(rng.normal()), 0, int(rng.integers(0, 1 << n))))
    if n >= 15:
        terms.append(W.PauliTerm(0.7, (1 << n) - 1 - 7, 5))  # X on every high qubit: a pass of its own
    s = gpu_state(qs, psi, dtype)
    want = oracle.expect_pauli(start(psi, dtype), terms)
    got = s.expect_pauli(terms)
    assert abs(got - want) <= EXPECT_TOL[dtype] * sum(abs(t.coeff) for t in terms), (got, want)
    # the state is unchanged
    assert np.array_equal(s.to_numpy(), psi.astype(s.to_numpy().dtype))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [6, 7, 13, 20, 22])
@pytest.mark.parametrize("kind", ["zz_classes", "zz_split", "xy_stages", "scattered"])
def test_expect_pauli_stage_and_class_layouts(qs, dtype, n, kind):
    # complex64 tile passes in their several layouts: a one-group
    # Hamiltonian of Z-Z classes at distances 1..7 with their own weights
    # (row evaluation), single-qubit X and Y terms on every qubit (register
    # stages, 16-byte pair reads where qubit 0 is a stage bit), and X terms
    # on high qubits far enough apart that the tile is no single TMA box
    # (per-thread copies); 6 qubits: tiles below the TMA size.  zz_split:
    # more two-Z terms than one group holds (64), so the diagonal terms form
    # several class groups in one pass, plus single-X terms.  22 qubits:
    # 512 complex64 tiles of 2^13, so CTAs run several tiles each (the
    # double-buffered copies reuse their buffers)
    rng = np.random.default_rng(1000 * n + len(kind))
    terms = []
    if kind == "zz_split":
        for d in range(1, 9):
            for i in range(n - d):
                terms.append(W.PauliTerm(0.1 * d - 0.35, 0, (1 << i) | (1 << (i + d))))
        terms += [W.PauliTerm(float(rng.normal()), 1 << q, 0) for q in range(0, n, 3)]
    elif kind == "zz_classes":
        for d in (1, 2, 3, 5, 7):
            w = float(rng.normal())
            for i in range(n - d):
                if rng.random() < 0.7:
                    terms.append(W.PauliTerm(w, 0, (1 << i) | (1 << (i + d))))
    elif kind == "xy_stages":
        for q in range(n):
            x = 1 << q
            terms.append(W.PauliTerm(float(rng.normal()), x, x if rng.random() < 0.4 else 0))
    else:
        for q in range(5, n, 2):
            terms.append(W.PauliTerm(float(rng.normal()), 1 << q, 0))
        terms.append(W.PauliTerm(0.25, 0, (1 << n) - 1))
    psi = W.random_state(n, 12000 + 10 * n + len(kind))
    s = gpu_state(qs, psi, dtype)
    want = oracle.expect_pauli(start(psi, dtype), terms)
    got = s.expect_pauli(terms)
    assert abs(got - want) <= EXPECT_TOL[dtype] * sum(abs(t.coeff) for t in terms), (got, want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_copy_from_host_async_then_plan(qs, dtype):
    # the queued copy lands before work queued behind it on the state's
    # stream: a plan run right after the call sees the copied state, bit for
    # bit the same as after the synchronous copy
    import torch
    n = 14
    psi = W.random_state(n, 77).astype(np.complex64 if dtype == "c64" else np.complex128)
    host = torch.from_numpy(psi.copy()).pin_memory()
    circ = qs.Circuit(W.brick(n, 6, 2))
    a = qs.State(n, dtype).copy_from_host_async(host.data_ptr())
    p = qs.Plan(circ, n, dtype, mode=qs.PLAN_FUSED, fuse_qubits=6 if dtype == "c64" else 5)
    a.run(p)
    b = qs.State(n, dtype).from_numpy(psi)
    b.run(p)
    assert np.array_equal(a.to_numpy(), b.to_numpy())
