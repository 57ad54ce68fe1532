"""GPU parity of computational-basis measurement (§II-A) against the oracle.

* qs_probabilities: marginals of 1 to 6 qubits (bit i of the outcome =
  qubits[i]) within 1e-13 absolute of the oracle (FP64 sums in different
  orders), both dtypes.  The complex64 state's oracle input is its FP32
  values widened, so the squares are the same.
* qs_sample: every sample x is a valid inverse of the oracle's cumulative
  distribution F (a sequential FP64 sum in index order): p_x > 0 and
  F(x - 1) - eps <= u T < F(x) + eps, eps the rounding bound of the two
  sums; where u T is farther than eps from every boundary, x is the oracle's
  own sample.  Sizes from 1 qubit (fewer amplitudes than lanes) to many
  superchunks, states with zero amplitudes and zero runs, edge uniforms 0
  and 1 - 2^-53; bit-exact closed forms for dyadic and basis states.
* qs_measure: the outcome is the one its probabilities decide, the collapsed
  state equals the oracle's collapse and has norm 1.
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


def gpu_state(qs, psi, dtype):
    n = int(psi.size).bit_length() - 1
    s = qs.State(n, dtype)
    s.from_numpy(psi.astype(np.complex64 if dtype == "c64" else np.complex128))
    return s


def widened(psi, dtype):
    return psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi.copy()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,qubits", [(1, [0]), (5, [3]), (5, [4, 0]), (12, [0, 11, 5]), (12, [7, 2, 9, 1]),
                                      (17, [16, 3, 8, 0, 12]), (17, [1, 2, 3, 4, 5, 6]), (6, [5, 4, 3, 2, 1, 0])])
def test_probabilities_vs_oracle(qs, dtype, n, qubits):
    psi = W.random_state(n, 50 + n)
    s = gpu_state(qs, psi, dtype)
    got = s.probabilities(qubits)
    want = oracle.probabilities(widened(psi, dtype), qubits)
    assert np.max(np.abs(got - want)) <= 1e-13
    # the state is unchanged
    assert np.array_equal(s.to_numpy(), psi.astype(s.to_numpy().dtype))


def uniforms(count, seed):
    u = np.random.default_rng(seed).random(count)
    return np.concatenate([[0.0, 1.0 - 2.0 ** -53, 0.5], u])


def check_samples(psi, u, got, min_clear=0.5):
    """Validity of GPU samples against the oracle's CDF.

    eps bounds the difference between the two computations of a partial sum
    of the p_x, relative to T: the oracle's sequential FP64 sum errs by at
    most N 2^-53 T; the GPU's FP64 prefix of superchunk and chunk sums by at
    most N 2^-53 T as well, and its double-float sums (relative error about
    2^-41 after 32 x 32 x 32 additions, plus 2^-45 from splitting complex128
    values into float pairs) by less than 2^14 2^-53 T.
    """
    F = oracle.cdf(psi)
    N, T = F.size, F[-1]
    eps = (2 * N + 2 ** 14) * 2.0 ** -53 * T
    p = psi.real ** 2 + psi.imag ** 2
    x = got.astype(np.int64)
    assert np.all((x >= 0) & (x < N))
    assert np.all(p[x] > 0)
    t = u * T
    below = np.where(x > 0, F[np.maximum(x - 1, 0)], 0.0)
    assert np.all(below - eps <= t), np.max(below - eps - t)
    assert np.all(t < F[x] + eps), np.max(t - F[x] - eps)
    want = oracle.sample(psi, u).astype(np.int64)
    wbelow = np.where(want > 0, F[np.maximum(want - 1, 0)], 0.0)
    clear = (t > wbelow + eps) & (t < F[want] - eps)
    assert np.array_equal(x[clear], want[clear])
    assert clear.mean() >= min_clear, clear.mean()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 3, 5, 10, 11, 14, 18, 21])
def test_sample_valid_inverse_cdf(qs, dtype, n):
    psi = W.random_state(n, 60 + n)
    if n >= 3:
        psi[1::3] = 0  # zero amplitudes in every lane range
    if n >= 16:
        psi[(1 << 15):(3 << 15)] = 0  # two whole superchunks of zeros
    if n >= 3:
        psi /= np.linalg.norm(psi)
    s = gpu_state(qs, psi, dtype)
    u = uniforms(3000, 70 + n)
    check_samples(widened(psi, dtype), u, s.sample(u))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sample_24q_valid(qs, dtype):
    # many superchunks (2^9), a state made by a circuit
    n = 24
    s = qs.State(n, dtype)
    s.run(qs.Plan(qs.Circuit(W.brick(n, 4, 71)), n, dtype, mode=qs.PLAN_TILED))
    psi = s.to_numpy().astype(np.complex128)
    u = uniforms(20000, 72)
    check_samples(psi, u, s.sample(u))


def test_sample_sparse_tail(qs):
    # only the first and a middle amplitude are nonzero: uniforms whose
    # u T rounds to T must still land on the last nonzero amplitude
    n = 17
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 0.6
    psi[12345] = 0.8j
    s = gpu_state(qs, psi, "c128")
    u = np.array([0.0, 0.3, 0.3599999, 0.3600001, 0.5, 0.99, 1.0 - 2.0 ** -53])
    got = s.sample(u)
    assert np.array_equal(got, np.where(u < 0.36, 0, 12345).astype(np.uint64))
    check_samples(psi, u, got, min_clear=0.0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sample_closed_forms(qs, dtype):
    # uniform dyadic state: floor(u 2^n); basis state: x0 always
    n = 12
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=complex)
    u = uniforms(2000, 73)
    assert np.array_equal(gpu_state(qs, psi, dtype).sample(u), np.floor(u * (1 << n)).astype(np.uint64))
    x0 = 3001
    s = qs.State(n, dtype)
    s.set_basis(x0)
    assert np.all(s.sample(u) == x0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_measure_matches_oracle_collapse(qs, dtype):
    n = 10
    psi = W.random_state(n, 80)
    for q, u in ((0, 0.1), (4, 0.9), (9, 0.37), (6, 0.75)):
        start = widened(psi, dtype)
        p = oracle.probabilities(start, [q])
        if abs(u * p.sum() - p[0]) < 1e-9:
            continue  # too close to the boundary for the two sums to agree on the side
        s = gpu_state(qs, psi, dtype)
        o, prob = s.measure(q, u)
        assert o == (0 if u * p.sum() < p[0] else 1)
        assert abs(prob - p[o] / p.sum()) <= 1e-12
        want = start.copy()
        oracle.collapse(want, q, o, p[o])
        got = s.to_numpy().astype(np.complex128)
        tol = 1e-12 if dtype == "c128" else 4e-6 * np.max(np.abs(want))
        assert np.max(np.abs(got - want)) <= tol
        assert abs(np.vdot(got, got).real - 1.0) <= (1e-12 if dtype == "c128" else 1e-6)


def test_measure_ghz_and_errors(qs):
    n = 8
    s = qs.State(n, "c128")
    s.run(qs.Plan(qs.Circuit(W.ghz(n)), n, "c128", mode=qs.PLAN_UNFUSED))
    o, prob = s.measure(3, 0.2)
    assert o == 0 and abs(prob - 0.5) <= 1e-12
    want = np.zeros(1 << n)
    want[0] = 1.0
    assert np.max(np.abs(s.to_numpy() - want)) <= 1e-12
    # a second measurement of another qubit is certain
    assert s.measure(5, 0.999) == (0, 1.0)
    with pytest.raises(qs.QSError):
        s.measure(n, 0.5)
    with pytest.raises(qs.QSError):
        s.measure(0, 1.0)
    with pytest.raises(qs.QSError):
        s.probabilities([1, 1])
    with pytest.raises(qs.QSError):
        s.sample([0.5, -0.1])
    z = qs.State(n, "c64")
    z.from_numpy(np.zeros(1 << n, dtype=np.complex64))
    with pytest.raises(qs.QSError):
        z.sample([0.5])
