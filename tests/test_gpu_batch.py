"""Batched persistent execution against the oracle.

Mixed circuit sizes (single-tile and multi-pass circuits in one launch),
both dtypes, graph replay, runs on current contents, the autotuner, and the
bounded dependency wait (a test hook makes every wait demand tiles that
never arrive; the run must end with QS_ETIMEOUT and leave the GPU usable).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from fidelity import check_c64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs
    return qs


def circuits_for(sizes, seed):
    out = []
    for i, n in enumerate(sizes):
        if i % 3 == 0:
            out.append(W.hea(n, 3, seed + i)[0])
        elif i % 3 == 1:
            out.append(W.brick(n, 6, seed + i))
        else:
            out.append(W.qft(n) + W.qsb(n, seed + i, sets=1))
    return out


def check(got, want, dtype, gates=None):
    if dtype == "c128":
        assert np.max(np.abs(got - want)) <= 1e-12
    else:
        check_c64(got, want, gates=gates)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_matches_oracle(qs, dtype):
    sizes = [4, 9, 12, 13, 14, 15, 16, 10, 5, 14]
    circs = circuits_for(sizes, 100)
    b = qs.Batch(sizes, circs, dtype=dtype)
    b.run(init_zero=True)
    b.sync()
    for i, (n, c) in enumerate(zip(sizes, circs)):
        want = oracle.zero_state(n)
        oracle.run_circuit(want, c)
        check(b.state(i).cpu().numpy(), want, dtype, gates=len(c))
    st = b.stats()
    assert st["circuits"] == len(sizes) and st["passes"] >= len(sizes)
    # replay (graph) twice more: same result from |0>
    b.run(True).run(True)
    b.sync()
    assert b.stats()["graph"] == 1
    for i, (n, c) in enumerate(zip(sizes, circs)):
        want = oracle.zero_state(n)
        oracle.run_circuit(want, c)
        check(b.state(i).cpu().numpy(), want, dtype, gates=len(c))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_with_fused_circuits(qs, dtype):
    # circuits of at least 14 qubits run as fused tensor-core plans on side
    # streams (more of them than streams), the rest in the persistent
    # launch; every circuit against the oracle, from |0> and on current
    # contents, over graph replays
    sizes = [14, 9, 15, 16, 12, 14, 15, 16, 14, 15, 10, 16]
    circs = circuits_for(sizes, 300)
    b = qs.Batch(sizes, circs, dtype=dtype, fuse_min_qubits=14)
    st = b.stats()
    assert st["circuits"] == len(sizes)
    wants = []
    for n, c in zip(sizes, circs):
        w = oracle.zero_state(n)
        oracle.run_circuit(w, c)
        wants.append(w)
    for _ in range(2):
        b.run(init_zero=True)
        b.sync()
        for i, c in enumerate(circs):
            check(b.state(i).cpu().numpy(), wants[i], dtype, gates=len(c))
    assert b.stats()["graph"] == 1
    # every circuit fused (no persistent launch at all)
    big = [i for i, n in enumerate(sizes) if n >= 14]
    b2 = qs.Batch([sizes[i] for i in big], [circs[i] for i in big], dtype=dtype, fuse_min_qubits=14)
    b2.run(True)
    b2.sync()
    for j, i in enumerate(big):
        check(b2.state(j).cpu().numpy(), wants[i], dtype, gates=len(circs[i]))
    # on current contents: the inverse circuits take every state back to |0>
    inv = qs.Batch(sizes, [W.inverse(c) for c in circs], dtype=dtype, fuse_min_qubits=14)
    inv.buffer.copy_(b.buffer)
    inv.run(init_zero=False)
    inv.sync()
    for i, n in enumerate(sizes):
        check(inv.state(i).cpu().numpy(), oracle.zero_state(n), dtype, gates=2 * len(circs[i]))


def test_batch_on_current_contents(qs):
    # circuits then their inverses as a second batch acting on the results
    sizes = [6, 11, 15]
    circs = circuits_for(sizes, 200)
    fwd = qs.Batch(sizes, circs, dtype="c128")
    fwd.run(True)
    fwd.sync()
    inv = qs.Batch(sizes, [W.inverse(c) for c in circs], dtype="c128")
    inv.buffer.copy_(fwd.buffer)
    inv.run(init_zero=False)
    inv.sync()
    for i, n in enumerate(sizes):
        got = inv.state(i).cpu().numpy()
        assert abs(got[0] - 1) <= 1e-12 and np.max(np.abs(got[1:])) <= 1e-12


def test_batch_tile_options_and_autotune(qs):
    sizes = [8, 12, 14, 16]
    circs = circuits_for(sizes, 300)
    for opts in (dict(tile_qubits=11, slot_qubits=4), dict(tile_qubits=12, slot_qubits=3, groups_per_thread=2)):
        b = qs.Batch(sizes, circs, dtype="c64", **opts)
        b.run(True)
        b.sync()
        for i, (n, c) in enumerate(zip(sizes, circs)):
            want = oracle.zero_state(n)
            oracle.run_circuit(want, c)
            check(b.state(i).cpu().numpy(), want, "c64", gates=len(c))
    b = qs.Batch(sizes, circs, dtype="c64", autotune=True)
    assert b.tuned_ms is not None and b.tuned_ms > 0
    b.run(True)
    b.sync()
    want = oracle.zero_state(16)
    oracle.run_circuit(want, circs[3])
    check(b.state(3).cpu().numpy(), want, "c64", gates=len(circs[3]))


def test_batch_wait_times_out_cleanly(qs):
    sizes = [15, 16]  # multi-pass circuits: second passes wait on the first
    circs = circuits_for(sizes, 400)
    b = qs.Batch(sizes, circs, dtype="c64", reserved=(1,))
    b.run(True)
    with pytest.raises(qs.QSError) as ei:
        b.sync()
    assert ei.value.code == qs.QS_ETIMEOUT
    # the context still works
    s = qs.State(8, "c128")
    s.apply_1q(3, np.array([[0, 1], [1, 0]]))
    assert abs(s.to_numpy()[8] - 1) == 0
