"""The autotuners on the GPU.

qs_plan_autotune times dense blocks of k = 4, 5, 6 (complex128: 4, 5) and
tile shapes on the caller's state and returns the fastest; the plan it
picks must still match the oracle.  Results are cached under a hash of the
circuit, n, dtype and GPU: a second call returns at once with the same
answer, and a cache file carries the results to a fresh load.  The batch
tuner keys on the actual circuits, so two different batches of equal size
are tuned separately.
"""
import time

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


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_plan_autotune_picks_a_correct_plan_and_caches(qs, dtype, tmp_path):
    n = 18
    circ = W.brick(n, 20, 51)
    c = qs.Circuit(circ)
    cache = tmp_path / "tune.txt"
    qs.set_tune_cache(str(cache))
    s = qs.State(n, dtype)
    opts, ms = qs.autotune(c, s)
    assert ms > 0 and opts.mode in (qs.PLAN_FUSED, qs.PLAN_TILED)
    if opts.mode == qs.PLAN_FUSED:
        assert 4 <= opts.fuse_qubits <= (6 if dtype == "c64" else 5)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("qs-tune-v3 ") and " plan " in lines[0]
    # the chosen plan is correct
    want = oracle.zero_state(n)
    oracle.run_circuit(want, circ)
    s.set_basis(0)
    s.run(qs.Plan(c, n, dtype, **qs.plan_kwargs(opts)))
    got = s.to_numpy()
    if dtype == "c128":
        assert np.max(np.abs(got - want)) <= 1e-12
    else:
        check_c64(got, want, gates=len(circ))
    # cached in memory: the same answer at once, no timing runs
    t0 = time.perf_counter()
    opts2, ms2 = qs.autotune(c, s)
    assert time.perf_counter() - t0 < 0.05
    assert qs.plan_kwargs(opts2) == qs.plan_kwargs(opts) and ms2 == pytest.approx(ms)
    # and through the file after a reload
    qs.set_tune_cache(str(cache))
    t0 = time.perf_counter()
    opts3, ms3 = qs.autotune(c, s)
    assert time.perf_counter() - t0 < 0.05
    assert qs.plan_kwargs(opts3) == qs.plan_kwargs(opts) and ms3 == pytest.approx(ms, rel=1e-5)
    assert len(cache.read_text().splitlines()) == 1
    qs.set_tune_cache(None)


def test_batch_autotune_keys_on_the_circuits(qs, tmp_path):
    # equal count, sizes and gate totals, different angles: tuned apart
    cache = tmp_path / "tune.txt"
    qs.set_tune_cache(str(cache))
    sizes = [10, 12, 14]
    for seed in (1, 2):
        circs = [W.hea(n, 3, seed * 100 + i)[0] for i, n in enumerate(sizes)]
        b = qs.Batch(sizes, circs, dtype="c64", autotune=True)
        assert b.tuned_ms is not None and b.tuned_ms > 0
    lines = [x for x in cache.read_text().splitlines() if " batch " in x]
    assert len(lines) == 2 and lines[0].split()[1] != lines[1].split()[1]
    qs.set_tune_cache(None)
