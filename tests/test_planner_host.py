"""The fusion planner's host arithmetic, without a GPU.

A QS_PLAN_FUSED plan replayed block by block with the oracle (apply_dense of
each block's matrix on its qubits, qs_plan_step_matrix / qs_plan_step_qubits)
must equal the circuit run gate by gate by the oracle.  This pins the
planner's block products (each absorbed gate multiplied onto the rows of the
running product, CNOT / SWAP / CZ / CP as row moves and scalings), the
widening of complex64 blocks with idle qubits, and the gate order across
blocks, independently of the kernels that later apply the blocks.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def qs():
    import paper_2203_16044_gb300 as qs
    return qs


def every_kind(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(60):
        name = ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "P", "U3", "CNOT", "CZ", "CP", "SWAP"][i % 15]
        prm = tuple(float(v) for v in rng.uniform(-3, 3, W.N_PARAMS.get(name, 0)))
        nq = 1 if name in W.ONE_QUBIT else 2
        out.append(W.Gate(name, tuple(int(v) for v in rng.permutation(n)[:nq]), prm))
    return out


CIRCUITS = [
    ("brick", 9, lambda: W.brick(9, 10, 1)),
    ("qft", 8, lambda: W.qft(8)),
    ("qsb", 8, lambda: W.qsb(8, 3, sets=3)),
    ("qv", 9, lambda: W.qv_like(9, 4, 2)),
    ("hea", 8, lambda: W.hea(8, 3, 4)[0]),
    ("every_kind", 7, lambda: every_kind(7, 5)),
]


@pytest.mark.parametrize("search", [1, 0])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("name,n,make", CIRCUITS, ids=[c[0] for c in CIRCUITS])
def test_fused_plan_replays_circuit(qs, dtype, k, name, n, make, search):
    circ = make()
    p = qs.Plan(qs.Circuit(circ), n, dtype, mode=qs.PLAN_FUSED, fuse_qubits=k, search=search)
    psi = W.random_state(n, 100 + n + k)
    got = psi.copy()
    for i, (kind, _) in enumerate(p.step_info()):
        assert kind == "block", kind
        q = p.step_qubits(i)
        M = p.step_matrix(i)
        assert M.shape == (1 << len(q), 1 << len(q)) and len(q) <= k + (3 if dtype == "c64" else 0)
        oracle.apply_dense(got, q, M)
    want = psi.copy()
    oracle.run_circuit(want, circ)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_block_order_search(qs, dtype):
    # a wider search never gives more passes than the greedy order (the
    # planner keeps the greedy schedule when it is cheaper), and on brick
    # circuits it gives fewer; every gate is still applied exactly once (the
    # replay test above checks the products)
    fewer = 0
    for n, circ in ((16, W.brick(16, 24, 6)), (14, W.qft(14)), (15, W.qsb(15, 2, sets=4)), (14, W.qv_like(14, 6, 1))):
        c = qs.Circuit(circ)
        passes = [qs.Plan(c, n, dtype, mode=qs.PLAN_FUSED, fuse_qubits=6, search=s).stats()["passes"] for s in (1, 4, 16)]
        assert passes[1] <= passes[0] and passes[2] <= passes[0], passes
        fewer += passes[2] < passes[0]
    assert fewer >= 1
    with pytest.raises(RuntimeError):
        qs.Plan(qs.Circuit(W.brick(8, 2, 1)), 8, dtype, mode=qs.PLAN_FUSED, fuse_qubits=5, search=257)


def test_wide_search_is_deterministic(qs):
    # widths of 16 and more expand the beam's states on host threads; the
    # merge runs in state order, so repeated builds give the same blocks,
    # and the width-64 plan of a brick circuit is no longer than width 16's
    circ = W.brick(20, 30, 6)
    c = qs.Circuit(circ)

    def blocks(search):
        p = qs.Plan(c, 20, "c64", mode=qs.PLAN_FUSED, fuse_qubits=6, search=search)
        return [tuple(sorted(p.step_qubits(i))) for i in range(p.stats()["passes"])]

    first = blocks(64)
    for _ in range(3):
        assert blocks(64) == first
    assert len(first) <= len(blocks(16))
    assert blocks(0) == first  # the default width is 64


def test_plan_kwargs_round_trip(qs):
    # the options an autotuner returns build a plan again (batch-only fields
    # such as fuse_min_qubits are left out)
    o = qs.PlanOpts(mode=qs.PLAN_FUSED, fuse_qubits=6, search=4, fuse_min_qubits=18)
    kw = qs.plan_kwargs(o)
    assert "fuse_min_qubits" not in kw and kw["fuse_qubits"] == 6 and kw["search"] == 4
    circ = W.brick(10, 4, 1)
    p = qs.Plan(qs.Circuit(circ), 10, "c64", **kw)
    assert p.stats()["gates"] == len(circ) and p.stats()["passes"] >= 1


def test_step_matrix_errors(qs):
    p = qs.Plan(qs.Circuit(W.brick(6, 2, 1)), 6, "c64", mode=qs.PLAN_UNFUSED)
    with pytest.raises(qs.QSError):
        p.step_matrix(0)  # a gate step, not a block
    p = qs.Plan(qs.Circuit(W.brick(6, 2, 1)), 6, "c64", mode=qs.PLAN_FUSED, fuse_qubits=4)
    with pytest.raises(qs.QSError):
        p.step_matrix(p.stats()["passes"])


ROUTED = [("qsb", 14, lambda: W.qsb(14, 3, sets=2)), ("brick", 15, lambda: W.brick(15, 8, 4)),
          ("qv", 14, lambda: W.qv_like(14, 4, 5)), ("hadamard", 13, lambda: W.hadamard_bench(13))]


def _compose_exchanges(p, n):
    # where each physical bit position ends up after all exchange passes
    pos = list(range(n))
    passes = []
    for i, (kind, b) in enumerate(p.step_info()):
        if kind != "swap":
            continue
        q = p.step_qubits(i)
        pairs = list(zip(q[0::2], q[1::2]))
        flat = [x for pr in pairs for x in pr]
        assert len(set(flat)) == len(flat), "pairs of one pass must be disjoint"
        assert all(0 <= x < n for x in flat)
        s = len(pairs)
        N = 2.0 ** n
        assert b == pytest.approx(2 * N * 8 * (1 - 2.0 ** -s))  # complex64 plans here
        passes.append(pairs)
        for a_, b_ in pairs:
            pos[a_], pos[b_] = pos[b_], pos[a_]
    return pos, passes


@pytest.mark.parametrize("name,n,make", ROUTED, ids=[r[0] for r in ROUTED])
@pytest.mark.parametrize("mode", ["swap", "permute"])
def test_routed_plans_end_in_logical_order(qs, name, n, make, mode):
    # the swap-insertion and fused-permutation policies (§III-D): every
    # exchange pass has disjoint pairs and the fused-swap traffic
    # 2 N S (1 - 2^-s); without SWAP gates in the circuit the passes compose
    # to the identity (the state ends in logical order); the tile passes
    # hold only the tile_qubits lowest qubits
    circ = make()
    m = 6
    md = qs.PLAN_SWAP if mode == "swap" else qs.PLAN_PERMUTE
    p = qs.Plan(qs.Circuit(circ), n, "c64", mode=md, tile_qubits=m)
    pos, passes = _compose_exchanges(p, n)
    assert pos == list(range(n))
    assert passes, "a circuit on more than the tile's qubits needs exchanges"
    if mode == "swap":
        # one pair per pass except the final return to logical order
        assert sum(len(x) == 1 for x in passes) >= len(passes) - 2
    assert p.stats()["gates"] == len(circ)


def test_fused_permutation_moves_less_than_swaps(qs):
    # on the QSB circuit the fused swaps need fewer exchange passes and fewer
    # bytes than one swap per remote target (§III-D)
    n, m = 16, 8
    circ = W.qsb(n, 9, sets=3)
    res = {}
    for mode, md in (("swap", qs.PLAN_SWAP), ("permute", qs.PLAN_PERMUTE)):
        p = qs.Plan(qs.Circuit(circ), n, "c64", mode=md, tile_qubits=m)
        ex = [b for k, b in p.step_info() if k == "swap"]
        res[mode] = (len(ex), sum(ex), p.stats()["passes"])
    assert res["permute"][0] < res["swap"][0]
    assert res["permute"][1] < res["swap"][1]
    assert res["permute"][2] < res["swap"][2]


def test_routed_qft_swaps_are_relabellings(qs):
    # SWAP gates of the circuit cost no pass: the exchanges compose to the
    # bit reversal that the QFT's final swaps perform
    n = 12
    p = qs.Plan(qs.Circuit(W.qft(n)), n, "c64", mode=qs.PLAN_PERMUTE, tile_qubits=6)
    pos, _ = _compose_exchanges(p, n)
    assert pos == [n - 1 - q for q in range(n)]


def test_circuit_hash_keys_the_tuner(qs, tmp_path):
    # the autotuner's circuit key: equal for equal gate lists, different when
    # any angle bit, qubit, n or dtype differs (no GPU needed)
    a = W.brick(10, 3, 1)
    h = qs.circuit_hash(qs.Circuit(a), 10, "c64")
    assert h == qs.circuit_hash(qs.Circuit(W.brick(10, 3, 1)), 10, "c64")
    b = list(a)
    g = b[5]
    b[5] = W.Gate(g.name, g.qubits, (g.params[0] + 2.0 ** -40,) + tuple(g.params[1:]), g.param_index)
    assert qs.circuit_hash(qs.Circuit(b), 10, "c64") != h
    assert qs.circuit_hash(qs.Circuit(a), 11, "c64") != h
    assert qs.circuit_hash(qs.Circuit(a), 10, "c128") != h
    assert qs.circuit_hash(qs.Circuit(W.brick(10, 3, 2)), 10, "c64") != h
    # cache files: absent, well formed, garbage -- all accepted
    qs.set_tune_cache(str(tmp_path / "none.txt"))
    f = tmp_path / "c.txt"
    f.write_text("qs-tune-v3 0123456789abcdef plan 2 0 0 0 0 0 6 0 0 1.5\nnot a cache line\n")
    qs.set_tune_cache(str(f))
    qs.set_tune_cache(None)
