"""The paper's distributed scheme (§III-B global-qubit operations, §III-D
fused swap) emulated on CPU ranks (gloo, 127.0.0.1): oracle/sharded.py.

* The 4-qubit worked example of §III-D (Hadamard and RX on every qubit, the
  two higher qubits global, complex double): the bytes actually sent between
  the four ranks are the paper's 1,024 (gates on global qubits), 512 (swap
  gates) and 384 (fused swaps), tests/golden/fused_swap_traffic.json.
* Brick and QV-shaped circuits on 2 and 4 ranks: the gathered state equals
  the single-process oracle's bit for bit (the ranks run the same per-pair
  arithmetic), and every fused swap of s qubits sends 2^(n+4) (1 - 2^-s)
  bytes over all ranks.
* Double buffering of the fused-swap exchange (§III-E): the same bytes and
  the same state.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def example_circuit():
    import workloads as W
    out = []
    for q in range(4):
        out.append(W.Gate("H", (q,)))
        out.append(W.Gate("RX", (q,), (0.3 + 0.2 * q,)))
    return out


def _worker(rank, world, port, q, job):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import workloads as W
        from oracle.sharded import ShardedState
        res = {}
        if job == "example":
            for policy in ("direct", "swap", "fused"):
                st = ShardedState(4)
                for g in example_circuit():
                    st.apply(g, policy)
                st.restore()
                res[policy] = (st.total_sent(), st.gather())
        elif job[0] == "buffered":
            _, n, circ = job
            for chunks in (1, 4):
                st = ShardedState(n, chunks=chunks)
                for g in circ:
                    st.apply(g, "fused")
                st.restore()
                res[chunks] = (st.total_sent(), st.gather(), len(st.history))
        else:
            n, circ = job
            for policy in ("fused", "swap"):
                st = ShardedState(n)
                for g in circ:
                    st.apply(g, policy)
                nswaps = [s for _, _, s in st.history]
                res[policy] = (st.total_sent(), st.gather(), nswaps)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def run_ranks(world, job):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q, job)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out[0]


def test_fused_swap_worked_example_traffic():
    import oracle
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "fused_swap_traffic.json")))
    res = run_ranks(4, "example")
    want = oracle.zero_state(4)
    oracle.run_circuit(want, example_circuit())
    assert res["direct"][0] == golden["bytes_original_circuit"]
    assert res["swap"][0] == golden["bytes_swapped_circuit"]
    assert res["fused"][0] == golden["bytes_fused_swap_circuit"]
    for policy in ("direct", "swap", "fused"):
        assert np.array_equal(res[policy][1], want), policy


@pytest.mark.parametrize("world,kind", [(2, "brick"), (4, "brick"), (4, "qv")])
def test_sharded_circuits_match_oracle(world, kind):
    import oracle
    import workloads as W
    n = 10
    circ = W.brick(n, 8, 90) if kind == "brick" else W.qv_like(n, 4, 91)
    res = run_ranks(world, (n, circ))
    want = oracle.zero_state(n)
    oracle.run_circuit(want, circ)
    p = world.bit_length() - 1
    for policy in ("fused", "swap"):
        sent, got, swaps = res[policy]
        assert np.array_equal(got, want), policy
        assert sent == sum(int(2 ** (n + 4) * (1 - 2.0 ** -s)) for s in swaps)
        if policy == "fused":
            assert swaps and all(s == p for s in swaps)


def test_double_buffered_fused_swap():
    # §III-E: the exchanges in 4 pieces per partner through two buffer
    # pairs move the same bytes and give the same state as in one piece
    import oracle
    import workloads as W
    n = 10
    circ = W.brick(n, 6, 92)
    res = run_ranks(4, ("buffered", n, circ))
    want = oracle.zero_state(n)
    oracle.run_circuit(want, circ)
    assert res[1][0] == res[4][0] > 0
    assert np.array_equal(res[1][1], want) and np.array_equal(res[4][1], want)
