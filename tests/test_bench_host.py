"""Host-side pieces of bench.py (no GPU): which kernel each plan step is
attributed to in the roofline."""
import pytest

import workloads as W


@pytest.fixture(scope="module")
def qs():
    import paper_2203_16044_gb300 as qs
    return qs


def test_step_kernel_labels(qs):
    import bench
    n = 14
    p = qs.Plan(qs.Circuit(W.brick(n, 12, 3)), n, "c64", mode=qs.PLAN_FUSED, fuse_qubits=6)
    seen = set()
    for i, (kind, _) in enumerate(p.step_info()):
        lab = bench.step_kernel(p, i, kind)
        if kind != "block":
            assert lab == kind
            continue
        q = sorted(p.step_qubits(i))
        if q[0] >= 2 and q == list(range(q[0], q[0] + len(q))):
            want = "k_fused_umma_tma<%d,window>" % len(q)
        elif q == list(range(len(q))):
            want = "k_fused_umma_tma<%d,rows>" % len(q)
        else:
            want = "k_fused_umma<%d>" % len(q)
        assert lab == want
        seen.add(want.split("<")[0] + ("," + want.split(",")[1] if "," in want else ""))
    # a brick plan has windows from qubit 2 up and a block on the lowest
    # qubits
    assert {"k_fused_umma_tma,window>", "k_fused_umma_tma,rows>"} <= seen
    # complex128: 4- and 5-qubit blocks run on k_fused_c128 (rows, windows
    # from qubit 1 up, gathered sets; fewer than 128 groups always gather),
    # 6-qubit requests are narrowed to 5, smaller blocks stay on k_dense
    for n, fq in ((14, 5), (14, 6), (13, 4), (8, 4)):
        p128 = qs.Plan(qs.Circuit(W.brick(n, 12, 3)), n, "c128", mode=qs.PLAN_FUSED, fuse_qubits=fq)
        for i, (kind, _) in enumerate(p128.step_info()):
            if kind != "block":
                continue
            q = sorted(p128.step_qubits(i))
            k = len(q)
            assert k <= 5
            lab = bench.step_kernel(p128, i, kind)
            if k < 4:
                assert lab == "k_dense<%d>" % k
            elif n - k < 7:
                assert lab == "k_fused_c128<%d,gather>" % k
            elif q == list(range(k)):
                assert lab == "k_fused_c128<%d,rows>" % k
            elif q[0] >= 1 and q == list(range(q[0], q[0] + k)):
                assert lab == "k_fused_c128<%d,window>" % k
            else:
                assert lab == "k_fused_c128<%d,gather>" % k


def test_planner_widens_complex64_blocks_to_windows(qs):
    # host-only: every complex64 tensor-core block whose touched qubits fit in
    # a window of at most k consecutive qubits is widened to such a window of
    # at least 4 qubits, starting at 0 or at 2 and above (the shapes the TMA
    # kernel takes); the widened block still holds all the qubits its gates
    # touch, and the plan's gate count is unchanged
    import workloads as W
    for n, k, circ in ((14, 6, W.brick(14, 12, 3)), (13, 5, W.qv_like(13, 6, 5)), (12, 4, W.qsb(12, 7, sets=3))):
        p = qs.Plan(qs.Circuit(circ), n, "c64", mode=qs.PLAN_FUSED, fuse_qubits=k)
        assert p.stats()["gates"] == len(circ)
        for i, (kind, _) in enumerate(p.step_info()):
            if kind != "block":
                continue
            q = sorted(p.step_qubits(i))
            assert 4 <= len(q) <= k
            if q[-1] - q[0] + 1 == len(q):  # a window
                assert q[0] == 0 or q[0] >= 2 or q[-1] + 1 >= n or len(q) == k
