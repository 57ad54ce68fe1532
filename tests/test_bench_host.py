"""Host-side pieces of bench.py (no GPU): which kernel each plan step is
attributed to in the roofline."""
import pytest

import workloads as W


@pytest.fixture(scope="module")
def qs():
    import paper_2203_16044_gb300 as qs
    return qs


def _runs(q, n):
    # maximal runs of block / non-block qubits over 0..n-1, counted directly
    cls = [b in set(q) for b in range(n)]
    return sum(1 for b in range(n) if b == 0 or cls[b] != cls[b - 1])


def test_step_kernel_labels(qs):
    import bench
    # with at most 5 runs of block and other qubits: sets starting with the
    # run 0..a-1 (a >= 4; 3 for complex128) take the rows form of the TMA
    # kernel ("rows" for 0..k-1, "lowrun" otherwise), other sets with qubit 0
    # outside or in the run 0, 1 its box form ("window" when consecutive);
    # other sets, and blocks with fewer than 128 groups, the per-thread
    # gather kernel.  complex128 k = 4, 5 alike (k_fused_c128), 6-qubit
    # requests narrowed to 5.
    seen = set()
    for dtype, n, fq, circ in (("c64", 14, 6, W.brick(14, 12, 3)), ("c64", 14, 6, W.qft(14)),
                               ("c64", 15, 5, W.qv_like(15, 6, 2)), ("c64", 9, 4, W.brick(9, 6, 1)),
                               ("c128", 14, 5, W.brick(14, 12, 3)), ("c128", 14, 6, W.qft(14)),
                               ("c128", 13, 4, W.qv_like(13, 6, 3)), ("c128", 8, 4, W.brick(8, 12, 3))):
        p = qs.Plan(qs.Circuit(circ), n, dtype, mode=qs.PLAN_FUSED, fuse_qubits=fq)
        name, gather = ("k_fused_c128", "k_fused_c128<%d,gather>") if dtype == "c128" else \
            ("k_fused_umma_tma", "k_fused_umma<%d>")
        for i, (kind, _) in enumerate(p.step_info()):
            lab = bench.step_kernel(p, i, kind)
            if kind != "block":
                assert lab == kind
                continue
            q = sorted(p.step_qubits(i))
            k = len(q)
            assert k <= (5 if dtype == "c128" else 6)
            low = len([j for j in range(k) if q[j] == j and all(q[x] == x for x in range(j))])
            if k < 4:
                want = "k_dense<%d>" % k
            elif n - k < 7 or _runs(q, n) > 5:
                want = gather % k
            elif low >= (3 if dtype == "c128" else 4):
                want = "%s<%d,%s>" % (name, k, "rows" if low == k else "lowrun")
            elif low in (0, 2):
                want = "%s<%d,%s>" % (name, k, "window" if q[-1] - q[0] + 1 == k else "box")
            else:
                want = gather % k
            assert lab == want, (dtype, n, q, lab)
            seen.add(want.split("<")[0] + "," + (want.split(",")[1] if "," in want else "gather"))
    assert {"k_fused_umma_tma,window>", "k_fused_umma_tma,rows>", "k_fused_umma_tma,box>",
            "k_fused_c128,window>", "k_fused_c128,rows>"} <= seen, seen


def test_planner_widens_complex64_blocks_to_windows(qs):
    # host-only: every complex64 tensor-core block whose touched qubits fit in
    # a window of at most k consecutive qubits is widened to such a window of
    # at least 4 qubits (the shapes the TMA kernel takes); the widened block
    # still holds all the qubits its gates touch, and the plan's gate count
    # is unchanged
    import workloads as W
    for n, k, circ in ((14, 6, W.brick(14, 12, 3)), (13, 5, W.qv_like(13, 6, 5)), (12, 4, W.qsb(12, 7, sets=3))):
        p = qs.Plan(qs.Circuit(circ), n, "c64", mode=qs.PLAN_FUSED, fuse_qubits=k)
        assert p.stats()["gates"] == len(circ)
        for i, (kind, _) in enumerate(p.step_info()):
            if kind != "block":
                continue
            q = sorted(p.step_qubits(i))
            assert 4 <= len(q) <= k
