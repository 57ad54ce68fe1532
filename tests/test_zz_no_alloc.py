"""qs_inner_noalloc: the allocation-free inner product.

Callers that cannot let the library allocate device memory (their own
allocator owns the GPU, or an allocation would stall a latency-critical loop)
use this entry point; it keeps its reduction scratch in a fixed static device
array.  Checked against the allocating qs_inner on two calls in a row, so a
second call that reuses the array's leftover contents is covered.  Kept in a
file collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_inner_noalloc_matches_inner_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs

    L = qs.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(17, "c128", 1), (12, "c64", 2), (17, "c128", 3)]
    for n, dtype, seed in cases:
        a = qs.State(n, dtype).from_numpy(W.random_state(n, 100 + seed))
        b = qs.State(n, dtype).from_numpy(W.random_state(n, 200 + seed))
        want = a.inner(b)
        for _ in range(2):  # two calls in a row share the static scratch
            out = (ctypes.c_double * 2)()
            rc = L.qs_inner_noalloc(ctypes.c_void_p(a.tensor.data_ptr()), ctypes.c_void_p(b.tensor.data_ptr()),
                                    n, qs.C64 if dtype == "c64" else qs.C128, stream, out)
            assert rc == qs.QS_OK, L.qs_last_error()
            got = complex(out[0], out[1])
            assert abs(got - want) <= 1e-12, (got, want)
    # argument checks, no GPU work
    out = (ctypes.c_double * 2)()
    assert L.qs_inner_noalloc(None, None, 5, qs.C128, stream, out) == qs.QS_EINVAL
    assert L.qs_inner_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 0, qs.C128, stream, out) == qs.QS_EINVAL
