"""qs_inner_noalloc: the allocation-free inner product.

Callers that cannot let the library allocate device memory (their own
allocator owns the GPU, or an allocation would stall a latency-critical loop)
use this entry point; it keeps its reduction scratch in a fixed static device
array.  Checked on two calls in a row (the second reuses the array's leftover
contents) against the oracle's inner product and against the allocating
qs_inner; at 24 qubits and at the 34-qubit maximum the grid reaches its cap
of 4 CTAs per SM, the largest number of partial sums the array must hold.
Kept in a file collected last so that a failure here does not hide the other
tests.
"""
import ctypes
import gc

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _call(qs, L, a_ptr, b_ptr, n, dtype, stream):
    out = (ctypes.c_double * 2)()
    rc = L.qs_inner_noalloc(ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr), n,
                            qs.C64 if dtype == "c64" else qs.C128, stream, out)
    assert rc == qs.QS_OK, L.qs_last_error()
    return complex(out[0], out[1])


def test_inner_noalloc_matches_oracle_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_16044_gb300 as qs

    L = qs.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the first call on the device looks the array up (and loads the module)
    warm = qs.State(4, "c64")
    _call(qs, L, warm.tensor.data_ptr(), warm.tensor.data_ptr(), 4, "c64", stream)
    cases = [(17, "c128", 1), (12, "c64", 2), (24, "c64", 3), (24, "c128", 4), (5, "c128", 5)]
    for n, dtype, seed in cases:
        pa, pb = W.random_state(n, 100 + seed), W.random_state(n, 200 + seed)
        a = qs.State(n, dtype).from_numpy(pa)
        b = qs.State(n, dtype).from_numpy(pb)
        # the oracle's inputs are the values the GPU holds (complex64 widened)
        wa = pa.astype(np.complex64).astype(np.complex128) if dtype == "c64" else pa
        wb = pb.astype(np.complex64).astype(np.complex128) if dtype == "c64" else pb
        want = oracle.inner(wa, wb)
        lib_inner = a.inner(b)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):  # two calls in a row share the static scratch
            got = _call(qs, L, a.tensor.data_ptr(), b.tensor.data_ptr(), n, dtype, stream)
            # FP64 sums of 2^n products of unit-norm vectors, different orders
            assert abs(got - want) <= 1e-12, (n, dtype, got, want)
            assert abs(got - lib_inner) <= 1e-12, (n, dtype, got, lib_inner)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "qs_inner_noalloc changed the device's free memory"
        del a, b
    # argument checks, no GPU work
    out = (ctypes.c_double * 2)()
    assert L.qs_inner_noalloc(None, None, 5, qs.C128, stream, out) == qs.QS_EINVAL
    assert L.qs_inner_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 0, qs.C128, stream, out) == qs.QS_EINVAL
    assert L.qs_inner_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 35, qs.C64, stream, out) == qs.QS_EINVAL


def test_inner_noalloc_34_qubits():
    # the largest state (2^34 complex64 amplitudes, 128 GiB) with every
    # amplitude 2^-17: <a|a> = 2^34 2^-34 = 1, exact in FP64 whatever the
    # summation order; the grid is at its cap of 4 CTAs per SM
    import torch
    import paper_2203_16044_gb300 as qs

    gc.collect()
    torch.cuda.empty_cache()
    n = 34
    L = qs.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    a = torch.full((1 << n,), complex(2.0 ** -17, 0.0), dtype=torch.complex64, device="cuda")
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            got = _call(qs, L, a.data_ptr(), a.data_ptr(), n, "c64", stream)
            assert got == 1.0, got
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        del a
        torch.cuda.empty_cache()
