"""Complex64 state checks shared by the GPU tests.

The stated tolerance is on the unnormalised infidelity 1 - |<a|b>|^2.  That
form goes negative when the complex64 state's norm exceeds 1, which can hide
a real error of the same size, so every check also bounds the normalised
infidelity 1 - |<a|b>|^2 / (<a|a> <b|b>) (never negative, by Cauchy-Schwarz)
and the norm difference |<a|a> - <b|b>|.

Norm tolerance: 1e-6, or for a circuit of G gates computed gate by gate in
FP32, 4 2^-24 sqrt(G) if larger.  Each gate's matrix rounded to FP32 is
unitary only to about 2^-23 (every entry rounded by 2^-24 relative), so each
gate scales the norm by 1 + O(2^-23) with a sign that varies from gate to
gate: a random walk of G steps.  (Tensor-core block plans restore each
group's norm and stay far inside 1e-6.)
"""
import numpy as np

C64_INFIDELITY = 1e-5
C64_NORM = 1e-6


def c64_metrics(got, want):
    """(stated infidelity, normalised infidelity, norm difference) of a
    complex64 result against a reference, in FP64."""
    a = np.asarray(got).astype(np.complex128, copy=False)
    b = np.asarray(want).astype(np.complex128, copy=False)
    ov = abs(np.vdot(a, b)) ** 2
    na, nb = np.vdot(a, a).real, np.vdot(b, b).real
    return 1.0 - ov, 1.0 - ov / (na * nb), abs(na - nb)


def norm_tol_for(gates=None):
    if not gates:
        return C64_NORM
    return max(C64_NORM, 4 * 2.0 ** -24 * gates ** 0.5)


def check_c64(got, want, tol=C64_INFIDELITY, gates=None):
    norm_tol = norm_tol_for(gates)
    stated, normalised, dnorm = c64_metrics(got, want)
    assert stated <= tol, ("infidelity", stated)
    assert normalised <= tol, ("normalised infidelity", normalised)
    assert dnorm <= norm_tol, ("norm difference", dnorm)
    return stated, normalised, dnorm


def torch_c64_metrics(t64, t128):
    """The same three numbers for two device tensors (complex64 result,
    complex128 reference), computed on the GPU in FP64."""
    import torch
    a = t64.to(torch.complex128)
    ov = abs(torch.vdot(a, t128).item()) ** 2
    na, nb = torch.vdot(a, a).real.item(), torch.vdot(t128, t128).real.item()
    del a
    return 1.0 - ov, 1.0 - ov / (na * nb), abs(na - nb)


def check_c64_torch(t64, t128, tol=C64_INFIDELITY, gates=None):
    norm_tol = norm_tol_for(gates)
    stated, normalised, dnorm = torch_c64_metrics(t64, t128)
    assert stated <= tol, ("infidelity", stated)
    assert normalised <= tol, ("normalised infidelity", normalised)
    assert dnorm <= norm_tol, ("norm difference", dnorm)
    return stated, normalised, dnorm
