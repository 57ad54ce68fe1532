"""Python binding of libqs, the GB300 state-vector gate engine.

Argument marshalling only: every operation is one call into the C ABI
declared in include/qs.h, and every step on the state runs in the library's
CUDA kernels.  PyTorch provides device memory (state vectors are torch
complex64/complex128 tensors wrapped with ``qs_wrap``) and streams (each call
is enqueued on ``torch.cuda.current_stream()``).

There is no CPU fallback: importing this package raises if libqs.so has not
been built (``python -m paper_2203_16044_gb300.build`` or
``__graft_entry__.build()``), and operations need a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libqs.so not found at {LIB_PATH}; build it with `python -m paper_2203_16044_gb300.build` "
        "(the package has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
C64, C128 = 0, 1
PLAN_UNFUSED, PLAN_TILED, PLAN_FUSED, PLAN_SWAP, PLAN_PERMUTE = 0, 1, 2, 3, 4

GATE_KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5, "RX": 6, "RY": 7, "RZ": 8, "P": 9,
             "U3": 10, "CNOT": 16, "CZ": 17, "CP": 18, "SWAP": 19}

_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)
_up = ctypes.POINTER(ctypes.c_uint64)
_int = ctypes.c_int


class PlanOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tile_qubits", ctypes.c_int), ("low_qubits", ctypes.c_int),
                ("slot_qubits", ctypes.c_int), ("groups_per_thread", ctypes.c_int), ("dense", ctypes.c_int),
                ("fuse_qubits", ctypes.c_int), ("search", ctypes.c_int), ("fuse_min_qubits", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("dtype", ctypes.c_int), ("gates", ctypes.c_int), ("passes", ctypes.c_int),
                ("hbm_bytes", ctypes.c_double), ("metric_bytes", ctypes.c_double), ("stages", ctypes.c_int),
                ("dense_stages", ctypes.c_int)]


_SIGS = {
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_version": ([], ctypes.c_char_p),
    "qs_alloc": ([_int, _int, ctypes.POINTER(_vp)], _int),
    "qs_wrap": ([_int, _int, _vp, ctypes.POINTER(_vp)], _int),
    "qs_free": ([_vp], _int),
    "qs_set_stream": ([_vp, _vp], _int),
    "qs_sync": ([_vp], _int),
    "qs_data": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)], _int),
    "qs_set_basis": ([_vp, ctypes.c_uint64], _int),
    "qs_copy_to_host": ([_vp, _vp], _int),
    "qs_copy_from_host": ([_vp, _vp], _int),
    "qs_copy_from_host_async": ([_vp, _vp], _int),
    "qs_apply_1q": ([_vp, _int, _dp], _int),
    "qs_apply_controlled": ([_vp, _ip, _int, _int, _dp], _int),
    "qs_apply_diag": ([_vp, _ip, _int, _dp], _int),
    "qs_apply_fused": ([_vp, _ip, _int, _dp], _int),
    "qs_permute_qubits": ([_vp, _ip], _int),
    "qs_fused_swap": ([_vp, _int, _int, _int], _int),
    "qs_norm2": ([_vp, _dp], _int),
    "qs_inner": ([_vp, _vp, _dp], _int),
    "qs_expect_pauli": ([_vp, _int, _up, _up, _dp, _dp], _int),
    "qs_expect_pauli_passes": ([_int, _int, _int, _up, _up, ctypes.POINTER(ctypes.c_int)], _int),
    "qs_inner_noalloc": ([_vp, _vp, _int, _int, _vp, _dp], _int),
    "qs_plan_autotune": ([_vp, _vp, ctypes.POINTER(PlanOpts), _dp], _int),
    "qs_tune_cache_file": ([ctypes.c_char_p], _int),
    "qs_circuit_hash": ([_vp, _int, _int, ctypes.POINTER(ctypes.c_uint64)], _int),
    "qs_circuit_create": ([ctypes.POINTER(_vp)], _int),
    "qs_circuit_destroy": ([_vp], _int),
    "qs_circuit_add": ([_vp, _int, _ip, _int, _dp, _int], _int),
    "qs_circuit_add_many": ([_vp, _int, _ip, _ip, _dp, _ip], _int),
    "qs_circuit_size": ([_vp, _ip], _int),
    "qs_plan_build": ([_vp, _int, _int, ctypes.POINTER(PlanOpts), ctypes.POINTER(_vp)], _int),
    "qs_plan_stats_get": ([_vp, ctypes.POINTER(PlanStats)], _int),
    "qs_plan_destroy": ([_vp], _int),
    "qs_run_plan": ([_vp, _vp], _int),
    "qs_plan_step_info": ([_vp, _int, _ip, _dp], _int),
    "qs_plan_step_qubits": ([_vp, _int, _ip, _int, _ip], _int),
    "qs_plan_step_matrix": ([_vp, _int, _dp, ctypes.c_size_t, _ip], _int),
    "qs_probabilities": ([_vp, _ip, _int, _dp], _int),
    "qs_measure": ([_vp, _int, ctypes.c_double, _ip, _dp], _int),
    "qs_sample": ([_vp, ctypes.c_uint64, _dp, ctypes.POINTER(ctypes.c_uint64)], _int),
    "qs_run_plan_profiled": ([_vp, _vp, ctypes.POINTER(ctypes.c_float), _int], _int),
    "qs_adjoint_grad": ([_vp, _vp, _dp, _int, _int, _int, _up, _up, _dp, _dp, _dp], _int),
    "qs_batch_create": ([_int, _ip, _int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(PlanOpts), _vp,
                         ctypes.POINTER(_vp)], _int),
    "qs_batch_run": ([_vp, _int], _int),
    "qs_batch_sync": ([_vp], _int),
    "qs_batch_stats_get": ([_vp, ctypes.c_void_p], _int),
    "qs_batch_destroy": ([_vp], _int),
    "qs_batch_autotune": ([_int, _ip, _int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, ctypes.POINTER(PlanOpts),
                           _dp], _int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class QSError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.qs_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(code: int, where: str) -> None:
    if code != QS_OK:
        raise QSError(code, where)


def lib() -> ctypes.CDLL:
    return _lib


def version() -> str:
    return _lib.qs_version().decode()


def _darr(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _iarr(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def _torch():
    import torch
    return torch


def _stream_ptr():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class State:
    """A 2^n-amplitude state vector in GPU memory.

    ``tensor`` is a 1-D torch tensor (complex64 or complex128) that owns the
    memory; the library handle wraps it.  Initialised to |0...0> unless
    ``tensor`` is given (then its contents are kept)."""

    def __init__(self, n: int, dtype: str = "c128", device=None, tensor=None):
        torch = _torch()
        if dtype not in ("c64", "c128"):
            raise ValueError("dtype must be 'c64' or 'c128'")
        self.n = int(n)
        self.dtype = dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        if tensor is None:
            dev = torch.device(device if device is not None else "cuda")
            tensor = torch.zeros(1 << self.n, dtype=tdt, device=dev)
            tensor[0] = 1
        else:
            if tensor.dtype != tdt or tensor.numel() != (1 << self.n) or not tensor.is_cuda or not tensor.is_contiguous():
                raise ValueError("tensor must be a contiguous CUDA tensor of 2^n amplitudes of the given dtype")
        self.tensor = tensor
        h = _vp()
        with torch.cuda.device(tensor.device):
            _check(_lib.qs_wrap(self.n, C64 if dtype == "c64" else C128, ctypes.c_void_p(tensor.data_ptr()),
                                ctypes.byref(h)), "qs_wrap")
        self._h = h

    @property
    def handle(self):
        return self._h

    def _bind(self):
        _check(_lib.qs_set_stream(self._h, _stream_ptr()), "qs_set_stream")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.qs_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state --------------------------------------------------------------
    def set_basis(self, x: int) -> "State":
        _check(_lib.qs_set_basis(self._bind(), int(x)), "qs_set_basis")
        return self

    def probabilities(self, qubits: Sequence[int]) -> np.ndarray:
        """Marginal Born-rule probabilities of the given qubits (qs_probabilities):
        entry r has bit i = qubits[i]."""
        q = _iarr(qubits)
        out = np.zeros(1 << len(q), dtype=np.float64)
        _check(_lib.qs_probabilities(self._bind(), _iptr(q), len(q), _dptr(out)), "qs_probabilities")
        return out

    def measure(self, q: int, u: float):
        """Measure qubit q with the uniform u in [0, 1) (qs_measure); the state
        collapses.  Returns (outcome, probability of the outcome)."""
        o = ctypes.c_int()
        p = ctypes.c_double()
        _check(_lib.qs_measure(self._bind(), int(q), float(u), ctypes.byref(o), ctypes.byref(p)), "qs_measure")
        return o.value, p.value

    def sample(self, u) -> np.ndarray:
        """Basis-state samples for the uniforms u in [0, 1) (qs_sample); the
        state is unchanged."""
        uu = np.ascontiguousarray(u, dtype=np.float64).ravel()
        out = np.zeros(uu.size, dtype=np.uint64)
        _check(_lib.qs_sample(self._bind(), uu.size, _dptr(uu), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
               "qs_sample")
        return out

    def to_numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex64 if self.dtype == "c64" else np.complex128)
        _check(_lib.qs_copy_to_host(self._bind(), out.ctypes.data_as(_vp)), "qs_copy_to_host")
        return out

    def from_numpy(self, a: np.ndarray) -> "State":
        a = np.ascontiguousarray(a, dtype=np.complex64 if self.dtype == "c64" else np.complex128)
        if a.size != (1 << self.n):
            raise ValueError("size mismatch")
        _check(_lib.qs_copy_from_host(self._bind(), a.ctypes.data_as(_vp)), "qs_copy_from_host")
        return self

    def copy_from_host_async(self, ptr: int) -> "State":
        """Queue the copy of 2^n amplitudes from host address ptr (pinned
        memory, kept unchanged until the stream passes the copy) on the
        state's stream and return (qs_copy_from_host_async)."""
        _check(_lib.qs_copy_from_host_async(self._bind(), _vp(int(ptr))), "qs_copy_from_host_async")
        return self

    def sync(self) -> None:
        _check(_lib.qs_sync(self._bind()), "qs_sync")

    # -- gates ----------------------------------------------------------------
    def apply_1q(self, q: int, U) -> "State":
        u = _darr(np.asarray(U).reshape(2, 2))
        _check(_lib.qs_apply_1q(self._bind(), int(q), _dptr(u)), "qs_apply_1q")
        return self

    def apply_controlled(self, controls: Sequence[int], target: int, U) -> "State":
        c = _iarr(controls)
        u = _darr(np.asarray(U).reshape(2, 2))
        _check(_lib.qs_apply_controlled(self._bind(), _iptr(c), len(c), int(target), _dptr(u)), "qs_apply_controlled")
        return self

    def apply_diag(self, qubits: Sequence[int], d) -> "State":
        q = _iarr(qubits)
        dd = _darr(np.asarray(d).reshape(-1))
        _check(_lib.qs_apply_diag(self._bind(), _iptr(q), len(q), _dptr(dd)), "qs_apply_diag")
        return self

    def apply_fused(self, qubits: Sequence[int], M) -> "State":
        q = _iarr(qubits)
        m = _darr(np.asarray(M).reshape(1 << len(q), 1 << len(q)))
        _check(_lib.qs_apply_fused(self._bind(), _iptr(q), len(q), _dptr(m)), "qs_apply_fused")
        return self

    def permute_qubits(self, perm: Sequence[int]) -> "State":
        p = _iarr(perm)
        if len(p) != self.n:
            raise ValueError("perm must have n entries")
        _check(_lib.qs_permute_qubits(self._bind(), _iptr(p)), "qs_permute_qubits")
        return self

    def fused_swap(self, p: int, q: int, s: int) -> "State":
        _check(_lib.qs_fused_swap(self._bind(), int(p), int(q), int(s)), "qs_fused_swap")
        return self

    # -- reductions -----------------------------------------------------------
    def norm2(self) -> float:
        out = ctypes.c_double()
        _check(_lib.qs_norm2(self._bind(), ctypes.byref(out)), "qs_norm2")
        return out.value

    def inner(self, other: "State") -> complex:
        out = (ctypes.c_double * 2)()
        other._bind()
        _check(_lib.qs_inner(self._bind(), other._h, out), "qs_inner")
        return complex(out[0], out[1])

    def expect_pauli(self, terms) -> float:
        xm = np.ascontiguousarray([t.xmask for t in terms], dtype=np.uint64)
        zm = np.ascontiguousarray([t.zmask for t in terms], dtype=np.uint64)
        cf = np.ascontiguousarray([t.coeff for t in terms], dtype=np.float64)
        out = ctypes.c_double()
        _check(_lib.qs_expect_pauli(self._bind(), len(terms), xm.ctypes.data_as(_up), zm.ctypes.data_as(_up),
                                    _dptr(cf), ctypes.byref(out)), "qs_expect_pauli")
        return out.value

    def run(self, plan: "Plan") -> "State":
        _check(_lib.qs_run_plan(self._bind(), plan.handle), "qs_run_plan")
        return self

    def run_profiled(self, plan: "Plan") -> np.ndarray:
        """Run the plan and return the device time of every step (ms)."""
        k = plan.stats()["passes"]
        ms = (ctypes.c_float * max(k, 1))()
        _check(_lib.qs_run_plan_profiled(self._bind(), plan.handle, ms, k), "qs_run_plan_profiled")
        return np.array(ms[:k], dtype=np.float64)


class Circuit:
    """Host-side gate list (qs_circuit)."""

    def __init__(self, gates=()):
        h = _vp()
        _check(_lib.qs_circuit_create(ctypes.byref(h)), "qs_circuit_create")
        self._h = h
        self.add_many(gates)

    def add_many(self, gates):
        """Append a sequence of gates (objects with name, qubits, params and
        optionally param_index) in one call."""
        gates = list(gates)
        if not gates:
            return
        m = len(gates)
        kinds = np.empty(m, dtype=np.int32)
        qubits = np.zeros((m, 2), dtype=np.int32)
        params = np.zeros((m, 3), dtype=np.float64)
        pidx = np.full(m, -1, dtype=np.int32)
        for i, g in enumerate(gates):
            kinds[i] = GATE_KIND[g.name]
            q = g.qubits
            qubits[i, 0] = q[0]
            if len(q) > 1:
                qubits[i, 1] = q[1]
            if len(g.params):
                params[i, :len(g.params)] = g.params
            pidx[i] = getattr(g, "param_index", -1)
        _check(_lib.qs_circuit_add_many(self._h, m, _iptr(kinds), _iptr(qubits), _dptr(params), _iptr(pidx)),
               "qs_circuit_add_many")

    @property
    def handle(self):
        return self._h

    def add(self, name: str, qubits: Sequence[int], params: Sequence[float] = (), param_index: int = -1):
        q = _iarr(qubits)
        p = np.ascontiguousarray(params if len(params) else [0.0], dtype=np.float64)
        _check(_lib.qs_circuit_add(self._h, GATE_KIND[name], _iptr(q), len(q), _dptr(p), int(param_index)),
               "qs_circuit_add")

    def __len__(self):
        n = ctypes.c_int()
        _check(_lib.qs_circuit_size(self._h, ctypes.byref(n)), "qs_circuit_size")
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.qs_circuit_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_kwargs(opts: PlanOpts) -> dict:
    """PlanOpts as keyword arguments of Plan."""
    return {f: getattr(opts, f) for f, _ in PlanOpts._fields_ if f not in ("reserved", "fuse_min_qubits")}


def autotune(circuit: "Circuit", state: "State"):
    """qs_plan_autotune: (PlanOpts, ms) of the fastest plan shape for this
    circuit on this state (whose contents are overwritten); cached."""
    best = PlanOpts()
    ms = ctypes.c_double()
    _check(_lib.qs_plan_autotune(circuit.handle, state._bind(), ctypes.byref(best), ctypes.byref(ms)),
           "qs_plan_autotune")
    return best, ms.value


def set_tune_cache(path) -> None:
    """qs_tune_cache_file: persist autotuning results in `path` (None: in
    memory only) and load those it holds."""
    _check(_lib.qs_tune_cache_file(None if path is None else os.fsencode(path)), "qs_tune_cache_file")


def circuit_hash(circuit: "Circuit", n: int, dtype: str) -> int:
    out = ctypes.c_uint64()
    _check(_lib.qs_circuit_hash(circuit.handle, int(n), C64 if dtype == "c64" else C128, ctypes.byref(out)),
           "qs_circuit_hash")
    return out.value


class Plan:
    """A circuit compiled for (n, dtype) into HBM passes (qs_plan)."""

    def __init__(self, circuit: Circuit, n: int, dtype: str = "c128", mode: int = PLAN_TILED,
                 tile_qubits: int = 0, low_qubits: int = 0, slot_qubits: int = 0, groups_per_thread: int = 0,
                 dense: int = 0, fuse_qubits: int = 0, search: int = 0):
        opts = PlanOpts(mode=mode, tile_qubits=tile_qubits, low_qubits=low_qubits, slot_qubits=slot_qubits,
                        groups_per_thread=groups_per_thread, dense=dense, fuse_qubits=fuse_qubits, search=search)
        h = _vp()
        _check(_lib.qs_plan_build(circuit.handle, int(n), C64 if dtype == "c64" else C128, ctypes.byref(opts),
                                  ctypes.byref(h)), "qs_plan_build")
        self._h = h
        self.n = n
        self.dtype = dtype

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = PlanStats()
        _check(_lib.qs_plan_stats_get(self._h, ctypes.byref(s)), "qs_plan_stats_get")
        return {"n": s.n, "dtype": s.dtype, "gates": s.gates, "passes": s.passes, "hbm_bytes": s.hbm_bytes,
                "metric_bytes": s.metric_bytes, "stages": s.stages, "dense_stages": s.dense_stages}

    STEP_KINDS = ("1q", "ctrl", "diag", "swap", "tile", "block")

    def step_info(self):
        """[(kind, algorithmic HBM bytes)] for every pass of the plan."""
        out = []
        for i in range(self.stats()["passes"]):
            k, b = ctypes.c_int(), ctypes.c_double()
            _check(_lib.qs_plan_step_info(self._h, i, ctypes.byref(k), ctypes.byref(b)), "qs_plan_step_info")
            out.append((self.STEP_KINDS[k.value], b.value))
        return out

    def step_qubits(self, i: int) -> list:
        """The qubits of plan step i (block: bit j of its matrix index is
        qubit j; gate: controls, then target; bit-pair exchange pass: its
        pairs a0, b0, a1, b1, ...; tile pass: [])."""
        q = (ctypes.c_int * 34)()
        cnt = ctypes.c_int()
        _check(_lib.qs_plan_step_qubits(self._h, int(i), q, 34, ctypes.byref(cnt)), "qs_plan_step_qubits")
        return list(q[:cnt.value])

    def step_matrix(self, i: int) -> np.ndarray:
        """The complex matrix of dense-block step i (bit j of its index is
        step_qubits(i)[j])."""
        buf = np.zeros(2 * 4 ** 6, dtype=np.float64)
        k = ctypes.c_int()
        _check(_lib.qs_plan_step_matrix(self._h, int(i), _dptr(buf), buf.size, ctypes.byref(k)), "qs_plan_step_matrix")
        D = 1 << k.value
        return buf[:2 * D * D].view(np.complex128).reshape(D, D).copy()

    def close(self):
        if getattr(self, "_h", None):
            _lib.qs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_circuit(state: State, gates, mode: int = PLAN_TILED, **kw) -> dict:
    """Compile ``gates`` (workload Gate records) for the state and run them."""
    c = Circuit(gates)
    p = Plan(c, state.n, state.dtype, mode=mode, **kw)
    state.run(p)
    return p.stats()


def _terms(terms):
    xm = np.ascontiguousarray([t.xmask for t in terms], dtype=np.uint64)
    zm = np.ascontiguousarray([t.zmask for t in terms], dtype=np.uint64)
    cf = np.ascontiguousarray([t.coeff for t in terms], dtype=np.float64)
    return xm, zm, cf


def expect_pauli_passes(n: int, dtype: str, terms) -> int:
    """Reads of the whole state that State.expect_pauli makes for these
    terms on an n-qubit state (host only; qs_expect_pauli_passes)."""
    xm, zm, _ = _terms(terms)
    out = ctypes.c_int()
    code = C64 if dtype == "c64" else C128 if dtype == "c128" else -1
    _check(_lib.qs_expect_pauli_passes(n, code, len(xm), xm.ctypes.data_as(_up), zm.ctypes.data_as(_up),
                                       ctypes.byref(out)), "qs_expect_pauli_passes")
    return out.value


def adjoint_grad(state: State, circuit: Circuit, theta, terms):
    """Energies and adjoint gradients for a batch of parameter sets.

    theta: (batch, nparam) or (nparam,) array of angles.  Returns
    (energy[batch], grad[batch, nparam]) as float64 numpy arrays (squeezed to
    match a 1-D theta).  The state's contents are overwritten."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    single = th.ndim == 1
    th2 = th.reshape(1, -1) if single else th
    batch, nparam = th2.shape
    xm, zm, cf = _terms(terms)
    energy = np.zeros(batch, dtype=np.float64)
    grad = np.zeros((batch, max(nparam, 1)), dtype=np.float64)
    _check(_lib.qs_adjoint_grad(state._bind(), circuit.handle, _dptr(th2), nparam, batch, len(terms),
                                xm.ctypes.data_as(_up), zm.ctypes.data_as(_up), _dptr(cf), _dptr(energy),
                                _dptr(grad)), "qs_adjoint_grad")
    grad = grad[:, :nparam]
    return (energy[0], grad[0]) if single else (energy, grad)


def expectation_fn():
    """torch.autograd.Function computing E(theta) with the adjoint gradient.

    Usage: E = expectation_fn().apply(theta, state, circuit, terms) with theta
    a float64 tensor of shape (nparam,) or (batch, nparam); E.backward()
    fills theta.grad.  Forward runs the adjoint sweep once (energy and
    gradient together, on the GPU) and keeps the gradient for backward."""
    torch = _torch()

    class _Expectation(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, state, circuit, terms):
            e, g = adjoint_grad(state, circuit, theta.detach().cpu().numpy(), terms)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(e, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            if g.dim() == 1:
                return grad_out * g, None, None, None
            return grad_out[:, None] * g, None, None, None

    return _Expectation


class BatchStats(ctypes.Structure):
    _fields_ = [("circuits", ctypes.c_int), ("units", ctypes.c_int), ("passes", ctypes.c_int), ("grid", ctypes.c_int),
                ("graph", ctypes.c_int), ("reserved", ctypes.c_int), ("hbm_bytes", ctypes.c_double),
                ("metric_bytes", ctypes.c_double)]


class Batch:
    """Many independent circuits run by one persistent launch (qs_batch).

    ``sizes``: qubit count of each circuit; ``gate_lists``: workload Gate
    lists.  The states live in one torch buffer (``self.buffer``) owned by
    this object; ``state(i)`` returns circuit i's vector (a view).  opts:
    PlanOpts fields as keywords (tile_qubits, slot_qubits, ...), or
    ``autotune=True`` to let the library pick them by timing."""

    def __init__(self, sizes, gate_lists, dtype: str = "c64", autotune: bool = False, **opts):
        torch = _torch()
        self.sizes = [int(n) for n in sizes]
        self.dtype = dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        self.offsets = []
        off = 0
        for n in self.sizes:
            self.offsets.append(off)
            off += 1 << n
        self.buffer = torch.zeros(off, dtype=tdt, device="cuda")
        self.circuits = [Circuit(g) for g in gate_lists]
        count = len(self.sizes)
        self._n = (ctypes.c_int * count)(*self.sizes)
        self._ptrs = (_vp * count)(*[self.buffer[o:].data_ptr() for o in self.offsets])
        self._circ = (_vp * count)(*[c.handle.value for c in self.circuits])
        # a stream of its own: the legacy default stream cannot be captured
        # into a CUDA graph
        self._tstream = torch.cuda.Stream()
        self._tstream.wait_stream(torch.cuda.current_stream())
        self._stream = ctypes.c_void_p(self._tstream.cuda_stream)
        dt = C64 if dtype == "c64" else C128
        po = PlanOpts(mode=PLAN_TILED, **opts)
        self.tuned_ms = None
        if autotune:
            best = PlanOpts()
            ms = ctypes.c_double()
            _check(_lib.qs_batch_autotune(count, self._n, dt, self._ptrs, self._circ, self._stream, ctypes.byref(best),
                                          ctypes.byref(ms)), "qs_batch_autotune")
            po, self.tuned_ms = best, ms.value
        self.opts = po
        h = _vp()
        _check(_lib.qs_batch_create(count, self._n, dt, self._ptrs, self._circ, ctypes.byref(po), self._stream,
                                    ctypes.byref(h)), "qs_batch_create")
        self._h = h

    def run(self, init_zero: bool = True) -> "Batch":
        """Enqueue one run on the batch's stream, after the work already
        queued on the caller's current stream."""
        torch = _torch()
        self._tstream.wait_stream(torch.cuda.current_stream())
        _check(_lib.qs_batch_run(self._h, 1 if init_zero else 0), "qs_batch_run")
        return self

    def sync(self) -> None:
        """Wait for the batch and check it (QSError QS_ETIMEOUT if a bounded
        wait gave up); later work on the current stream is ordered after it."""
        torch = _torch()
        _check(_lib.qs_batch_sync(self._h), "qs_batch_sync")
        torch.cuda.current_stream().wait_stream(self._tstream)

    def state(self, i: int):
        return self.buffer[self.offsets[i]:self.offsets[i] + (1 << self.sizes[i])]

    def stats(self) -> dict:
        s = BatchStats()
        _check(_lib.qs_batch_stats_get(self._h, ctypes.byref(s)), "qs_batch_stats_get")
        return {f: getattr(s, f) for f, _ in BatchStats._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            _lib.qs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
