"""CPU emulation of the paper's distributed state vector (§III-B, §III-D).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by tests, never by
the product path.

2^p ranks (torch.distributed, gloo backend, CPU) each hold 2^m amplitudes,
m = n - p: the amplitudes whose global bits (physical qubits m .. n-1) equal
the rank's bits.  Operations on local qubits (physical 0 .. m-1) run on the
rank's chunk with the oracle's own kernels (the per-pair arithmetic is the
same as on the whole state, so results are bit-identical to a single-process
oracle run).  What this module adds is only the data movement between ranks,
in the two forms of the paper, with every byte sent counted:

* a gate on a global qubit (§III-B): each rank exchanges its whole chunk with
  the partner that differs in that qubit's bit (2^(n+4) bytes per gate over
  all ranks, complex double);
* a fused swap (§III-D, Listing 1): swap(p + i, q + i) for i < s with one
  range global and one local; each rank keeps the 1/2^s of its chunk whose
  local field equals its own global field and trades one block of
  2^(m-s) amplitudes with each of its 2^s - 1 partners (2^(n+4) (1 - 2^-s)
  bytes over all ranks).

Instead of moving qubits back after a swap, the emulation keeps the map
phys[logical qubit] -> physical position; `restore` swaps back to the
identity map, and `gather` assembles the logical state on rank 0.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import apply_1q, gate_matrix, run_circuit


class ShardedState:
    def __init__(self, n: int, x0: int = 0, chunks: int = 1):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        R = dist.get_world_size()
        p = R.bit_length() - 1
        if (1 << p) != R or p >= n:
            raise ValueError("need 2^p ranks with p < n")
        self.n, self.p, self.m = n, p, n - p
        self.local = np.zeros(1 << self.m, dtype=np.complex128)
        if (x0 >> self.m) == self.rank:
            self.local[x0 & ((1 << self.m) - 1)] = 1.0
        self.phys = list(range(n))  # phys[logical] = physical position
        self.history = []           # fused swaps done, (glob, loc, s)
        self.sent = 0               # bytes this rank has sent
        self.chunks = chunks        # > 1: double-buffered fused swaps (§III-E)

    # ---- communication ---------------------------------------------------
    def _sendrecv(self, partner: int, send: np.ndarray) -> np.ndarray:
        import torch
        out = torch.empty(send.size * 2, dtype=torch.float64)
        src = torch.from_numpy(np.ascontiguousarray(send).view(np.float64).copy())
        reqs = [self.dist.isend(src, partner), self.dist.irecv(out, partner)]
        for r in reqs:
            r.wait()
        self.sent += send.size * 16
        return out.numpy().view(np.complex128)

    # ---- gates -----------------------------------------------------------
    def _gate_local(self, name: str, phys_qubits: Sequence[int], params: Sequence[float]):
        from workloads import Gate
        run_circuit(self.local, [Gate(name, tuple(phys_qubits), tuple(params))])

    def apply_global_1q(self, name: str, logical: int, params: Sequence[float] = ()):
        """A one-qubit gate on a global qubit, §III-B: the whole chunk is
        exchanged with the partner rank, and this rank's half of every pair
        is computed by the oracle's one-qubit kernel on the two chunks
        stacked as one (m + 1)-qubit state (the global bit on top)."""
        g = self.phys[logical]
        if g < self.m:
            raise ValueError("qubit is local")
        bit = (self.rank >> (g - self.m)) & 1
        partner = self.rank ^ (1 << (g - self.m))
        theirs = self._sendrecv(partner, self.local)
        pair = np.concatenate([theirs, self.local] if bit else [self.local, theirs])
        apply_1q(pair, self.m, gate_matrix(name, params))
        M = 1 << self.m
        self.local = pair[M:].copy() if bit else pair[:M].copy()

    def fused_swap(self, glob: int, loc: int, s: int, record: bool = True):
        """Physical global qubits glob .. glob+s-1 exchanged with local ones
        loc .. loc+s-1 (Listing 1 with one range on each side).  An amplitude
        of rank r at local index x goes to the rank whose global field is x's
        local field, at the index whose local field is r's global field."""
        m = self.m
        if not (glob >= m and glob + s <= self.n and loc >= 0 and loc + s <= m):
            raise ValueError("need a global range and a local range")
        a = glob - m
        fmask = (1 << s) - 1
        w = (self.rank >> a) & fmask                        # this rank's global field
        idx = np.arange(1 << m, dtype=np.int64)
        field = (idx >> loc) & fmask                         # each amplitude's local field
        new = np.empty_like(self.local)
        keep = field == w
        new[keep] = self.local[keep]
        if self.chunks > 1:
            self._exchange_double_buffered(new, field, w, a, s)
        else:
            for d in range(1, 1 << s):
                v = w ^ d
                partner = (self.rank & ~(fmask << a)) | (v << a)
                send = self.local[field == v]                    # these move to the rank with field v
                recv = self._sendrecv(partner, send)            # the partner's amplitudes whose field is w
                # on arrival their local field becomes the partner's global field v
                new[field == v] = recv
        self.local = new
        for lq, ph in enumerate(self.phys):
            if glob <= ph < glob + s:
                self.phys[lq] = loc + (ph - glob)
            elif loc <= ph < loc + s:
                self.phys[lq] = glob + (ph - loc)
        if record:
            self.history.append((glob, loc, s))

    def _exchange_double_buffered(self, new, field, w, a, s):
        """The exchanges of a fused swap with double buffering (§III-E): each
        partner's block goes in `chunks` pieces through two send / receive
        buffer pairs; the transfer of piece j is in flight while piece j - 1
        is scattered into place and piece j + 1 is gathered, and the first
        piece for the next partner is posted before the last scatter of the
        current one."""
        import torch
        fmask = (1 << s) - 1
        pieces = []  # (partner, send piece, destination index array)
        for d in range(1, 1 << s):
            v = w ^ d
            partner = (self.rank & ~(fmask << a)) | (v << a)
            idx = np.nonzero(field == v)[0]
            for part in np.array_split(idx, self.chunks):
                pieces.append((partner, part))
        bufs = [None, None]  # (requests, receive buffer, destination indices)

        def post(j):
            partner, part = pieces[j]
            src = torch.from_numpy(np.ascontiguousarray(self.local[part]).view(np.float64).copy())  # gather
            out = torch.empty(part.size * 2, dtype=torch.float64)
            reqs = [self.dist.isend(src, partner), self.dist.irecv(out, partner)]
            self.sent += part.size * 16
            bufs[j % 2] = (reqs, out, part, src)

        def finish(j):
            reqs, out, part, _ = bufs[j % 2]
            for r in reqs:
                r.wait()
            new[part] = out.numpy().view(np.complex128)  # scatter
            bufs[j % 2] = None

        if pieces:
            post(0)
            for j in range(len(pieces)):
                if j + 1 < len(pieces):
                    post(j + 1)
                finish(j)

    def swap_gate(self, glob: int, loc: int):
        """A single swap of a global and a local qubit (a fused swap of one)."""
        self.fused_swap(glob, loc, 1)

    def apply(self, gate, policy: str = "fused"):
        """Apply one circuit gate.  Gates on local qubits run in place.  A
        gate touching global qubits: policy "direct" (one-qubit gates only,
        §III-B), "swap" (one swap gate per global qubit, with a local qubit
        the gate does not use), "fused" (one fused swap of all p global
        qubits with a range of p local qubits the gate does not use)."""
        ph = [self.phys[q] for q in gate.qubits]
        glob = [x for x in ph if x >= self.m]
        if glob:
            if policy == "direct":
                if len(gate.qubits) != 1:
                    raise ValueError("direct: one-qubit gates only")
                self.apply_global_1q(gate.name, gate.qubits[0], gate.params)
                return
            busy = set(x for x in ph if x < self.m)
            if policy == "swap":
                for g in glob:
                    loc = max(x for x in range(self.m) if x not in busy)
                    self.swap_gate(g, loc)
                    busy.add(loc)
            elif policy == "fused":
                loc = max(b for b in range(self.m - self.p + 1)
                          if not any(b <= x < b + self.p for x in busy))
                self.fused_swap(self.m, loc, self.p)
            else:
                raise ValueError(policy)
            ph = [self.phys[q] for q in gate.qubits]
        self._gate_local(gate.name, ph, gate.params)

    def restore(self):
        """Move every qubit back to its own position (phys = identity): the
        swaps done so far, each its own inverse, undone in reverse order."""
        for glob, loc, s in reversed(self.history):
            self.fused_swap(glob, loc, s, record=False)
        self.history = []
        if self.phys != list(range(self.n)):
            raise RuntimeError("restore left a permutation")

    # ---- results ---------------------------------------------------------
    def gather(self):
        """The logical state on rank 0 (None elsewhere)."""
        import torch
        R = 1 << self.p
        chunk = torch.from_numpy(self.local.view(np.float64).copy())
        if self.rank == 0:
            parts = [torch.empty_like(chunk) for _ in range(R)]
            self.dist.gather(chunk, gather_list=parts, dst=0)
            full = np.concatenate([t.numpy().view(np.complex128) for t in parts])
            if self.phys == list(range(self.n)):
                return full
            # physical index -> logical index: logical bit q sits at phys[q]
            x = np.arange(1 << self.n, dtype=np.int64)
            logical = np.zeros_like(x)
            for q, ph in enumerate(self.phys):
                logical |= ((x >> ph) & 1) << q
            out = np.empty_like(full)
            out[logical] = full
            return out
        self.dist.gather(chunk, dst=0)
        return None

    def total_sent(self) -> int:
        import torch
        t = torch.tensor([self.sent], dtype=torch.int64)
        self.dist.all_reduce(t)
        return int(t.item())


def run_sharded(n: int, circuit: Sequence, policy: str = "fused", restore: bool = False, x0: int = 0,
                chunks: int = 1):
    """Run a circuit on the emulated ranks; returns (state on rank 0 or None,
    total bytes sent over all ranks)."""
    st = ShardedState(n, x0, chunks)
    for g in circuit:
        st.apply(g, policy)
    if restore:
        st.restore()
    total = st.total_sent()
    return st.gather(), total
