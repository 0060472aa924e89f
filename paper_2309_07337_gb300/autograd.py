"""Differentiable halo exchange: the persistent neighbourhood all-to-all-v as a
torch.autograd.Function.

The exchange is linear (every receive slot copies one source element), so its adjoint is
the reverse exchange: each source element receives the sum of the gradients of the
receive slots that read it.  Forward and backward are two persistent requests of the
library (gbx_neighbor_alltoallv_init, gbx_backward_init); each call re-binds them to the
caller's tensors (gbx_request_bind, no copy) and completes them stream-ordered
(gbx_wait_stream), so autograd never blocks the host.  The backward sums in a fixed
order, so gradients are bitwise reproducible.  Each call returns a fresh tensor; only the
entries the exchange leaves unwritten are zeroed (none at all for a receive buffer that the
blocks cover completely).
"""
from __future__ import annotations

import torch

from . import DTYPE_CODES, DevicePattern, Exchange, backward_init

_TORCH = {"f32": torch.float32, "f64": torch.float64}


class DistributedHalo:
    """Forward / backward requests of one pattern.  `halo = exchange(x)` maps the send
    buffer of all ranks (x) to the receive buffer of all ranks and is differentiable in x.
    Receive slots no block writes are zero in the output; source elements no slot reads get
    a zero gradient."""

    def __init__(self, p, algorithm: str = "standard", info: str = "", device="cuda"):
        if p.dtype not in _TORCH:
            raise ValueError("differentiation needs an f32 or f64 payload")
        self.p = p
        self.dtype = _TORCH[p.dtype]
        esz = torch.empty((), dtype=self.dtype).element_size()
        self.n_send = p.sendbuf_bytes // esz
        self.n_recv = p.recvbuf_bytes // esz
        x = torch.zeros(self.n_send, dtype=self.dtype, device=device)
        h = torch.zeros(self.n_recv, dtype=self.dtype, device=device)
        self.dp = DevicePattern(p, device)
        self.fwd = Exchange(p, x, h, algorithm=algorithm, info=info, dp=self.dp)
        gh = torch.zeros(self.n_recv, dtype=self.dtype, device=device)
        gx = torch.zeros(self.n_send, dtype=self.dtype, device=device)
        self.bwd = backward_init(self.fwd.request, gh, gx, accumulate=False, info=info)
        assert DTYPE_CODES[p.dtype] in (1, 2)
        # Outputs are fresh tensors every call (autograd may hold several at once), but only
        # the entries the exchange does not write are zeroed: the receive slots no block
        # covers, and the source elements no slot reads.
        cover, read = _coverage(p, esz)
        self.recv_zero = _zero_plan(cover, device)
        self.send_zero = _zero_plan(read, device)

    def run_forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        out = _fresh(self.n_recv, self.dtype, x.device, self.recv_zero)
        r = self.fwd.request
        r.bind(x, out)
        r.start()
        r.wait_stream()
        return out

    def run_backward(self, g: torch.Tensor) -> torch.Tensor:
        g = g.contiguous()
        gx = _fresh(self.n_send, self.dtype, g.device, self.send_zero)
        self.bwd.bind(g, gx)
        self.bwd.start()
        self.bwd.wait_stream()
        return gx

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        return HaloExchange.apply(x, self)


def _coverage(p, esz):
    """Boolean masks over the receive buffer (slots some block writes) and the send buffer
    (elements some slot reads), in units of the payload type, from the pattern's arrays."""
    import numpy as np
    cpe = p.elem_size // esz
    cnt = np.asarray(p.sendcounts, dtype=np.int64)
    owner = np.repeat(np.arange(p.P), np.diff(np.asarray(p.out_ptr)))
    first = np.cumsum(cnt) - cnt
    V = int(cnt.sum())
    k = np.arange(V) - np.repeat(first, cnt)
    slot = np.repeat(np.asarray(p.sdispls, dtype=np.int64), cnt) + k
    r = np.repeat(owner, cnt)
    el = slot if p.send_idx is None else \
        np.asarray(p.send_idx, dtype=np.int64)[np.asarray(p.send_slot_ptr)[r] + slot]
    src0 = (np.asarray(p.send_base)[r] // esz + el * cpe)
    rcnt = np.asarray(p.recvcounts, dtype=np.int64)
    in_owner = np.repeat(np.arange(p.P), np.diff(np.asarray(p.in_ptr)))
    rfirst = np.cumsum(rcnt) - rcnt
    rk = np.arange(int(rcnt.sum())) - np.repeat(rfirst, rcnt)
    dst0 = np.asarray(p.recv_base)[np.repeat(in_owner, rcnt)] // esz + \
        (np.repeat(np.asarray(p.rdispls, dtype=np.int64), rcnt) + rk) * cpe
    cover = np.zeros(p.recvbuf_bytes // esz, dtype=bool)
    read = np.zeros(p.sendbuf_bytes // esz, dtype=bool)
    for c in range(cpe):
        cover[dst0 + c] = True
        read[src0 + c] = True
    return cover, read


def _zero_plan(written, device):
    """What a fresh output needs before the exchange: None (every entry is written), the
    device indices of the unwritten entries, or "all" when they are most of the buffer
    (a full zero fill is then cheaper than an indexed one)."""
    import numpy as np
    miss = np.flatnonzero(~written)
    if len(miss) == 0:
        return None
    if 4 * len(miss) > len(written):
        return "all"
    return torch.from_numpy(miss.astype(np.int64)).to(device)


def _fresh(n, dtype, device, plan):
    if plan is None:
        return torch.empty(n, dtype=dtype, device=device)
    if isinstance(plan, str):
        return torch.zeros(n, dtype=dtype, device=device)
    out = torch.empty(n, dtype=dtype, device=device)
    out.index_fill_(0, plan, 0)
    return out


class HaloExchange(torch.autograd.Function):
    """y = E x with E the exchange's 0/1 map; dL/dx = E^T dL/dy by the reverse exchange."""

    @staticmethod
    def forward(ctx, x, halo: DistributedHalo):
        if x.dtype != halo.dtype or x.numel() != halo.n_send:
            raise ValueError("x must be the pattern's whole send buffer in its payload type")
        ctx.halo = halo
        return halo.run_forward(x)

    @staticmethod
    def backward(ctx, g):
        return ctx.halo.run_backward(g), None
