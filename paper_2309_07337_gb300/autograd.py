"""Differentiable halo exchange: the persistent neighbourhood all-to-all-v as a
torch.autograd.Function.

The exchange is linear (every receive slot copies one source element), so its adjoint is
the reverse exchange: each source element receives the sum of the gradients of the
receive slots that read it.  Forward and backward are two persistent requests of the
library (gbx_neighbor_alltoallv_init, gbx_backward_init); each call re-binds them to the
caller's tensors (gbx_request_bind, no copy) and completes them stream-ordered
(gbx_wait_stream), so autograd never blocks the host.  The backward sums in a fixed
order, so gradients are bitwise reproducible.
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

    def run_forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        out = torch.zeros(self.n_recv, dtype=self.dtype, device=x.device)
        r = self.fwd.request
        r.bind(x, out)
        r.start()
        r.wait_stream()
        return out

    def run_backward(self, g: torch.Tensor) -> torch.Tensor:
        g = g.contiguous()
        gx = torch.zeros(self.n_send, dtype=self.dtype, device=g.device)
        self.bwd.bind(g, gx)
        self.bwd.start()
        self.bwd.wait_stream()
        return gx

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        return HaloExchange.apply(x, self)


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
