"""Helpers of the GPU tests: run the library on a pattern, compare with the oracle."""
import numpy as np
import torch

import oracle
import paper_2309_07337_gb300 as gbx
from paper_2309_07337_gb300 import patterns as pt


def dev_bytes(a: np.ndarray) -> torch.Tensor:
    b = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
    if not b.flags.writeable:
        b = b.copy()
    return torch.from_numpy(b).cuda()


def forward(p, send_bytes, algorithm="standard", info="", recv_init=None, dp=None):
    """Runs one start/wait; returns (receive bytes, Exchange)."""
    send = dev_bytes(send_bytes)
    recv = dev_bytes(recv_init) if recv_init is not None else \
        torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.Exchange(p, send, recv, algorithm=algorithm, info=info, dp=dp)
    ex.start()
    ex.wait()
    ex.send, ex.recv = send, recv
    return recv.cpu().numpy(), ex


def backward(ex, grad_recv_bytes, grad_send_init=None, accumulate=False, info=""):
    p = ex.p
    gr = dev_bytes(grad_recv_bytes)
    gs = dev_bytes(grad_send_init) if grad_send_init is not None else \
        torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
    b = gbx.backward_init(ex.request, gr, gs, accumulate=accumulate, info=info)
    b.start()
    b.wait()
    return gs.cpu().numpy(), b


def payload(p, seed):
    """Finite values for float patterns (so sums are meaningful), raw bytes otherwise."""
    rng = np.random.default_rng(seed)
    if p.dtype == "f64":
        return rng.standard_normal(p.sendbuf_bytes // 8)
    if p.dtype == "f32":
        return rng.standard_normal(p.sendbuf_bytes // 4).astype(np.float32)
    return pt.random_bytes(p.sendbuf_bytes, seed)


def grad_payload(p, seed):
    rng = np.random.default_rng(seed)
    if p.dtype == "f64":
        return rng.standard_normal(p.recvbuf_bytes // 8)
    return rng.standard_normal(p.recvbuf_bytes // 4).astype(np.float32)


def assert_bytes_equal(got, want, what=""):
    got = np.asarray(got).view(np.uint8).reshape(-1)
    want = np.asarray(want).view(np.uint8).reshape(-1)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{what}: {len(bad)} bytes differ, first at {bad[:8]}")
