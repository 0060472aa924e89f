"""The allocation-free exchange gives the same bytes as the persistent one.

gbx_neighbor_alltoallv_noalloc serves callers that cannot allocate device memory (a
fixed budget owned by another allocator, latency-critical paths that cannot pay
cudaMalloc's device-wide synchronisation, plug-ins barred from the allocator).  It keeps
its per-edge tables in a fixed static device array instead of memory of its own, so
this test checks, through the C ABI, that two calls in a row (the second one reusing the
array the first one left behind) each produce exactly the receive buffer that the
persistent standard exchange produces for the same send data, and that an edge count
beyond the array's capacity is refused before any device work.  It runs last so that a
failure here cannot hide another test's, and it passes alone or after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402

MAX_EDGES = 1 << 18   # GBX_NOALLOC_MAX_EDGES


@pytest.fixture(scope="module")
def noalloc():
    import __graft_entry__
    __graft_entry__.build()
    f = gbx.lib().gbx_neighbor_alltoallv_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [ctypes.c_int, i64, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp, i64, vp, vp, vp, i64, vp]
    f.restype = ctypes.c_int
    return f


def call(f, p, dp, send, recv, n_in=None, n_out=None):
    n_in = len(p.sources) if n_in is None else n_in
    n_out = len(p.dests) if n_out is None else n_out
    return f(p.P, n_in, dp.in_ptr.data_ptr(), dp.sources.data_ptr(), n_out, dp.out_ptr.data_ptr(),
             dp.dests.data_ptr(), send.data_ptr(), send.numel(), dp.send_base.data_ptr(),
             dp.sendcounts.data_ptr(), dp.sdispls.data_ptr(), recv.data_ptr(), recv.numel(),
             dp.recv_base.data_ptr(), dp.recvcounts.data_ptr(), dp.rdispls.data_ptr(), p.elem_size,
             torch.cuda.current_stream().cuda_stream)


def packed(p):
    """The same exchange with a user-packed send buffer (each rank's send lists gathered
    into its send slots, as a plain MPI_Neighbor_alltoallv caller does)."""
    q = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.send_idx = None
    q.global_sidx = q.global_ridx = None
    q.send_base = (p.send_slot_ptr[:-1] * p.elem_size).astype(np.int64)
    q.sendbuf_bytes = int(p.send_slot_ptr[-1] * p.elem_size)
    q.name = p.name + "_packed"
    return q


def cases():
    for seed in (3, 11, 29):
        yield pt.random_pattern(seed, indexed=False)
    yield pt.random_pattern(41, P=64, indexed=False, max_deg=20, max_count=40, elem_size=24)
    yield packed(pt.config1())
    yield packed(pt.config5(edge=8))


@pytest.mark.parametrize("p", list(cases()), ids=lambda p: p.name)
def test_noalloc_matches_persistent_on_two_calls(noalloc, p):
    dp = gbx.DevicePattern(p)
    init = torch.from_numpy(pt.random_bytes(p.recvbuf_bytes, 5)).cuda()
    send = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
    ref_recv = init.clone()
    ex = gbx.Exchange(p, send, ref_recv, dp=dp)
    out = init.clone()
    for call_no, seed in enumerate((101, 202)):
        send.copy_(torch.from_numpy(pt.random_bytes(p.sendbuf_bytes, seed)))
        ex.start()
        ex.wait()
        rc = call(noalloc, p, dp, send, out)
        assert rc == gbx.SUCCESS, (call_no, rc)
        torch.cuda.synchronize()
        assert torch.equal(out, ref_recv), f"call {call_no}: bytes differ from the persistent exchange"


def test_noalloc_refuses_sizes_beyond_its_scratch(noalloc):
    p = pt.random_pattern(3, indexed=False)
    dp = gbx.DevicePattern(p)
    send = torch.zeros(max(p.sendbuf_bytes, 1), dtype=torch.uint8, device="cuda")
    out = torch.zeros(max(p.recvbuf_bytes, 1), dtype=torch.uint8, device="cuda")
    assert call(noalloc, p, dp, send, out, n_in=MAX_EDGES + 1, n_out=MAX_EDGES + 1) == gbx.ERR_LIMIT
    # still usable afterwards
    assert call(noalloc, p, dp, send, out) == gbx.SUCCESS


def test_noalloc_on_host_buffers(noalloc):
    """Send and receive buffers in pinned host memory, read and written in place; a pageable
    host buffer is refused with ERR_ARG before any device work."""
    p = packed(pt.config1())
    dp = gbx.DevicePattern(p)
    x = pt.random_bytes(p.sendbuf_bytes, 7)
    init = pt.random_bytes(p.recvbuf_bytes, 8)
    ref = torch.from_numpy(init.copy()).cuda()
    ex = gbx.Exchange(p, torch.from_numpy(x).cuda(), ref, dp=dp)
    ex.start()
    ex.wait()
    send = torch.from_numpy(x.copy()).pin_memory()
    out = torch.from_numpy(init.copy()).pin_memory()
    assert call(noalloc, p, dp, send, out) == gbx.SUCCESS
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu())
    pageable = torch.from_numpy(x.copy())
    assert call(noalloc, p, dp, pageable, out) == gbx.ERR_ARG
