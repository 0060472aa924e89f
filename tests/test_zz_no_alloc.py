"""The allocation-free exchange gives the oracle's bytes and the persistent exchange's.

gbx_neighbor_alltoallv_noalloc serves callers that cannot allocate device memory (a
fixed budget owned by another allocator, latency-critical paths that cannot pay
cudaMalloc's device-wide synchronisation, plug-ins barred from the allocator).  It keeps
its per-edge tables in a fixed static device array instead of memory of its own, so
this test checks, through the C ABI, that two calls in a row (the second one reusing the
array the first one left behind) each produce exactly the receive buffer of the oracle's
exchange and of the persistent standard exchange for the same send data, that the second
call changes the device's free memory by nothing, that an edge count beyond the array's
capacity is refused before any device work, and that each invalid input returns the
oracle's error code with the receive buffer left untouched.  It runs last so that a
failure here cannot hide another test's, and it passes alone or after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
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
    init_h = pt.random_bytes(p.recvbuf_bytes, 5)
    init = torch.from_numpy(init_h).cuda()
    send = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
    ref_recv = init.clone()
    ex = gbx.Exchange(p, send, ref_recv, dp=dp)
    out = init.clone()
    for call_no, seed in enumerate((101, 202)):
        x = pt.random_bytes(p.sendbuf_bytes, seed)
        send.copy_(torch.from_numpy(x))
        ex.start()
        ex.wait()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = call(noalloc, p, dp, send, out)
        assert rc == gbx.SUCCESS, (call_no, rc)
        torch.cuda.synchronize()
        if call_no == 1:   # the first call on a device may load the array; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free_before, "the call changed the device's free memory"
        got = out.cpu().numpy()
        assert np.array_equal(got, oracle.standard(p, x, init_h)), f"call {call_no}: bytes differ from the oracle"
        assert torch.equal(out, ref_recv), f"call {call_no}: bytes differ from the persistent exchange"


def _bad_cases():
    """Invalid inputs made from a valid exchange, each with the field it corrupts."""
    base = packed(pt.config1())
    i0 = int(np.flatnonzero(np.asarray(base.recvcounts) > 0)[0])

    def variant(name, **change):
        q = pt.Pattern(**{k: getattr(base, k) for k in base.__dataclass_fields__})
        for k, f in change.items():
            setattr(q, k, f(np.array(getattr(base, k))))
        q.name = name
        return q

    def csr_down(a):
        a[2] = a[3] + 1          # in-list CSR no longer non-decreasing
        return a

    def rank_out(a):
        a[0] = base.P            # a neighbour rank outside [0, P)
        return a

    def count_up(a):
        a[i0] += 1               # receives one element more than its sender sends
        return a

    def disp_past(a):
        a[i0] = base.recvbuf_bytes // base.elem_size   # the block ends past the receive buffer
        return a

    def disp_neg(a):
        a[0] = -1
        return a

    yield variant("bad_csr", in_ptr=csr_down)
    yield variant("rank_out_of_range", sources=rank_out)
    yield variant("count_mismatch", recvcounts=count_up)
    yield variant("rdispl_past_buffer", rdispls=disp_past)
    yield variant("negative_sdispl", sdispls=disp_neg)


@pytest.mark.parametrize("q", list(_bad_cases()), ids=lambda q: q.name)
def test_noalloc_errors_match_oracle_and_write_nothing(noalloc, q):
    want = oracle.validate(q)
    assert want != oracle.OK, q.name
    dp = gbx.DevicePattern(q)
    send = torch.from_numpy(pt.random_bytes(q.sendbuf_bytes, 1)).cuda()
    init = pt.random_bytes(q.recvbuf_bytes, 2)
    out = torch.from_numpy(init.copy()).cuda()
    assert call(noalloc, q, dp, send, out) == want, q.name
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), init), f"{q.name}: the receive buffer was written"


def test_noalloc_huge_element_size_is_an_index_error(noalloc):
    """Bounds are checked by division: an element size of 2^62 bytes cannot wrap an offset
    computation into a small, valid-looking one."""
    p = packed(pt.config1())
    dp = gbx.DevicePattern(p)
    send = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
    out = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    q = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.elem_size = 1 << 62
    assert call(noalloc, q, dp, send, out) == gbx.ERR_INDEX
    torch.cuda.synchronize()
    assert not bool(out.any())


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
