"""GPU: the partitioned (early-bird) exchange against the oracle: the receive buffer after
any subset of ready send partitions, the arrival flags of the receive partitions, the
whole exchange once every partition is marked, stream-ordered producers and consumers,
and the state errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from gpu_util import assert_bytes_equal, dev_bytes  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _aligned_cuts(rng, base, total, s, n):
    """n partitions of a buffer whose rank regions start at `base` (increasing): cuts at
    element boundaries of some region (or at its ends), so no element is split."""
    ends = np.append(base[1:], total)
    cand = [np.arange(b, e + 1, s) for b, e in zip(base, ends) if e >= b] + [np.array([0, total])]
    cand = np.unique(np.concatenate(cand))
    pick = np.sort(rng.choice(cand, size=n - 1, replace=True))
    return np.concatenate([[0], pick, [total]]).astype(np.int64)


def elem_cuts(rng, p, n):
    return _aligned_cuts(rng, p.send_base, p.sendbuf_bytes, p.elem_size, n)


def recv_cuts(rng, p, n):
    return _aligned_cuts(rng, p.recv_base, p.recvbuf_bytes, p.elem_size, n)


def make(p, x, init, pc, rc, info=""):
    send = dev_bytes(x)
    recv = dev_bytes(init)
    ex = gbx.Exchange(p, send, recv, "standard")
    pr = gbx.partitioned_init(ex.request, pc, rc, info=info)
    return ex, pr, send, recv


@pytest.mark.parametrize("seed", range(24))
def test_partial_states_and_arrivals_match_oracle(seed):
    rng = np.random.default_rng(seed)
    p = pt.random_pattern(900 + seed, P=int(rng.integers(2, 40)))
    x = pt.random_bytes(p.sendbuf_bytes, seed)
    init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
    n, nr = int(rng.integers(1, 9)), int(rng.integers(1, 6))
    pc, rc = elem_cuts(rng, p, n), recv_cuts(rng, p, nr)
    ex, pr, send, recv = make(p, x, init, pc, rc)
    for epoch in range(2):
        recv.copy_(torch.from_numpy(init))
        pr.start()
        order = rng.permutation(n)
        first = order[: int(rng.integers(0, n + 1))]
        for k in first:
            pr.pready(int(k))
        torch.cuda.synchronize()
        ready = np.zeros(n, np.uint8)
        ready[first] = 1
        assert_bytes_equal(recv.cpu().numpy(), oracle.standard_partial(p, pc, ready, x, init),
                           f"{p.name} epoch {epoch} partial")
        want_arr = oracle.arrived(p, pc, ready, rc)
        assert [pr.parrived(j) for j in range(nr)] == [bool(a) for a in want_arr]
        if len(first) < n:
            with pytest.raises(gbx.GbxError) as e:
                pr.wait()
            assert e.value.code == gbx.ERR_STATE
        for k in order[len(first):]:
            pr.pready(int(k))
        pr.wait()
        assert_bytes_equal(recv.cpu().numpy(), oracle.standard(p, x, init), f"{p.name} epoch {epoch} full")


def test_stream_ordered_producer_and_consumer():
    """Each partition is produced by a kernel on a side stream and marked ready on that
    stream; a consumer stream waits for one receive partition and copies it out.  Every
    value moved is the produced one."""
    p = pt.config5(edge=8, comps=4)
    n = 8
    region = p.sendbuf_bytes // n
    pc = np.array([min(k * region // p.elem_size * p.elem_size, p.sendbuf_bytes) for k in range(n)] +
                  [p.sendbuf_bytes], np.int64)
    rc = np.array([0, p.recv_base[p.P // 2], p.recvbuf_bytes], np.int64)
    x0 = np.zeros(p.sendbuf_bytes // 8)
    ex, pr, send, recv = make(p, x0, np.zeros(p.recvbuf_bytes, np.uint8), pc, rc)
    xs = send.view(torch.float64)
    prod = torch.cuda.Stream()
    cons = torch.cuda.Stream()
    out = torch.zeros(int(rc[2] - rc[1]), dtype=torch.uint8, device="cuda")
    pr.start()
    with torch.cuda.stream(prod):
        for k in range(n):
            lo, hi = int(pc[k]) // 8, int(pc[k + 1]) // 8
            torch.cuda._sleep(200_000)           # a slow producer
            xs[lo:hi] = torch.arange(lo, hi, dtype=torch.float64, device="cuda") * 0.5
            pr.pready(k, prod)
    pr.parrived_stream(1, cons)
    with torch.cuda.stream(cons):
        out.copy_(recv[int(rc[1]):int(rc[2])])
    pr.wait()
    torch.cuda.synchronize()
    want = oracle.standard(p, np.arange(p.sendbuf_bytes // 8) * 0.5)
    assert_bytes_equal(recv.cpu().numpy(), want, "full")
    assert_bytes_equal(out.cpu().numpy(), want[int(rc[1]):int(rc[2])], "consumer copy")


def test_partitions_over_datatype_exchange():
    """Partitioned over a neighbourhood all-to-all-w (component-major stencil)."""
    w = pt.stencil_w((32, 32, 32), (4, 4, 2), ppn=8, comps=3, layout="soa")
    x = pt.random_bytes(w.sendbuf_bytes, 3)
    send = dev_bytes(x)
    recv = torch.zeros(w.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.WExchange(w, send, recv)
    plane = w.sendbuf_bytes // w.P // 3                 # one component plane of one rank
    pc = np.arange(0, w.sendbuf_bytes + 1, plane, dtype=np.int64)
    pr = gbx.partitioned_init(ex.request, pc, [0, w.recvbuf_bytes])
    pr.start()
    for k in range(len(pc) - 1):
        pr.pready(k)
    pr.wait()
    assert_bytes_equal(recv.cpu().numpy(), oracle.alltoallw(w, x), "w partitioned")


def test_state_and_argument_errors():
    p = pt.random_pattern(5, P=8)
    x = pt.random_bytes(p.sendbuf_bytes, 1)
    init = np.zeros(p.recvbuf_bytes, np.uint8)
    pc = np.array([0, p.sendbuf_bytes], np.int64)
    rc = np.array([0, p.recvbuf_bytes], np.int64)
    ex, pr, send, recv = make(p, x, init, pc, rc)

    def code(f, *a):
        with pytest.raises(gbx.GbxError) as e:
            f(*a)
        return e.value.code

    assert code(pr.pready, 0) == gbx.ERR_STATE          # before start
    pr.start()
    assert code(pr.parrived_stream, 0) == gbx.ERR_STATE  # its partition not marked
    pr.pready(0)
    assert code(pr.pready, 0) == gbx.ERR_STATE          # twice in one epoch
    assert code(pr.pready, 1) == gbx.ERR_ARG
    pr.wait()
    assert code(gbx.startall, [pr]) == gbx.ERR_UNSUPPORTED
    # cuts that do not cover the buffer, decrease, or split a sent element
    for bad in ([0, p.sendbuf_bytes - 1], [1, p.sendbuf_bytes], [0, 8, 4, p.sendbuf_bytes]):
        assert code(gbx.partitioned_init, ex.request, bad, rc) == gbx.ERR_ARG
    if p.elem_size > 1 and p.sendcounts.sum() > 0:
        # the oracle decides which cut splits an element that is sent
        rng = np.random.default_rng(0)
        for _ in range(20):
            c = int(rng.integers(1, p.sendbuf_bytes))
            want = None
            try:
                oracle.standard_partial(p, [0, c, p.sendbuf_bytes], [1, 1], x)
                want = 0
            except oracle.OracleError as e:
                want = e.code
            if want == 0:
                gbx.partitioned_init(ex.request, [0, c, p.sendbuf_bytes], rc).free()
            else:
                assert code(gbx.partitioned_init, ex.request, [0, c, p.sendbuf_bytes], rc) == want
    q = pt.random_pattern(6, P=8)
    xq = pt.random_bytes(q.sendbuf_bytes, 2)
    loc = gbx.Exchange(q, dev_bytes(xq), torch.zeros(q.recvbuf_bytes, dtype=torch.uint8, device="cuda"), "locality")
    assert code(gbx.partitioned_init, loc.request, [0, q.sendbuf_bytes], [0, q.recvbuf_bytes]) == gbx.ERR_UNSUPPORTED


def test_config5_slabs():
    """512^3 stencil (the benchmarked exchange) in 8 send partitions of 512 ranks each and
    8 receive partitions: marked in reverse order, the result equals the index-list
    exchange byte for byte; each receive partition arrives only after its feeders."""
    p = pt.config5()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    x = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    h1 = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    h2 = torch.zeros_like(h1)
    dp = gbx.DevicePattern(p)
    ex = gbx.Exchange(p, x, h1, "standard", dp=dp)
    ex2 = gbx.Exchange(p, x, h2, "standard", dp=dp, graph=ex.graph)
    n = 8
    pc = np.array([p.send_base[k * p.P // n] if k < n else p.sendbuf_bytes for k in range(n + 1)], np.int64)
    rc = np.array([p.recv_base[k * p.P // n] if k < n else p.recvbuf_bytes for k in range(n + 1)], np.int64)
    pr = gbx.partitioned_init(ex2.request, pc, rc)
    ex.start()
    ex.wait()
    pr.start()
    for k in reversed(range(n)):
        pr.pready(k)
    pr.wait()
    assert torch.equal(h1.view(torch.uint8), h2.view(torch.uint8))
    assert pr.info()["launches"] == n
