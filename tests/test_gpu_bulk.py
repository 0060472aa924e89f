"""GPU: the bulk form (contiguous pieces moved through shared memory by the bulk-copy
engine, cp.async.bulk with mbarrier completion) gives the oracle's bytes wherever it
applies: the locality form's node-pair blocks, user-packed standard exchanges, messages
longer than one piece, datatype exchanges cut into contiguous runs, and batches; no bounded
wait gives up."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from gpu_util import assert_bytes_equal, dev_bytes, forward, payload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    gbx.device_status()          # start from a clean status word


@pytest.fixture(autouse=True)
def status_clean():
    yield
    assert gbx.device_status() == 0, "a bounded wait of the bulk kernel gave up"


@pytest.mark.parametrize("info", ["bulk=2", "bulk=2;graph=0", "bulk=2;autotune=0", "bulk=1"])
def test_locality_node_pair_blocks(info):
    p = pt.config5(edge=8, comps=2)
    x = payload(p, 4)
    want = oracle.standard(p, x)
    got, ex = forward(p, x, "locality", info=info)
    assert_bytes_equal(got, want, info)
    ex.start()
    ex.wait()
    assert_bytes_equal(ex.recv.cpu().numpy(), want, info + " again")


@pytest.mark.parametrize("seed,s", [(1, 16), (2, 32), (3, 48), (4, 64), (5, 128), (6, 4096)])
def test_packed_standard_exchange(seed, s):
    p = pt.random_pattern(seed, P=24, elem_size=s, indexed=False, gaps=False, max_count=40)
    x = pt.random_bytes(p.sendbuf_bytes, seed)
    init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
    got, _ = forward(p, x, "standard", info="bulk=2", recv_init=init)
    assert_bytes_equal(got, oracle.standard(p, x, init), p.name)


def test_messages_longer_than_a_piece():
    """Dense all-to-all-v, 8 ranks, 700 points of 64 bytes (44.8 KB) per rank pair: every
    message is two pieces, the second one short."""
    P, c, s = 8, 700, 64
    r = np.arange(P, dtype=np.int64)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    cnt = np.full(P * P, c)
    disp = np.tile(r * c, P)
    base = torch.from_numpy(r * P * c * s).cuda()
    x = pt.random_bytes(P * P * c * s, 9)
    send = dev_bytes(x)
    recv = torch.zeros_like(send)
    comm = gbx.Comm(P, 4)
    req = gbx.alltoallv_init(comm, send, base, t32(cnt), t32(disp), recv, base, t32(cnt), t32(disp), s, gbx.BYTES,
                             info="bulk=2")
    req.start()
    req.wait()
    want = x.reshape(P, P, c * s).transpose(1, 0, 2).reshape(-1)   # recv[d][r] = send[r][d]
    assert_bytes_equal(recv.cpu().numpy(), want, "dense")


def test_datatype_runs_and_batch():
    w = pt.stencil_w((32, 32, 32), (4, 4, 2), ppn=8, comps=4, layout="aos")
    x = pt.random_bytes(w.sendbuf_bytes, 2)
    recv = torch.zeros(w.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.WExchange(w, dev_bytes(x), recv, info="bulk=2")
    ex.start()
    ex.wait()
    assert_bytes_equal(recv.cpu().numpy(), oracle.alltoallw(w, x), "w aos")
    # a batch of bulk-form requests (locality node-pair blocks of two patterns)
    pats = [pt.config5(edge=4, comps=2), pt.config5(edge=8, comps=4)]
    exs = []
    for k, p in enumerate(pats):
        xs = payload(p, k)
        send = dev_bytes(xs)
        rb = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        exs.append((gbx.Exchange(p, send, rb, "locality", info="bulk=2"), rb, oracle.standard(p, xs)))
    reqs = [e.request for e, _, _ in exs]
    gbx.startall(reqs)
    gbx.waitall(reqs)
    for e, rb, want in exs:
        assert_bytes_equal(rb.cpu().numpy(), want, "batched bulk")


def test_full_size_locality_bulk():
    """512^3: the locality form with bulk node-pair blocks equals the standard form."""
    p = pt.config5()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    x = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    h1 = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    h2 = torch.zeros_like(h1)
    dp = gbx.DevicePattern(p)
    a = gbx.Exchange(p, x, h1, "standard", dp=dp)
    b = gbx.Exchange(p, x, h2, "locality", dp=dp, graph=a.graph, info="bulk=2")
    a.start(); a.wait()
    b.start(); b.wait()
    assert torch.equal(h1.view(torch.uint8), h2.view(torch.uint8))
