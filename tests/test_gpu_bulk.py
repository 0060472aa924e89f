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
from gpu_util import assert_bytes_equal, backward, dev_bytes, forward, grad_payload, payload  # noqa: E402


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


SCATTER = 1 << 9


@pytest.mark.parametrize("seed,s", [(11, 16), (12, 32), (13, 64), (14, 128), (15, 4096)])
def test_backward_scatter_form(seed, s):
    """The reverse exchange's one-term rows in the scatter form (source windows read by the
    bulk-copy engine, scattered to their destinations by threads) give the oracle's bytes,
    alone and beside the folded rows, with and without accumulation (an accumulating
    backward folds every row, so it must equal the oracle too)."""
    for p in (pt.random_pattern(seed, P=24, elem_size=s, dtype="f64", gaps=False, max_count=12, max_deg=8),
              pt.config5(edge=4, comps=s // 8) if s <= 128 else None):
        if p is None:
            continue
        x = payload(p, 1)
        g = grad_payload(p, 2)
        old = payload(p, 3)
        for alg, form in (("standard", 0), ("locality", 1)):
            _, ex = forward(p, x, alg)
            got, b = backward(ex, g, info="bulk=2")
            assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg} s={s}")
            if alg == "standard" and p.volume > 0:   # one-term rows all read the one gradient buffer
                assert b.info()["copy_forms"] & SCATTER, (p.name, b.info()["copy_forms"])
            got, _ = backward(ex, g, old, accumulate=True, info="bulk=2")
            assert_bytes_equal(got, oracle.backward(p, g, old, form=form, accumulate=True),
                               f"{p.name} {alg} s={s} acc")


@pytest.mark.parametrize("info", ["bulk=2;graph=0", "bulk=2;autotune=0", "bulk=2;split_order=source", "bulk=1",
                                  "bulk=2;split_order=dest", "bulk=2;block=128", "bulk=2;block=256",
                                  "bulk=2;block=512", "bulk=2;block=1024"])
def test_backward_scatter_info_variants(info):
    """Every scatter-kernel shape (block=128/256/512/1024 select threads x stages x CTAs per
    SM), eager and graph launches, and the orders that leave the form out."""
    p = pt.config5(edge=8, comps=4)
    x = payload(p, 5)
    g = grad_payload(p, 6)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        gs = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
        b = gbx.backward_init(ex.request, dev_bytes(g), gs, info=info)
        want = oracle.backward(p, g, form=form)
        for rep in range(2):
            b.start()
            b.wait()
            assert_bytes_equal(gs.cpu().numpy(), want, f"{alg} {info} start {rep}")
        if info.startswith("bulk=2") and alg == "standard":   # destination order has no scatter form
            assert bool(b.info()["copy_forms"] & SCATTER) == ("dest" not in info)


def test_backward_scatter_batch_and_full_size():
    """Two scatter-form backwards in one batch; then the 512^3 backward in the scatter form
    equals the default backward (which the exchange tests pin to the oracle) bit for bit."""
    pats = [pt.config5(edge=4, comps=2), pt.config5(edge=8, comps=4)]
    reqs, outs = [], []
    for k, p in enumerate(pats):
        _, ex = forward(p, payload(p, k), "standard")
        g = grad_payload(p, 10 + k)
        gs = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
        b = gbx.backward_init(ex.request, dev_bytes(g), gs, info="bulk=2")
        reqs.append(b)
        outs.append((gs, oracle.backward(p, g, form=0), ex))
    gbx.startall(reqs)
    gbx.waitall(reqs)
    for gs, want, _ in outs:
        assert_bytes_equal(gs.cpu().numpy(), want, "batched scatter backward")
    del reqs, outs
    p = pt.config5()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(8)
    x = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    h = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    ex = gbx.Exchange(p, x, h, "standard")
    g = torch.randn(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    g1 = torch.zeros_like(x)
    g2 = torch.zeros_like(x)
    b1 = gbx.backward_init(ex.request, g, g1)
    b2 = gbx.backward_init(ex.request, g, g2, info="bulk=2")
    assert b2.info()["copy_forms"] & SCATTER
    b1.start(); b1.wait()
    b2.start(); b2.wait()
    assert torch.equal(g1.view(torch.uint8), g2.view(torch.uint8))
