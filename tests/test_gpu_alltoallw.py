"""GPU: the persistent neighbourhood all-to-all-w (per-edge nested strided datatypes)
against the oracle, byte for byte: random datatypes of every shape, stencil halos through
point-major and component-major field layouts, error codes, the reverse exchange and the
info variants."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from gpu_util import assert_bytes_equal, dev_bytes, forward  # noqa: E402
import pins  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_w(w, send_bytes, recv_init=None, info="", dw=None):
    send = dev_bytes(send_bytes)
    recv = dev_bytes(recv_init) if recv_init is not None else \
        torch.zeros(w.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.WExchange(w, send, recv, info=info, dw=dw)
    ex.start()
    ex.wait()
    ex.send, ex.recv = send, recv
    return recv.cpu().numpy(), ex


def floats(n_bytes, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "f64":
        return rng.standard_normal(n_bytes // 8)
    return rng.standard_normal(n_bytes // 4).astype(np.float32)


@pytest.mark.parametrize("seed", range(40))
def test_random_datatypes_match_oracle(seed):
    w = pt.random_wpattern(seed)
    sb = pt.random_bytes(w.sendbuf_bytes, seed)
    init = pt.random_bytes(w.recvbuf_bytes, seed + 1)
    want = oracle.alltoallw(w, sb, init)
    got, ex = run_w(w, sb, init)
    assert_bytes_equal(got, want, w.name)
    ex.start()
    ex.wait()
    assert_bytes_equal(ex.recv.cpu().numpy(), want, w.name + " second start")


@pytest.mark.parametrize("seed", range(6))
def test_random_datatypes_many_tiles(seed):
    """Messages of hundreds of items over 64 ranks: many tiles and a ragged tail."""
    w = pt.random_wpattern(500 + seed, P=64, max_deg=10, max_items=60, max_el=40)
    sb = pt.random_bytes(w.sendbuf_bytes, seed)
    init = pt.random_bytes(w.recvbuf_bytes, seed + 7)
    got, ex = run_w(w, sb, init)
    assert_bytes_equal(got, oracle.alltoallw(w, sb, init), w.name)
    assert ex.info()["V"] * ex.info()["elem_size"] == int(w.message_bytes().sum())


@pytest.mark.parametrize("info", ["flat=0", "min_run=0", "graph=0", "vec=4", "block=128", "autotune=0",
                                  "flat=0;min_run=0;block=1024"])
def test_info_variants_identical(info):
    for w in (pt.random_wpattern(77, P=32, dtype="f64", max_items=30, max_el=20),
              pt.stencil_w((32, 32, 32), (4, 4, 2), ppn=8, comps=3, layout="soa")):
        sb = pt.random_bytes(w.sendbuf_bytes, 5)
        init = pt.random_bytes(w.recvbuf_bytes, 6)
        got, _ = run_w(w, sb, init, info=info)
        assert_bytes_equal(got, oracle.alltoallw(w, sb, init), f"{w.name} {info}")


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_stencil_halo_through_datatypes(layout):
    """27-point halo of a 64^3 grid over 4^3 ranks, 8 fp64 per point: the datatype form
    over either field layout receives exactly what the index-list exchange receives."""
    w = pt.stencil_w((64, 64, 64), (4, 4, 4), ppn=16, comps=8, layout=layout)
    p = w.meta["v_pattern"]
    x = pt.stencil_field(p, 3)
    npts = int(np.prod(p.meta["blk"]))
    xs = x if layout == "aos" else pt.soa_from_aos(x, p.P, npts, 8)
    got, ex = run_w(w, xs)
    assert_bytes_equal(got, oracle.alltoallw(w, xs), "oracle")
    got_v, _ = forward(p, x)
    assert_bytes_equal(got, got_v, "index-list exchange")
    assert ex.info()["elem_size"] == (16 if layout == "aos" else 8)


def test_stencil_soa_large_and_backward():
    """256^3 grid over 16^3 ranks (P = 4096), 8 fp64 per point, component-major field:
    forward equals the point-major index-list exchange; the reverse exchange of the
    component-major form, transposed back, equals the index-list backward bit for bit
    (both sum each point's terms in destination rank, receive position order)."""
    w = pt.stencil_w((256, 256, 256), (16, 16, 16), ppn=64, comps=8, layout="soa")
    p = w.meta["v_pattern"]
    npts = int(np.prod(p.meta["blk"]))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    x = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    xs = x.view(p.P, npts, 8).transpose(1, 2).contiguous().view(-1)
    hw = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    hv = torch.zeros_like(hw)
    ew = gbx.WExchange(w, xs, hw)
    ev = gbx.Exchange(p, x, hv)
    ew.start(); ew.wait()
    ev.start(); ev.wait()
    assert torch.equal(hw.view(torch.uint8), hv.view(torch.uint8))
    g = torch.randn(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    gw = torch.zeros_like(xs)
    gv = torch.zeros_like(x)
    bw = gbx.backward_init(ew.request, g, gw)
    bv = gbx.backward_init(ev.request, g, gv)
    bw.start(); bw.wait()
    bv.start(); bv.wait()
    back = gw.view(p.P, 8, npts).transpose(1, 2).contiguous().view(-1)
    assert torch.equal(back.view(torch.uint8), gv.view(torch.uint8))


@pytest.mark.parametrize("seed", range(16))
def test_backward_matches_oracle(seed):
    w = pt.random_wpattern(300 + seed, dtype="f64" if seed % 2 else "f32", P=24, max_items=8, max_el=10)
    x = floats(w.sendbuf_bytes, w.dtype, seed)
    _, ex = run_w(w, x)
    g = floats(w.recvbuf_bytes, w.dtype, seed + 1)
    old = floats(w.sendbuf_bytes, w.dtype, seed + 2)
    for acc in (False, True):
        gs = dev_bytes(old)
        b = gbx.backward_init(ex.request, dev_bytes(g), gs, accumulate=acc)
        b.start()
        b.wait()
        assert_bytes_equal(gs.cpu().numpy(), oracle.alltoallw_backward(w, g, old, accumulate=acc),
                           f"{w.name} accumulate={acc}")


def test_w_with_one_contiguous_type_equals_v():
    for seed in (3, 8, 13):
        p = pt.random_pattern(seed, indexed=False)
        w = pt.w_from_v(p)
        sb = pt.random_bytes(p.sendbuf_bytes, seed)
        init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
        got_w, _ = run_w(w, sb, init)
        got_v, _ = forward(p, sb, recv_init=init)
        assert_bytes_equal(got_w, got_v, p.name)


def _error_cases():
    w, g = pins.load_wgolden("alltoallw_vector.json")
    for k, case in enumerate(g["error_cases"]):
        yield f"golden{k}", pins.apply_change(w, case["change"])
    base = pt.random_wpattern(41, P=12)
    busy = np.flatnonzero((base.recvcounts > 0) & (base.type_sizes()[base.recvtypes] > 0))
    assert len(busy) >= 2
    q = pins.apply_change(base, {})
    q.recvcounts[busy[0]] += 1
    yield "count", q
    q = pins.apply_change(base, {})
    q.rdispls[busy[-1]] = base.recvbuf_bytes
    yield "bound", q
    q = pins.apply_change(base, {})
    q.sendtypes[0] = len(base.types)
    yield "type_index", q
    # two non-empty messages into one rank at the same address
    owner = np.repeat(np.arange(base.P), np.diff(base.in_ptr))
    for d in range(base.P):
        mine = busy[owner[busy] == d]
        if len(mine) >= 2:
            q = pins.apply_change(base, {})
            q.rdispls[mine[1]] = q.rdispls[mine[0]]
            yield "overlap", q
            break


@pytest.mark.parametrize("case", list(_error_cases()), ids=lambda c: c[0])
def test_error_codes_match_oracle(case):
    _, w = case
    want = oracle.alltoallw_validate(w)
    assert want != 0
    sb = np.zeros(max(int(w.sendbuf_bytes), 1), np.uint8)[: w.sendbuf_bytes]
    with pytest.raises(gbx.GbxError) as e:
        run_w(w, sb)
    assert e.value.code == want


def test_unsupported_algorithms_and_byte_backward():
    w = pt.random_wpattern(5, dtype="bytes", P=8)
    sb = pt.random_bytes(w.sendbuf_bytes, 1)
    for alg in ("locality", "auto"):
        with pytest.raises(gbx.GbxError) as e:
            run_w(w, sb, info=f"algorithm={alg}")
        assert e.value.code == gbx.ERR_UNSUPPORTED
    _, ex = run_w(w, sb)
    with pytest.raises(gbx.GbxError) as e:
        gbx.backward_init(ex.request, torch.zeros(max(w.recvbuf_bytes, 1), dtype=torch.uint8, device="cuda"),
                          torch.zeros(max(w.sendbuf_bytes, 1), dtype=torch.uint8, device="cuda"))
    assert e.value.code == gbx.ERR_ARG
