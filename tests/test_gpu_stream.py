"""GPU: the stream form of the flat copies (index arrays copied into shared memory by the
bulk-copy engine, a ring of stages between one producer warp and the consumer warps) gives
the oracle's bytes wherever it applies, forced with info stream=2: the standard exchange on
random patterns (element sizes 4 to 4,096 bytes, ragged last tiles, multigraphs, receive
gaps), the locality form's gathers, the reverse exchange's two-index copy, batches pooling
several patterns into one stream launch, host-resident buffers, and the SpMV halo and the
stencil at full size."""
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

STREAM = 1 << 10
STREAM2 = 1 << 11


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    gbx.device_status()


@pytest.fixture(autouse=True)
def status_clean():
    yield
    assert gbx.device_status() == 0, "a bounded wait of the stream kernel gave up"


@pytest.mark.parametrize("seed", range(24))
def test_random_standard_forward(seed):
    """Packed receive buffers (the flat form applies, so the stream form must run) for even
    seeds; receive gaps and unaligned regions (segments, the stream form left out) for odd."""
    s = [4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 4096][seed % 12]
    packed = seed % 2 == 0
    p = pt.random_pattern(3000 + seed, elem_size=s, max_count=300 if s <= 64 else 20, gaps=not packed)
    x = pt.random_bytes(p.sendbuf_bytes, seed)
    init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
    want = oracle.standard(p, x, init)
    for info in ("stream=2", "stream=2;block=512", "stream=2;block=128", "stream=2;graph=0;max_ctas=3"):
        got, ex = forward(p, x, "standard", info=info, recv_init=init)
        assert_bytes_equal(got, want, f"{p.name} {info}")
        if packed and p.volume > 0:
            assert ex.info()["copy_forms"] & STREAM, (p.name, info, ex.info()["copy_forms"])


@pytest.mark.parametrize("seed", range(12))
def test_random_locality_forward(seed):
    p = pt.random_pattern(3100 + seed, elem_size=[8, 16, 64][seed % 3], gaps=seed % 4 == 3)
    x = pt.random_bytes(p.sendbuf_bytes, seed)
    init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
    got, _ = forward(p, x, "locality", info="stream=2", recv_init=init)
    assert_bytes_equal(got, oracle.standard(p, x, init), p.name)


@pytest.mark.parametrize("seed", range(12))
def test_random_backward_two_index(seed):
    dt = "f64" if seed % 2 else "f32"
    p = pt.random_pattern(3200 + seed, dtype=dt)
    x = payload(p, seed)
    g = grad_payload(p, seed + 5)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        got, b = backward(ex, g, info="stream=2;bulk=0")
        assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg}")


def test_batch_pools_patterns_into_one_stream_launch():
    pats = [pt.random_pattern(3300 + k, elem_size=8, max_count=200, gaps=False) for k in range(6)]
    items = []
    for k, p in enumerate(pats):
        x = pt.random_bytes(p.sendbuf_bytes, k)
        init = pt.random_bytes(p.recvbuf_bytes, k + 50)
        send, recv = dev_bytes(x), dev_bytes(init)
        ex = gbx.Exchange(p, send, recv, "standard", info="stream=2")
        items.append((p, x, init, send, recv, ex))
    reqs = [it[5].request for it in items]
    for _ in range(2):
        gbx.startall(reqs)
        gbx.waitall(reqs)
    for p, x, init, _, recv, _ in items:
        assert_bytes_equal(recv.cpu().numpy(), oracle.standard(p, x, init), p.name)


def test_host_resident_buffers():
    p = pt.random_pattern(3400, elem_size=16, max_count=100, gaps=False)
    x = pt.random_bytes(p.sendbuf_bytes, 1)
    init = pt.random_bytes(p.recvbuf_bytes, 2)
    send = torch.from_numpy(x.copy()).pin_memory()
    recv = torch.from_numpy(init.copy()).pin_memory()
    ex = gbx.Exchange(p, send, recv, "standard", info="stream=2")
    ex.start()
    ex.wait()
    assert_bytes_equal(recv.numpy(), oracle.standard(p, x, init), p.name)


def test_spmv_halo_full_size():
    p = pt.config2()
    x = pt.spmv_x(p, 3)
    want = oracle.standard(p, x)
    for alg in ("standard", "locality"):
        for info in ("stream=2", "stream=2;block=128"):   # tuned shape; the narrow one-chunk shape
            got, ex = forward(p, x, alg, info=info)
            assert ex.info()["copy_forms"] & STREAM
            assert_bytes_equal(got, want, f"{alg} {info}")


def test_stencil_256cube_forward_backward():
    p = pt.config5(edge=16)
    x = payload(p, 11)
    g = grad_payload(p, 12)
    got, ex = forward(p, x, "standard", info="stream=2")
    assert_bytes_equal(got, oracle.standard(p, x), "forward")
    gs, b = backward(ex, g, info="stream=2;bulk=0")
    assert b.info()["copy_forms"] & STREAM2
    assert_bytes_equal(gs, oracle.backward(p, g, form=0), "backward")


@pytest.mark.parametrize("seed", range(10))
def test_stream_fold_every_row(seed):
    """The stream form of the fold (records and term lists staged in shared memory, a row's
    gradient loads issued together) with every row folded (single_split=0), in both orders,
    and accumulating."""
    dt = "f64" if seed % 2 else "f32"
    p = pt.random_pattern(3500 + seed, dtype=dt, max_count=40)
    x = payload(p, seed)
    g = grad_payload(p, seed + 5)
    old = payload(p, seed + 9)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        got, b = backward(ex, g, info="stream=2;single_split=0")
        assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg}")
        got, b = backward(ex, g, grad_send_init=old, accumulate=True, info="stream=2;autotune=0")
        assert_bytes_equal(got, oracle.backward(p, g, grad_send=old, form=form, accumulate=True),
                           f"{p.name} {alg} accumulate")


@pytest.mark.parametrize("alg,form", [("standard", 0), ("locality", 1)])
def test_stream_fold_spmv_and_stencil(alg, form):
    """fp32 one-element rows (the SpMV halo's reverse, many terms per row) and 64-byte fp64
    rows (the 256^3 stencil's edges and corners), stream fold forced."""
    for p, seed in ((pt.config4(n=1 << 16, P=128, ppn=32), 21), (pt.config5(edge=16), 22)):
        x = payload(p, seed)
        g = grad_payload(p, seed + 1)
        _, ex = forward(p, x, alg)
        got, b = backward(ex, g, info="stream=2")
        assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg}")
