"""GPU: a bounded device wait that gives up fails the request instead of passing silently.
The kernels that wait on their own asynchronous copies (the bulk-copy form and the scatter
form) take the spin limit of their main waits from info wait_limit; with a limit of 0 every
main wait gives up at once, deterministically, while the waits that drain copies already in
flight keep their full limit, so the kernel still ends with no copy outstanding.  Nothing
here waits on a flag that never comes: the copies complete, the kernel only stops waiting
for them.  Each case checks that the start reports GBX_ERR_DEVICE_WAIT, that the request can
be started again, and that the context stays usable (a default request right after gives
the oracle's bytes)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from gpu_util import assert_bytes_equal, dev_bytes, grad_payload, payload  # noqa: E402

GIVE_UP = "autotune=0;wait_limit=0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    gbx.device_status()


def _expect_device_wait(fn):
    with pytest.raises(gbx.GbxError) as e:
        fn()
    assert e.value.code == gbx.ERR_DEVICE_WAIT, e.value.code


def test_bulk_form_wait_gives_up():
    p = pt.config5(edge=4, comps=2)            # 16-byte points: node-pair blocks in the bulk form
    x = payload(p, 4)
    want = oracle.standard(p, x)
    send = dev_bytes(x)
    recv = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.Exchange(p, send, recv, "locality", info="bulk=2;" + GIVE_UP)
    assert ex.info()["copy_forms"] & (1 << 8), "the bulk form is not in the program"
    for _ in range(2):                         # inactive after the report, and startable again
        ex.start()
        _expect_device_wait(ex.wait)
    assert ex.request.test()                   # reported once: the word is clear now
    assert gbx.device_status() == 1            # the process-wide aggregate saw it too
    ok = torch.zeros_like(recv)
    good = gbx.Exchange(p, send, ok, "locality", info="bulk=2", dp=ex.dp, graph=ex.graph)
    good.start()
    good.wait()
    assert_bytes_equal(ok.cpu().numpy(), want, "default limit after a failed start")
    assert gbx.device_status() == 0


def test_scatter_form_wait_gives_up():
    p = pt.config5(edge=4, comps=2)
    x = payload(p, 5)
    g = grad_payload(p, 6)
    send = dev_bytes(x)
    recv = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.Exchange(p, send, recv, "standard")
    gr = dev_bytes(g)
    gx = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
    b = gbx.backward_init(ex.request, gr, gx, info="bulk=2;" + GIVE_UP)
    assert b.info()["copy_forms"] & (1 << 9), "the scatter form is not in the program"
    b.start()
    _expect_device_wait(b.wait)
    # completed on a stream instead: the next host completion call reports it
    b.start()
    b.wait_stream()
    torch.cuda.synchronize()
    _expect_device_wait(b.wait)
    assert gbx.device_status() == 1
    gx2 = torch.zeros_like(gx)
    b2 = gbx.backward_init(ex.request, gr, gx2, info="bulk=2")
    b2.start()
    b2.wait()
    assert_bytes_equal(gx2.cpu().numpy(), oracle.backward(p, g, form=0), "default limit after a failed start")
    assert gbx.device_status() == 0


def test_batch_reports_every_member():
    """A pooled bulk launch that gives up leaves pieces of any member unfinished: every
    request of the batch reports it (the batch takes the first request's limit)."""
    p = pt.config5(edge=4, comps=2)
    x = payload(p, 7)
    send = dev_bytes(x)
    outs = [torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    a = gbx.Exchange(p, send, outs[0], "locality", info="bulk=2;" + GIVE_UP)
    b = gbx.Exchange(p, send, outs[1], "locality", info="bulk=2;autotune=0", dp=a.dp, graph=a.graph)
    gbx.startall([a.request, b.request])
    _expect_device_wait(lambda: gbx.waitall([a.request, b.request]))
    assert a.request.test() and b.request.test()   # both waited, both clear now
    gbx.device_status()
    gbx.startall([b.request])                       # b alone keeps its default limit
    gbx.waitall([b.request])
    assert_bytes_equal(outs[1].cpu().numpy(), oracle.standard(p, x), "member started alone")
    assert gbx.device_status() == 0
