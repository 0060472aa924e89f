"""GPU: config 3 at full size -- 64 uneven SpMV halo patterns (rows 2^14..2^20, P 64..1024,
8-32 nnz/row, fp32 and fp64) started together by one startall (one CUDA graph, fused
launches per kernel class), in the launch configuration the benchmark times.  Every
pattern's receive buffer is compared byte for byte with the oracle's exchange, and every
pattern's gradient from the batched reverse exchange (one startall of the 64 backward
requests) with the oracle's backward in the order of its form."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from gpu_util import assert_bytes_equal  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_config3_batched_full_size():
    pats = pt.config3_torch(64, device="cuda")
    assert len(pats) == 64 and {q.dtype for q in pats} == {"f32", "f64"}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 30)
    items = []
    for j, q in enumerate(pats):
        dt = torch.float64 if q.dtype == "f64" else torch.float32
        esz = 8 if q.dtype == "f64" else 4
        sb = torch.randn(q.sendbuf_bytes // esz, device="cuda", dtype=dt, generator=gen)
        rb = torch.full((q.recvbuf_bytes // esz,), -7.0, device="cuda", dtype=dt)
        gr = torch.randn(q.recvbuf_bytes // esz, device="cuda", dtype=dt, generator=gen)
        gx = torch.full_like(sb, 3.0)   # elements no slot reads keep this value
        alg = "locality" if j % 3 == 0 else "standard"
        ex = gbx.Exchange(q, sb, rb, alg, dp=gbx.DevicePattern(q))
        b = gbx.backward_init(ex.request, gr, gx)
        items.append((q, sb, rb, gr, gx, ex, b, alg))
    fwd = [it[5].request for it in items]
    bwd = [it[6] for it in items]
    for _ in range(2):                   # a second start must give the same bytes
        gbx.startall(fwd)
        gbx.waitall(fwd)
        gbx.startall(bwd)
        gbx.waitall(bwd)
    host = [(q, sb.cpu().numpy(), rb.cpu().numpy(), gr.cpu().numpy(), gx.cpu().numpy(), alg)
            for q, sb, rb, gr, gx, _, _, alg in items]
    del items, fwd, bwd

    def check(h):
        q, x, got, g, got_g, alg = h
        init = np.full(len(got), -7.0, dtype=got.dtype)
        assert_bytes_equal(got, oracle.standard(q, x, init), q.name)
        g0 = np.full(len(got_g), 3.0, dtype=got_g.dtype)
        want_g = oracle.backward(q, g, g0, form=0 if alg == "standard" else 1)
        assert_bytes_equal(got_g, want_g, q.name + " backward " + alg)
        return q.volume

    # the oracle is C called through ctypes, which releases the GIL: one pattern per thread
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as pool:
        vols = list(pool.map(check, host))
    assert sum(vols) == sum(h[0].volume for h in host)
