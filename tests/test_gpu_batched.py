"""GPU: config 3 at full size -- 64 uneven SpMV halo patterns (rows 2^14..2^20, P 64..1024,
8-32 nnz/row, fp32 and fp64) started together by one startall (one CUDA graph, fused
launches per kernel class), in the launch configuration the benchmark times; every
pattern's receive buffer is compared with the same pattern run alone, and a sample of
patterns (the largest, the smallest and two more of each payload type) with the oracle."""
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
    for q in pats:
        dt = torch.float64 if q.dtype == "f64" else torch.float32
        n = q.sendbuf_bytes // (8 if q.dtype == "f64" else 4)
        sb = torch.randn(n, device="cuda", dtype=dt, generator=gen)
        rb = torch.full((q.recvbuf_bytes // sb.element_size(),), -7.0, device="cuda", dtype=dt)
        alone = rb.clone()
        dq = gbx.DevicePattern(q)
        ex = gbx.Exchange(q, sb, rb, "locality" if len(items) % 3 == 0 else "standard", dp=dq)
        ex2 = gbx.Exchange(q, sb, alone, "standard", info="graph=0", dp=dq, graph=ex.graph)
        ex2.start()
        ex2.wait()
        items.append((q, sb, rb, alone, ex, ex2))
    reqs = [it[4].request for it in items]
    for _ in range(2):
        gbx.startall(reqs)
        gbx.waitall(reqs)
    for q, sb, rb, alone, *_ in items:
        assert torch.equal(rb.view(torch.uint8), alone.view(torch.uint8)), q.name
    by_size = sorted(range(64), key=lambda j: pats[j].volume)
    f32 = [j for j in by_size if pats[j].dtype == "f32"]
    f64 = [j for j in by_size if pats[j].dtype == "f64"]
    sample = {by_size[0], by_size[-1], f32[len(f32) // 2], f32[-1], f64[len(f64) // 2], f64[0]}
    for j in sorted(sample):
        q, sb, rb = items[j][0], items[j][1], items[j][2]
        init = np.full(q.recvbuf_bytes // sb.element_size(), -7.0, dtype=sb.cpu().numpy().dtype)
        want = oracle.standard(q, sb.cpu().numpy(), init)
        assert_bytes_equal(rb.cpu().numpy(), want, q.name)
