"""GPU parity: the CUDA path against the CPU oracle, byte for byte, through the C ABI."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2309_07337_gb300 as gbx  # noqa: E402
import pins  # noqa: E402
from gpu_util import (assert_bytes_equal, backward, dev_bytes, forward, grad_payload,  # noqa: E402
                      payload)
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


# ------------------------------------------------------------------- golden
@pytest.mark.parametrize("name", ["ring3.json", "multigraph.json", "locality_dedup.json",
                                  "backward_order.json", "backward_order2.json"])
def test_golden_forward(name):
    g = pins.load_golden(name)
    algs = ["standard"] + (["locality"] if g.global_sidx is not None else [])
    for alg in algs:
        got, _ = forward(g, g.sendbuf, alg, recv_init=g.recv_init)
        assert_bytes_equal(got, np.array(g.expected_recv, dtype=g.vt), f"{name} {alg}")


@pytest.mark.parametrize("name", ["locality_dedup.json", "backward_order.json", "backward_order2.json"])
def test_golden_backward(name):
    g = pins.load_golden(name)
    gr = np.array(g.grad_recv, dtype=np.float64)
    for alg, key in (("standard", "standard"), ("locality", "node_blocked")):
        _, ex = forward(g, g.sendbuf, alg, recv_init=g.recv_init)
        got, _ = backward(ex, gr)
        want = getattr(g, f"expected_grad_{key}", None) or g.expected_grad_send
        assert_bytes_equal(got, np.array(want, dtype=np.float64), f"{name} {alg}")
        if hasattr(g, "grad_send_init"):
            got, _ = backward(ex, gr, np.array(g.grad_send_init), accumulate=True)
            assert_bytes_equal(got, np.array(getattr(g, f"expected_grad_{key}_accumulate")), f"{name} {alg} acc")


def test_golden_locality_stats():
    g = pins.load_golden("locality_dedup.json")
    _, ex = forward(g, g.sendbuf, "locality", recv_init=g.recv_init)
    info = ex.info()
    for k, v in g.expected_stats.items():
        assert info[k] == v, (k, info[k], v)


# ---------------------------------------------------------- random patterns
@pytest.mark.parametrize("seed", range(60))
def test_random_forward(seed):
    p = pt.random_pattern(seed)
    x = pt.random_bytes(p.sendbuf_bytes, seed + 1)
    init = pt.random_bytes(p.recvbuf_bytes, seed + 2)
    want = oracle.standard(p, x, init)
    for alg in ("standard", "locality"):
        got, ex = forward(p, x, alg, recv_init=init)
        assert_bytes_equal(got, want, f"{p.name} {alg}")
        info = ex.info()
        assert info["V"] == p.volume


@pytest.mark.parametrize("seed", range(30))
def test_random_backward(seed):
    dt = "f64" if seed % 2 else "f32"
    p = pt.random_pattern(1000 + seed, dtype=dt)
    x = payload(p, seed)
    g = grad_payload(p, seed + 5)
    old = payload(p, seed + 9)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        got, _ = backward(ex, g)
        assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg}")
        got, _ = backward(ex, g, old, accumulate=True)
        assert_bytes_equal(got, oracle.backward(p, g, old, form=form, accumulate=True), f"{p.name} {alg} acc")


# ------------------------------------------------------------------ configs
def _config_case(p, seed, algs=("standard", "locality"), backward_too=True):
    x = payload(p, seed)
    want = oracle.standard(p, x)
    for alg in algs:
        got, ex = forward(p, x, alg)
        assert_bytes_equal(got, want, f"{p.name} {alg}")
        if backward_too and p.dtype in ("f32", "f64"):
            g = grad_payload(p, seed + 1)
            got, _ = backward(ex, g)
            assert_bytes_equal(got, oracle.backward(p, g, form=0 if alg == "standard" else 1),
                               f"{p.name} {alg} backward")
    return ex


def test_config1_stencil2d():
    ex = _config_case(pt.config1(), pt.SEED + 1)
    assert ex.info()["E"] == 48


def test_config2_spmv_halo_full():
    _config_case(pt.config2(), pt.SEED + 2)


def test_config4_small_copy_f32():
    _config_case(pt.config4(n=4096, P=64), pt.SEED + 4)


def test_config5_reduced_128cube():
    _config_case(pt.config5(edge=8), pt.SEED + 5)


def test_config5_message_size_sweep_small():
    for comps in (1, 2, 4, 16):
        _config_case(pt.config5(edge=4, comps=comps), pt.SEED + 5 + comps, backward_too=comps == 2)


def test_config5_full_512cube():
    """The full 512^3 27-point stencil (8.59 GB field, 1.6 GB halo) in the launch
    configuration the benchmark times (persistent request, CUDA graph, tuned shape)."""
    p = pt.config5()
    x = pt.stencil_field(p, pt.SEED + 5)
    want = oracle.standard(p, x)
    for alg in ("standard", "locality"):
        got, ex = forward(p, x, alg)
        assert_bytes_equal(got, want, f"{p.name} {alg}")
        del ex
        torch.cuda.empty_cache()


# ---------------------------------------------------------------- behaviour
def test_shapes_and_graph_modes_identical():
    p = pt.config5(edge=4, comps=3)
    x = payload(p, 3)
    want = oracle.standard(p, x)
    for info in ("graph=0", "autotune=0", "vec=8;block=128", "vec=4;block=1024", "vec=8;block=512;graph=0",
                 "min_run=0", "min_run=1;vec=8", "min_run=2;block=256", "piece=32", "piece=7;min_run=0",
                 "piece=1;vec=4", "flat=1", "flat=0", "flat=1;block=128;min_run=0"):
        for alg in ("standard", "locality"):
            got, _ = forward(p, x, alg, info=info)
            assert_bytes_equal(got, want, f"{info} {alg}")


def test_auto_picks_a_form_with_identical_output():
    p = pt.config2(n=1 << 16, P=64)
    x = payload(p, 4)
    got, ex = forward(p, x, "auto")
    assert_bytes_equal(got, oracle.standard(p, x), "auto")
    assert ex.info()["algorithm"] in (0, 1)


def test_repeated_starts_and_rebind():
    p = pt.random_pattern(77, elem_size=8, indexed=True)
    x1, x2 = pt.random_bytes(p.sendbuf_bytes, 1), pt.random_bytes(p.sendbuf_bytes, 2)
    got, ex = forward(p, x1, "locality")
    for _ in range(3):
        ex.start()
        ex.wait()
    assert_bytes_equal(ex.recv.cpu().numpy(), oracle.standard(p, x1), "repeat")
    s2 = dev_bytes(x2)
    r2 = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex.request.bind(s2, r2)
    ex.start()
    ex.wait()
    assert_bytes_equal(r2.cpu().numpy(), oracle.standard(p, x2), "rebound")


def test_start_on_active_request_and_test():
    p = pt.config1()
    _, ex = forward(p, payload(p, 1))
    ex.start()
    with pytest.raises(gbx.GbxError) as e:
        ex.start()
    assert e.value.code == gbx.ERR_ACTIVE
    ex.wait()
    assert ex.request.test()


def test_wait_timeout_returns_error_then_completes():
    """Failure detection without a GPU fault: the stream is held by a bounded sleep kernel
    longer than the request's timeout; wait reports GBX_ERR_TIMEOUT, the request stays
    active, and a later wait completes it."""
    p = pt.config1()
    x = payload(p, 2)
    send = dev_bytes(x)
    recv = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.Exchange(p, send, recv, info="timeout_ms=100")
    torch.cuda._sleep(2_000_000_000)   # a bounded spin of 2e9 SM cycles: about 1 s at 2 GHz
    ex.start()
    with pytest.raises(gbx.GbxError) as e:
        ex.wait()
    assert e.value.code == gbx.ERR_TIMEOUT
    torch.cuda.synchronize()
    ex.wait()
    assert_bytes_equal(recv.cpu().numpy(), oracle.standard(p, x), "after timeout")


def test_startall_mixed_sizes_matches_individual():
    pats = [pt.random_pattern(500 + i, elem_size=[4, 8, 24, 64, 3][i % 5]) for i in range(10)]
    xs = [pt.random_bytes(p.sendbuf_bytes, i) for i, p in enumerate(pats)]
    exs = []
    for p, x in zip(pats, xs):
        send = dev_bytes(x)
        recv = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        ex = gbx.Exchange(p, send, recv, algorithm="locality" if len(exs) % 2 else "standard")
        ex.send, ex.recv = send, recv
        exs.append(ex)
    reqs = [e.request for e in exs]
    for _ in range(2):
        for e in exs:
            e.recv.zero_()
        gbx.startall(reqs)
        gbx.waitall(reqs)
        for p, x, e in zip(pats, xs, exs):
            assert_bytes_equal(e.recv.cpu().numpy(), oracle.standard(p, x), f"batched {p.name}")


@pytest.mark.parametrize("seed", range(4))
def test_startall_random_forward_and_backward_batch(seed):
    """One gbx_startall of random forward requests (both forms, fp32 and fp64, indexed and
    packed sends) and the backward requests of the same patterns (accumulating on every other
    one), started together twice: every receive buffer equals the oracle's exchange and every
    gradient the oracle's reverse exchange in the order of its form, byte for byte."""
    pats = [pt.random_pattern(1300 + 10 * seed + i, dtype="f64" if i % 2 else "f32", indexed=bool(i % 3))
            for i in range(8)]
    items = []
    for i, q in enumerate(pats):
        alg, form = ("locality", 1) if i % 2 == 0 else ("standard", 0)
        x = payload(q, 50 + i)
        g = grad_payload(q, 60 + i)
        old = payload(q, 70 + i)
        acc = i % 4 >= 2
        send, recv = dev_bytes(x), torch.zeros(q.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        ex = gbx.Exchange(q, send, recv, algorithm=alg)
        gr, gs = dev_bytes(g), dev_bytes(old)
        b = gbx.backward_init(ex.request, gr, gs, accumulate=acc)
        items.append((q, x, g, old, acc, form, recv, gs, ex, b))
    reqs = [it[8].request for it in items] + [it[9] for it in items]
    for rep in range(2):
        for q, x, g, old, acc, form, recv, gs, ex, b in items:
            recv.zero_()
            gs.copy_(dev_bytes(old))
        gbx.startall(reqs)
        gbx.waitall(reqs)
        for q, x, g, old, acc, form, recv, gs, ex, b in items:
            assert_bytes_equal(recv.cpu().numpy(), oracle.standard(q, x), f"{q.name} forward #{rep}")
            want = oracle.backward(q, g, old, form=form, accumulate=acc)
            assert_bytes_equal(gs.cpu().numpy(), want, f"{q.name} backward acc={acc} #{rep}")


def test_startall_rebind_moves_batch_to_new_buffers():
    """A batch keeps its launches across rebinds: every request of a started batch is rebound
    to new buffers, first as aligned as the old ones, then offset by half an element (accepted
    only where the request's tuned vector allows it); each start writes the oracle's bytes into
    the buffers bound at that moment."""
    pats = [pt.random_pattern(540 + i, elem_size=[8, 16, 64, 4][i % 4]) for i in range(8)]
    xs = [pt.random_bytes(p.sendbuf_bytes, 40 + i) for i, p in enumerate(pats)]
    bound = [torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda") for p in pats]
    exs = [gbx.Exchange(p, dev_bytes(x), r, algorithm="locality" if i % 2 else "standard")
           for i, (p, x, r) in enumerate(zip(pats, xs, bound))]
    reqs = [e.request for e in exs]

    def run(tag):
        for r in bound:
            r.fill_(0x5A)
        gbx.startall(reqs)
        gbx.waitall(reqs)
        for p, x, r in zip(pats, xs, bound):
            init = np.full(p.recvbuf_bytes, 0x5A, dtype=np.uint8)   # gaps keep this byte
            assert_bytes_equal(r.cpu().numpy(), oracle.standard(p, x, init), f"{tag} {p.name}")

    run("first")
    for i, (p, x) in enumerate(zip(pats, xs)):
        s2 = dev_bytes(x)
        r2 = torch.empty(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        reqs[i].bind(s2, r2)
        bound[i] = r2
    run("rebound")
    moved = 0
    for i, (p, x) in enumerate(zip(pats, xs)):
        off = p.elem_size // 2
        s3 = torch.empty(p.sendbuf_bytes + off, dtype=torch.uint8, device="cuda")
        r3 = torch.empty(p.recvbuf_bytes + off, dtype=torch.uint8, device="cuda")
        s3[off:].copy_(dev_bytes(x))
        try:
            reqs[i].bind(s3[off:], r3[off:])
        except gbx.GbxError as e:
            assert e.code == gbx.ERR_ARG   # the request's vector needs more alignment
            continue
        bound[i] = r3[off:]
        moved += 1
    run(f"offset ({moved} of {len(reqs)} moved)")


def test_host_buffers_end_to_end():
    p = pt.config1()
    x = payload(p, 5)
    send = dev_bytes(x)
    recv = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    ex = gbx.Exchange(p, send, recv)
    hs = torch.from_numpy(x.view(np.uint8).copy()).pin_memory()
    hr = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8).pin_memory()
    ex.request.start_host(hs, hr)
    assert_bytes_equal(hr.numpy(), oracle.standard(p, x), "host buffers")


def test_host_buffers_pipelined_steps():
    """Stream-ordered host-buffer starts over two request sets (standard and locality forward
    over one uploaded field, backward with an uploaded gradient), four steps with different
    inputs in flight together: every step's read-back equals the oracle's."""
    p = pt.config5(edge=4, comps=2)
    steps = 4
    xs = [payload(p, 20 + k) for k in range(steps)]
    gs = [grad_payload(p, 40 + k) for k in range(steps)]
    hx = [torch.from_numpy(x.view(np.uint8).copy()).pin_memory() for x in xs]
    hg = [torch.from_numpy(g.view(np.uint8).copy()).pin_memory() for g in gs]
    out = [[torch.zeros(n, dtype=torch.uint8).pin_memory() for n in (p.recvbuf_bytes, p.recvbuf_bytes,
                                                                       p.sendbuf_bytes)] for _ in range(steps)]
    sets = []
    for k in range(2):
        field = torch.zeros(p.sendbuf_bytes, dtype=torch.uint8, device="cuda")
        h1 = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        h2 = torch.zeros_like(h1)
        g = torch.zeros(p.recvbuf_bytes, dtype=torch.uint8, device="cuda")
        gf = torch.zeros_like(field)
        a = gbx.Exchange(p, field, h1, "standard")
        b = gbx.Exchange(p, field, h2, "locality")
        sets.append((a, b, gbx.backward_init(a.request, g, gf), (field, h1, h2, g, gf)))
    side = torch.cuda.Stream()
    for k in range(steps):
        a, b, bw, _ = sets[k % 2]
        a.request.start_host_async(hx[k], out[k][0])
        b.request.start_host_async(None, out[k][1])
        bw.start_host_async(hg[k], out[k][2])
        for r in (a.request, b.request, bw):
            r.wait_stream(side)          # completes without ordering the requests' stream
    torch.cuda.synchronize()
    for k in range(steps):
        want = oracle.standard(p, xs[k])
        assert_bytes_equal(out[k][0].numpy(), want, f"step {k} standard")
        assert_bytes_equal(out[k][1].numpy(), want, f"step {k} locality")
        assert_bytes_equal(out[k][2].numpy(), oracle.backward(p, gs[k], form=0), f"step {k} backward")
    # a plain start after host starts is ordered after their read-back
    a, _, _, bufs = sets[0]
    a.start()
    a.wait()
    assert_bytes_equal(bufs[1].cpu().numpy(), oracle.standard(p, xs[2]), "plain start after host starts")


# ------------------------------------------------------------------- errors
def _error_cases():
    base = pins.load_golden("ring3.json")

    def mod(**kw):
        g = pins.load_golden("ring3.json")
        for k, (i, v) in kw.items():
            a = getattr(g, k).copy()
            a[i] = v
            setattr(g, k, a)
        return g
    yield "rank", mod(dests=(0, 5))
    yield "unmatched", mod(dests=(0, 2))
    yield "count", mod(recvcounts=(0, 3))
    yield "rdispl_past_end", mod(rdispls=(3, 9))
    yield "negative_sdispl", mod(sdispls=(1, -1))
    yield "overlap", mod(rdispls=(1, 1))
    yield "not_csr", mod(in_ptr=(1, 4))
    p = pt.spmv_halo(600, 4, 2, 6, seed=1, dtype="f64", band=80)
    q = dataclasses.replace(p)
    q.send_idx = p.send_idx.copy()
    q.send_idx[3] = 10 ** 6
    yield "send_idx", q
    q = dataclasses.replace(p)
    q.global_ridx = p.global_ridx.copy()
    q.global_ridx[5] += 1
    yield "gidx", q
    del base


@pytest.mark.parametrize("case", list(_error_cases()), ids=lambda c: c[0])
def test_error_codes_match_oracle(case):
    _, g = case
    want = oracle.validate(g)
    assert want != 0
    sb = np.zeros(max(int(g.sendbuf_bytes), 1), np.uint8)[: g.sendbuf_bytes]
    with pytest.raises(gbx.GbxError) as e:
        forward(g, sb, "standard")
    assert e.value.code == want


@pytest.mark.parametrize("info", ["", "single_split=0", "flat=0", "vec=8;block=128", "single_split=0;block=1024",
                                  "max_ctas=7", "max_ctas=1;bulk=2",
                                  "split_order=source", "split_order=source;vec=8", "split_order=dest",
                                  "bulk=2"])
def test_backward_modes_identical(info):
    """Every backward program shape (single-term rows split out or folded, flat or segment
    copies, any launch shape) gives the oracle's bytes."""
    for p in (pt.config5(edge=4, comps=2), pt.random_pattern(321, dtype="f32"), pt.config4(n=4096, P=64)):
        x = payload(p, 1)
        g = grad_payload(p, 2)
        old = payload(p, 3)
        for alg, form in (("standard", 0), ("locality", 1)):
            _, ex = forward(p, x, alg, info=info)
            got, _ = backward(ex, g, info=info)
            assert_bytes_equal(got, oracle.backward(p, g, form=form), f"{p.name} {alg} {info}")
            got, _ = backward(ex, g, old, accumulate=True, info=info)
            assert_bytes_equal(got, oracle.backward(p, g, old, form=form, accumulate=True),
                               f"{p.name} {alg} {info} acc")


def test_accumulating_backward_init_leaves_gradient_untouched():
    """Init of an accumulating backward must not launch into the caller's gradient buffer
    (the autotuner never trial-runs it); the first start adds exactly once."""
    p = pt.config5(edge=4, comps=2)
    x = payload(p, 1)
    g = grad_payload(p, 2)
    old = payload(p, 3)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        gr = dev_bytes(g)
        gs = dev_bytes(old.copy())
        b = gbx.backward_init(ex.request, gr, gs, accumulate=True)
        torch.cuda.synchronize()
        assert_bytes_equal(gs.cpu().numpy(), old, f"{alg}: init changed the gradient buffer")
        b.start()
        b.wait()
        assert_bytes_equal(gs.cpu().numpy(), oracle.backward(p, g, old, form=form, accumulate=True), alg)


def _dup_pattern(seed):
    """A random pattern in which one inter-node send slot is given the global index of
    another slot of the same node pair that reads different bytes (receive indices
    dropped), so the locality form would send the first slot's value for both."""
    p = pt.random_pattern(seed, indexed=True, P=24, ppn=4)
    x = pt.random_bytes(p.sendbuf_bytes, seed)
    owner = np.repeat(np.arange(p.P), np.diff(p.out_ptr))
    seen = {}
    for e in range(len(p.dests)):
        r, d = int(owner[e]), int(p.dests[e])
        if r // p.ppn == d // p.ppn:
            continue
        for k in range(int(p.sendcounts[e])):
            slot = int(p.send_slot_ptr[r] + p.sdispls[e] + k)
            off = int(p.send_base[r] + p.send_idx[slot] * p.elem_size)
            key = (r // p.ppn, d // p.ppn)
            if key in seen:
                s0, o0 = seen[key]
                if o0 != off and not np.array_equal(x[o0:o0 + p.elem_size], x[off:off + p.elem_size]):
                    q = pt.Pattern(**{k_: getattr(p, k_) for k_ in p.__dataclass_fields__})
                    q.global_sidx = p.global_sidx.copy()
                    q.global_sidx[slot] = p.global_sidx[s0]
                    q.global_ridx = None
                    q.recv_slot_ptr = None
                    return q, x
            else:
                seen[key] = (slot, off)
    return None, None


@pytest.mark.parametrize("seed", [3, 8, 21])
def test_check_dup_reports_conflicting_global_indices(seed):
    q, x = _dup_pattern(seed)
    if q is None:
        pytest.skip("no inter-node pair with two distinct slots")
    with pytest.raises(oracle.OracleError) as oe:
        oracle.locality(q, x)
    assert oe.value.code == gbx.ERR_DUP
    with pytest.raises(gbx.GbxError) as e:
        forward(q, x, "locality", info="check_dup=1")
    assert e.value.code == gbx.ERR_DUP
    forward(q, x, "locality")            # without the debug check init does not read the payload
    # consistent indices pass the check and change nothing
    p = pt.config5(edge=4, comps=2)
    xs = payload(p, 1)
    got, _ = forward(p, xs, "locality", info="check_dup=1")
    assert_bytes_equal(got, oracle.standard(p, xs), "check_dup on a valid pattern")


def test_config5_full_512cube_backward():
    """The backward of the full 512^3 exchange, both forms, against the oracle bit for bit
    (fp64 gradients; each form in its own fixed summation order)."""
    p = pt.config5()
    x = pt.stencil_field(p, pt.SEED + 5)
    g = grad_payload(p, 77)
    for alg, form in (("standard", 0), ("locality", 1)):
        _, ex = forward(p, x, alg)
        got, b = backward(ex, g)
        assert_bytes_equal(got, oracle.backward(p, g, form=form), f"full backward {alg}")
        del ex, b
        torch.cuda.empty_cache()


def test_backward_bit_identical_over_100_starts_512cube():
    """Determinism of the reverse exchange at full size, in the launch configuration the
    benchmark times: 100 starts of each form's backward give the same field gradient, bit for
    bit (fixed summation order, no atomics), and it is the oracle's."""
    p = pt.config5()
    x = torch.from_numpy(pt.stencil_field(p, pt.SEED + 5)).cuda()
    halo = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    g_np = grad_payload(p, 78)
    g = torch.from_numpy(g_np).cuda()
    dp = gbx.DevicePattern(p)
    for alg, form in (("standard", 0), ("locality", 1)):
        ex = gbx.Exchange(p, x, halo, alg, dp=dp)
        gx = torch.zeros_like(x)
        b = gbx.backward_init(ex.request, g, gx)
        b.start()
        b.wait()
        first = gx.clone()
        for _ in range(100):
            gx.zero_()   # (source points no slot reads keep the initial zeros)
            b.start()
            b.wait()
            assert torch.equal(gx.view(torch.uint8), first.view(torch.uint8)), f"{alg}: a start changed the gradient"
        assert_bytes_equal(first.cpu().numpy(), oracle.backward(p, g_np, form=form), f"{alg} vs oracle")
        del ex, b, gx, first
        torch.cuda.empty_cache()


def _explicit(P, ppn, out_lists, in_lists, s, send_base, recv_base, sendbuf_bytes, recvbuf_bytes, dtype="bytes"):
    """Pattern from per-rank lists: out_lists[r] = [(d, count, sdispl)], in_lists[d] = [(r, count, rdispl)]."""
    def csr(lists):
        return np.concatenate([[0], np.cumsum([len(l) for l in lists])]).astype(np.int32)
    flat = lambda lists, j: np.array([t[j] for l in lists for t in l], np.int32)
    return pt.Pattern(name="explicit", P=P, ppn=ppn, in_ptr=csr(in_lists), sources=flat(in_lists, 0),
                      out_ptr=csr(out_lists), dests=flat(out_lists, 0), sendcounts=flat(out_lists, 1),
                      sdispls=flat(out_lists, 2), recvcounts=flat(in_lists, 1), rdispls=flat(in_lists, 2),
                      elem_size=s, dtype=dtype, send_base=np.array(send_base, np.int64),
                      recv_base=np.array(recv_base, np.int64), sendbuf_bytes=sendbuf_bytes,
                      recvbuf_bytes=recvbuf_bytes)


def _degenerate_cases():
    # one rank sending to itself
    yield "self", _explicit(1, 1, [[(0, 5, 0)]], [[(0, 5, 2)]], 8, [0], [0], 40, 64, "f64")
    # a graph with no edges
    yield "no_edges", _explicit(4, 2, [[], [], [], []], [[], [], [], []], 8, [0] * 4, [0] * 4, 8, 8)
    # edges that all carry nothing
    yield "zero_counts", _explicit(3, 1, [[(1, 0, 0)], [(2, 0, 3)], [(0, 0, 1)]],
                                   [[(2, 0, 0)], [(0, 0, 1)], [(1, 0, 0)]], 4, [0, 8, 16], [0, 8, 16], 24, 24)
    # one large element per message
    yield "elem_4096", _explicit(2, 1, [[(1, 1, 0)], [(0, 1, 1)]], [[(1, 1, 0)], [(0, 1, 1)]], 4096,
                                 [0, 8192], [0, 8192], 16384, 16384)
    # one-byte elements at odd offsets, two nodes, a repeated neighbour
    yield "bytes_odd", _explicit(4, 2, [[(3, 3, 1), (3, 2, 0)], [], [(0, 1, 2)], [(1, 4, 0)]],
                                 [[(2, 1, 0)], [(3, 4, 3)], [], [(0, 3, 0), (0, 2, 5)]], 1,
                                 [1, 7, 11, 13], [3, 5, 14, 17], 19, 27)


@pytest.mark.parametrize("case", list(_degenerate_cases()), ids=lambda c: c[0])
def test_degenerate_patterns(case):
    _, p = case
    assert oracle.validate(p) == 0
    x = pt.random_bytes(p.sendbuf_bytes, 1) if p.dtype == "bytes" else payload(p, 1)
    init = pt.random_bytes(p.recvbuf_bytes, 2)
    want = oracle.standard(p, x, init)
    for alg in ("standard", "locality"):
        got, ex = forward(p, x, alg, recv_init=init)
        assert_bytes_equal(got, want, f"{case[0]} {alg}")
        ex.start()
        ex.wait()
        if p.dtype == "f64":
            g = grad_payload(p, 3)
            got, _ = backward(ex, g)
            assert_bytes_equal(got, oracle.backward(p, g, form=0 if alg == "standard" else 1), f"{case[0]} bwd")


def test_element_offsets_beyond_int32():
    """One-byte elements in a 2.15 GB send buffer: rank 1's elements lie past 2^31 elements,
    which the flat form's 31-bit element indices cannot name, so those copies take the
    segment form (64-bit offsets).  Both forms give the oracle's bytes, twice."""
    base1 = (1 << 31) + 4096
    sendbuf = base1 + 65536
    p = _explicit(2, 1, [[(1, 1000, 0)], [(0, 3000, 100), (1, 500, 20000)]],
                  [[(1, 3000, 0)], [(0, 1000, 0), (1, 500, 1000)]], 1, [0, base1], [0, 4096], sendbuf, 8192)
    assert oracle.validate(p) == 0
    x = np.zeros(sendbuf, np.uint8)
    x[:4096] = pt.random_bytes(4096, 7)
    x[base1:] = pt.random_bytes(65536, 8)
    init = pt.random_bytes(p.recvbuf_bytes, 9)
    want = oracle.standard(p, x, init)
    send = dev_bytes(x)
    for alg in ("standard", "locality"):
        recv = dev_bytes(init)
        ex = gbx.Exchange(p, send, recv, alg)
        for rep in range(2):
            ex.start()
            ex.wait()
            assert_bytes_equal(recv.cpu().numpy(), want, f"{alg} start {rep}")
    del send
    torch.cuda.empty_cache()


@pytest.mark.parametrize("seed", [0, 1])
def test_host_resident_buffers(seed):
    """Send and receive buffers, and the backward's gradients, in pinned host memory: the
    kernels read and write them in place over the host link.  Both forms and the backward
    give the oracle's bytes, graph-captured, eager and batched, also with bulk=2, whose
    bulk-copy forms then stay on the device-resident aggregates (no scatter form on host
    gradients)."""
    p = pt.config5(edge=4, comps=2) if seed == 0 else pt.random_pattern(77, P=24, dtype="f64")
    x = payload(p, 3)
    init = pt.random_bytes(p.recvbuf_bytes, 4)
    want = oracle.standard(p, x, init)
    send = torch.from_numpy(x.view(np.uint8).copy()).pin_memory()
    for alg, form in (("standard", 0), ("locality", 1)):
        for info in ("", "bulk=2", "graph=0"):
            recv = torch.from_numpy(init.copy()).pin_memory()
            ex = gbx.Exchange(p, send, recv, alg, info=info)
            for rep in range(2):
                ex.start()
                ex.wait()
                assert_bytes_equal(recv.numpy(), want, f"{alg} {info} start {rep}")
            recv.copy_(torch.from_numpy(init))
            gbx.startall([ex.request])
            gbx.waitall([ex.request])
            assert_bytes_equal(recv.numpy(), want, f"{alg} {info} batched")
            g = grad_payload(p, 5)
            old = payload(p, 6)
            gr = torch.from_numpy(g.view(np.uint8).copy()).pin_memory()
            for acc in (False, True):
                gs = torch.from_numpy(old.view(np.uint8).copy()).pin_memory()
                b = gbx.backward_init(ex.request, gr, gs, accumulate=acc, info=info)
                b.start()
                b.wait()
                assert not b.info()["copy_forms"] & (1 << 9), "scatter form on host gradients"
                assert_bytes_equal(gs.numpy(), oracle.backward(p, g, old, form=form, accumulate=acc),
                                   f"{alg} {info} backward acc={acc}")


def test_rebind_bulk_form_to_host_is_refused():
    p = pt.random_pattern(3, P=24, elem_size=32, indexed=False, gaps=False, max_count=40)
    x = pt.random_bytes(p.sendbuf_bytes, 3)
    got, ex = forward(p, x, "standard", info="bulk=2")
    assert_bytes_equal(got, oracle.standard(p, x), "device buffers")
    assert ex.info()["copy_forms"] & (1 << 8)
    host = torch.from_numpy(x.copy()).pin_memory()
    with pytest.raises(gbx.GbxError) as e:
        ex.request.bind(host, None)
    assert e.value.code == gbx.ERR_UNSUPPORTED
    ex.start()                      # still bound to its device buffers
    ex.wait()
    assert_bytes_equal(ex.recv.cpu().numpy(), oracle.standard(p, x), "after the refused bind")


def test_pageable_host_buffers_are_refused():
    """Pageable host memory is not addressable by the kernels: init and bind refuse it with
    ERR_ARG before anything runs."""
    import ctypes
    p = pt.config1()
    x = payload(p, 1)
    got, ex = forward(p, x)
    pageable = np.zeros(p.sendbuf_bytes, np.uint8)
    rc = gbx.lib().gbx_request_bind(ex.request.handle, ctypes.c_void_p(pageable.ctypes.data), None)
    assert rc == gbx.ERR_ARG
    ex.start()
    ex.wait()
    assert_bytes_equal(ex.recv.cpu().numpy(), oracle.standard(p, x), "still bound to its device buffers")
    dp = ex.dp
    h = ctypes.c_void_p()
    rc = gbx.lib().gbx_neighbor_alltoallv_init(
        ctypes.c_void_p(pageable.ctypes.data), p.sendbuf_bytes, dp.send_base.data_ptr(), dp.sendcounts.data_ptr(),
        dp.sdispls.data_ptr(), None, None, ex.recv.data_ptr(), p.recvbuf_bytes, dp.recv_base.data_ptr(),
        dp.recvcounts.data_ptr(), dp.rdispls.data_ptr(), None, p.elem_size, gbx.DTYPE_CODES[p.dtype], None, None,
        ex.graph.handle, None, None, ctypes.byref(h))
    assert rc == gbx.ERR_ARG and not h.value


@pytest.mark.parametrize("info", ["", "bulk=2", "flat=0", "graph=0;max_ctas=5"])
def test_guard_bands_untouched(info):
    """Every form writes only inside the buffers bound to it: 4 KB bands of random bytes just
    before and after the receive buffer and the gradient buffer are unchanged after the
    forward and the backward, and the bytes inside match the oracle (receive slots and
    gradient elements no block writes keep their old bytes)."""
    G = 4096
    for p in (pt.config5(edge=4, comps=2), pt.random_pattern(123, P=24, dtype="f64")):
        x = payload(p, 1)
        g = grad_payload(p, 2)
        send = dev_bytes(x)
        for alg, form in (("standard", 0), ("locality", 1)):
            big = torch.from_numpy(pt.random_bytes(p.recvbuf_bytes + 2 * G, 9)).cuda()
            before = big.clone()
            recv = big[G:G + p.recvbuf_bytes]
            ex = gbx.Exchange(p, send, recv, alg, info=info)
            ex.start()
            ex.wait()
            assert torch.equal(big[:G], before[:G]) and torch.equal(big[G + p.recvbuf_bytes:],
                                                                    before[G + p.recvbuf_bytes:]), f"{alg} recv guard"
            assert_bytes_equal(recv.cpu().numpy(), oracle.standard(p, x, before[G:G + p.recvbuf_bytes].cpu().numpy()),
                               f"{alg} {info} forward")
            gbig = torch.from_numpy(pt.random_bytes(p.sendbuf_bytes + 2 * G, 10)).cuda()
            gbefore = gbig.clone()
            gs = gbig[G:G + p.sendbuf_bytes]
            b = gbx.backward_init(ex.request, dev_bytes(g), gs, info=info)
            b.start()
            b.wait()
            assert torch.equal(gbig[:G], gbefore[:G]) and torch.equal(gbig[G + p.sendbuf_bytes:],
                                                                      gbefore[G + p.sendbuf_bytes:]), f"{alg} grad guard"
            old = gbefore[G:G + p.sendbuf_bytes].cpu().numpy()
            assert_bytes_equal(gs.cpu().numpy(), oracle.backward(p, g, old, form=form), f"{alg} {info} backward")
