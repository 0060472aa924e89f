"""GPU: neighbor_alltoall / allgather / allgatherv and the dense alltoallv, each against the
oracle's derived collectives (oracle.neighbor_pattern / neighbor_allgatherv / alltoallv_pattern,
whose counts and displacements come from the MPI definitions in oracle.c)."""
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


def _graph_of(p):
    comm = gbx.Comm(p.P, p.ppn)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    return comm, gbx.DistGraph(comm, t(p.in_ptr), t(p.sources), t(p.out_ptr), t(p.dests))


def _problem(p, region_send, region_recv, s):
    """p's graph with packed per-rank regions of the given sizes (in elements) and element
    size s: the argument of the oracle's derived collectives."""
    g = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    g.elem_size = s
    g.dtype = "bytes"
    g.send_base = (np.concatenate([[0], np.cumsum(region_send)[:-1]]) * s).astype(np.int64)
    g.recv_base = (np.concatenate([[0], np.cumsum(region_recv)[:-1]]) * s).astype(np.int64)
    g.sendbuf_bytes = int(np.sum(region_send) * s)
    g.recvbuf_bytes = int(np.sum(region_recv) * s)
    return g


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("kind", ["alltoall", "allgather"])
def test_neighbor_alltoall_and_allgather(seed, kind):
    p = pt.random_pattern(seed)
    s, count = int([1, 8, 24][seed % 3]), 3 + seed
    deg_out = np.diff(p.out_ptr)
    deg_in = np.diff(p.in_ptr)
    region_send = deg_out * count if kind == "alltoall" else np.full(p.P, count)
    g = _problem(p, np.maximum(region_send, 1), np.maximum(deg_in * count, 1), s)
    x = pt.random_bytes(g.sendbuf_bytes, seed)
    init = pt.random_bytes(g.recvbuf_bytes, seed + 9)
    q = oracle.neighbor_pattern(g, kind, count=count)
    want = oracle.standard(q, x, init)
    comm, gr = _graph_of(p)
    send = torch.from_numpy(x.copy()).cuda()
    recv = torch.from_numpy(init.copy()).cuda()
    sb = torch.from_numpy(g.send_base).cuda()
    rb = torch.from_numpy(g.recv_base).cuda()
    f = gbx.neighbor_alltoall_init if kind == "alltoall" else gbx.neighbor_allgather_init
    r = f(send, sb, recv, rb, count, gr, s)
    r.start()
    r.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, f"{kind} seed {seed}")
    # locality-aware form: values named by their source elements, so an allgather sends each
    # element once per remote node; same bytes, the oracle's statistics
    recv2 = torch.from_numpy(init.copy()).cuda()
    r2 = f(send, sb, recv2, rb, count, gr, s, info="algorithm=locality")
    r2.start()
    r2.wait()
    assert_bytes_equal(recv2.cpu().numpy(), want, f"{kind} seed {seed} locality")
    st = oracle.locality_stats(q)
    i = r2.info()
    assert {k: i[k] for k in ("U", "node_pairs", "V_inter", "msgs_step1", "msgs_step3")} == \
        {k: st[k] for k in ("U", "node_pairs", "V_inter", "msgs_step1", "msgs_step3")}


def test_neighbor_allgatherv():
    p = pt.random_pattern(17)
    s = 8
    rng = np.random.default_rng(4)
    rank_count = rng.integers(0, 6, size=p.P)
    E = len(p.dests)
    rc = rank_count[p.sources]                       # each in-edge receives its sender's count
    rd = np.zeros(E, np.int64)
    for d in range(p.P):                             # packed in in-list order
        lo, hi = p.in_ptr[d], p.in_ptr[d + 1]
        rd[lo:hi] = np.concatenate([[0], np.cumsum(rc[lo:hi])[:-1]]) if hi > lo else []
    region_recv = np.array([rc[p.in_ptr[d]:p.in_ptr[d + 1]].sum() for d in range(p.P)])
    g = _problem(p, np.maximum(rank_count, 1), np.maximum(region_recv, 1), s)
    x = pt.random_bytes(g.sendbuf_bytes, 2)
    want = oracle.neighbor_allgatherv(g, rank_count, rc, rd, x)
    comm, gr = _graph_of(p)
    send = torch.from_numpy(x.copy()).cuda()
    recv = torch.zeros(g.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    r = gbx.neighbor_allgatherv_init(send, torch.from_numpy(g.send_base).cuda(), t32(rank_count), recv,
                                     torch.from_numpy(g.recv_base).cuda(), t32(rc), t32(rd), gr, s)
    r.start()
    r.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, "allgatherv")
    # a receive count that differs from the sender's is MPI_ERR_TRUNCATE, as in the oracle
    bad = rc.copy()
    if len(bad):
        bad[0] += 1
        with pytest.raises(oracle.OracleError) as oe:
            oracle.neighbor_allgatherv(g, rank_count, bad, rd, x)
        with pytest.raises(gbx.GbxError) as e:
            gbx.neighbor_allgatherv_init(send, torch.from_numpy(g.send_base).cuda(), t32(rank_count), recv,
                                         torch.from_numpy(g.recv_base).cuda(), t32(bad), t32(rd), gr, s)
        assert e.value.code == oe.value.code == gbx.ERR_TRUNCATE


def test_alltoall_displacement_overflow():
    """Rank 0 lists three out-neighbours; with count = 2^30 its third block would start at
    element 2^31, beyond the int32 displacements: the oracle and the library both refuse the
    call with ERR_UNSUPPORTED (before any buffer is checked, so the buffers are tiny)."""
    P = 4
    p = pt.Pattern(name="wide", P=P, ppn=P, in_ptr=np.array([0, 0, 1, 2, 3], np.int32),
                   sources=np.zeros(3, np.int32), out_ptr=np.array([0, 3, 3, 3, 3], np.int32),
                   dests=np.array([1, 2, 3], np.int32), sendcounts=None, sdispls=None, recvcounts=None,
                   rdispls=None, elem_size=1, dtype="bytes", send_base=np.zeros(P, np.int64),
                   recv_base=np.zeros(P, np.int64), sendbuf_bytes=16, recvbuf_bytes=16)
    with pytest.raises(oracle.OracleError) as oe:
        oracle.neighbor_pattern(p, "alltoall", count=1 << 30)
    comm, gr = _graph_of(p)
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    z = torch.zeros(P, dtype=torch.int64, device="cuda")
    with pytest.raises(gbx.GbxError) as e:
        gbx.neighbor_alltoall_init(buf, z, buf.clone(), z, 1 << 30, gr, 1)
    assert e.value.code == oe.value.code == gbx.ERR_UNSUPPORTED


@pytest.mark.parametrize("P,ppn", [(1, 1), (7, 3), (64, 8)])
def test_dense_alltoallv(P, ppn):
    rng = np.random.default_rng(P)
    s = 8
    cnt = rng.integers(0, 5, size=(P, P))            # cnt[r, d] elements from r to d
    sd = np.zeros((P, P), np.int64)
    rd = np.zeros((P, P), np.int64)
    for r in range(P):
        sd[r] = np.concatenate([[0], np.cumsum(cnt[r])[:-1]])
    for d in range(P):
        rd[d] = np.concatenate([[0], np.cumsum(cnt[:, d])[:-1]])
    region_send = np.maximum(cnt.sum(1), 1)
    region_recv = np.maximum(cnt.sum(0), 1)
    send_base = (np.concatenate([[0], np.cumsum(region_send)[:-1]]) * s).astype(np.int64)
    recv_base = (np.concatenate([[0], np.cumsum(region_recv)[:-1]]) * s).astype(np.int64)
    p = oracle.alltoallv_pattern(P, ppn, cnt, sd, cnt.T, rd, send_base, recv_base, s, int(region_send.sum() * s),
                                 int(region_recv.sum() * s), dtype="f64")
    x = rng.standard_normal(p.sendbuf_bytes // 8)
    want = oracle.standard(p, x)
    comm = gbx.Comm(P, ppn)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    send = torch.from_numpy(x).cuda()
    recv = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    r = gbx.alltoallv_init(comm, send, torch.from_numpy(p.send_base).cuda(), t32(p.sendcounts), t32(p.sdispls),
                           recv, torch.from_numpy(p.recv_base).cuda(), t32(p.recvcounts), t32(p.rdispls), s,
                           gbx.F64)
    for _ in range(2):
        r.start()
        r.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, f"alltoallv P={P}")
    # differentiable too: the backward of the dense exchange equals the oracle's
    g = torch.randn(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    gx = torch.zeros_like(send)
    b = gbx.backward_init(r, g, gx)
    b.start()
    b.wait()
    assert_bytes_equal(gx.cpu().numpy(), oracle.backward(p, g.cpu().numpy(), form=0), f"alltoallv backward P={P}")

    # locality-aware dense traffic: one aggregate per node pair; the reverse follows the
    # three steps (node-blocked order)
    recv2 = torch.zeros_like(recv)
    r2 = gbx.alltoallv_init(comm, send, torch.from_numpy(p.send_base).cuda(), t32(p.sendcounts), t32(p.sdispls),
                            recv2, torch.from_numpy(p.recv_base).cuda(), t32(p.recvcounts), t32(p.rdispls), s,
                            gbx.F64, info="algorithm=locality")
    r2.start()
    r2.wait()
    assert_bytes_equal(recv2.cpu().numpy(), want, f"alltoallv locality P={P}")
    st = oracle.locality_stats(p)
    assert r2.info()["U"] == st["U"] and r2.info()["node_pairs"] == st["node_pairs"]
    gx2 = torch.zeros_like(send)
    b2 = gbx.backward_init(r2, g, gx2)
    b2.start()
    b2.wait()
    assert_bytes_equal(gx2.cpu().numpy(), oracle.backward(p, g.cpu().numpy(), form=1),
                       f"alltoallv locality backward P={P}")


@pytest.mark.parametrize("seed", range(12))
def test_locality_without_global_indices(seed):
    """Index-list exchanges given no global indices: the locality form names values by
    their source elements (repeated elements are aggregated once per node pair)."""
    p = pt.random_pattern(700 + seed, dtype="f64" if seed % 2 else "f32")
    q = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.global_sidx = q.global_ridx = None
    if q.send_idx is None:
        q.send_slot_ptr = None
    rng = np.random.default_rng(seed)
    vt = np.float64 if p.dtype == "f64" else np.float32
    x = rng.standard_normal(p.sendbuf_bytes // np.dtype(vt).itemsize).astype(vt)
    want, st = oracle.locality(q, x)
    dq = gbx.DevicePattern(q)
    send = torch.from_numpy(x).cuda()
    recv = torch.zeros(max(p.recvbuf_bytes, 1) // np.dtype(vt).itemsize, dtype=send.dtype, device="cuda")
    recv = recv[: p.recvbuf_bytes // np.dtype(vt).itemsize]
    ex = gbx.Exchange(q, send, recv, "locality", dp=dq)
    ex.start()
    ex.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, q.name)
    i = ex.info()
    for k in ("U", "node_pairs", "V_direct", "V_inter", "msgs_step1", "msgs_step3"):
        assert i[k] == st[k], (k, i[k], st[k])
    g = rng.standard_normal(len(recv)).astype(vt)
    gx = torch.zeros_like(send)
    b = gbx.backward_init(ex.request, torch.from_numpy(g).cuda(), gx)
    b.start()
    b.wait()
    assert_bytes_equal(gx.cpu().numpy(), oracle.backward(q, g, form=1), q.name + " backward")
