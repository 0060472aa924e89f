"""GPU: neighbor_alltoall / allgather / allgatherv and the dense alltoallv, each against the
oracle's neighbourhood all-to-all-v run on the equivalent counts and displacements written
out from the MPI definitions on the host."""
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


def _explicit(p, send_counts_of_edge, sdispl_of_edge, recvcount_of_edge, rdispl_of_edge, region_send, region_recv, s):
    """The equivalent neighbourhood all-to-all-v problem (packed regions, byte bases)."""
    q = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.sendcounts = send_counts_of_edge.astype(np.int32)
    q.sdispls = sdispl_of_edge.astype(np.int32)
    q.recvcounts = recvcount_of_edge.astype(np.int32)
    q.rdispls = rdispl_of_edge.astype(np.int32)
    q.elem_size = s
    q.send_base = (np.concatenate([[0], np.cumsum(region_send)[:-1]]) * s).astype(np.int64)
    q.recv_base = (np.concatenate([[0], np.cumsum(region_recv)[:-1]]) * s).astype(np.int64)
    q.sendbuf_bytes = int(np.sum(region_send) * s)
    q.recvbuf_bytes = int(np.sum(region_recv) * s)
    q.send_slot_ptr = q.send_idx = q.recv_slot_ptr = q.global_sidx = q.global_ridx = None
    return q


def _pos_in_list(ptr):
    return np.concatenate([np.arange(ptr[r + 1] - ptr[r]) for r in range(len(ptr) - 1)] + [np.zeros(0, int)]).astype(np.int64)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("kind", ["alltoall", "allgather"])
def test_neighbor_alltoall_and_allgather(seed, kind):
    p = pt.random_pattern(seed)
    s, count = int([1, 8, 24][seed % 3]), 3 + seed
    out_owner = np.repeat(np.arange(p.P), np.diff(p.out_ptr))
    in_owner = np.repeat(np.arange(p.P), np.diff(p.in_ptr))
    deg_out = np.diff(p.out_ptr)
    deg_in = np.diff(p.in_ptr)
    E = len(p.dests)
    jo = _pos_in_list(p.out_ptr)
    ji = _pos_in_list(p.in_ptr)
    cnt = np.full(E, count)
    sd = jo * count if kind == "alltoall" else np.zeros(E, np.int64)
    region_send = deg_out * count if kind == "alltoall" else np.full(p.P, count)
    q = _explicit(p, cnt, sd, np.full(E, count), ji * count, np.maximum(region_send, 1), np.maximum(deg_in * count, 1), s)
    x = pt.random_bytes(q.sendbuf_bytes, seed)
    init = pt.random_bytes(q.recvbuf_bytes, seed + 9)
    want = oracle.standard(q, x, init)
    comm, g = _graph_of(p)
    send = torch.from_numpy(x.copy()).cuda()
    recv = torch.from_numpy(init.copy()).cuda()
    sb = torch.from_numpy(q.send_base).cuda()
    rb = torch.from_numpy(q.recv_base).cuda()
    f = gbx.neighbor_alltoall_init if kind == "alltoall" else gbx.neighbor_allgather_init
    r = f(send, sb, recv, rb, count, g, s)
    r.start()
    r.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, f"{kind} seed {seed}")
    # locality-aware form: values named by their source elements, so an allgather sends each
    # element once per remote node; same bytes, the oracle's statistics
    recv2 = torch.from_numpy(init.copy()).cuda()
    r2 = f(send, sb, recv2, rb, count, g, s, info="algorithm=locality")
    r2.start()
    r2.wait()
    assert_bytes_equal(recv2.cpu().numpy(), want, f"{kind} seed {seed} locality")
    st = oracle.locality_stats(q)
    i = r2.info()
    assert {k: i[k] for k in ("U", "node_pairs", "V_inter", "msgs_step1", "msgs_step3")} == \
        {k: st[k] for k in ("U", "node_pairs", "V_inter", "msgs_step1", "msgs_step3")}
    del out_owner, in_owner


def test_neighbor_allgatherv():
    p = pt.random_pattern(17)
    s = 8
    rng = np.random.default_rng(4)
    rank_count = rng.integers(0, 6, size=p.P)
    E = len(p.dests)
    in_owner = np.repeat(np.arange(p.P), np.diff(p.in_ptr))
    rc = rank_count[p.sources]                       # each in-edge receives its sender's count
    rd = np.zeros(E, np.int64)
    for d in range(p.P):                             # packed in in-list order
        lo, hi = p.in_ptr[d], p.in_ptr[d + 1]
        rd[lo:hi] = np.concatenate([[0], np.cumsum(rc[lo:hi])[:-1]]) if hi > lo else []
    region_recv = np.array([rc[p.in_ptr[d]:p.in_ptr[d + 1]].sum() for d in range(p.P)])
    q = _explicit(p, rank_count[np.repeat(np.arange(p.P), np.diff(p.out_ptr))], np.zeros(E, np.int64), rc, rd,
                  np.maximum(rank_count, 1), np.maximum(region_recv, 1), s)
    x = pt.random_bytes(q.sendbuf_bytes, 2)
    want = oracle.standard(q, x)
    comm, g = _graph_of(p)
    send = torch.from_numpy(x.copy()).cuda()
    recv = torch.zeros(q.recvbuf_bytes, dtype=torch.uint8, device="cuda")
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    r = gbx.neighbor_allgatherv_init(send, torch.from_numpy(q.send_base).cuda(), t32(rank_count), recv,
                                     torch.from_numpy(q.recv_base).cuda(), t32(rc), t32(rd), g, s)
    r.start()
    r.wait()
    assert_bytes_equal(recv.cpu().numpy(), want, "allgatherv")
    # a receive count that differs from the sender's is MPI_ERR_TRUNCATE
    bad = rc.copy()
    if len(bad):
        bad[0] += 1
        with pytest.raises(gbx.GbxError) as e:
            gbx.neighbor_allgatherv_init(send, torch.from_numpy(q.send_base).cuda(), t32(rank_count), recv,
                                         torch.from_numpy(q.recv_base).cuda(), t32(bad), t32(rd), g, s)
        assert e.value.code == gbx.ERR_TRUNCATE
    del in_owner


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
    ptr = (np.arange(P + 1) * P).astype(np.int32)
    ranks = np.tile(np.arange(P), P).astype(np.int32)
    p = pt.Pattern(name="dense", P=P, ppn=ppn, in_ptr=ptr, sources=ranks, out_ptr=ptr, dests=ranks,
                   sendcounts=cnt.reshape(-1).astype(np.int32), sdispls=sd.reshape(-1).astype(np.int32),
                   recvcounts=cnt.T.reshape(-1).astype(np.int32), rdispls=rd.reshape(-1).astype(np.int32),
                   elem_size=s, dtype="f64", send_base=np.zeros(P, np.int64), recv_base=np.zeros(P, np.int64),
                   sendbuf_bytes=0, recvbuf_bytes=0)
    p.send_base = (np.concatenate([[0], np.cumsum(region_send)[:-1]]) * s).astype(np.int64)
    p.recv_base = (np.concatenate([[0], np.cumsum(region_recv)[:-1]]) * s).astype(np.int64)
    p.sendbuf_bytes = int(region_send.sum() * s)
    p.recvbuf_bytes = int(region_recv.sum() * s)
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
