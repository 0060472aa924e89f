"""GPU: the differentiable halo exchange (torch.autograd.Function over the library's
forward and reverse exchanges), checked by gradcheck, the dense transpose, finite
differences and the oracle, alone and inside a distributed SpMV y = A x (config 4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2309_07337_gb300 import patterns as pt  # noqa: E402
from paper_2309_07337_gb300.autograd import DistributedHalo  # noqa: E402
from gpu_util import assert_bytes_equal  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _dense_exchange(p):
    """0/1 matrix of the exchange [receive element, send element] from the oracle's
    forward on element ids (pinned separately against brute force)."""
    vt = np.float64 if p.dtype == "f64" else np.float32
    n_send = p.sendbuf_bytes // np.dtype(vt).itemsize
    n_recv = p.recvbuf_bytes // np.dtype(vt).itemsize
    ids = np.arange(n_send, dtype=np.float64)
    q = pt.Pattern(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    scale = 8 // np.dtype(vt).itemsize
    q.elem_size = p.elem_size * scale
    q.send_base = p.send_base * scale
    q.recv_base = p.recv_base * scale
    q.sendbuf_bytes = p.sendbuf_bytes * scale
    q.recvbuf_bytes = p.recvbuf_bytes * scale
    r = np.frombuffer(oracle.standard(q, ids, np.full(n_recv, -1.0)).tobytes(), np.float64).astype(np.int64)
    E = np.zeros((n_recv, n_send))
    ok = r >= 0
    E[np.nonzero(ok)[0], r[ok]] = 1.0
    return E


@pytest.mark.parametrize("alg", ["standard", "locality"])
def test_gradcheck_fp64_tiny(alg):
    p = pt.stencil((8, 8), (2, 2), ppn=2, comps=1, dtype="f64", neighbors="all")
    halo = DistributedHalo(p, algorithm=alg)
    x = torch.randn(halo.n_send, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(halo, (x,), eps=1e-6, atol=1e-9, rtol=1e-7)


def assert_near_transpose(got, ref, mag, tol, what):
    """Element by element against the dense transpose: |got_i - ref_i| <= tol * mag_i, where
    ref_i is the exact sum of the terms feeding element i and mag_i the sum of their
    magnitudes; exactly 0 where no term feeds it.  Without cancellation (all terms of one
    sign) mag_i = |ref_i|, so this is the relative bound tol * |ref_i|.  With cancellation a
    bound relative to |ref_i| holds for no floating-point summation order; the rounding error
    of any order of k terms is at most (k-1) u mag_i (u = 2^-24 in fp32, 2^-53 in fp64)."""
    got = np.asarray(got, dtype=np.float64)
    none = mag == 0
    assert np.all(got[none] == 0), f"{what}: elements fed by no term are not zero"
    err = np.abs(got - ref)
    bad = np.flatnonzero(~none & (err > tol * mag))
    assert len(bad) == 0, f"{what}: {len(bad)} elements off, first {bad[:5]}, rel {(err / np.maximum(mag, 1e-300))[bad[:5]]}"


def _small_spmv(dtype):
    """The 4096-row copy of the config-4 matrix (64 ranks, 32 per node) in fp32 or fp64."""
    if dtype == "f32":
        return pt.config4(n=4096, P=64, ppn=32)
    return pt.spmv_halo(4096, 64, 32, 20, pt.SEED + 2, "f64", name="cfg4_spmv_n4096_P64_f64", keep_matrix=True)


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-12)])
@pytest.mark.parametrize("alg,form", [("standard", 0), ("locality", 1)])
def test_exchange_backward_equals_oracle_and_dense_transpose(alg, form, dtype, tol):
    p = _small_spmv(dtype)
    vt = np.float32 if dtype == "f32" else np.float64
    halo = DistributedHalo(p, algorithm=alg)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(pt.spmv_x(p, 1)).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(halo.n_recv).astype(vt)).cuda()
    h = halo(x)
    assert_bytes_equal(h.detach().cpu().numpy(), oracle.standard(p, x.detach().cpu().numpy()), "forward")
    (h * w).sum().backward()
    g = x.grad.cpu().numpy()
    assert_bytes_equal(g, oracle.backward(p, w.cpu().numpy(), form=form), "backward vs oracle")
    E = _dense_exchange(p)
    wn = w.cpu().numpy().astype(np.float64)
    assert_near_transpose(g, E.T @ wn, E.T @ np.abs(wn), tol, f"{alg} {dtype} backward vs dense transpose")


def test_fresh_outputs_zero_only_unwritten_entries():
    """Receive slots no block covers and source elements no slot reads come back as zeros
    even when the caching allocator hands back memory full of NaNs; the rest is the
    oracle's, bit for bit."""
    for seed in (5, 21, 40):
        p = pt.random_pattern(seed, dtype="f64")
        halo = DistributedHalo(p, algorithm="standard")
        rng = np.random.default_rng(seed)
        x = torch.from_numpy(rng.standard_normal(halo.n_send)).cuda().requires_grad_(True)
        w = torch.from_numpy(rng.standard_normal(halo.n_recv)).cuda()
        for _ in range(2):
            junk = torch.full((max(halo.n_send, halo.n_recv) * 2,), float("nan"), dtype=torch.float64, device="cuda")
            del junk
            x.grad = None
            h = halo(x)
            (h * w).sum().backward()
            assert_bytes_equal(h.detach().cpu().numpy(), oracle.standard(p, x.detach().cpu().numpy()), p.name)
            assert_bytes_equal(x.grad.cpu().numpy(), oracle.backward(p, w.cpu().numpy(), form=0), p.name + " grad")


def _spmv_operators(p, seed):
    """Sparse operators of the distributed y = A x: on-rank columns read x, off-rank
    columns read the receiving rank's halo slot of that column."""
    n, rs, cols = p.meta["n"], p.meta["row_starts"], p.meta["cols"]
    nnz = cols.shape[1]
    vals = np.random.default_rng(seed).standard_normal(cols.shape).astype(np.float32)
    rows = np.repeat(np.arange(n), nnz)
    c = cols.reshape(-1)
    v = vals.reshape(-1)
    ro = np.searchsorted(rs, rows, side="right") - 1
    co = np.searchsorted(rs, c, side="right") - 1
    on = ro == co
    slot = np.zeros(len(c), dtype=np.int64)
    for d in np.unique(ro[~on]):
        sel = (~on) & (ro == d)
        hc = p.global_ridx[p.recv_slot_ptr[d]:p.recv_slot_ptr[d + 1]]
        slot[sel] = p.recv_slot_ptr[d] + np.searchsorted(hc, c[sel])
        assert np.array_equal(hc[slot[sel] - p.recv_slot_ptr[d]], c[sel])
    n_recv = int(p.recv_slot_ptr[-1])
    A_loc = torch.sparse_coo_tensor(torch.from_numpy(np.stack([rows[on], c[on]])), torch.from_numpy(v[on]),
                                    (n, n)).coalesce().cuda()
    A_halo = torch.sparse_coo_tensor(torch.from_numpy(np.stack([rows[~on], slot[~on]])), torch.from_numpy(v[~on]),
                                     (n, n_recv)).coalesce().cuda()
    dense = np.zeros((n, n))
    np.add.at(dense, (rows, c), v.astype(np.float64))
    return A_loc, A_halo, dense


@pytest.mark.parametrize("alg", ["standard", "locality"])
def test_distributed_spmv_dense_transpose_and_finite_differences(alg):
    """The 4096-row copy of config 4: y = A_loc x + A_halo halo(x) against the dense A,
    dL/dx against A^T w, and central differences along random directions (fp32)."""
    p = pt.config4(n=4096, P=64, ppn=32)
    halo = DistributedHalo(p, algorithm=alg)
    A_loc, A_halo, dense = _spmv_operators(p, 7)
    x0 = torch.from_numpy(pt.spmv_x(p, 2)).cuda()
    w = torch.from_numpy(np.random.default_rng(5).standard_normal(p.meta["n"]).astype(np.float32)).cuda()

    def y_of(x):
        return (torch.sparse.mm(A_loc, x[:, None]) + torch.sparse.mm(A_halo, halo(x)[:, None]))[:, 0]

    x = x0.clone().requires_grad_(True)
    y = y_of(x)
    xn = x0.cpu().numpy().astype(np.float64)
    assert_near_transpose(y.detach().cpu().numpy(), dense @ xn, np.abs(dense) @ np.abs(xn), 1e-5, "y = A x")
    (y * w).sum().backward()
    wn = w.cpu().numpy().astype(np.float64)
    g = x.grad.cpu().numpy().astype(np.float64)
    assert_near_transpose(g, dense.T @ wn, np.abs(dense).T @ np.abs(wn), 1e-5, "dL/dx = A^T w")
    rng = np.random.default_rng(11)
    with torch.no_grad():
        for _ in range(3):
            v = torch.from_numpy(rng.standard_normal(len(x0)).astype(np.float32)).cuda()
            h = 1e-2 * float(x0.abs().max())
            fp = float((y_of(x0 + h * v).double() * w.double()).sum())
            fm = float((y_of(x0 - h * v).double() * w.double()).sum())
            fd = (fp - fm) / (2 * h)
            an = float(np.dot(g, v.cpu().numpy().astype(np.float64)))
            assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-6), (fd, an)


def test_config4_full_size_forward_backward():
    """2^20 rows over 1024 ranks, fp32: the autograd path equals the oracle bit for bit."""
    p = pt.config4()
    halo = DistributedHalo(p, algorithm="standard")
    x = torch.from_numpy(pt.spmv_x(p, 4)).cuda().requires_grad_(True)
    w = torch.randn(halo.n_recv, dtype=torch.float32, device="cuda")
    h = halo(x)
    assert_bytes_equal(h.detach().cpu().numpy(), oracle.standard(p, x.detach().cpu().numpy()), "forward")
    (h * w).sum().backward()
    assert_bytes_equal(x.grad.cpu().numpy(), oracle.backward(p, w.cpu().numpy(), form=0), "backward")


def test_backward_is_deterministic():
    p = pt.config4(n=1 << 16, P=128, ppn=32)
    halo = DistributedHalo(p, algorithm="locality")
    w = torch.randn(halo.n_recv, dtype=torch.float32, device="cuda")
    first = halo.run_backward(w)
    for _ in range(20):
        assert torch.equal(halo.run_backward(w), first)
