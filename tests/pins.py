"""Checks that pin the CPU oracle to facts outside itself.

Each check takes an oracle library handle (the real one, or a build with a planted
mistake in the mutation test) and raises AssertionError when the oracle disagrees with:
  * hand-worked golden cases (tests/golden/*.json, each with its citation);
  * brute force: a stencil halo equals the global grid read at the ghost coordinates,
    an SpMV halo equals x[off-rank columns of the rank's rows];
  * invariants: list-order permutation, locality form == standard form, idempotence;
  * closed-form counts from the stencil geometry;
  * the adjoint: backward == dense transpose of the forward's 0/1 map, exactly for
    integer data, and finite differences.
"""
from __future__ import annotations

import itertools
import json
import os
import types

import numpy as np

import oracle
from paper_2309_07337_gb300 import patterns as pt

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_ARR = {"in_ptr": np.int32, "sources": np.int32, "out_ptr": np.int32, "dests": np.int32,
        "sendcounts": np.int32, "sdispls": np.int32, "recvcounts": np.int32,
        "rdispls": np.int32, "send_base": np.int64, "recv_base": np.int64,
        "send_slot_ptr": np.int64, "send_idx": np.int32, "recv_slot_ptr": np.int64,
        "global_sidx": np.int64, "global_ridx": np.int64}


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    ns = types.SimpleNamespace()
    for k, v in g.items():
        setattr(ns, k, np.array(v, dtype=_ARR[k]) if k in _ARR else v)
    for k in _ARR:
        if not hasattr(ns, k):
            setattr(ns, k, None)
    vt = np.int32 if g["values"] == "i4" else np.float64
    ns.vt = vt
    ns.sendbuf = np.array(g["send_values"], dtype=vt)
    ns.recv_init = np.array(g["recv_init"], dtype=vt)
    ns.dtype = "f64" if vt == np.float64 else "bytes"
    return ns


def as_values(b, vt):
    return np.frombuffer(np.ascontiguousarray(b).tobytes(), dtype=vt)


# ------------------------------------------------------------------ golden ----

def check_golden_forward(lib):
    for name in ("ring3.json", "multigraph.json", "locality_dedup.json", "backward_order.json"):
        g = load_golden(name)
        got = as_values(oracle.standard(g, g.sendbuf, g.recv_init, lib=lib), g.vt)
        assert np.array_equal(got, np.array(g.expected_recv, dtype=g.vt)), name
        if g.global_sidx is not None:
            got2, _ = oracle.locality(g, g.sendbuf, g.recv_init, lib=lib)
            assert np.array_equal(as_values(got2, g.vt), np.array(g.expected_recv, dtype=g.vt)), name


def check_golden_multigraph_truncate(lib):
    g = load_golden("multigraph.json")
    g.recvcounts = g.recvcounts[::-1].copy()   # first listing now expects 2 elements
    assert oracle.validate(g, lib=lib) == g.swapped_recvcounts_error


def check_golden_locality(lib):
    g = load_golden("locality_dedup.json")
    st = oracle.locality_stats(g, lib=lib)
    assert st == g.expected_stats, st
    a, b, gi, rep = oracle.locality_layout(g, lib=lib)
    lay = g.expected_layout
    assert a.tolist() == lay["a"] and b.tolist() == lay["b"]
    assert gi.tolist() == lay["gidx"] and rep.tolist() == lay["rep"]
    gr = np.array(g.grad_recv, dtype=np.float64)
    for form in (0, 1):
        got = as_values(oracle.backward(g, gr, form=form, lib=lib), np.float64)
        assert np.array_equal(got, np.array(g.expected_grad_send)), (form, got)


def check_golden_backward_order(lib):
    for name in ("backward_order.json", "backward_order2.json"):
        g = load_golden(name)
        got = as_values(oracle.standard(g, g.sendbuf, g.recv_init, lib=lib), np.float64)
        assert got.tolist() == g.expected_recv, name
        gr = np.array(g.grad_recv, dtype=np.float64)
        old = np.array(g.grad_send_init, dtype=np.float64)
        for form, key in ((0, "standard"), (1, "node_blocked")):
            got = as_values(oracle.backward(g, gr, form=form, lib=lib), np.float64)
            assert got.tolist() == g.__dict__[f"expected_grad_{key}"], (name, key, got)
            got = as_values(oracle.backward(g, gr, old, form=form, accumulate=True, lib=lib),
                            np.float64)
            assert got.tolist() == g.__dict__[f"expected_grad_{key}_accumulate"], (name, key, got)


# ------------------------------------------------------------- brute force ----

def ghost_expected(p, field):
    """Receive region of every rank, read straight from the assembled global grid at
    the ghost-layer coordinates (neighbour directions in ascending rank order)."""
    grid, ranks, blk, comps = p.meta["grid"], p.meta["ranks"], p.meta["blk"], p.meta["comps"]
    D = len(grid)
    npts = int(np.prod(blk))
    f = field.reshape(p.P, npts, comps)
    G = np.zeros(tuple(reversed(grid)) + (comps,), dtype=field.dtype)
    rc_all = []
    for r in range(p.P):
        rc = []
        q = r
        for ax in range(D):
            rc.append(q % ranks[ax])
            q //= ranks[ax]
        rc_all.append(rc)
        sl = tuple(slice(rc[ax] * blk[ax], (rc[ax] + 1) * blk[ax]) for ax in reversed(range(D)))
        G[sl] = f[r].reshape(tuple(reversed(blk)) + (comps,))
    out = []
    for r in range(p.P):
        rc = rc_all[r]
        parts = []
        for dd in itertools.product((-1, 0, 1), repeat=D):
            dd = tuple(reversed(dd))
            if not any(dd):
                continue
            if p.meta["neighbors"] == "faces" and sum(map(abs, dd)) != 1:
                continue
            if any(not (0 <= rc[ax] + dd[ax] < ranks[ax]) for ax in range(D)):
                continue
            rngs = []
            for ax in range(D):
                o = rc[ax] * blk[ax]
                if dd[ax] == -1:
                    rngs.append(np.array([o - 1]))
                elif dd[ax] == 1:
                    rngs.append(np.array([o + blk[ax]]))
                else:
                    rngs.append(np.arange(o, o + blk[ax]))
            idx = np.meshgrid(*[rngs[ax] for ax in reversed(range(D))], indexing="ij")
            parts.append(G[tuple(i.reshape(-1) for i in idx)])
        out.append(np.concatenate(parts) if parts else np.zeros((0, comps), field.dtype))
    return out


def check_bruteforce_stencil(lib):
    for grid, ranks, ppn, comps, nb in (((24, 16), (3, 2), 4, 1, "all"),
                                        ((16, 16), (4, 4), 4, 1, "faces"),
                                        ((12, 8, 8), (3, 2, 2), 5, 2, "all")):
        p = pt.stencil(grid, ranks, ppn=ppn, comps=comps, dtype="f64", neighbors=nb)
        x = pt.stencil_field(p, 11)
        exp = ghost_expected(p, x)
        for fn in (oracle.standard, lambda *a, **k: oracle.locality(*a, **k)[0]):
            got = as_values(fn(p, x, lib=lib), np.float64).reshape(-1, comps)
            for r in range(p.P):
                lo = p.recv_base[r] // p.elem_size
                assert np.array_equal(got[lo: lo + len(exp[r])], exp[r]), (grid, r)


def check_bruteforce_spmv(lib):
    for n, P, ppn, nnz, band, dt in ((4096, 16, 4, 12, 300, "f64"), (3000, 7, 3, 9, 200, "f32")):
        p = pt.spmv_halo(n, P, ppn, nnz, seed=5, dtype=dt, band=band, keep_matrix=True)
        x = pt.spmv_x(p, 6)
        rs = pt.row_starts(n, P)
        cols = p.meta["cols"]
        for fn in (oracle.standard, lambda *a, **k: oracle.locality(*a, **k)[0]):
            got = as_values(fn(p, x, lib=lib), x.dtype)
            for r in range(P):
                c = np.unique(cols[rs[r]:rs[r + 1]])
                off = c[(c < rs[r]) | (c >= rs[r + 1])]
                lo = p.recv_base[r] // p.elem_size
                assert np.array_equal(got[lo: lo + len(off)], x[off]), (n, r)


def check_permutation_invariance(lib):
    p = pt.spmv_halo(2048, 9, 4, 10, seed=8, dtype="f64", band=200)
    x = pt.spmv_x(p, 9)
    ref = oracle.standard(p, x, lib=lib)
    rng = np.random.default_rng(3)
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    for side, ptr, cols in (("out", "out_ptr", ("dests", "sendcounts", "sdispls")),
                            ("in", "in_ptr", ("sources", "recvcounts", "rdispls"))):
        perm = np.concatenate([lo + rng.permutation(hi - lo) for lo, hi in
                               zip(getattr(p, ptr)[:-1], getattr(p, ptr)[1:])])
        for c in cols:
            setattr(q, c, getattr(p, c)[perm])
    got = oracle.standard(q, x, lib=lib)
    assert np.array_equal(got, ref)
    got2, st2 = oracle.locality(q, x, lib=lib)
    assert np.array_equal(got2, ref)
    # list order is not part of the problem: every count is invariant too
    assert st2 == oracle.locality_stats(p, lib=lib)


def check_idempotent_and_untouched(lib):
    p = pt.spmv_halo(1024, 5, 2, 8, seed=4, dtype="f64", band=150)
    x = pt.spmv_x(p, 2)
    # widen the receive buffer with a sentinel tail no block covers
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.recvbuf_bytes = p.recvbuf_bytes + 64
    init = np.full(q.recvbuf_bytes, 0xAB, dtype=np.uint8)
    a = oracle.standard(q, x, init, lib=lib)
    b = oracle.standard(q, x, a, lib=lib)
    assert np.array_equal(a, b)
    assert (a[p.recvbuf_bytes:] == 0xAB).all()
    assert int(np.sum(p.sendcounts)) == int(np.sum(p.recvcounts))


# ------------------------------------------------------------ closed forms ----

def stencil_counts(ranks, blk, ppn, neighbors="all"):
    """Edge and element counts of a box-stencil halo from its geometry alone."""
    D = len(ranks)
    P = int(np.prod(ranks))
    rc = np.indices(tuple(reversed(ranks))).reshape(D, -1)[::-1]
    node = np.arange(P) // ppn
    stride = np.array([1, ranks[0], ranks[0] * (ranks[1] if D > 1 else 1)][:D])
    E = V = Vx = Mx = 0
    pairs = set()
    per_rb = {}
    dirs = [tuple(reversed(d)) for d in itertools.product((-1, 0, 1), repeat=D)
            if any(d) and (neighbors == "all" or sum(map(abs, d)) == 1)]
    for dd in dirs:
        ok = np.ones(P, dtype=bool)
        for ax in range(D):
            ok &= (rc[ax] + dd[ax] >= 0) & (rc[ax] + dd[ax] < ranks[ax])
        src = np.nonzero(ok)[0]
        dst = src + int((np.array(dd) * stride).sum())
        tsz = int(np.prod([blk[ax] if dd[ax] == 0 else 1 for ax in range(D)]))
        inter = node[src] != node[dst]
        E += len(src)
        V += len(src) * tsz
        Vx += int(inter.sum()) * tsz
        Mx += int(inter.sum())
        for a, b in set(zip(node[src[inter]].tolist(), node[dst[inter]].tolist())):
            pairs.add((a, b))
        for r, b in zip(src[inter].tolist(), node[dst[inter]].tolist()):
            per_rb.setdefault((r, b), []).append(dd)
    # distinct points per (source rank, destination node): a point of boundary type t
    # (per axis -1 at 0, +1 at n-1, 0 inside) lies in the send list of delta iff every
    # axis has delta = 0 or delta = t.
    types_ = list(itertools.product((-1, 0, 1), repeat=D))
    tcount = {t: int(np.prod([1 if t[ax] else blk[ax] - 2 for ax in range(D)])) for t in types_}
    U = 0
    for dl in per_rb.values():
        for t in types_:
            if any(all(d[ax] == 0 or d[ax] == t[ax] for ax in range(D)) for d in dl):
                U += tcount[t]
    # leaders (the reading adopted for the aggregation): node pair (a, b) gathers at rank
    # a*ppn + (b mod size(a)) and scatters from rank b*ppn + (a mod size(b)); every
    # stencil point has one owner, so the representative of a value is its sender.
    def size(a):
        return min(ppn, P - a * ppn)
    m1 = sum(1 for (r, b) in per_rb if r != (r // ppn) * ppn + b % size(r // ppn))
    seen3 = set()
    for (r, b), dl in per_rb.items():
        for dd in dl:
            d = r + int((np.array(dd) * stride).sum())
            seen3.add((r // ppn, d))
    m3 = sum(1 for (a, d) in seen3 if d != (d // ppn) * ppn + a % size(d // ppn))
    return dict(E=E, V=V, V_inter=Vx, V_direct=V - Vx, msgs_inter=Mx, msgs_intra=E - Mx,
                node_pairs=len(pairs), U=U, msgs_step1=m1, msgs_step3=m3)


def check_closed_forms_small(lib):
    for grid, ranks, ppn, nb in (((256, 256), (4, 4), 4, "faces"),
                                 ((40, 24, 16), (5, 3, 2), 6, "all"),
                                 ((32, 32, 32), (4, 4, 4), 8, "all")):
        p = pt.stencil(grid, ranks, ppn=ppn, comps=1, dtype="f64", neighbors=nb)
        blk = tuple(g // r for g, r in zip(grid, ranks))
        want = stencil_counts(ranks, blk, ppn, nb)
        got = oracle.locality_stats(p, lib=lib)
        for k, v in want.items():
            assert got[k] == v, (grid, k, got[k], v)


def bytes1(p):
    """The same pattern with one-byte elements (counts are independent of the size)."""
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    s = p.elem_size
    q.elem_size = 1
    q.send_base = p.send_base // s
    q.recv_base = p.recv_base // s
    q.sendbuf_bytes = p.sendbuf_bytes // s
    q.recvbuf_bytes = p.recvbuf_bytes // s
    return q


# ------------------------------------------------------------------ adjoint ----

def forward_map(p, lib, form=0):
    """Source element read by each receive element (-1 where no block writes):
    the forward run on element ids, which fp64 carries exactly."""
    comps = p.elem_size // (8 if p.dtype == "f64" else 4)
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.elem_size = comps * 8
    q.send_base = p.send_base // p.elem_size * q.elem_size
    q.recv_base = p.recv_base // p.elem_size * q.elem_size
    q.sendbuf_bytes = p.sendbuf_bytes // p.elem_size * q.elem_size
    q.recvbuf_bytes = p.recvbuf_bytes // p.elem_size * q.elem_size
    ids = np.arange(q.sendbuf_bytes // 8, dtype=np.float64)
    init = np.full(q.recvbuf_bytes // 8, -1.0)
    if form == 0:
        r = oracle.standard(q, ids, init, lib=lib)
    else:
        r, _ = oracle.locality(q, ids, init, lib=lib)
    return as_values(r, np.float64).astype(np.int64)


def dense_transpose(p, src_of, g):
    """E^T g with E the 0/1 matrix [receive component, send component]."""
    n_send = p.sendbuf_bytes // (8 if p.dtype == "f64" else 4)
    E = np.zeros((len(src_of), n_send))
    cov = src_of >= 0
    E[np.nonzero(cov)[0], src_of[cov]] = 1.0
    return E.T @ g.astype(np.float64), cov


def adjoint_cases():
    yield pt.stencil((12, 8), (3, 2), ppn=4, comps=2, dtype="f64", neighbors="all")
    yield pt.stencil((8, 8, 4), (2, 2, 2), ppn=3, comps=1, dtype="f32", neighbors="all")
    yield pt.spmv_halo(1500, 6, 4, 9, seed=21, dtype="f32", band=120)
    yield pt.spmv_halo(1200, 5, 2, 7, seed=22, dtype="f64", band=100)


def check_adjoint_dense(lib):
    rng = np.random.default_rng(17)
    for p in adjoint_cases():
        vt = np.float64 if p.dtype == "f64" else np.float32
        src_of = forward_map(p, lib)
        assert np.array_equal(src_of, forward_map(p, lib, form=1))
        # integer-valued gradients: every order sums exactly
        gi = rng.integers(-8, 9, size=len(src_of)).astype(vt)
        want, cov = dense_transpose(p, src_of, np.where(src_of >= 0, gi, 0))
        touched = np.zeros(len(want), dtype=bool)
        touched[src_of[cov]] = True
        for form in (0, 1):
            got = as_values(oracle.backward(p, gi, form=form, lib=lib), vt)
            assert np.array_equal(got[touched], want[touched].astype(vt)), (p.name, form)
            assert (got[~touched] == 0).all()
        # random positive data: within the rounding of a short sum
        gr = rng.uniform(0.5, 1.5, size=len(src_of)).astype(vt)
        want, _ = dense_transpose(p, src_of, np.where(src_of >= 0, gr, 0))
        tol = 1e-12 if vt == np.float64 else 1e-5
        for form in (0, 1):
            got = as_values(oracle.backward(p, gr, form=form, lib=lib), vt).astype(np.float64)
            assert np.allclose(got[touched], want[touched], rtol=tol, atol=0), (p.name, form)


def check_accumulate_and_untouched(lib):
    rng = np.random.default_rng(5)
    for p in adjoint_cases():
        vt = np.float64 if p.dtype == "f64" else np.float32
        n_recv = p.recvbuf_bytes // np.dtype(vt).itemsize
        n_send = p.sendbuf_bytes // np.dtype(vt).itemsize
        g = rng.standard_normal(n_recv).astype(vt)
        old = rng.standard_normal(n_send).astype(vt)
        src_of = forward_map(p, lib)
        touched = np.zeros(n_send, dtype=bool)
        touched[src_of[src_of >= 0]] = True
        for form in (0, 1):
            plain = as_values(oracle.backward(p, g, old, form=form, lib=lib), vt)
            acc = as_values(oracle.backward(p, g, old, form=form, accumulate=True, lib=lib), vt)
            assert np.array_equal(plain[~touched], old[~touched])
            assert np.array_equal(acc[~touched], old[~touched])
            assert np.array_equal(acc[touched], (old[touched] + plain[touched]).astype(vt))


def check_finite_difference(lib):
    """Linear map: the central difference of L(x) = <w, forward(x)> along v equals
    <backward(w), v>; checked in fp32 within 1e-3 relative."""
    rng = np.random.default_rng(9)
    p = pt.spmv_halo(2000, 8, 4, 10, seed=31, dtype="f32", band=150)
    x = pt.spmv_x(p, 3)
    nrecv = p.recvbuf_bytes // 4
    w = rng.standard_normal(nrecv).astype(np.float32)
    cov = forward_map(p, lib) >= 0
    w[~cov] = 0
    for form in (0, 1):
        g = as_values(oracle.backward(p, w, form=form, lib=lib), np.float32).astype(np.float64)
        for _ in range(3):
            v = rng.standard_normal(len(x)).astype(np.float32)
            h = np.float32(1e-2 * np.abs(x).max())

            def L(z):
                return float(np.dot(w.astype(np.float64),
                                    as_values(oracle.standard(p, z, lib=lib), np.float32)))
            fd = (L((x + h * v).astype(np.float32)) - L((x - h * v).astype(np.float32))) / (2 * h)
            an = float(np.dot(g, v.astype(np.float64)))
            assert abs(fd - an) <= 1e-3 * max(abs(an), 1e-6), (form, fd, an)


# ------------------------------------------------------------------ errors ----

def check_error_codes(lib):
    def ring():
        return load_golden("ring3.json")

    g = ring()
    assert oracle.validate(g, lib=lib) == 0
    g = ring(); g.dests = g.dests.copy(); g.dests[0] = 5
    assert oracle.validate(g, lib=lib) == oracle.ERR_RANK
    g = ring(); g.dests = g.dests.copy(); g.dests[0] = 2          # r0 lists 2 twice
    assert oracle.validate(g, lib=lib) == oracle.ERR_TRUNCATE
    g = ring(); g.recvcounts = g.recvcounts.copy(); g.recvcounts[0] = 3
    assert oracle.validate(g, lib=lib) == oracle.ERR_TRUNCATE
    g = ring(); g.rdispls = g.rdispls.copy(); g.rdispls[3] = 9     # rank 2 block past the end
    assert oracle.validate(g, lib=lib) == oracle.ERR_INDEX
    g = ring(); g.sdispls = g.sdispls.copy(); g.sdispls[1] = -1
    assert oracle.validate(g, lib=lib) == oracle.ERR_INDEX
    g = ring(); g.rdispls = g.rdispls.copy(); g.rdispls[1] = 1     # rank 0 blocks overlap
    assert oracle.validate(g, lib=lib) == oracle.ERR_OVERLAP
    g = ring(); g.in_ptr = g.in_ptr.copy(); g.in_ptr[1] = 4        # not a CSR
    assert oracle.validate(g, lib=lib) == oracle.ERR_ARG
    # send index lists: out-of-range element
    p = pt.spmv_halo(600, 4, 2, 6, seed=1, dtype="f64", band=80)
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.send_idx = p.send_idx.copy()
    q.send_idx[3] = 10 ** 6
    assert oracle.validate(q, lib=lib) == oracle.ERR_INDEX
    # receive global index that disagrees with the matched send index
    q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    q.global_ridx = p.global_ridx.copy()
    q.global_ridx[5] += 1
    assert oracle.validate(q, lib=lib) == oracle.ERR_GIDX
    # one global index carried by different bytes from two ranks of one node
    g = load_golden("locality_dedup.json")
    g.global_sidx = g.global_sidx.copy()
    g.global_sidx[2] = 100        # rank 1's value now claims index 100, with other bytes
    g.global_ridx = g.global_ridx.copy()
    g.global_ridx[g.global_ridx == 102] = 100
    assert oracle.validate(g, lib=lib) == 0
    try:
        oracle.locality(g, g.sendbuf, lib=lib)
        raise AssertionError("duplicate index with different bytes accepted")
    except oracle.OracleError as e:
        assert e.code == oracle.ERR_DUP
    sb = g.sendbuf.copy()
    sb[2] = sb[0]                  # same bytes: legal, sent once
    r, st = oracle.locality(g, sb, lib=lib)
    assert st["U"] == 4


# ------------------------------------------- locality without global indices ----

def check_locality_names_values_by_source_element(lib):
    """Without global indices a value is its source element: for generator patterns whose
    indices name source elements, dropping them changes no byte, no statistic and no
    aggregate layout; an element sent to every rank of a node crosses the node pair once."""
    for seed in (2, 5, 7, 12, 19, 33):
        p = pt.random_pattern(seed, indexed=bool(seed % 2))
        if p.global_sidx is None:
            continue
        q = types.SimpleNamespace(**{k: getattr(p, k) for k in p.__dataclass_fields__})
        q.global_sidx = q.global_ridx = None
        if p.send_idx is None:
            q.send_slot_ptr = None
        x = pt.random_bytes(p.sendbuf_bytes, seed)
        a, sa = oracle.locality(p, x, lib=lib)
        b, sb = oracle.locality(q, x, lib=lib)
        assert np.array_equal(a, b) and sa == sb, (seed, sa, sb)
        la, lb = oracle.locality_layout(p, lib=lib), oracle.locality_layout(q, lib=lib)
        assert all(np.array_equal(la[j], lb[j]) for j in (0, 1, 3)), seed
    # rank 0 sends its elements 0..2 to every rank of node 1 (ranks 4..7), ppn 4
    star = types.SimpleNamespace(
        P=8, ppn=4, in_ptr=np.array([0, 0, 0, 0, 0, 1, 2, 3, 4], np.int32), sources=np.zeros(4, np.int32),
        out_ptr=np.array([0, 4, 4, 4, 4, 4, 4, 4, 4], np.int32), dests=np.array([4, 5, 6, 7], np.int32),
        sendcounts=np.full(4, 3, np.int32), sdispls=np.zeros(4, np.int32), recvcounts=np.full(4, 3, np.int32),
        rdispls=np.zeros(4, np.int32), send_base=np.zeros(8, np.int64), recv_base=np.arange(8, dtype=np.int64) * 24,
        send_slot_ptr=None, send_idx=None, recv_slot_ptr=None, global_sidx=None, global_ridx=None,
        elem_size=8, sendbuf_bytes=24, recvbuf_bytes=192)
    x = np.array([1.5, -2.0, 4.25])
    got, st = oracle.locality(star, x, lib=lib)
    assert st["V"] == 12 and st["V_inter"] == 12 and st["U"] == 3 and st["node_pairs"] == 1, st
    assert np.array_equal(as_values(got, np.float64)[12:], np.tile(x, 4))


# ---------------------------------------------------- partitioned exchange ----

def ghost_sources(p):
    """Byte offset of the source point of every receive element of a stencil pattern, per
    rank, read from the global grid assembled from each point's own offset."""
    npts = int(np.prod(p.meta["blk"]))
    comps = p.meta["comps"]
    offs = p.send_base[:, None] + np.arange(npts)[None, :] * p.elem_size
    ids = np.repeat(offs.reshape(-1, 1), comps, axis=1).astype(np.float64).reshape(-1)
    return [g[:, 0].astype(np.int64) for g in ghost_expected(p, ids)]


def _cuts(rng, n_elems, s, n):
    """n partitions of a buffer of n_elems elements of s bytes, cut at element boundaries
    (some possibly empty)."""
    c = np.sort(rng.integers(0, n_elems + 1, size=n - 1)) * s
    return np.concatenate([[0], c, [n_elems * s]]).astype(np.int64)


def check_partitioned_bruteforce(lib):
    """Only the elements whose source point lies in a ready send partition have moved; a
    receive partition has arrived when all its elements have; all partitions ready is the
    whole exchange; the order in which partitions move does not matter."""
    rng = np.random.default_rng(23)
    for grid, ranks, comps, dt in (((12, 8), (3, 2), 2, "f64"), ((8, 8, 8), (2, 2, 2), 1, "f32")):
        p = pt.stencil(grid, ranks, ppn=2, comps=comps, dtype=dt, neighbors="all")
        vt = np.float64 if dt == "f64" else np.float32
        x = pt.stencil_field(p, 3)
        xb = x.view(np.uint8)
        src = ghost_sources(p)
        full = oracle.standard(p, x, lib=lib)
        init = pt.random_bytes(p.recvbuf_bytes, 4)
        s = p.elem_size
        for trial in range(6):
            n, nr = int(rng.integers(1, 7)), int(rng.integers(1, 5))
            cuts = _cuts(rng, p.sendbuf_bytes // s, s, n)
            rcuts = _cuts(rng, p.recvbuf_bytes // s, s, nr)
            ready = rng.integers(0, 2, size=n).astype(np.uint8)
            part = lambda off, c: int(np.searchsorted(c, off, side="right") - 1)
            want = init.copy()
            arr = np.ones(nr, np.uint8)
            for r in range(p.P):
                for k, so in enumerate(src[r]):
                    ro = int(p.recv_base[r]) + k * s
                    if ready[part(so, cuts)]:
                        want[ro: ro + s] = xb[so: so + s]
                    else:
                        arr[part(ro, rcuts)] = 0
            got = oracle.standard_partial(p, cuts, ready, x, init, lib=lib)
            assert np.array_equal(got, want), (grid, trial)
            assert np.array_equal(oracle.arrived(p, cuts, ready, rcuts, lib=lib), arr), (grid, trial)
            rest = 1 - ready
            both = oracle.standard_partial(p, cuts, rest, x, got, lib=lib)
            assert np.array_equal(both, oracle.standard(p, x, init, lib=lib)), (grid, trial)
            assert oracle.arrived(p, cuts, np.ones(n, np.uint8), rcuts, lib=lib).all()
        assert np.array_equal(oracle.standard_partial(p, [0, p.sendbuf_bytes], [1], x, lib=lib), full)
        # a boundary inside an element that is sent, and malformed pointers, are errors
        sent = int(src[0][0])
        for bad in ([0, sent + 1, p.sendbuf_bytes], [0, p.sendbuf_bytes - s], [s, p.sendbuf_bytes],
                    [0, 3 * s, 2 * s, p.sendbuf_bytes]):
            try:
                oracle.standard_partial(p, bad, np.ones(len(bad) - 1, np.uint8), x, lib=lib)
                raise AssertionError(f"accepted partition pointers {bad}")
            except oracle.OracleError as e:
                assert e.code == oracle.ERR_ARG


# -------------------------------------------------------- all-to-all-w ----

def load_wgolden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    w = pt.WPattern(
        name=name, P=g["P"], ppn=1, in_ptr=np.array(g["in_ptr"], np.int32), sources=np.array(g["sources"], np.int32),
        out_ptr=np.array(g["out_ptr"], np.int32), dests=np.array(g["dests"], np.int32),
        sendcounts=np.array(g["sendcounts"], np.int32), sdispls=np.array(g["sdispls"], np.int64),
        sendtypes=np.array(g["sendtypes"], np.int32), recvcounts=np.array(g["recvcounts"], np.int32),
        rdispls=np.array(g["rdispls"], np.int64), recvtypes=np.array(g["recvtypes"], np.int32),
        types=np.array(g["types"], np.int64), send_base=np.array(g["send_base"], np.int64),
        recv_base=np.array(g["recv_base"], np.int64), sendbuf_bytes=g["sendbuf_bytes"],
        recvbuf_bytes=g["recvbuf_bytes"], dtype="bytes")
    return w, g


def apply_change(w, change):
    q = pt.WPattern(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in w.__dict__.items()})
    for k, v in change.items():
        if k == "types_row":
            q.types[v[0]] = v[1]
        else:
            setattr(q, k, np.array(v, dtype=getattr(w, k).dtype))
    return q


def check_w_golden(lib):
    w, g = load_wgolden("alltoallw_vector.json")
    sb = np.array(g["send_values"], np.uint8)
    got = oracle.alltoallw(w, sb, np.array(g["recv_init"], np.uint8), lib=lib)
    assert got.tolist() == g["expected_recv"], got.tolist()
    for case in g["error_cases"]:
        assert oracle.alltoallw_validate(apply_change(w, case["change"]), lib=lib) == case["expected"], case


def w_brute(w, sendbuf, recv_init):
    """The all-to-all-w written as nested loops over each type map (item, level 2,
    level 1, level 0, byte), paired by the t-th occurrence rule read off the lists."""
    out = np.array(recv_init, dtype=np.uint8, copy=True)
    T = w.types
    occ_in = {}
    for d in range(w.P):
        for i in range(w.in_ptr[d], w.in_ptr[d + 1]):
            occ_in.setdefault((int(w.sources[i]), d), []).append(i)
    seen = {}

    def offsets(t, count):
        bl, c0, c1, c2, s0, s1, s2, ext = (int(x) for x in T[t])
        res = []
        for it in range(count):
            for k2 in range(c2):
                for k1 in range(c1):
                    for k0 in range(c0):
                        for b in range(bl):
                            res.append(it * ext + k2 * s2 + k1 * s1 + k0 * s0 + b)
        return res
    for r in range(w.P):
        for e in range(w.out_ptr[r], w.out_ptr[r + 1]):
            d = int(w.dests[e])
            n = seen.get((r, d), 0)
            seen[(r, d)] = n + 1
            i = occ_in[(r, d)][n]
            so = offsets(w.sendtypes[e], int(w.sendcounts[e]))
            ro = offsets(w.recvtypes[i], int(w.recvcounts[i]))
            assert len(so) == len(ro)
            for a, b in zip(so, ro):
                out[w.recv_base[d] + w.rdispls[i] + b] = sendbuf[w.send_base[r] + w.sdispls[e] + a]
    return out


def check_w_bruteforce_random(lib):
    for seed in range(12):
        w = pt.random_wpattern(seed, max_deg=3, max_items=3, max_el=6)
        sb = pt.random_bytes(w.sendbuf_bytes, seed)
        init = pt.random_bytes(w.recvbuf_bytes, seed + 100)
        got = oracle.alltoallw(w, sb, init, lib=lib)
        assert np.array_equal(got, w_brute(w, sb, init)), w.name
        # idempotent, and the bytes received are the bytes sent
        assert np.array_equal(oracle.alltoallw(w, sb, got, lib=lib), got)
        assert int(w.message_bytes().sum()) == int((w.recvcounts.astype(np.int64) *
                                                    w.type_sizes()[w.recvtypes]).sum())


def check_w_reduces_to_v(lib):
    """With one contiguous element type the all-to-all-w is the all-to-all-v."""
    for seed in (1, 4, 9, 17, 23):
        p = pt.random_pattern(seed, indexed=False)
        w = pt.w_from_v(p)
        sb = pt.random_bytes(p.sendbuf_bytes, seed)
        init = pt.random_bytes(p.recvbuf_bytes, seed + 1)
        assert np.array_equal(oracle.alltoallw(w, sb, init, lib=lib), oracle.standard(p, sb, init, lib=lib))
        bad = pt.random_pattern(seed, indexed=False)
        if len(bad.recvcounts):
            bad.recvcounts = bad.recvcounts.copy()
            bad.recvcounts[0] += 1
            assert oracle.alltoallw_validate(pt.w_from_v(bad), lib=lib) == oracle.validate(bad, lib=lib)


def check_w_stencil_bruteforce(lib):
    """A stencil halo through datatypes over the point-major and the component-major
    field equals the global grid read at the ghost coordinates."""
    for grid, ranks, ppn, comps in (((12, 8, 8), (3, 2, 2), 4, 3), ((16, 12), (4, 3), 4, 2)):
        for layout in ("aos", "soa"):
            w = pt.stencil_w(grid, ranks, ppn, comps=comps, dtype="f64", layout=layout)
            p = w.meta["v_pattern"]
            x = pt.stencil_field(p, 13)
            npts = int(np.prod(p.meta["blk"]))
            xs = x if layout == "aos" else pt.soa_from_aos(x, p.P, npts, comps)
            got = as_values(oracle.alltoallw(w, xs, lib=lib), np.float64).reshape(-1, comps)
            exp = ghost_expected(p, x)
            for r in range(p.P):
                lo = p.recv_base[r] // p.elem_size
                assert np.array_equal(got[lo: lo + len(exp[r])], exp[r]), (grid, layout, r)


def w_forward_map(w, lib):
    """Source payload element of every receive payload element (-1 if none), from the
    forward on element ids (the forward is pinned by the checks above)."""
    vt = np.float64 if w.dtype == "f64" else np.float32
    n_send, n_recv = w.sendbuf_bytes // vt().itemsize, w.recvbuf_bytes // vt().itemsize
    ids = np.arange(n_send, dtype=vt)
    got = as_values(oracle.alltoallw(w, ids, np.full(n_recv, -1, vt), lib=lib), vt)
    return got.astype(np.int64), vt


def check_w_adjoint(lib):
    """Backward == transpose of the forward map, exactly on integer-valued gradients;
    accumulate adds; elements no message reads are untouched."""
    for seed in range(20, 32):
        w = pt.random_wpattern(seed, dtype="f64" if seed % 2 else "f32")
        src, vt = w_forward_map(w, lib)
        rng = np.random.default_rng(seed)
        g = rng.integers(-8, 9, size=len(src)).astype(vt)
        old = rng.integers(-8, 9, size=w.sendbuf_bytes // vt().itemsize).astype(vt)
        ref = np.zeros(len(old), np.float64)
        hit = np.zeros(len(old), bool)
        ok = src >= 0
        np.add.at(ref, src[ok], g[ok].astype(np.float64))
        hit[src[ok]] = True
        got = as_values(oracle.alltoallw_backward(w, g, old, lib=lib), vt)
        assert np.array_equal(got[hit], ref[hit].astype(vt)), w.name
        assert np.array_equal(got[~hit], old[~hit]), w.name
        acc = as_values(oracle.alltoallw_backward(w, g, old, accumulate=True, lib=lib), vt)
        assert np.array_equal(acc[hit], (old[hit] + ref[hit]).astype(vt)), w.name
        assert np.array_equal(acc[~hit], old[~hit]), w.name


# ------------------------------------------------------ derived collectives ----

def _coll_problem(c):
    """A golden collective case as the oracle's argument (graph, bases, buffers; bytes)."""
    g = types.SimpleNamespace(name=c["name"], P=c["P"], ppn=c["ppn"], elem_size=c["elem_size"], dtype="bytes")
    for k in ("in_ptr", "sources", "out_ptr", "dests"):
        setattr(g, k, np.array(c[k], np.int32) if k in c else None)
    g.send_base = np.array(c["send_base"], np.int64)
    g.recv_base = np.array(c["recv_base"], np.int64)
    g.sendbuf = np.array(c["send_values"], np.uint8)
    g.recv_init = np.array(c["recv_init"], np.uint8)
    g.sendbuf_bytes, g.recvbuf_bytes = len(g.sendbuf), len(g.recv_init)
    return g


def _coll_run(c, lib):
    g = _coll_problem(c)
    if c["kind"] == "alltoall":
        return oracle.neighbor_alltoall(g, c["count"], g.sendbuf, g.recv_init, lib=lib)
    if c["kind"] == "allgather":
        return oracle.neighbor_allgather(g, c["count"], g.sendbuf, g.recv_init, lib=lib)
    if c["kind"] == "allgatherv":
        return oracle.neighbor_allgatherv(g, c["sendcount"], c["recvcounts"], c["rdispls"], g.sendbuf, g.recv_init,
                                          lib=lib)
    return oracle.alltoallv(g.P, g.ppn, c["sendcounts"], c["sdispls"], c["recvcounts"], c["rdispls"], g.send_base,
                            g.recv_base, g.elem_size, g.sendbuf, g.recvbuf_bytes, g.recv_init, lib=lib)


def check_collectives_golden(lib):
    with open(os.path.join(GOLDEN, "collectives.json")) as f:
        gold = json.load(f)
    cases = {c["name"]: c for c in gold["cases"]}
    for c in gold["cases"]:
        got = _coll_run(c, lib)
        assert np.array_equal(got, np.array(c["expected_recv"], np.uint8)), c["name"]
    for e in gold["errors"]:
        c = dict(cases[e["of"]], **e["change"]) if "of" in e else e
        try:
            _coll_run(c, lib)
            code = 0
        except oracle.OracleError as x:
            code = x.code
        assert code == e["expected_error"], (e["name"], code)


def _listing_pairs(p):
    """(in-edge i, receiver d, position of i in d's in-list, sender r, position in r's
    out-list of the listing it pairs with): the t-th listing of r by d pairs with the t-th
    listing of d by r, found by scanning the lists."""
    out = []
    for d in range(p.P):
        seen = {}
        for i in range(p.in_ptr[d], p.in_ptr[d + 1]):
            r = int(p.sources[i])
            t = seen.get(r, 0)
            seen[r] = t + 1
            js = [j for j in range(p.out_ptr[r + 1] - p.out_ptr[r]) if p.dests[p.out_ptr[r] + j] == d]
            out.append((i, d, i - p.in_ptr[d], r, js[t]))
    return out


def _packed_layout(rng, sizes):
    """Displacements placing blocks of the given sizes one after another in a random order."""
    order = rng.permutation(len(sizes))
    disp = np.zeros(len(sizes), np.int64)
    acc = 0
    for k in order:
        disp[k] = acc
        acc += sizes[k]
    return disp, acc


def check_collectives_bruteforce(lib):
    """Every derived collective on random multigraphs equals its MPI definition, written out
    element by element from the listing pairs."""
    for seed in (3, 11, 19, 26):
        p = pt.random_pattern(seed)
        P, s = p.P, [1, 4, 8, 2][seed % 4]
        rng = np.random.default_rng(seed)
        deg_out, deg_in = np.diff(p.out_ptr), np.diff(p.in_ptr)
        pairs = _listing_pairs(p)
        for kind in ("alltoall", "allgather", "allgatherv"):
            count = 1 + seed % 3
            sendcount = rng.integers(0, 4, P)
            region_send = {"alltoall": deg_out * count, "allgather": np.full(P, count), "allgatherv": sendcount}[kind]
            rcnt = np.array([sendcount[p.sources[i]] if kind == "allgatherv" else count
                             for i in range(len(p.sources))], np.int64)
            rd = np.zeros(len(p.sources), np.int64)
            region_recv = np.zeros(P, np.int64)
            for d in range(P):
                lo, hi = p.in_ptr[d], p.in_ptr[d + 1]
                if kind == "allgatherv":
                    rd[lo:hi], region_recv[d] = _packed_layout(rng, rcnt[lo:hi])
                else:
                    region_recv[d] = (hi - lo) * count
            g = types.SimpleNamespace(name=f"{kind}{seed}", P=P, ppn=p.ppn, in_ptr=p.in_ptr, sources=p.sources,
                                      out_ptr=p.out_ptr, dests=p.dests, elem_size=s, dtype="bytes")
            g.send_base = np.concatenate([[0], np.cumsum(region_send)[:-1]]).astype(np.int64) * s
            g.recv_base = np.concatenate([[0], np.cumsum(region_recv + 1)[:-1]]).astype(np.int64) * s
            g.sendbuf_bytes = int(region_send.sum()) * s
            g.recvbuf_bytes = int((region_recv + 1).sum()) * s
            x = rng.integers(0, 256, g.sendbuf_bytes).astype(np.uint8)
            init = rng.integers(0, 256, g.recvbuf_bytes).astype(np.uint8)
            want = init.copy()
            for i, d, k, r, j in pairs:
                if kind == "alltoall":
                    src, n, dst = g.send_base[r] + j * count * s, count * s, g.recv_base[d] + k * count * s
                elif kind == "allgather":
                    src, n, dst = g.send_base[r], count * s, g.recv_base[d] + k * count * s
                else:
                    src, n, dst = g.send_base[r], sendcount[r] * s, g.recv_base[d] + rd[i] * s
                want[dst:dst + n] = x[src:src + n]
            if kind == "alltoall":
                got = oracle.neighbor_alltoall(g, count, x, init, lib=lib)
            elif kind == "allgather":
                got = oracle.neighbor_allgather(g, count, x, init, lib=lib)
            else:
                got = oracle.neighbor_allgatherv(g, sendcount, rcnt, rd, x, init, lib=lib)
            assert np.array_equal(got, want), (kind, seed)
    for P in (1, 3, 6):
        rng = np.random.default_rng(100 + P)
        s = 4
        cnt = rng.integers(0, 4, (P, P))
        sd = np.zeros((P, P), np.int64)
        rd = np.zeros((P, P), np.int64)
        region_send, region_recv = np.zeros(P, np.int64), np.zeros(P, np.int64)
        for r in range(P):
            sd[r], region_send[r] = _packed_layout(rng, cnt[r])
        for d in range(P):
            rd[d], region_recv[d] = _packed_layout(rng, cnt[:, d])
        send_base = np.concatenate([[0], np.cumsum(region_send)[:-1]]).astype(np.int64) * s
        recv_base = np.concatenate([[0], np.cumsum(region_recv)[:-1]]).astype(np.int64) * s
        x = rng.integers(0, 256, int(region_send.sum()) * s).astype(np.uint8)
        want = np.zeros(int(region_recv.sum()) * s, np.uint8)
        for r in range(P):
            for d in range(P):
                n = cnt[r, d] * s
                src, dst = send_base[r] + sd[r, d] * s, recv_base[d] + rd[d, r] * s
                want[dst:dst + n] = x[src:src + n]
        got = oracle.alltoallv(P, 2, cnt, sd, cnt.T, rd, send_base, recv_base, s, x, len(want), lib=lib)
        assert np.array_equal(got, want), ("alltoallv", P)


ALL_CHECKS = [check_collectives_golden, check_collectives_bruteforce,
              check_partitioned_bruteforce, check_locality_names_values_by_source_element, check_w_golden, check_w_bruteforce_random, check_w_reduces_to_v,
              check_w_stencil_bruteforce, check_w_adjoint,
              check_golden_forward, check_golden_multigraph_truncate, check_golden_locality,
              check_golden_backward_order, check_bruteforce_stencil, check_bruteforce_spmv,
              check_permutation_invariance, check_idempotent_and_untouched,
              check_closed_forms_small, check_adjoint_dense, check_accumulate_and_untouched,
              check_finite_difference, check_error_codes]
