"""CPU oracle for the neighbourhood all-to-all-v data movement (test infrastructure).

Only tests/, __graft_entry__.smoke() and the CPU-baseline / reference legs of bench.py
may import this package.  The GPU library never does, and the two share no code.

The arithmetic lives in oracle.c (plain C, built with gcc by build()).  What it
follows, from "MPI Advance: Open-Source Message Passing Optimizations" (arXiv
2309.07337):
  * section 2.2, Listings 3-4: persistent MPI_Neighbor_alltoallv over a communicator
    from MPI_Dist_graph_create_adjacent, with the MPI standard's meaning
    (orc_match, orc_standard);
  * section 2.2, last paragraph, and section 1: locality-aware aggregation with
    unique global indices, one message per node pair (orc_locality);
  * the reverse exchange (the transpose of the forward 0/1 map) in two fixed
    summation orders (orc_backward);
  * the neighbourhood all-to-all-w (section 2.2's neighbourhood collectives with one
    datatype per edge, MPI standard meaning) and its reverse (orc_alltoallw,
    orc_alltoallw_backward);
  * the partitioned (early-bird) exchange of section 2.3: the state after a subset of
    send partitions has moved, and which receive partitions have arrived
    (orc_standard_partial, orc_arrived);
  * the other neighbourhood collectives (MPI_Neighbor_alltoall, _allgather, _allgatherv:
    section 2.2's drop-in replacements) and MPIX_Alltoallv over the whole communicator
    (section 2.1, Listing 2), each as the neighbourhood all-to-all-v whose counts and
    displacements the MPI standard fixes (orc_derive_neighbor, orc_complete_graph).

Parity is pinned by tests/test_oracle_pins.py against brute-force global indexing,
hand-worked golden cases, invariants and closed-form counts.  The backward's bit
pattern under non-integer data follows the fixed orders documented in oracle.c, a
convention rather than something the paper fixes: within those orders it is pinned by
integer-valued (exactly summed) data and by the dense transpose within rounding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import types

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_ARG, ERR_RANK, ERR_TRUNCATE, ERR_INDEX, ERR_DUP, ERR_GIDX = 0, 1, 2, 3, 4, 5, 6
ERR_NOMEM, ERR_UNSUPPORTED, ERR_OVERLAP = 10, 11, 13
DTYPES = {"bytes": 0, "f32": 1, "f64": 2}

_lib = None


def build(force: bool = False, extra_flags=()) -> str:
    """Compiles oracle.c with gcc (plain IEEE arithmetic, no contraction)."""
    out = _LIB if not extra_flags else os.path.join(
        _HERE, "liboracle_" + "_".join(f.strip("-").replace("=", "") for f in extra_flags) + ".so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", *extra_flags, "-o", out + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    return out


class _Pattern(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_int), ("ppn", ctypes.c_int),
        ("in_ptr", ctypes.c_void_p), ("sources", ctypes.c_void_p),
        ("out_ptr", ctypes.c_void_p), ("dests", ctypes.c_void_p),
        ("sendcounts", ctypes.c_void_p), ("sdispls", ctypes.c_void_p),
        ("recvcounts", ctypes.c_void_p), ("rdispls", ctypes.c_void_p),
        ("send_base", ctypes.c_void_p), ("recv_base", ctypes.c_void_p),
        ("send_slot_ptr", ctypes.c_void_p), ("send_idx", ctypes.c_void_p),
        ("recv_slot_ptr", ctypes.c_void_p),
        ("global_sidx", ctypes.c_void_p), ("global_ridx", ctypes.c_void_p),
        ("elem_size", ctypes.c_int64), ("sendbuf_bytes", ctypes.c_int64),
        ("recvbuf_bytes", ctypes.c_int64),
    ]


class _WPattern(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_int),
        ("in_ptr", ctypes.c_void_p), ("sources", ctypes.c_void_p),
        ("out_ptr", ctypes.c_void_p), ("dests", ctypes.c_void_p),
        ("sendcounts", ctypes.c_void_p), ("sendtypes", ctypes.c_void_p), ("sdispls", ctypes.c_void_p),
        ("recvcounts", ctypes.c_void_p), ("recvtypes", ctypes.c_void_p), ("rdispls", ctypes.c_void_p),
        ("send_base", ctypes.c_void_p), ("recv_base", ctypes.c_void_p),
        ("types", ctypes.c_void_p), ("ntypes", ctypes.c_int),
        ("sendbuf_bytes", ctypes.c_int64), ("recvbuf_bytes", ctypes.c_int64),
    ]


def load(path: str | None = None):
    global _lib
    if path is not None:
        lib = ctypes.CDLL(path)
    else:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
    P = ctypes.POINTER(_Pattern)
    vp = ctypes.c_void_p
    lib.orc_match.argtypes = [P, vp]
    lib.orc_validate.argtypes = [P]
    lib.orc_standard.argtypes = [P, vp, vp]
    lib.orc_locality.argtypes = [P, vp, vp, vp]
    lib.orc_locality_stats.argtypes = [P, vp]
    lib.orc_locality_layout.argtypes = [P, vp, vp, vp, vp]
    lib.orc_backward.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    W = ctypes.POINTER(_WPattern)
    lib.orc_alltoallw_validate.argtypes = [W]
    lib.orc_alltoallw.argtypes = [W, vp, vp]
    lib.orc_alltoallw_backward.argtypes = [W, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.orc_standard_partial.argtypes = [P, ctypes.c_int, vp, vp, vp, vp]
    lib.orc_arrived.argtypes = [P, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp]
    lib.orc_derive_neighbor.argtypes = [P, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.orc_complete_graph.argtypes = [ctypes.c_int, vp, vp]
    for f in ("orc_standard_partial", "orc_arrived", "orc_derive_neighbor", "orc_complete_graph"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("orc_match", "orc_validate", "orc_standard", "orc_locality",
              "orc_locality_stats", "orc_locality_layout", "orc_backward",
              "orc_alltoallw_validate", "orc_alltoallw", "orc_alltoallw_backward"):
        getattr(lib, f).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def _arr(a, dt):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=dt)


class _Marshalled:
    """Keeps the contiguous copies alive while the C struct points at them."""

    def __init__(self, p):
        self.keep = {}
        s = _Pattern()
        s.P, s.ppn = int(p.P), int(p.ppn)
        for name, dt in (("in_ptr", np.int32), ("sources", np.int32), ("out_ptr", np.int32),
                         ("dests", np.int32), ("sendcounts", np.int32), ("sdispls", np.int32),
                         ("recvcounts", np.int32), ("rdispls", np.int32),
                         ("send_base", np.int64), ("recv_base", np.int64),
                         ("send_slot_ptr", np.int64), ("send_idx", np.int32),
                         ("recv_slot_ptr", np.int64), ("global_sidx", np.int64),
                         ("global_ridx", np.int64)):
            a = _arr(getattr(p, name, None), dt)
            self.keep[name] = a
            setattr(s, name, None if a is None else a.ctypes.data)
        s.elem_size = int(p.elem_size)
        s.sendbuf_bytes = int(p.sendbuf_bytes)
        s.recvbuf_bytes = int(p.recvbuf_bytes)
        self.struct = s

    def ref(self):
        return ctypes.byref(self.struct)


def _bytes_view(buf):
    b = np.ascontiguousarray(buf)
    return b, b.view(np.uint8).reshape(-1)


def match(p, lib=None):
    lib = lib or load()
    m = _Marshalled(p)
    out = np.zeros(max(int(p.out_ptr[-1]), 1), dtype=np.int64)
    rc = lib.orc_match(m.ref(), out.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out[: int(p.out_ptr[-1])]


def validate(p, lib=None) -> int:
    """Error code the exchange would raise for this pattern (0 = valid)."""
    lib = lib or load()
    return lib.orc_validate(_Marshalled(p).ref())


def standard(p, sendbuf, recvbuf=None, lib=None):
    """Standard exchange; returns the receive buffer (a copy of recvbuf if given, so
    that uncovered bytes keep their old value, else zeros)."""
    lib = lib or load()
    m = _Marshalled(p)
    _, sb = _bytes_view(sendbuf)
    out = np.zeros(int(p.recvbuf_bytes), dtype=np.uint8) if recvbuf is None else \
        np.array(np.ascontiguousarray(recvbuf).view(np.uint8).reshape(-1), copy=True)
    rc = lib.orc_standard(m.ref(), sb.ctypes.data, out.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out


def locality(p, sendbuf, recvbuf=None, lib=None):
    """Three-step locality-aware exchange; returns (receive bytes, stats dict)."""
    lib = lib or load()
    m = _Marshalled(p)
    _, sb = _bytes_view(sendbuf)
    out = np.zeros(int(p.recvbuf_bytes), dtype=np.uint8) if recvbuf is None else \
        np.array(np.ascontiguousarray(recvbuf).view(np.uint8).reshape(-1), copy=True)
    st = np.zeros(16, dtype=np.int64)
    rc = lib.orc_locality(m.ref(), sb.ctypes.data, out.ctypes.data, st.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out, _stats(st)


STAT_NAMES = ("V", "E", "E_nonzero", "V_direct", "V_inter", "U", "node_pairs",
              "msgs_inter", "msgs_intra", "msgs_step1", "msgs_step3")


def _stats(st):
    return {k: int(st[i]) for i, k in enumerate(STAT_NAMES)}


def locality_stats(p, lib=None):
    lib = lib or load()
    st = np.zeros(16, dtype=np.int64)
    rc = lib.orc_locality_stats(_Marshalled(p).ref(), st.ctypes.data)
    if rc:
        raise OracleError(rc)
    return _stats(st)


def locality_layout(p, lib=None):
    """Aggregate order: arrays (a, b, gidx, rep_rank), one entry per aggregate slot."""
    lib = lib or load()
    st = locality_stats(p, lib)
    n = max(st["U"], 1)
    a = np.zeros(n, np.int32)
    b = np.zeros(n, np.int32)
    g = np.zeros(n, np.int64)
    r = np.zeros(n, np.int32)
    rc = lib.orc_locality_layout(_Marshalled(p).ref(), a.ctypes.data, b.ctypes.data,
                                 g.ctypes.data, r.ctypes.data)
    if rc:
        raise OracleError(rc)
    u = st["U"]
    return a[:u], b[:u], g[:u], r[:u]


def backward(p, grad_recv, grad_send=None, form=0, accumulate=False, dtype=None, lib=None):
    """Reverse exchange; form 0 = standard order, 1 = node-blocked (three-step) order.
    Returns the new grad_send bytes (a copy of grad_send, or zeros)."""
    lib = lib or load()
    m = _Marshalled(p)
    _, gr = _bytes_view(grad_recv)
    out = np.zeros(int(p.sendbuf_bytes), dtype=np.uint8) if grad_send is None else \
        np.array(np.ascontiguousarray(grad_send).view(np.uint8).reshape(-1), copy=True)
    dt = DTYPES[dtype or p.dtype]
    rc = lib.orc_backward(m.ref(), int(form), dt, int(bool(accumulate)), gr.ctypes.data,
                          out.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out


class _WMarshalled:
    """C view of an all-to-all-w problem (patterns.WPattern)."""

    def __init__(self, w):
        self.keep = {}
        s = _WPattern()
        s.P = int(w.P)
        for name, dt in (("in_ptr", np.int32), ("sources", np.int32), ("out_ptr", np.int32),
                         ("dests", np.int32), ("sendcounts", np.int32), ("sendtypes", np.int32),
                         ("sdispls", np.int64), ("recvcounts", np.int32), ("recvtypes", np.int32),
                         ("rdispls", np.int64), ("send_base", np.int64), ("recv_base", np.int64)):
            a = _arr(getattr(w, name), dt)
            self.keep[name] = a
            setattr(s, name, a.ctypes.data if a is not None and a.size else None)
        t = np.ascontiguousarray(np.asarray(w.types, dtype=np.int64).reshape(-1, 8))
        self.keep["types"] = t
        s.types = t.ctypes.data if t.size else None
        s.ntypes = int(t.shape[0])
        s.sendbuf_bytes = int(w.sendbuf_bytes)
        s.recvbuf_bytes = int(w.recvbuf_bytes)
        self.struct = s

    def ref(self):
        return ctypes.byref(self.struct)


def alltoallw_validate(w, lib=None) -> int:
    """Error code the all-to-all-w would raise (0 = valid)."""
    lib = lib or load()
    return lib.orc_alltoallw_validate(_WMarshalled(w).ref())


def alltoallw(w, sendbuf, recvbuf=None, lib=None):
    """Neighbourhood all-to-all-w; returns the receive bytes (a copy of recvbuf if
    given, else zeros)."""
    lib = lib or load()
    m = _WMarshalled(w)
    _, sb = _bytes_view(sendbuf)
    out = np.zeros(int(w.recvbuf_bytes), dtype=np.uint8) if recvbuf is None else \
        np.array(np.ascontiguousarray(recvbuf).view(np.uint8).reshape(-1), copy=True)
    rc = lib.orc_alltoallw(m.ref(), sb.ctypes.data if sb.size else None, out.ctypes.data if out.size else None)
    if rc:
        raise OracleError(rc)
    return out


def alltoallw_backward(w, grad_recv, grad_send=None, accumulate=False, dtype=None, lib=None):
    """Reverse all-to-all-w in the standard order; returns the new grad_send bytes."""
    lib = lib or load()
    m = _WMarshalled(w)
    _, gr = _bytes_view(grad_recv)
    out = np.zeros(int(w.sendbuf_bytes), dtype=np.uint8) if grad_send is None else \
        np.array(np.ascontiguousarray(grad_send).view(np.uint8).reshape(-1), copy=True)
    rc = lib.orc_alltoallw_backward(m.ref(), DTYPES[dtype or w.dtype], int(bool(accumulate)),
                                    gr.ctypes.data if gr.size else None, out.ctypes.data if out.size else None)
    if rc:
        raise OracleError(rc)
    return out


def standard_partial(p, part_ptr, ready, sendbuf, recvbuf=None, lib=None):
    """Standard exchange restricted to elements whose source lies in a ready send
    partition (part_ptr: byte boundaries, ready: one flag per partition)."""
    lib = lib or load()
    m = _Marshalled(p)
    _, sb = _bytes_view(sendbuf)
    out = np.zeros(int(p.recvbuf_bytes), dtype=np.uint8) if recvbuf is None else \
        np.array(np.ascontiguousarray(recvbuf).view(np.uint8).reshape(-1), copy=True)
    pp = np.ascontiguousarray(part_ptr, dtype=np.int64)
    rd = np.ascontiguousarray(ready, dtype=np.uint8)
    rc = lib.orc_standard_partial(m.ref(), len(pp) - 1, pp.ctypes.data, rd.ctypes.data,
                                  sb.ctypes.data if sb.size else None, out.ctypes.data if out.size else None)
    if rc:
        raise OracleError(rc)
    return out


def arrived(p, part_ptr, ready, rpart_ptr, lib=None):
    """Per receive partition: 1 when all of its values come from ready send partitions."""
    lib = lib or load()
    m = _Marshalled(p)
    pp = np.ascontiguousarray(part_ptr, dtype=np.int64)
    rpp = np.ascontiguousarray(rpart_ptr, dtype=np.int64)
    rd = np.ascontiguousarray(ready, dtype=np.uint8)
    out = np.zeros(len(rpp) - 1, dtype=np.uint8)
    rc = lib.orc_arrived(m.ref(), len(pp) - 1, pp.ctypes.data, rd.ctypes.data, len(rpp) - 1, rpp.ctypes.data,
                         out.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out


# ------------------------------------------------ derived neighbourhood collectives

_PATTERN_KEYS = ("name", "P", "ppn", "in_ptr", "sources", "out_ptr", "dests", "sendcounts", "sdispls",
                 "recvcounts", "rdispls", "send_base", "recv_base", "send_slot_ptr", "send_idx",
                 "recv_slot_ptr", "global_sidx", "global_ridx", "elem_size", "sendbuf_bytes",
                 "recvbuf_bytes", "dtype")


def _explicit(g, sendcounts, sdispls, recvcounts, rdispls):
    """The neighbourhood all-to-all-v problem of g's graph, bases and buffers with the given
    per-edge arrays, user-packed (no send lists, no global indices)."""
    q = types.SimpleNamespace(**{k: getattr(g, k, None) for k in _PATTERN_KEYS})
    q.sendcounts = np.ascontiguousarray(sendcounts, dtype=np.int32)
    q.sdispls = np.ascontiguousarray(sdispls, dtype=np.int32)
    q.recvcounts = np.ascontiguousarray(recvcounts, dtype=np.int32)
    q.rdispls = np.ascontiguousarray(rdispls, dtype=np.int32)
    q.send_slot_ptr = q.send_idx = q.recv_slot_ptr = q.global_sidx = q.global_ridx = None
    q.dtype = q.dtype or "bytes"
    return q


def neighbor_pattern(g, kind, count=0, sendcount=None, recvcounts=None, rdispls=None, lib=None):
    """The all-to-all-v problem equal to MPI_Neighbor_<kind> on g (its graph, per-rank byte
    bases, element size and buffer sizes): kind "alltoall" or "allgather" with `count`,
    or "allgatherv" with the per-rank `sendcount` and the caller's per-in-edge `recvcounts`
    and `rdispls`.  The counts and displacements come from orc_derive_neighbor."""
    lib = lib or load()
    mode = {"alltoall": 0, "allgather": 1, "allgatherv": 2}[kind]
    E, Ein = int(g.out_ptr[-1]), int(g.in_ptr[-1])
    sc, sd = np.zeros(max(E, 1), np.int32), np.zeros(max(E, 1), np.int32)
    rc, rd = np.zeros(max(Ein, 1), np.int32), np.zeros(max(Ein, 1), np.int32)
    rk = None if sendcount is None else np.ascontiguousarray(sendcount, dtype=np.int32)
    m = _Marshalled(types.SimpleNamespace(**{k: getattr(g, k, None) for k in _PATTERN_KEYS}))
    err = lib.orc_derive_neighbor(m.ref(), mode, int(count), None if rk is None else rk.ctypes.data,
                                  sc.ctypes.data, sd.ctypes.data, rc.ctypes.data, rd.ctypes.data)
    if err:
        raise OracleError(err)
    if mode == 2:
        rc, rd = recvcounts, rdispls
    return _explicit(g, sc[:E], sd[:E], np.asarray(rc)[:Ein], np.asarray(rd)[:Ein])


def neighbor_alltoall(g, count, sendbuf, recvbuf=None, lib=None):
    """MPI_Neighbor_alltoall on g; returns the receive bytes (see neighbor_pattern)."""
    return standard(neighbor_pattern(g, "alltoall", count=count, lib=lib), sendbuf, recvbuf, lib=lib)


def neighbor_allgather(g, count, sendbuf, recvbuf=None, lib=None):
    """MPI_Neighbor_allgather on g; returns the receive bytes."""
    return standard(neighbor_pattern(g, "allgather", count=count, lib=lib), sendbuf, recvbuf, lib=lib)


def neighbor_allgatherv(g, sendcount, recvcounts, rdispls, sendbuf, recvbuf=None, lib=None):
    """MPI_Neighbor_allgatherv on g; returns the receive bytes."""
    q = neighbor_pattern(g, "allgatherv", sendcount=sendcount, recvcounts=recvcounts, rdispls=rdispls, lib=lib)
    return standard(q, sendbuf, recvbuf, lib=lib)


def alltoallv_pattern(P, ppn, sendcounts, sdispls, recvcounts, rdispls, send_base, recv_base, elem_size,
                      sendbuf_bytes, recvbuf_bytes, dtype="bytes", lib=None):
    """The neighbourhood all-to-all-v problem equal to MPIX_Alltoallv over P ranks: the
    complete graph of orc_complete_graph with the P x P matrices (row-major by rank:
    sendcounts[r*P + d] from r to d, recvcounts[d*P + r] at d from r) as per-edge arrays."""
    lib = lib or load()
    ptr = np.zeros(P + 1, np.int32)
    ranks = np.zeros(max(P * P, 1), np.int32)
    err = lib.orc_complete_graph(int(P), ptr.ctypes.data, ranks.ctypes.data)
    if err:
        raise OracleError(err)
    g = types.SimpleNamespace(name="alltoallv", P=int(P), ppn=int(ppn), in_ptr=ptr, sources=ranks[:P * P],
                              out_ptr=ptr, dests=ranks[:P * P], send_base=np.asarray(send_base, np.int64),
                              recv_base=np.asarray(recv_base, np.int64), elem_size=int(elem_size),
                              sendbuf_bytes=int(sendbuf_bytes), recvbuf_bytes=int(recvbuf_bytes), dtype=dtype)
    return _explicit(g, np.ravel(sendcounts), np.ravel(sdispls), np.ravel(recvcounts), np.ravel(rdispls))


def alltoallv(P, ppn, sendcounts, sdispls, recvcounts, rdispls, send_base, recv_base, elem_size, sendbuf,
              recvbuf_bytes, recvbuf=None, lib=None):
    """MPIX_Alltoallv over P ranks; returns the receive bytes."""
    sb = np.ascontiguousarray(sendbuf).view(np.uint8).reshape(-1)
    q = alltoallv_pattern(P, ppn, sendcounts, sdispls, recvcounts, rdispls, send_base, recv_base, elem_size,
                          sb.size, recvbuf_bytes, lib=lib)
    return standard(q, sb, recvbuf, lib=lib)
