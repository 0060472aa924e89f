"""GB300-native persistent neighbourhood all-to-all-v over emulated ranks in one GPU.

Thin Python binding of the C ABI in include/gbx.h (libgbx.so, built in-tree by
build.py): argument marshalling only, every step of the exchange runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU fallback:
using the binding without the built library raises.

Names follow MPI Advance (arXiv 2309.07337) section 2.2, Listing 4:
dist_graph_create_adjacent, neighbor_alltoallv_init, start, wait.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbx.so")

SUCCESS, ERR_ARG, ERR_RANK, ERR_TRUNCATE, ERR_INDEX, ERR_DUP, ERR_GIDX = 0, 1, 2, 3, 4, 5, 6
ERR_ACTIVE, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM, ERR_UNSUPPORTED, ERR_INTERNAL, ERR_OVERLAP = 7, 8, 9, 10, 11, 12, 13
ERR_LIMIT, ERR_STATE, ERR_DEVICE_WAIT = 14, 15, 16
BYTES, F32, F64 = 0, 1, 2
ALG_STANDARD, ALG_LOCALITY = 0, 1
DTYPE_CODES = {"bytes": BYTES, "f32": F32, "f64": F64}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_pvp = ctypes.POINTER(ctypes.c_void_p)


class RequestInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("kind", "algorithm", "levels", "launches", "use_graph", "vec_bytes", "block", "unroll")] + \
               [(n, ctypes.c_int64) for n in
                ("elem_size", "V", "E", "E_nonzero", "V_direct", "V_inter", "U", "node_pairs",
                 "msgs_inter", "msgs_intra", "msgs_step1", "msgs_step3", "rows", "terms",
                 "user_bytes", "algo_bytes", "device_bytes", "copy_forms")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def lib():
    """The loaded libgbx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(or python -m paper_2309_07337_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "gbx_comm_create": [ctypes.c_int, ctypes.c_int, _pvp],
        "gbx_comm_free": [_pvp],
        "gbx_dist_graph_create_adjacent": [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp,
                                           ctypes.c_char_p, ctypes.c_int, _vp, _pvp],
        "gbx_graph_free": [_pvp],
        "gbx_neighbor_alltoallv_init": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp,
                                        _vp, _vp, _i64, ctypes.c_int, _vp, _vp, _vp,
                                        ctypes.c_char_p, _vp, _pvp],
        "gbx_backward_init": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_char_p, _vp, _pvp],
        "gbx_neighbor_alltoall_init": [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.c_int, _i64, ctypes.c_int, _vp,
                                       ctypes.c_char_p, _vp, _pvp],
        "gbx_neighbor_allgather_init": [_vp, _i64, _vp, _vp, _i64, _vp, ctypes.c_int, _i64, ctypes.c_int, _vp,
                                        ctypes.c_char_p, _vp, _pvp],
        "gbx_neighbor_allgatherv_init": [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, ctypes.c_int, _vp,
                                         ctypes.c_char_p, _vp, _pvp],
        "gbx_alltoallv_init": [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, ctypes.c_int,
                               ctypes.c_char_p, _vp, _pvp],
        "gbx_partitioned_init": [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_char_p, _vp, _pvp],
        "gbx_pready": [_vp, ctypes.c_int, _vp],
        "gbx_parrived": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
        "gbx_parrived_stream": [_vp, ctypes.c_int, _vp],
        "gbx_neighbor_alltoallw_init": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                                        _vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_char_p, _vp, _pvp],
        "gbx_device_status": [ctypes.POINTER(ctypes.c_int)],
        "gbx_start": [_vp],
        "gbx_wait": [_vp],
        "gbx_test": [_vp, ctypes.POINTER(ctypes.c_int)],
        "gbx_wait_stream": [_vp, _vp],
        "gbx_startall": [ctypes.c_int, _pvp],
        "gbx_waitall": [ctypes.c_int, _pvp],
        "gbx_request_bind": [_vp, _vp, _vp],
        "gbx_start_host": [_vp, _vp, _vp],
        "gbx_start_host_async": [_vp, _vp, _vp],
        "gbx_request_get_info": [_vp, ctypes.POINTER(RequestInfo)],
        "gbx_request_free": [_pvp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.gbx_error_string.argtypes = [ctypes.c_int]
    L.gbx_error_string.restype = ctypes.c_char_p
    L.gbx_version.argtypes = []
    L.gbx_version.restype = ctypes.c_int
    _lib = L
    return L


class GbxError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        msg = lib().gbx_error_string(code).decode()
        super().__init__(f"{where}: gbx error {code} ({msg})" if where else f"gbx error {code} ({msg})")
        self.code = code


def _check(rc: int, where: str):
    if rc != SUCCESS:
        raise GbxError(rc, where)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device arrays must be contiguous CUDA tensors"
    return t.data_ptr()


def _buf(t) -> Optional[int]:
    """A data buffer: a contiguous CUDA tensor, or a contiguous pinned CPU tensor, which the
    kernels then read or write in place over the host link."""
    if t is None:
        return None
    assert t.is_contiguous() and (t.is_cuda or t.is_pinned()), \
        "data buffers must be contiguous CUDA tensors or pinned CPU tensors"
    return t.data_ptr()


def _nbytes(t) -> int:
    return 0 if t is None else t.numel() * t.element_size()


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Comm:
    """Emulated communicator: P ranks, ranks_per_node consecutive ranks per node."""

    def __init__(self, P: int, ranks_per_node: int):
        h = ctypes.c_void_p()
        _check(lib().gbx_comm_create(int(P), int(ranks_per_node), ctypes.byref(h)), "comm_create")
        self.handle, self.P, self.ppn = h, int(P), int(ranks_per_node)

    def free(self):
        if self.handle:
            lib().gbx_comm_free(ctypes.byref(self.handle))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class DistGraph:
    """MPI_Dist_graph_create_adjacent over all ranks (CSR in/out lists, int32 CUDA tensors)."""

    def __init__(self, comm: Comm, in_ptr, sources, out_ptr, dests, stream=None):
        h = ctypes.c_void_p()
        _check(lib().gbx_dist_graph_create_adjacent(
            comm.handle, sources.numel(), _ptr(in_ptr), _ptr(sources), None,
            dests.numel(), _ptr(out_ptr), _ptr(dests), None, None, 0, _stream_handle(stream),
            ctypes.byref(h)), "dist_graph_create_adjacent")
        self.handle, self.comm = h, comm

    def free(self):
        if self.handle:
            lib().gbx_graph_free(ctypes.byref(self.handle))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Request:
    """Persistent request: start() / wait() (MPIX_Start / MPIX_Wait)."""

    def __init__(self, handle, keep=()):
        self.handle = handle
        self._keep = list(keep)   # bound buffers stay alive as long as the request

    def start(self):
        _check(lib().gbx_start(self.handle), "start")

    def wait(self):
        _check(lib().gbx_wait(self.handle), "wait")

    def test(self) -> bool:
        f = ctypes.c_int(0)
        _check(lib().gbx_test(self.handle, ctypes.byref(f)), "test")
        return bool(f.value)

    def wait_stream(self, stream=None):
        _check(lib().gbx_wait_stream(self.handle, _stream_handle(stream)), "wait_stream")

    def pready(self, partition: int, stream=None):
        """Partitioned request: partition `partition` of the send buffer is ready; its
        moves are enqueued on `stream` (default: the request's)."""
        _check(lib().gbx_pready(self.handle, int(partition), _stream_handle(stream)), "pready")

    def parrived(self, rpartition: int) -> bool:
        f = ctypes.c_int(0)
        _check(lib().gbx_parrived(self.handle, int(rpartition), ctypes.byref(f)), "parrived")
        return bool(f.value)

    def parrived_stream(self, rpartition: int, stream=None):
        """`stream` waits on the device until receive partition `rpartition` has landed."""
        _check(lib().gbx_parrived_stream(self.handle, int(rpartition), _stream_handle(stream)), "parrived_stream")

    def bind(self, src=None, dst=None):
        _check(lib().gbx_request_bind(self.handle, _buf(src), _buf(dst)), "bind")
        # the request now uses these buffers: keep them (and only the latest ones) alive
        if src is not None:
            self._bound_src = src
        if dst is not None:
            self._bound_dst = dst

    def start_host(self, host_src, host_dst):
        """One exchange on host tensors (copied in, exchanged, copied out)."""
        _check(lib().gbx_start_host(self.handle, host_src.data_ptr(), host_dst.data_ptr()), "start_host")

    def start_host_async(self, host_src=None, host_dst=None):
        """Stream-ordered exchange on host tensors (see gbx_start_host_async in include/gbx.h):
        None skips that copy.  The host tensors must stay alive until the request completes."""
        for t in (host_src, host_dst):
            assert t is None or (not t.is_cuda and t.is_contiguous()), "host buffers must be contiguous CPU tensors"
        _check(lib().gbx_start_host_async(self.handle, None if host_src is None else host_src.data_ptr(),
                                          None if host_dst is None else host_dst.data_ptr()), "start_host_async")
        self._host_keep = (host_src, host_dst)

    def info(self) -> dict:
        i = RequestInfo()
        _check(lib().gbx_request_get_info(self.handle, ctypes.byref(i)), "get_info")
        return i.as_dict()

    def free(self):
        if self.handle:
            lib().gbx_request_free(ctypes.byref(self.handle))
            self._keep = []

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def neighbor_alltoallv_init(sendbuf, send_base, sendcounts, sdispls, recvbuf, recv_base,
                            recvcounts, rdispls, graph: DistGraph, elem_size: int, dtype: int = BYTES,
                            send_slot_ptr=None, send_idx=None, recv_slot_ptr=None,
                            global_sidx=None, global_ridx=None, info: str = "",
                            stream=None) -> Request:
    """MPIX_Neighbor_alltoallv_init over the emulated communicator (see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_neighbor_alltoallv_init(
        _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _ptr(sendcounts), _ptr(sdispls),
        _ptr(send_slot_ptr), _ptr(send_idx), _buf(recvbuf), _nbytes(recvbuf), _ptr(recv_base),
        _ptr(recvcounts), _ptr(rdispls), _ptr(recv_slot_ptr), int(elem_size), int(dtype),
        _ptr(global_sidx), _ptr(global_ridx), graph.handle, info.encode() if info else None,
        _stream_handle(stream), ctypes.byref(h)), "neighbor_alltoallv_init")
    return Request(h, keep=(sendbuf, recvbuf, graph))


def backward_init(forward: Request, grad_recv, grad_send, accumulate: bool = False,
                  info: str = "", stream=None) -> Request:
    """Reverse exchange of a forward request (see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_backward_init(forward.handle, _buf(grad_recv), _buf(grad_send),
                                   int(bool(accumulate)), info.encode() if info else None,
                                   _stream_handle(stream), ctypes.byref(h)), "backward_init")
    return Request(h, keep=(grad_recv, grad_send, forward))


def neighbor_alltoall_init(sendbuf, send_base, recvbuf, recv_base, count: int, graph: DistGraph,
                           elem_size: int, dtype: int = BYTES, info: str = "", stream=None) -> Request:
    """MPI_Neighbor_alltoall, persistent (see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_neighbor_alltoall_init(
        _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _buf(recvbuf), _nbytes(recvbuf), _ptr(recv_base),
        int(count), int(elem_size), int(dtype), graph.handle, info.encode() if info else None,
        _stream_handle(stream), ctypes.byref(h)), "neighbor_alltoall_init")
    return Request(h, keep=(sendbuf, recvbuf, graph))


def neighbor_allgather_init(sendbuf, send_base, recvbuf, recv_base, count: int, graph: DistGraph,
                            elem_size: int, dtype: int = BYTES, info: str = "", stream=None) -> Request:
    """MPI_Neighbor_allgather, persistent (see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_neighbor_allgather_init(
        _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _buf(recvbuf), _nbytes(recvbuf), _ptr(recv_base),
        int(count), int(elem_size), int(dtype), graph.handle, info.encode() if info else None,
        _stream_handle(stream), ctypes.byref(h)), "neighbor_allgather_init")
    return Request(h, keep=(sendbuf, recvbuf, graph))


def neighbor_allgatherv_init(sendbuf, send_base, sendcount, recvbuf, recv_base, recvcounts, rdispls,
                             graph: DistGraph, elem_size: int, dtype: int = BYTES, info: str = "",
                             stream=None) -> Request:
    """MPI_Neighbor_allgatherv, persistent (see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_neighbor_allgatherv_init(
        _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _ptr(sendcount), _buf(recvbuf), _nbytes(recvbuf),
        _ptr(recv_base), _ptr(recvcounts), _ptr(rdispls), int(elem_size), int(dtype), graph.handle,
        info.encode() if info else None, _stream_handle(stream), ctypes.byref(h)), "neighbor_allgatherv_init")
    return Request(h, keep=(sendbuf, recvbuf, graph))


def alltoallv_init(comm: Comm, sendbuf, send_base, sendcounts, sdispls, recvbuf, recv_base, recvcounts,
                   rdispls, elem_size: int, dtype: int = BYTES, info: str = "", stream=None) -> Request:
    """MPIX_Alltoallv over the emulated communicator, persistent (P x P arrays, see include/gbx.h)."""
    h = ctypes.c_void_p()
    _check(lib().gbx_alltoallv_init(
        comm.handle, _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _ptr(sendcounts), _ptr(sdispls),
        _buf(recvbuf), _nbytes(recvbuf), _ptr(recv_base), _ptr(recvcounts), _ptr(rdispls), int(elem_size),
        int(dtype), info.encode() if info else None, _stream_handle(stream), ctypes.byref(h)), "alltoallv_init")
    return Request(h, keep=(sendbuf, recvbuf, comm))


class Datatype(ctypes.Structure):
    """gbx_datatype_t: a block of `blocklen` bytes over three strided levels (innermost
    first), items `extent` bytes apart; all in bytes (see include/gbx.h)."""
    _fields_ = [("blocklen", ctypes.c_int64), ("count", ctypes.c_int64 * 3), ("stride", ctypes.c_int64 * 3),
                ("extent", ctypes.c_int64)]


def datatype_table(rows):
    """ctypes array of Datatype from rows (blocklen, count0, count1, count2, stride0,
    stride1, stride2, extent)."""
    rows = [tuple(int(x) for x in r) for r in rows]
    arr = (Datatype * max(len(rows), 1))()
    for k, r in enumerate(rows):
        arr[k].blocklen = r[0]
        arr[k].count[:] = r[1:4]
        arr[k].stride[:] = r[4:7]
        arr[k].extent = r[7]
    return arr, len(rows)


def neighbor_alltoallw_init(sendbuf, send_base, sendcounts, sdispls, sendtypes, recvbuf, recv_base, recvcounts,
                            rdispls, recvtypes, types, graph: DistGraph, dtype: int = BYTES, info: str = "",
                            stream=None) -> Request:
    """MPI_Neighbor_alltoallw, persistent: per-edge datatypes, byte displacements (see
    include/gbx.h).  `types`: rows (blocklen, count0, count1, count2, stride0, stride1,
    stride2, extent), copied at init; the per-edge arrays are device tensors."""
    arr, n = datatype_table(types)
    h = ctypes.c_void_p()
    _check(lib().gbx_neighbor_alltoallw_init(
        _buf(sendbuf), _nbytes(sendbuf), _ptr(send_base), _ptr(sendcounts), _ptr(sdispls), _ptr(sendtypes),
        _buf(recvbuf), _nbytes(recvbuf), _ptr(recv_base), _ptr(recvcounts), _ptr(rdispls), _ptr(recvtypes),
        ctypes.cast(arr, ctypes.c_void_p), int(n), int(dtype), graph.handle, info.encode() if info else None,
        _stream_handle(stream), ctypes.byref(h)), "neighbor_alltoallw_init")
    return Request(h, keep=(sendbuf, recvbuf, graph))


def partitioned_init(forward: Request, part_ptr, rpart_ptr, info: str = "", stream=None) -> Request:
    """Partitioned (early-bird) exchange over a standard-form forward request: send
    partitions = byte ranges part_ptr[k]..part_ptr[k+1] of its send buffer, receive
    partitions likewise over its receive buffer (host integer sequences; see include/gbx.h).
    Use start(), pready(k, stream) per ready partition, parrived(j) / parrived_stream(j),
    then wait()."""
    import numpy as np
    pp = np.ascontiguousarray(part_ptr, dtype=np.int64)
    rp = np.ascontiguousarray(rpart_ptr, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib().gbx_partitioned_init(forward.handle, len(pp) - 1, pp.ctypes.data, len(rp) - 1, rp.ctypes.data,
                                      info.encode() if info else None, _stream_handle(stream), ctypes.byref(h)),
           "partitioned_init")
    return Request(h, keep=(forward,))


def device_status() -> int:
    """Reads and clears the move kernels' device status word (1 = a bounded wait gave up)."""
    f = ctypes.c_int(0)
    _check(lib().gbx_device_status(ctypes.byref(f)), "device_status")
    return f.value


def _handles(reqs: Sequence[Request]):
    arr = (ctypes.c_void_p * len(reqs))(*[r.handle.value for r in reqs])
    return arr


def startall(reqs: Sequence[Request]):
    _check(lib().gbx_startall(len(reqs), _handles(reqs)), "startall")


def waitall(reqs: Sequence[Request]):
    _check(lib().gbx_waitall(len(reqs), _handles(reqs)), "waitall")


# --------------------------------------------------------------- conveniences

class DevicePattern:
    """A patterns.Pattern's integer arrays uploaded to the GPU (inputs only)."""

    FIELDS = (("in_ptr", "int32"), ("sources", "int32"), ("out_ptr", "int32"), ("dests", "int32"),
              ("sendcounts", "int32"), ("sdispls", "int32"), ("recvcounts", "int32"),
              ("rdispls", "int32"), ("send_base", "int64"), ("recv_base", "int64"),
              ("send_slot_ptr", "int64"), ("send_idx", "int32"), ("recv_slot_ptr", "int64"),
              ("global_sidx", "int64"), ("global_ridx", "int64"))

    def __init__(self, p, device="cuda"):
        import numpy as np
        import torch
        self.p = p
        for name, dt in self.FIELDS:
            a = getattr(p, name, None)
            setattr(self, name, None if a is None else
                    torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device))


class Exchange:
    """Communicator + graph + persistent request for one pattern and its buffers.
    Every array the pattern has is passed to the library (send lists, global indices)."""

    def __init__(self, p, sendbuf, recvbuf, algorithm="standard", info="", dp: DevicePattern = None,
                 stream=None, graph: DistGraph = None):
        self.p = p
        self.dp = dp or DevicePattern(p)
        self.comm = graph.comm if graph is not None else Comm(p.P, p.ppn)
        self.graph = graph or DistGraph(self.comm, self.dp.in_ptr, self.dp.sources, self.dp.out_ptr,
                                        self.dp.dests, stream)
        full = f"algorithm={algorithm}" + (";" + info if info else "")
        dp = self.dp
        self.request = neighbor_alltoallv_init(
            sendbuf, dp.send_base, dp.sendcounts, dp.sdispls, recvbuf, dp.recv_base, dp.recvcounts,
            dp.rdispls, self.graph, p.elem_size, DTYPE_CODES[p.dtype],
            send_slot_ptr=dp.send_slot_ptr, send_idx=dp.send_idx, recv_slot_ptr=dp.recv_slot_ptr,
            global_sidx=dp.global_sidx, global_ridx=dp.global_ridx, info=full, stream=stream)

    def start(self):
        self.request.start()

    def wait(self):
        self.request.wait()

    def info(self):
        return self.request.info()


class DeviceWPattern:
    """A patterns.WPattern's per-edge and per-rank arrays uploaded to the GPU."""

    FIELDS = (("in_ptr", "int32"), ("sources", "int32"), ("out_ptr", "int32"), ("dests", "int32"),
              ("sendcounts", "int32"), ("sdispls", "int64"), ("sendtypes", "int32"),
              ("recvcounts", "int32"), ("rdispls", "int64"), ("recvtypes", "int32"),
              ("send_base", "int64"), ("recv_base", "int64"))

    def __init__(self, w, device="cuda"):
        import numpy as np
        import torch
        self.w = w
        for name, dt in self.FIELDS:
            setattr(self, name, torch.from_numpy(np.ascontiguousarray(getattr(w, name), dtype=dt)).to(device))


class WExchange:
    """Communicator + graph + persistent all-to-all-w request for one WPattern."""

    def __init__(self, w, sendbuf, recvbuf, info="", dw: DeviceWPattern = None, stream=None,
                 graph: DistGraph = None):
        self.w = w
        self.dw = dw or DeviceWPattern(w)
        self.comm = graph.comm if graph is not None else Comm(w.P, w.ppn)
        self.graph = graph or DistGraph(self.comm, self.dw.in_ptr, self.dw.sources, self.dw.out_ptr,
                                        self.dw.dests, stream)
        d = self.dw
        self.request = neighbor_alltoallw_init(
            sendbuf, d.send_base, d.sendcounts, d.sdispls, d.sendtypes, recvbuf, d.recv_base, d.recvcounts,
            d.rdispls, d.recvtypes, w.types, self.graph, DTYPE_CODES[w.dtype], info=info, stream=stream)

    def start(self):
        self.request.start()

    def wait(self):
        self.request.wait()

    def info(self):
        return self.request.info()
