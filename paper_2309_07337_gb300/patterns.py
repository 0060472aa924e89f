"""Seeded synthetic communication patterns for the neighbourhood exchange.

This module only builds inputs: distributed-graph adjacency, per-edge counts and
displacements, send index lists, global indices and payload buffers, for the workloads
the exchange is measured on (halo exchanges of structured stencils and of a
row-partitioned sparse matrix-vector product, the applications that motivate
locality-aware neighbourhood collectives in section 1 of the MPI Advance paper).
It holds none of the exchange's own arithmetic: no edge matching, no data movement,
no aggregation.  Both the GPU path and the CPU oracle consume what it returns.

Conventions shared by every generator:
  * ranks are numbered row-major with x fastest; node(r) = r // ppn;
  * out- and in-neighbour lists are in ascending rank order;
  * each rank's send slots are its send lists concatenated in out-list order
    (sdispls packed), its receive slots the received blocks concatenated in in-list
    order (rdispls packed);
  * all ranks' regions live in one send buffer and one receive buffer, located by
    per-rank byte offsets;
  * numpy PCG64 streams seeded by the caller.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Pattern:
    """One neighbourhood all-to-all-v problem over P emulated ranks."""

    name: str
    P: int
    ppn: int
    in_ptr: np.ndarray          # int32 [P+1], CSR of in-lists
    sources: np.ndarray         # int32 [E]
    out_ptr: np.ndarray         # int32 [P+1], CSR of out-lists
    dests: np.ndarray           # int32 [E]
    sendcounts: np.ndarray      # int32 [E], aligned with dests
    sdispls: np.ndarray         # int32 [E]
    recvcounts: np.ndarray      # int32 [E], aligned with sources
    rdispls: np.ndarray         # int32 [E]
    elem_size: int              # bytes per element
    dtype: str                  # 'f64', 'f32' or 'bytes'
    send_base: np.ndarray       # int64 [P], byte offset of rank r's send region
    recv_base: np.ndarray       # int64 [P], byte offset of rank r's receive region
    sendbuf_bytes: int
    recvbuf_bytes: int
    send_slot_ptr: Optional[np.ndarray] = None   # int64 [P+1]
    send_idx: Optional[np.ndarray] = None        # int32 [send slots]
    recv_slot_ptr: Optional[np.ndarray] = None   # int64 [P+1]
    global_sidx: Optional[np.ndarray] = None     # int64 [send slots]
    global_ridx: Optional[np.ndarray] = None     # int64 [receive slots]
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.out_ptr[-1])

    @property
    def volume(self) -> int:
        """Elements moved by one exchange (V)."""
        return int(self.sendcounts.astype(np.int64).sum())

    def user_bytes(self) -> int:
        """Bytes a user sees moved: V elements read and V elements written."""
        return 2 * self.volume * self.elem_size


def _ptr_from_counts(counts: np.ndarray) -> np.ndarray:
    ptr = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    return ptr


def _segmented_exclusive(counts: np.ndarray, owner: np.ndarray, P: int) -> np.ndarray:
    """Exclusive running sum of counts restarting at every owner (edges sorted by owner)."""
    c = counts.astype(np.int64)
    run = np.cumsum(c) - c
    first = np.searchsorted(owner, np.arange(P), side="left")
    start_of = np.concatenate([run, [0]])[first]  # running sum at each owner's first edge
    return run - start_of[owner]


def _ragged_arange(counts: np.ndarray) -> np.ndarray:
    """concatenate([arange(c) for c in counts]) without a Python loop."""
    counts = counts.astype(np.int64)
    total = int(counts.sum())
    if total == 0:
        return np.zeros(0, dtype=np.int64)
    starts = np.cumsum(counts) - counts
    return np.arange(total, dtype=np.int64) - np.repeat(starts, counts)


def _assemble(name, P, ppn, out_src, out_dst, out_cnt, send_elem, send_gidx,
              in_dst, in_src, in_cnt, recv_gidx, elem_size, dtype, region_elems, meta):
    """Builds a Pattern from edge lists already sorted by (owner rank, list order).

    out_*: one entry per out-edge; send_elem/send_gidx: one per send slot, in out-edge
    order.  in_*: one per in-edge; recv_gidx: one per receive slot in in-edge order.
    region_elems[r]: number of elements in rank r's send region."""
    out_src = np.asarray(out_src, dtype=np.int64)
    in_dst = np.asarray(in_dst, dtype=np.int64)
    out_ptr = _ptr_from_counts(np.bincount(out_src, minlength=P)).astype(np.int32)
    in_ptr = _ptr_from_counts(np.bincount(in_dst, minlength=P)).astype(np.int32)
    sdispls = _segmented_exclusive(out_cnt, out_src, P)
    rdispls = _segmented_exclusive(in_cnt, in_dst, P)
    send_tot = np.bincount(out_src, weights=out_cnt, minlength=P).astype(np.int64)
    recv_tot = np.bincount(in_dst, weights=in_cnt, minlength=P).astype(np.int64)
    send_slot_ptr = _ptr_from_counts(send_tot)
    recv_slot_ptr = _ptr_from_counts(recv_tot)
    region_elems = np.asarray(region_elems, dtype=np.int64)
    send_base = (_ptr_from_counts(region_elems)[:-1] * elem_size).astype(np.int64)
    recv_base = (recv_slot_ptr[:-1] * elem_size).astype(np.int64)
    return Pattern(
        name=name, P=P, ppn=ppn,
        in_ptr=in_ptr, sources=np.asarray(in_src, dtype=np.int32),
        out_ptr=out_ptr, dests=np.asarray(out_dst, dtype=np.int32),
        sendcounts=np.asarray(out_cnt, dtype=np.int32), sdispls=sdispls.astype(np.int32),
        recvcounts=np.asarray(in_cnt, dtype=np.int32), rdispls=rdispls.astype(np.int32),
        elem_size=int(elem_size), dtype=dtype,
        send_base=send_base, recv_base=recv_base,
        sendbuf_bytes=int(region_elems.sum() * elem_size),
        recvbuf_bytes=int(recv_slot_ptr[-1] * elem_size),
        send_slot_ptr=send_slot_ptr, send_idx=np.asarray(send_elem, dtype=np.int32),
        recv_slot_ptr=recv_slot_ptr,
        global_sidx=np.asarray(send_gidx, dtype=np.int64),
        global_ridx=np.asarray(recv_gidx, dtype=np.int64),
        meta=meta)


# ------------------------------------------------------------------ stencils ---

def stencil(grid, ranks, ppn, comps=1, dtype="f64", neighbors="all", name=None, directions=None) -> Pattern:
    """Halo exchange of a structured grid split into equal rank blocks (no periodicity).

    grid, ranks: per-axis point and rank counts (x first), 2 or 3 axes.
    neighbors: 'faces' (5-point in 2D, 7-point in 3D) or 'all' (9- / 27-point).
    directions: optional subset of neighbour offsets (x first) to keep.
    Each point carries `comps` values stored together (one element of comps*8 or
    comps*4 bytes).  The send list towards direction delta is the boundary layer facing
    it (coordinate 0 where delta=-1, n-1 where delta=+1, all where delta=0), in
    ascending local point index; the global index of a point is its row-major index in
    the whole grid."""
    grid = tuple(int(g) for g in grid)
    ranks = tuple(int(r) for r in ranks)
    D = len(grid)
    assert D in (2, 3) and len(ranks) == D
    blk = tuple(g // r for g, r in zip(grid, ranks))
    assert all(b * r == g for b, r, g in zip(blk, ranks, grid))
    P = int(np.prod(ranks))
    esz = comps * (8 if dtype == "f64" else 4)
    npts = int(np.prod(blk))

    # directions in ascending neighbour-rank order: lexicographic in (dz, dy, dx)
    dirs = []
    for d in itertools.product((-1, 0, 1), repeat=D):
        dd = tuple(reversed(d))  # dd[0] = dx
        if any(dd) and (neighbors == "all" or sum(map(abs, dd)) == 1):
            if directions is None or dd in [tuple(x) for x in directions]:
                dirs.append(dd)

    # local coordinates of each local point (x fastest)
    loc = np.indices(tuple(reversed(blk))).reshape(D, -1)[::-1]  # loc[axis][point]
    templates = []
    for dd in dirs:
        m = np.ones(npts, dtype=bool)
        for ax in range(D):
            if dd[ax] == -1:
                m &= loc[ax] == 0
            elif dd[ax] == 1:
                m &= loc[ax] == blk[ax] - 1
        templates.append(np.nonzero(m)[0].astype(np.int64))
    tsize = np.array([len(t) for t in templates], dtype=np.int64)
    tpool = np.concatenate(templates)
    toff = _ptr_from_counts(tsize)[:-1]

    rc = np.indices(tuple(reversed(ranks))).reshape(D, -1)[::-1]  # rank coords[axis][rank]
    stride = [1, ranks[0], ranks[0] * ranks[1]][:D]
    dirs_a = np.array(dirs, dtype=np.int64)                         # [ndir, D]
    valid = np.ones((P, len(dirs)), dtype=bool)
    for ax in range(D):
        c = rc[ax][:, None] + dirs_a[None, :, ax]
        valid &= (c >= 0) & (c < ranks[ax])
    nbr = np.arange(P)[:, None] + (dirs_a * np.array(stride)).sum(1)[None, :]
    er, ed = np.nonzero(valid)                 # edges sorted by (rank, direction order)
    edst = nbr[er, ed]
    ecnt = tsize[ed]

    gstride = [1, grid[0], grid[0] * grid[1]][:D]

    def gidx_of(rank, local):
        g = np.zeros(len(local), dtype=np.int64)
        for ax in range(D):
            g += (rc[ax][rank] * blk[ax] + loc[ax][local]) * gstride[ax]
        return g

    k = _ragged_arange(ecnt)
    send_elem = tpool[np.repeat(toff[ed], ecnt) + k]
    send_rank = np.repeat(er, ecnt)
    send_gidx = gidx_of(send_rank, send_elem)

    # receive side: rank d hears from d+delta' (ascending order = same direction order);
    # the block from q = d + delta' is q's send list towards -delta'.
    opp = np.array([dirs.index(tuple(-x for x in dd)) for dd in dirs], dtype=np.int64)
    ir, idd = np.nonzero(valid)
    isrc = nbr[ir, idd]
    icnt = tsize[opp[idd]]
    k2 = _ragged_arange(icnt)
    recv_elem = tpool[np.repeat(toff[opp[idd]], icnt) + k2]
    recv_gidx = gidx_of(np.repeat(isrc, icnt), recv_elem)

    meta = dict(kind="stencil", grid=grid, ranks=ranks, blk=blk, comps=comps,
                neighbors=neighbors, dirs=dirs)
    return _assemble(name or f"stencil{D}d_{'x'.join(map(str, grid))}_P{P}_c{comps}",
                     P, ppn, er, edst, ecnt, send_elem, send_gidx,
                     ir, isrc, icnt, recv_gidx, esz, dtype, np.full(P, npts), meta)


def stencil_field(p: Pattern, seed: int) -> np.ndarray:
    """Send buffer of a stencil pattern: every rank's block, values U(-1, 1)."""
    rng = np.random.default_rng(seed)
    n = p.sendbuf_bytes // (8 if p.dtype == "f64" else 4)
    if p.dtype == "f64":
        return rng.uniform(-1.0, 1.0, size=n)
    return rng.uniform(-1.0, 1.0, size=n).astype(np.float32)


# -------------------------------------------------------------- SpMV halos ---

def row_starts(n: int, P: int) -> np.ndarray:
    """Contiguous row partition; the first n mod P ranks get one extra row."""
    base, extra = divmod(n, P)
    r = np.arange(P + 1, dtype=np.int64)
    return r * base + np.minimum(r, extra)


def spmv_columns(n: int, nnz: int, seed: int, band: int = 4096, band_frac: float = 0.8):
    """Column indices of a random sparse matrix: per row, round(band_frac*nnz) columns
    uniform in [i-band, i+band] (clipped to the matrix) and the rest uniform in [0, n);
    duplicates inside a row are redrawn from the same distribution."""
    rng = np.random.default_rng(seed)
    nb = int(round(band_frac * nnz))
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(rows - band, 0)
    hi = np.minimum(rows + band, n - 1)
    assert int((hi - lo + 1).min()) >= nb and n >= nnz, "band too narrow for nnz"
    cols = np.empty((n, nnz), dtype=np.int64)
    cols[:, :nb] = rng.integers(lo[:, None], hi[:, None] + 1, size=(n, nb))
    cols[:, nb:] = rng.integers(0, n, size=(n, nnz - nb))
    while True:
        order = np.argsort(cols, axis=1, kind="stable")
        srt = np.take_along_axis(cols, order, axis=1)
        dup_sorted = np.zeros_like(srt, dtype=bool)
        dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
        if not dup_sorted.any():
            break
        dup = np.zeros_like(dup_sorted)
        np.put_along_axis(dup, order, dup_sorted, axis=1)
        ri, ci = np.nonzero(dup)
        is_band = ci < nb
        cols[ri[is_band], ci[is_band]] = rng.integers(lo[ri[is_band]], hi[ri[is_band]] + 1)
        cols[ri[~is_band], ci[~is_band]] = rng.integers(0, n, size=int((~is_band).sum()))
    return cols


def spmv_halo(n: int, P: int, ppn: int, nnz: int, seed: int, dtype: str = "f64",
              band: int = 4096, band_frac: float = 0.8, name=None, keep_matrix=False) -> Pattern:
    """Halo exchange of y = A x with A row-partitioned over P ranks.

    Rank d receives the x entries of every column its rows touch outside its own row
    range (the off-rank columns, ascending global index = ascending owner); the owner
    sends them, in the same order, from its slice of x.  Global index = matrix column."""
    cols = spmv_columns(n, nnz, seed, band, band_frac)
    rs = row_starts(n, P)
    row_owner = np.repeat(np.arange(P, dtype=np.int64), np.diff(rs))
    col_owner = np.searchsorted(rs, cols, side="right") - 1
    off = col_owner != row_owner[:, None]
    d_of = np.broadcast_to(row_owner[:, None], cols.shape)[off]
    keys = np.sort(d_of * n + cols[off])             # sorted by (receiver, column)
    keys = keys[np.r_[True, keys[1:] != keys[:-1]]]
    rd = keys // n
    rcol = keys % n
    rq = np.searchsorted(rs, rcol, side="right") - 1  # owner of each received column
    # in-edges: runs of (d, q)
    ek = rd * P + rq
    starts = np.flatnonzero(np.r_[True, ek[1:] != ek[:-1]])
    in_dst = rd[starts]
    in_src = rq[starts]
    in_cnt = np.diff(np.r_[starts, len(ek)])
    # out-edges: the same (q -> d) blocks sorted by (q, d, column)
    o = np.lexsort((rcol, rd, rq))
    sq, sd, sc = rq[o], rd[o], rcol[o]
    ok = sq * P + sd
    ostarts = np.flatnonzero(np.r_[True, ok[1:] != ok[:-1]])
    out_src = sq[ostarts]
    out_dst = sd[ostarts]
    out_cnt = np.diff(np.r_[ostarts, len(ok)])
    send_elem = sc - rs[sq]
    esz = 8 if dtype == "f64" else 4
    meta = dict(kind="spmv", n=n, nnz=nnz, band=band, row_starts=rs, seed=seed)
    if keep_matrix:
        meta["cols"] = cols
    return _assemble(name or f"spmv_n{n}_P{P}_nnz{nnz}_{dtype}", P, ppn,
                     out_src, out_dst, out_cnt, send_elem, sc,
                     in_dst, in_src, in_cnt, rcol, esz, dtype, np.diff(rs), meta)


def spmv_x(p: Pattern, seed: int) -> np.ndarray:
    """Send buffer of an SpMV halo pattern: x ~ N(0, 1) in the pattern's precision."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(p.meta["n"])
    return x if p.dtype == "f64" else x.astype(np.float32)


def batched_specs(count: int, seed: int):
    """Sizes of the uneven batch: rows 2^k (k uniform in 14..20), P uniform in 64..1024,
    nnz/row uniform in 8..32, fp32 or fp64 with probability 1/2 each, 32 ranks per node."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        k = int(rng.integers(14, 21))
        P = int(rng.integers(64, 1025))
        nnz = int(rng.integers(8, 33))
        dt = "f32" if rng.random() < 0.5 else "f64"
        out.append(dict(n=1 << k, P=P, ppn=32, nnz=nnz, dtype=dt, seed=seed * 1000 + j))
    return out


# ------------------------------------------------------------ the workloads ---

SEED = 2309


def config1():
    """2D 5-point Laplacian halo: 256x256 grid, 4x4 ranks of 64x64, 4 ranks per node, fp64."""
    return stencil((256, 256), (4, 4), ppn=4, comps=1, dtype="f64", neighbors="faces",
                   name="cfg1_stencil2d_5pt_256sq_P16")


def config2(n=1 << 20, P=1024):
    """SpMV halo: 2^20 rows over 1024 ranks (32 per node), 20 nnz/row, fp64 x."""
    return spmv_halo(n, P, 32, 20, SEED + 2, "f64", name=f"cfg2_spmv_n{n}_P{P}")


def config3(count=64):
    """64 uneven SpMV halo patterns, mixed fp32 / fp64."""
    return [spmv_halo(s["n"], s["P"], s["ppn"], s["nnz"], s["seed"], s["dtype"],
                      name=f"cfg3_{j}_n{s['n']}_P{s['P']}_{s['dtype']}")
            for j, s in enumerate(batched_specs(count, SEED + 3))]


def config4(n=1 << 20, P=1024, ppn=32):
    """Differentiable halo: the config-2 matrix with fp32 values and fp32 x."""
    return spmv_halo(n, P, ppn, 20, SEED + 2, "f32", name=f"cfg4_spmv_n{n}_P{P}_f32",
                     keep_matrix=True)


def config5(edge=32, comps=8, R=16, ppn=64):
    """3D 27-point stencil: (R*edge)^3 grid over R^3 ranks, `comps` fp64 per point."""
    g = R * edge
    return stencil((g, g, g), (R, R, R), ppn=ppn, comps=comps, dtype="f64", neighbors="all",
                   name=f"cfg5_stencil3d_27pt_{g}cube_P{R ** 3}_c{comps}")


def restrict_to_receivers(p: Pattern, keep) -> Pattern:
    """Sub-problem of `p` in which only ranks in `keep` receive (a bounded sample of the
    same workload).  Buffers and displacements are unchanged; edges into other ranks
    are dropped from both lists."""
    keep_mask = np.zeros(p.P, dtype=bool)
    keep_mask[np.asarray(keep)] = True
    in_owner = np.repeat(np.arange(p.P), np.diff(p.in_ptr))
    out_owner = np.repeat(np.arange(p.P), np.diff(p.out_ptr))
    ki = keep_mask[in_owner]
    ko = keep_mask[p.dests]
    q = dataclasses.replace(p)
    q.name = p.name + f"_recv{int(keep_mask.sum())}"
    q.in_ptr = _ptr_from_counts(np.bincount(in_owner[ki], minlength=p.P)).astype(np.int32)
    q.sources = p.sources[ki]
    q.recvcounts = p.recvcounts[ki]
    q.rdispls = p.rdispls[ki]
    q.out_ptr = _ptr_from_counts(np.bincount(out_owner[ko], minlength=p.P)).astype(np.int32)
    q.dests = p.dests[ko]
    q.sendcounts = p.sendcounts[ko]
    q.sdispls = p.sdispls[ko]
    return q


# ----------------------------------------------------------- random patterns ---

def random_pattern(seed: int, P=None, ppn=None, elem_size=None, indexed=None, dtype=None,
                   max_deg=6, max_count=5, gaps=True) -> Pattern:
    """Random valid exchange for fuzzing: repeated neighbours (multigraph), self edges,
    zero-count edges, isolated ranks, in-lists in shuffled order (each sender's listings
    keep their relative order, as the multigraph rule pairs them by occurrence), receive
    blocks placed in random order with gaps, and byte gaps between rank regions so that
    offsets are not vector aligned.  Global indices name source elements, so equal
    indices always carry equal bytes."""
    rng = np.random.default_rng(seed)
    P = int(P if P is not None else rng.integers(1, 65))
    ppn = int(ppn if ppn is not None else rng.choice([1, 2, 3, 4, max(P, 1)]))
    if dtype is None:
        dtype = "bytes"
    if elem_size is None:
        elem_size = int(rng.choice([1, 2, 3, 4, 5, 8, 12, 16, 24, 64, 128])) if dtype == "bytes" else \
            (8 if dtype == "f64" else 4) * int(rng.choice([1, 2, 3, 4, 8]))
    s = int(elem_size)
    unit = 1 if dtype == "bytes" else (8 if dtype == "f64" else 4)   # gaps keep float data aligned
    indexed = bool(rng.integers(0, 2)) if indexed is None else bool(indexed)
    region = rng.integers(1, 21, size=P) if indexed else None
    outs = []   # per rank: list of (dest, count, send elements)
    for r in range(P):
        deg = int(rng.integers(0, max_deg + 1)) if rng.random() > 0.1 else 0
        lst = []
        for _ in range(deg):
            d = int(rng.integers(0, P))
            c = int(rng.integers(0, max_count + 1))
            els = rng.integers(0, region[r], size=c) if indexed else None
            lst.append((d, c, els))
        outs.append(lst)
    # send slots: packed in out-list order
    send_elem, send_rank_of_slot = [], []
    sdispls, out_src, out_dst, out_cnt = [], [], [], []
    for r in range(P):
        pos = 0
        for d, c, els in outs[r]:
            out_src.append(r); out_dst.append(d); out_cnt.append(c); sdispls.append(pos)
            send_elem.extend(els.tolist() if indexed else range(pos, pos + c))
            send_rank_of_slot.extend([r] * c)
            pos += c
    nslots = np.bincount(np.array(out_src, dtype=np.int64), weights=np.array(out_cnt), minlength=P).astype(np.int64) \
        if out_src else np.zeros(P, np.int64)
    send_slot_ptr = _ptr_from_counts(nslots)
    region_elems = region if indexed else np.maximum(nslots, 1)
    # send regions with byte gaps
    send_base = np.zeros(P, np.int64)
    off = int(rng.integers(0, 7)) * unit if gaps else 0
    for r in range(P):
        send_base[r] = off
        off += int(region_elems[r]) * s + (int(rng.integers(0, 7)) * unit if gaps else 0)
    sendbuf_bytes = off
    # element identity -> global index (equal index <=> same source element)
    elem_base = _ptr_from_counts(np.asarray(region_elems, np.int64))
    send_elem = np.asarray(send_elem, dtype=np.int64)
    srank = np.asarray(send_rank_of_slot, dtype=np.int64)
    gs = elem_base[srank] + send_elem if len(send_elem) else np.zeros(0, np.int64)
    # in-lists: every d lists its senders; shuffle but keep each sender's listings in order
    ins = [[] for _ in range(P)]
    e = 0
    for r in range(P):
        for t, (d, c, els) in enumerate(outs[r]):
            ins[d].append((r, c, e))
            e += 1
    in_dst, in_src, in_cnt, rdispls, rgidx_blocks = [], [], [], [], []
    recv_slots = np.zeros(P, np.int64)
    recv_g = []
    for d in range(P):
        lst = ins[d]
        # random interleaving that keeps per-sender order
        keys = rng.random(len(lst))
        by_sender = {}
        for i, (r, c, eid) in enumerate(lst):
            by_sender.setdefault(r, []).append(i)
        for r, idxs in by_sender.items():
            ks = np.sort(keys[idxs])
            for i, k in zip(idxs, ks):
                keys[i] = k
        order = np.argsort(keys, kind="stable")
        lst = [lst[i] for i in order]
        # receive blocks in a random order with gaps
        place = rng.permutation(len(lst))
        pos = 0
        disp = [0] * len(lst)
        for i in place:
            pos += int(rng.integers(0, 3)) if gaps else 0
            disp[i] = pos
            pos += lst[i][1]
        recv_slots[d] = pos + (int(rng.integers(0, 3)) if gaps else 0)
        g = np.full(recv_slots[d], -1, np.int64)
        for (r, c, eid), dp in zip(lst, disp):
            in_dst.append(d); in_src.append(r); in_cnt.append(c); rdispls.append(dp)
            so = send_slot_ptr[r] + sdispls[eid]
            g[dp:dp + c] = gs[so:so + c]
        recv_g.append(g)
    recv_slot_ptr = _ptr_from_counts(recv_slots)
    recv_base = np.zeros(P, np.int64)
    off = int(rng.integers(0, 7)) * unit if gaps else 0
    for d in range(P):
        recv_base[d] = off
        off += int(recv_slots[d]) * s + (int(rng.integers(0, 7)) * unit if gaps else 0)
    recvbuf_bytes = off
    out_ptr = _ptr_from_counts(np.bincount(np.array(out_src, np.int64), minlength=P) if out_src
                               else np.zeros(P, np.int64)).astype(np.int32)
    in_ptr = _ptr_from_counts(np.bincount(np.array(in_dst, np.int64), minlength=P) if in_dst
                              else np.zeros(P, np.int64)).astype(np.int32)
    return Pattern(
        name=f"random{seed}_P{P}_ppn{ppn}_s{s}_{'idx' if indexed else 'packed'}", P=P, ppn=ppn,
        in_ptr=in_ptr, sources=np.asarray(in_src, np.int32), out_ptr=out_ptr,
        dests=np.asarray(out_dst, np.int32), sendcounts=np.asarray(out_cnt, np.int32),
        sdispls=np.asarray(sdispls, np.int32), recvcounts=np.asarray(in_cnt, np.int32),
        rdispls=np.asarray(rdispls, np.int32), elem_size=s, dtype=dtype,
        send_base=send_base, recv_base=recv_base, sendbuf_bytes=int(sendbuf_bytes),
        recvbuf_bytes=int(recvbuf_bytes), send_slot_ptr=send_slot_ptr,
        send_idx=send_elem.astype(np.int32) if indexed else None,
        recv_slot_ptr=recv_slot_ptr, global_sidx=gs.astype(np.int64),
        global_ridx=np.concatenate(recv_g) if recv_g else np.zeros(0, np.int64),
        meta=dict(kind="random", seed=seed))


def random_bytes(n: int, seed: int) -> np.ndarray:
    """Arbitrary payload bytes (includes NaN, -0.0 and denormal bit patterns)."""
    return np.random.default_rng(seed).integers(0, 256, size=n, dtype=np.uint8)


# ------------------------------------------------- device-side SpMV generator ---

def spmv_halo_torch(n: int, P: int, ppn: int, nnz: int, seed: int, dtype: str = "f64",
                    band: int = 4096, band_frac: float = 0.8, device="cuda", name=None) -> Pattern:
    """The spmv_halo recipe drawn with torch (on the GPU when device='cuda'), for the
    large uneven batch whose numpy generation would take minutes.  Same distributions and
    layout; a different random stream than the numpy version for the same seed."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    nb = int(round(band_frac * nnz))
    rows = torch.arange(n, device=device, dtype=torch.int64)
    lo = torch.clamp(rows - band, min=0)
    width = torch.clamp(rows + band, max=n - 1) - lo + 1
    assert int(width.min()) >= nb and n >= nnz

    def draw_band(r):
        u = torch.rand(r.shape, generator=g, device=device, dtype=torch.float64)
        return lo[r] + torch.minimum((u * width[r]).to(torch.int64), width[r] - 1)

    cols = torch.empty((n, nnz), dtype=torch.int64, device=device)
    rr = rows[:, None].expand(n, nb)
    cols[:, :nb] = draw_band(rr)
    cols[:, nb:] = torch.randint(0, n, (n, nnz - nb), generator=g, device=device)
    while True:
        srt, order = torch.sort(cols, dim=1, stable=True)
        dup_sorted = torch.zeros_like(srt, dtype=torch.bool)
        dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
        if not bool(dup_sorted.any()):
            break
        dup = torch.zeros_like(dup_sorted)
        dup.scatter_(1, order, dup_sorted)
        ri, ci = torch.nonzero(dup, as_tuple=True)
        isb = ci < nb
        cols[ri[isb], ci[isb]] = draw_band(ri[isb])
        cols[ri[~isb], ci[~isb]] = torch.randint(0, n, (int((~isb).sum()),), generator=g, device=device)
    rs = torch.from_numpy(row_starts(n, P)).to(device)
    row_owner = torch.searchsorted(rs, rows, right=True) - 1
    col_owner = torch.searchsorted(rs, cols, right=True) - 1
    off = col_owner != row_owner[:, None]
    keys = (row_owner[:, None].expand_as(cols)[off] * n + cols[off])
    keys = torch.unique(keys)                       # sorted by (receiver, column)
    rd = keys // n
    rcol = keys % n
    rq = torch.searchsorted(rs, rcol, right=True) - 1
    ek = rd * P + rq
    starts = torch.nonzero(torch.cat([torch.ones(1, dtype=torch.bool, device=device), ek[1:] != ek[:-1]])).flatten()
    ends = torch.cat([starts[1:], torch.tensor([len(ek)], device=device)])
    in_dst, in_src, in_cnt = rd[starts], rq[starts], ends - starts
    okey = (rq * P + rd) * n + rcol
    o = torch.argsort(okey)
    sq, sd, sc = rq[o], rd[o], rcol[o]
    ok2 = sq * P + sd
    ostarts = torch.nonzero(torch.cat([torch.ones(1, dtype=torch.bool, device=device), ok2[1:] != ok2[:-1]])).flatten()
    oends = torch.cat([ostarts[1:], torch.tensor([len(ok2)], device=device)])
    out_src, out_dst, out_cnt = sq[ostarts], sd[ostarts], oends - ostarts
    send_elem = sc - rs[sq]
    c = lambda t: t.cpu().numpy()
    esz = 8 if dtype == "f64" else 4
    meta = dict(kind="spmv", n=n, nnz=nnz, band=band, row_starts=c(rs), seed=seed, generator="torch")
    return _assemble(name or f"spmv_n{n}_P{P}_nnz{nnz}_{dtype}", P, ppn, c(out_src), c(out_dst), c(out_cnt),
                     c(send_elem), c(sc), c(in_dst), c(in_src), c(in_cnt), c(rcol), esz, dtype,
                     np.diff(c(rs)), meta)


def config3_torch(count=64, device="cuda"):
    """The uneven batch drawn on the device (see spmv_halo_torch)."""
    return [spmv_halo_torch(s["n"], s["P"], s["ppn"], s["nnz"], s["seed"], s["dtype"], device=device,
                            name=f"cfg3_{j}_n{s['n']}_P{s['P']}_{s['dtype']}")
            for j, s in enumerate(batched_specs(count, SEED + 3))]


# ------------------------------------------------- neighbourhood all-to-all-w ---

# Datatype table columns: a block of `blocklen` bytes repeated over three strided levels
# (innermost first), items `extent` bytes apart (an hvector nested up to three times and
# resized, lower bound 0).
TYPE_COLUMNS = ("blocklen", "count0", "count1", "count2", "stride0", "stride1", "stride2", "extent")


def contiguous_type(nbytes: int) -> list:
    """One item = `nbytes` contiguous bytes."""
    return [nbytes, 1, 1, 1, nbytes, nbytes, nbytes, nbytes]


@dataclasses.dataclass
class WPattern:
    """One neighbourhood all-to-all-w problem: per edge a count, a byte displacement and
    a datatype (an index into `types`), on both sides."""

    name: str
    P: int
    ppn: int
    in_ptr: np.ndarray          # int32 [P+1]
    sources: np.ndarray         # int32 [E]
    out_ptr: np.ndarray         # int32 [P+1]
    dests: np.ndarray           # int32 [E]
    sendcounts: np.ndarray      # int32 [E] items, aligned with dests
    sdispls: np.ndarray         # int64 [E] bytes from the rank's send region
    sendtypes: np.ndarray       # int32 [E] rows of `types`
    recvcounts: np.ndarray      # int32 [E] items, aligned with sources
    rdispls: np.ndarray         # int64 [E] bytes from the rank's receive region
    recvtypes: np.ndarray       # int32 [E]
    types: np.ndarray           # int64 [ntypes, 8], columns TYPE_COLUMNS
    send_base: np.ndarray       # int64 [P]
    recv_base: np.ndarray       # int64 [P]
    sendbuf_bytes: int
    recvbuf_bytes: int
    dtype: str                  # payload type for the backward: 'f64', 'f32' or 'bytes'
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.out_ptr[-1])

    def type_sizes(self) -> np.ndarray:
        t = self.types.astype(np.int64)
        return t[:, 0] * t[:, 1] * t[:, 2] * t[:, 3]

    def message_bytes(self) -> np.ndarray:
        """Bytes of every out-edge's message."""
        return self.sendcounts.astype(np.int64) * self.type_sizes()[self.sendtypes]

    def user_bytes(self) -> int:
        return 2 * int(self.message_bytes().sum())


def w_from_v(p: Pattern, name=None) -> WPattern:
    """The all-to-all-v problem `p` (packed send buffers, no send index list) written as
    an all-to-all-w with one contiguous element type: counts unchanged, displacements in
    bytes."""
    assert p.send_idx is None, "a send index list has no all-to-all-w equivalent here"
    s = int(p.elem_size)
    E = int(p.out_ptr[-1])
    return WPattern(
        name=name or p.name + "_w", P=p.P, ppn=p.ppn, in_ptr=p.in_ptr.copy(), sources=p.sources.copy(),
        out_ptr=p.out_ptr.copy(), dests=p.dests.copy(), sendcounts=p.sendcounts.copy(),
        sdispls=p.sdispls.astype(np.int64) * s, sendtypes=np.zeros(E, np.int32),
        recvcounts=p.recvcounts.copy(), rdispls=p.rdispls.astype(np.int64) * s,
        recvtypes=np.zeros(E, np.int32), types=np.array([contiguous_type(s)], np.int64),
        send_base=p.send_base.copy(), recv_base=p.recv_base.copy(), sendbuf_bytes=int(p.sendbuf_bytes),
        recvbuf_bytes=int(p.recvbuf_bytes), dtype=p.dtype)


def stencil_w(grid, ranks, ppn, comps=1, dtype="f64", neighbors="all", layout="soa", name=None) -> WPattern:
    """The stencil halo exchange of `stencil(...)` with each message described by a
    datatype over the rank's field block instead of a send index list.

    layout 'aos': point-major field (a point's `comps` values together), the layout of
    `stencil`; layout 'soa': component-major field (component c of all the rank's points,
    then component c+1).  Every message is the boundary box facing its direction, sent
    as z-planes (items) of y-rows (level 2) of x-runs (level 1) of the point's components
    (level 0 for 'soa'; the block itself for 'aos'), i.e. in ascending local point order
    with components innermost.  Receive side: the ghost points packed point-major, as in
    `stencil`.  With the same values the receive buffer equals `stencil`'s."""
    p = stencil(grid, ranks, ppn, comps=comps, dtype=dtype, neighbors=neighbors)
    D = len(grid)
    blk = [g // r for g, r in zip(grid, ranks)] + [1] * (3 - D)
    rk = list(ranks) + [1] * (3 - D)
    nx, ny, nz = blk
    npts = nx * ny * nz
    vb = 8 if dtype == "f64" else 4
    esz = comps * vb

    def coords(r):
        return (r % rk[0], (r // rk[0]) % rk[1], r // (rk[0] * rk[1]))

    E = p.n_edges
    owner = np.repeat(np.arange(p.P), np.diff(p.out_ptr))
    types, key_of = [contiguous_type(esz)], {}
    sendtypes = np.zeros(E, np.int32)
    sendcounts = np.zeros(E, np.int32)
    sdispls = np.zeros(E, np.int64)
    for e in range(E):
        r, d = int(owner[e]), int(p.dests[e])
        cr, cd = coords(r), coords(d)
        box = []
        for ax in range(3):
            dd = cd[ax] - cr[ax]
            n = blk[ax]
            box.append((0, 1) if dd == -1 else (n - 1, 1) if dd == 1 else (0, n))
        (x0, lx), (y0, ly), (z0, lz) = box
        p0 = x0 + nx * (y0 + ny * z0)
        if layout == "soa":
            t = [vb, comps, lx, ly, npts * vb, vb, nx * vb, nx * ny * vb]
            sdispls[e] = p0 * vb
        else:
            t = [esz, lx, ly, 1, esz, nx * esz, 0, nx * ny * esz]
            sdispls[e] = p0 * esz
        k = tuple(t)
        if k not in key_of:
            key_of[k] = len(types)
            types.append(t)
        sendtypes[e] = key_of[k]
        sendcounts[e] = lz
    return WPattern(
        name=name or f"stencil{D}d_{layout}_{'x'.join(map(str, grid))}_P{p.P}_c{comps}", P=p.P, ppn=p.ppn,
        in_ptr=p.in_ptr, sources=p.sources, out_ptr=p.out_ptr, dests=p.dests, sendcounts=sendcounts,
        sdispls=sdispls, sendtypes=sendtypes, recvcounts=p.recvcounts.copy(),
        rdispls=p.rdispls.astype(np.int64) * esz, recvtypes=np.zeros(E, np.int32),
        types=np.array(types, np.int64), send_base=p.send_base.copy(), recv_base=p.recv_base.copy(),
        sendbuf_bytes=int(p.sendbuf_bytes), recvbuf_bytes=int(p.recvbuf_bytes), dtype=dtype,
        meta={"v_pattern": p, "layout": layout, "block": tuple(blk[:D]), "comps": comps})


def soa_from_aos(field: np.ndarray, P: int, npts: int, comps: int) -> np.ndarray:
    """Component-major copy of a point-major field of P equal rank blocks."""
    return np.ascontiguousarray(field.reshape(P, npts, comps).transpose(0, 2, 1)).reshape(-1)


def _divisors(n):
    return [k for k in range(1, n + 1) if n % k == 0]


def _random_type(rng, k_el, es, overlap_ok):
    """A datatype of k_el elements of es bytes; returns (row, span of one item).  Without
    overlap_ok no byte appears twice in one item or across items."""
    bl = int(rng.choice(_divisors(k_el)))
    rest = k_el // bl
    c = []
    for _ in range(2):
        f = int(rng.choice(_divisors(rest)))
        c.append(f)
        rest //= f
    c.append(rest)
    rng.shuffle(c)
    # nesting by stride magnitude: a random level order, each level stepping over the
    # span of the ones inside it (plus a gap), so blocks never collide
    order = rng.permutation(3)
    stride = [0, 0, 0]
    span = bl * es
    for lv in order:
        st = span + int(rng.integers(0, 3)) * es
        if overlap_ok and rng.random() < 0.2:
            st = int(rng.integers(0, span + 1)) // es * es
        stride[lv] = st
        span = span + (c[lv] - 1) * st
    ext = span + int(rng.integers(0, 3)) * es
    if overlap_ok and rng.random() < 0.2:
        ext = int(rng.integers(0, span + 1)) // es * es
    return [bl * es, c[0], c[1], c[2], stride[0], stride[1], stride[2], ext], span


def random_wpattern(seed: int, P=None, dtype=None, es=None, max_deg=5, max_items=4, max_el=12) -> WPattern:
    """Random valid all-to-all-w for fuzzing: multigraph and self edges, empty messages,
    send and receive datatypes of different shapes (levels nested in random order, gaps,
    overlapping reads on the send side), receive messages in random order with gaps.
    For f32/f64 every offset is a multiple of the payload size."""
    rng = np.random.default_rng(seed)
    P = int(P if P is not None else rng.integers(1, 25))
    ppn = int(rng.choice([1, 2, 4, max(P, 1)]))
    dtype = dtype or str(rng.choice(["bytes", "f32", "f64"]))
    if es is None:
        es = int(rng.choice([1, 2, 3, 8])) if dtype == "bytes" else (4 if dtype == "f32" else 8) * int(rng.choice([1, 2]))
    outs = [[int(rng.integers(0, P)) for _ in range(int(rng.integers(0, max_deg + 1)))] for _ in range(P)]
    types = []
    out_src, out_dst, scount, stype, sdisp, n_el = [], [], [], [], [], []
    send_need = np.zeros(P, np.int64)
    for r in range(P):
        for d in outs[r]:
            n = int(rng.integers(0, max_items + 1)) * int(rng.integers(1, max_el + 1)) if rng.random() > 0.1 else 0
            k_s = int(rng.choice(_divisors(n))) if n > 0 else int(rng.integers(1, 4))
            row, span = _random_type(rng, k_s, es, overlap_ok=True)
            ns = n // k_s if n > 0 else 0
            types.append(row)
            disp = int(rng.integers(0, 6)) * es
            out_src.append(r); out_dst.append(d); scount.append(ns); stype.append(len(types) - 1)
            sdisp.append(disp); n_el.append(n)
            if ns > 0:
                send_need[r] = max(send_need[r], disp + (ns - 1) * row[7] + span)
    E = len(out_src)
    send_base = np.zeros(P, np.int64)
    off = int(rng.integers(0, 3)) * es
    for r in range(P):
        send_base[r] = off
        off += int(send_need[r]) + int(rng.integers(0, 3)) * es
    sendbuf_bytes = off
    # in-lists: shuffled, each sender's listings in their order
    ins = [[] for _ in range(P)]
    for e in range(E):
        ins[out_dst[e]].append(e)
    in_src, rcount, rtype, rdisp, recv_size = [], [], [], [], np.zeros(P, np.int64)
    for d in range(P):
        lst = ins[d]
        keys = rng.random(len(lst))
        by_sender = {}
        for i, e in enumerate(lst):
            by_sender.setdefault(out_src[e], []).append(i)
        for idxs in by_sender.values():
            keys[idxs] = np.sort(keys[idxs])
        lst = [lst[i] for i in np.argsort(keys, kind="stable")]
        rows = []
        for e in lst:
            n = n_el[e]
            k_r = int(rng.choice(_divisors(n))) if n > 0 else int(rng.integers(1, 4))
            row, span = _random_type(rng, k_r, es, overlap_ok=False)
            nr = n // k_r if n > 0 else 0
            types.append(row)
            rows.append((e, nr, len(types) - 1, (nr - 1) * row[7] + span if nr > 0 else 0))
        place = rng.permutation(len(rows))
        pos = 0
        disp = [0] * len(rows)
        for i in place:
            pos += int(rng.integers(0, 3)) * es
            disp[i] = pos
            pos += rows[i][3]
        recv_size[d] = pos + int(rng.integers(0, 3)) * es
        for (e, nr, t, _), dp in zip(rows, disp):
            in_src.append(out_src[e]); rcount.append(nr); rtype.append(t); rdisp.append(dp)
    recv_base = np.zeros(P, np.int64)
    off = int(rng.integers(0, 3)) * es
    for d in range(P):
        recv_base[d] = off
        off += int(recv_size[d]) + int(rng.integers(0, 3)) * es
    in_cnt = np.bincount(np.array([out_dst[e] for d in range(P) for e in ins[d]], np.int64), minlength=P) \
        if E else np.zeros(P, np.int64)
    out_cnt = np.bincount(np.array(out_src, np.int64), minlength=P) if E else np.zeros(P, np.int64)
    types.append(contiguous_type(es))     # an unused row
    return WPattern(
        name=f"randw{seed}_P{P}_{dtype}_es{es}", P=P, ppn=ppn,
        in_ptr=_ptr_from_counts(in_cnt).astype(np.int32), sources=np.array(in_src, np.int32),
        out_ptr=_ptr_from_counts(out_cnt).astype(np.int32), dests=np.array(out_dst, np.int32),
        sendcounts=np.array(scount, np.int32), sdispls=np.array(sdisp, np.int64),
        sendtypes=np.array(stype, np.int32), recvcounts=np.array(rcount, np.int32),
        rdispls=np.array(rdisp, np.int64), recvtypes=np.array(rtype, np.int32), types=np.array(types, np.int64),
        send_base=send_base, recv_base=recv_base, sendbuf_bytes=int(sendbuf_bytes), recvbuf_bytes=int(off),
        dtype=dtype)
