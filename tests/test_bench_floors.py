"""CPU: the benchmark's 128-byte-line floors.  The locality form's aggregate count and direct
count agree with the oracle's locality statistics (distinct (sender node, receiver node,
global index) triples), and the standard, locality and backward floors agree with a
brute-force count of the lines on small patterns."""
import numpy as np
import pytest

import bench
import oracle
from paper_2309_07337_gb300 import patterns as pt


def _elements(p):
    """(sender, receiver, byte offset in the send buffer, global index) of every element, by
    plain loops over the edges."""
    out = []
    for r in range(p.P):
        for e in range(p.out_ptr[r], p.out_ptr[r + 1]):
            for k in range(int(p.sendcounts[e])):
                slot = int(p.sdispls[e]) + k
                sp = int(p.send_slot_ptr[r]) + slot if p.send_slot_ptr is not None else None
                el = slot if p.send_idx is None else int(p.send_idx[sp])
                g = int(p.global_sidx[sp]) if sp is not None and p.global_sidx is not None else None
                out.append((r, int(p.dests[e]), int(p.send_base[r]) + el * p.elem_size, g))
    return out


def _lines(offsets, s):
    return {o >> 7 for o in offsets} | {(o + s - 1) >> 7 for o in offsets}


PATTERNS = [pt.config1(), pt.config5(edge=4, R=4, ppn=8, comps=2)] + \
           [pt.random_pattern(700 + i, indexed=True) for i in range(6)]


@pytest.mark.parametrize("p", PATTERNS, ids=lambda p: p.name)
def test_standard_line_floor_brute_force(p):
    els = _elements(p)
    s = p.elem_size
    got = bench.line_floor(p)
    assert got["read_lines_bytes"] == 128 * len(_lines([o for _, _, o, _ in els], s))
    assert got["index_bytes"] == 4 * len(els) and got["write_bytes"] == s * len(els)


@pytest.mark.parametrize("p", PATTERNS, ids=lambda p: p.name)
def test_locality_line_floor_matches_oracle_and_brute_force(p):
    got = bench.locality_line_floor(p)
    st = oracle.locality_stats(p)
    assert got["U"] == st["U"] and got["V_direct"] == st["V_direct"]
    s = p.elem_size
    els = _elements(p)
    seen, inter_offs = set(), []
    for r, d, o, g in els:
        if r // p.ppn != d // p.ppn and (r // p.ppn, d // p.ppn, g) not in seen:
            seen.add((r // p.ppn, d // p.ppn, g))
            inter_offs.append(o)
    direct_offs = [o for r, d, o, _ in els if r // p.ppn == d // p.ppn]
    U, V = len(seen), len(els)
    assert got["step1"] == 128 * len(_lines(inter_offs, s)) + 4 * U + s * U
    assert got["step2"] == 2 * s * U
    assert got["step3"] == 128 * len(_lines(direct_offs, s)) + s * U + 4 * V + s * V
    assert got["total"] == got["step1"] + got["step2"] + got["step3"]


def _elements_with_receive(p):
    """(byte offset of the source element, byte offset of its receive slot) of every element,
    pairing the t-th listing of d by r with the t-th listing of r by d (plain loops)."""
    s = p.elem_size
    inl = {}   # (r, d) -> in-edge indices of d listing r, in list order
    for d in range(p.P):
        for j in range(p.in_ptr[d], p.in_ptr[d + 1]):
            inl.setdefault((int(p.sources[j]), d), []).append(j)
    seen = {}
    out = []
    for r in range(p.P):
        for e in range(p.out_ptr[r], p.out_ptr[r + 1]):
            d = int(p.dests[e])
            t = seen.get((r, d), 0)
            seen[(r, d)] = t + 1
            j = inl[(r, d)][t]
            for k in range(int(p.sendcounts[e])):
                slot = int(p.sdispls[e]) + k
                el = slot if p.send_idx is None else int(p.send_idx[int(p.send_slot_ptr[r]) + slot])
                out.append((int(p.send_base[r]) + el * s, int(p.recv_base[d]) + (int(p.rdispls[j]) + k) * s))
    return out


@pytest.mark.parametrize("p", PATTERNS, ids=lambda p: p.name)
def test_backward_line_floor_brute_force(p):
    s = p.elem_size
    els = _elements_with_receive(p)
    reads = {}
    for src, dst in els:
        reads.setdefault(src, []).append(dst)
    single = {src for src, d in reads.items() if len(d) == 1}
    V, rows = len(els), len(reads)
    algo = V * s + rows * s + 1000   # the program's index bytes: 1000 here
    got = bench.bwd_line_floor(p, {"algo_bytes": algo})
    one, two = got["one_pass"], got["two_pass"]
    assert one["rows"] == rows and one["index_bytes"] == 1000 == two["index_bytes"]
    assert one["read_bytes"] == 128 * len(_lines([d for _, d in els], s))
    assert one["write_lines_bytes"] == 128 * len(_lines(list(reads), s))
    assert two["read_bytes"] == 128 * (len(_lines([d for x, d in els if x in single], s)) +
                                       len(_lines([d for x, d in els if x not in single], s)))
    assert two["write_lines_bytes"] == 128 * (len(_lines(list(single), s)) +
                                              len(_lines([x for x in reads if x not in single], s)))
