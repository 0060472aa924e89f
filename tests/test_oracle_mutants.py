"""Pin strength: every plausible mistake planted in a copy of the oracle's source must
make at least one pin in tests/pins.py fail.  The mutants are built from temporary
copies of oracle/oracle.c (the committed oracle is never modified) and run in child
processes, on the CPU."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, text in oracle.c, replacement); the first occurrence is replaced
MUTANTS = [
    ("match_ignores_occurrence", "int64_t want = a + t;", "int64_t want = a;"),
    ("recv_uses_send_displacement",
     "int64_t dst = pt->recv_base[d] + (pt->rdispls[i] + k) * s;",
     "int64_t dst = pt->recv_base[d] + (pt->sdispls[e] + k) * s;"),
    ("send_index_list_ignored",
     "if (pt->send_idx) return pt->send_idx[pt->send_slot_ptr[r] + q];", "if (0) return 0;"),
    ("step3_reads_wrong_slot", "R + L.pos_of_t[x->t] * s", "R + x->t * s"),
    ("sign_error_f64_add", "z = x + y;", "z = x - y;"),
    ("backward_wrong_rank_offset", "t[n].val = grad_recv + pt->recv_base[d] + p * s;",
     "t[n].val = grad_recv + pt->recv_base[r] + p * s;"),
    ("backward_drops_terms", "add_elem(dtype, s, gacc, gacc, t[j].val);", "(void)0;"),
    ("send_leader_formula", "return a * pt->ppn + b % node_size(pt, a);",
     "return a * pt->ppn + a % node_size(pt, a);"),
    ("node_map_off_by_one", "static int node_of(const orc_pattern *pt, int r) { return r / pt->ppn; }",
     "static int node_of(const orc_pattern *pt, int r) { return (r + 1) / pt->ppn; }"),
    ("accumulate_overwrites", "if (accumulate) add_elem(dtype, s, out + row, out + row, racc);",
     "if (accumulate) memcpy(out + row, racc, (size_t)s);"),
    ("node_blocked_groups_lost", "t1[n].group = L.u[q].b;", "t1[n].group = 0;"),
    ("overlap_unchecked", "if (rr[x].lo < rr[x - 1].hi)", "if (0)"),
    ("count_mismatch_unchecked", "if (pt->recvcounts[i] != cnt || cnt < 0)", "if (cnt < 0)"),
    ("w_level_strides_swapped", "c1 * t->stride[1] + c0 * t->stride[0] + off",
     "c1 * t->stride[0] + c0 * t->stride[1] + off"),
    ("w_extent_ignored", "return item * t->extent + c2", "return item * type_size(t) + c2"),
    ("w_level_digits_reversed",
     "int64_t c0 = blk % t->count[0];\n    blk /= t->count[0];\n    int64_t c1 = blk % t->count[1];\n"
     "    int64_t c2 = blk / t->count[1];",
     "int64_t c2 = blk % t->count[2];\n    blk /= t->count[2];\n    int64_t c1 = blk % t->count[1];\n"
     "    int64_t c0 = blk / t->count[1];"),
    ("w_recv_through_send_type", "recvbuf[wp->recv_base[d] + wp->rdispls[i] + type_byte(Tr, b)] =",
     "recvbuf[wp->recv_base[d] + wp->rdispls[i] + type_byte(Ts, b)] ="),
    ("w_overlap_unchecked", "if (seen[da]) { err = ORC_ERR_OVERLAP; break; }", "if (0) { err = ORC_ERR_OVERLAP; break; }"),
    ("w_length_unchecked", "n != (int64_t)wp->recvcounts[i] * type_size(Tr)", "0"),
    ("w_backward_wrong_base", "t[n].val = grad_recv + da;", "t[n].val = grad_recv + (da - wp->recv_base[d]);"),
    ("values_named_by_send_slot", "pt->global_sidx[pt->send_slot_ptr[r] + q] : x->src_off;",
     "pt->global_sidx[pt->send_slot_ptr[r] + q] : q;"),
    ("partition_by_receive_offset", "sp[n] = part_of(npart, part_ptr, src, s);",
     "sp[n] = part_of(npart, part_ptr, dst < pt->sendbuf_bytes ? dst : 0, s);"),
    ("partition_straddle_accepted", "return off + s <= ptr[p + 1] ? p : -1;", "return p;"),
    ("arrival_ignores_readiness", "if (!ready[sp[n]]) arrived[rp[n]] = 0;", "(void)0;"),
    ("collective_receives_at_out_position", "int64_t k = i - g->in_ptr[d];  /* position",
     "int64_t k = i - g->out_ptr[d];  /* position"),
    ("alltoall_sends_from_zero", "int64_t disp = mode == 0 ? j * (int64_t)count : 0;", "int64_t disp = 0;"),
    ("allgather_sends_from_position", "mode == 0 ? j * (int64_t)count : 0", "mode <= 1 ? j * (int64_t)count : 0"),
    ("allgatherv_fixed_count", "sendcounts[e] = mode == 2 ? rank_count[r] : count;", "sendcounts[e] = count;"),
    ("alltoall_overflow_unchecked", "if (disp > INT32_MAX) err = ORC_ERR_UNSUPPORTED;\n            sendcounts",
     "if (0) err = ORC_ERR_UNSUPPORTED;\n            sendcounts"),
    ("dense_graph_reversed", "ranks[(int64_t)r * P + d] = d;", "ranks[(int64_t)r * P + d] = P - 1 - d;"),
    ("dedup_by_gidx_only", "if (p->a != q->a) return p->a < q->a ? -1 : 1;\n    if (p->b != q->b) return p->b < q->b ? -1 : 1;\n    if (p->gidx",
     "if (0) return 0;\n    if (0) return 0;\n    if (p->gidx"),
]

RUNNER = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, pins
lib = oracle.load({lib!r})
for check in pins.ALL_CHECKS:
    try:
        check(lib)
    except Exception as e:
        print("caught by", check.__name__, type(e).__name__)
        sys.exit(1)
print("survived")
sys.exit(0)
"""


def _build_and_run(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    so = os.path.join(tmp, f"lib{name}.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-w",
                    "-o", so, path], check=True)
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=so)
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                            stderr=subprocess.STDOUT, text=True)


def test_every_mutant_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        procs = [(m[0], _build_and_run(*m, tmp)) for m in MUTANTS]
        survivors = []
        for name, p in procs:
            out, _ = p.communicate(timeout=600)
            if p.returncode == 0:
                survivors.append(name)
        assert not survivors, f"mutants not caught by any pin: {survivors}"
