#!/usr/bin/env python
"""Benchmark of the persistent neighbourhood all-to-all-v on one GB300.

Workload (default): the 3D 27-point stencil halo exchange of a 512^3 grid split over
P = 4096 emulated ranks (16^3 blocks of 32^3 points, 64 ranks per node), 8 fp64
components per point (64-byte elements, U(-1,1) from a seed); V = 25,002,360 elements
per exchange from an 8.59 GB field.  Inputs are larger than L2, so no flush is needed.

One step = one start + wait of each of the three persistent requests of that pattern:
  * the standard exchange        (pack by send list + block copy + unpack, one kernel),
  * the locality-aware exchange  (direct + gather, node-pair block copy, redistribute),
  * the backward exchange        (reverse of the standard one, fixed-order sums).
value = (user-visible bytes of the three exchanges) / step time, where a forward moves
2*V*s user bytes and the backward reads V*s and writes rows*s.

End to end (`e2e`): the same step with every buffer in pinned host memory, bound to the
three requests, so the kernels read and write it in place over the host link; `e2e_staged`:
the step through gbx_start_host_async on device-bound requests (whole buffers copied up and
back, two buffer sets overlapping one step's uploads with the previous step's downloads).

Also reported (extras, on by default): per-form GB/s and roofline fractions, the fused
forward+backward vs plain (one launch and one host wait per exchange) factor, the
batched uneven-patterns (config 3: 64 SpMV halos, mixed fp32/fp64) vs plain factor, and
the SpMV halo (config 2) standard vs locality rates.

--impl reference times the CPU oracle (the only reference this build has) on the host's
cores: each step runs the three exchanges of the whole workload, the receivers split over one
oracle process per core.  The default run reports the oracle single-threaded and on all cores
as cpu_baseline.

Two other modes print their own JSON line instead of the step's:
  --sweep  message-size sweep of the stencil at P = 4096: block edge 8/16/32 points x 1..16
           fp64 per point, standard and locality forms, cold L2;
  --faces  the standard exchange per direction class (x, y, z faces; edges and corners) of
           the 512^3 stencil, with each class's 128-byte-line DRAM floor;
  --bwd-forms  the 512^3 backward (standard and locality order) in every program shape the
           library offers (tuned default, bulk forms off, scatter form forced, single-term
           rows folded, destination-ordered pairs), each checked bit for bit against the
           default.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2309_07337_gb300 import patterns as pt  # noqa: E402

METRIC = "neighbor_alltoallv effective GB/s (standard + locality-aware forward + backward per step)"
NOMINAL_HBM_GBPS = 8000.0   # GB300 HBM3e, nominal (~8 TB/s); the roofline uses the measured copy rate
UNIT = "GB/s"


def parse_args():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=100)
    a.add_argument("--warmup", type=int, default=5)
    a.add_argument("--impl", default="ours", choices=["ours", "reference"])
    a.add_argument("--e2e-steps", type=int, default=8)
    a.add_argument("--cpu-sample-ranks", type=int, default=4096,
                   help="receivers in the CPU-oracle baseline sample (4096 = the whole exchange)")
    a.add_argument("--no-extras", action="store_true")
    a.add_argument("--no-e2e", action="store_true")
    a.add_argument("--no-cpu", action="store_true")
    a.add_argument("--edge", type=int, default=32, help="block edge (32 = the 512^3 workload)")
    a.add_argument("--ranks", type=int, default=16, help="ranks per dimension (16 = the workload; 8 keeps the "
                                                         "32^3 blocks of the 512^3 case on a 256^3 grid, for "
                                                         "counter captures of a few GB)")
    a.add_argument("--sweep", action="store_true",
                   help="instead of the step: message-size sweep, comps 1..16 x block edge 8..32 at P=4096")
    a.add_argument("--bwd-forms", action="store_true",
                   help="time the backward in each program shape (own JSON line)")
    a.add_argument("--spmv", action="store_true",
                   help="instead of the step: the SpMV halo exchange (2^20 rows, P=1024) standard vs locality")
    a.add_argument("--batched", action="store_true",
                   help="instead of the step: the uneven 64-pattern batch, plain vs startall")
    a.add_argument("--reps", type=int, default=20, help="repetitions of the --spmv / --batched timings")
    a.add_argument("--count", type=int, default=64, help="patterns of the --batched batch (64 = the workload)")
    a.add_argument("--info", default="", help="extra info keys for the timed requests (e.g. form=10 to pin a "
                                             "copy form for a profiler run)")
    a.add_argument("--faces", action="store_true",
                   help="instead of the step: standard exchange per face / edge+corner subset of the 512^3 "
                        "stencil, with the 128-byte-line DRAM floor of each")
    return a.parse_args()


# ------------------------------------------------------------------- helpers
def workload(edge=32, ranks=16):
    p = pt.config5(edge=edge, R=ranks)
    return p


def workload_config(p, edge, world=1, ranks=16):
    """The workload's description, the same dict in both arms."""
    g = ranks * edge
    full = edge == 32 and ranks == 16
    return {"workload": f"stencil3d_27pt_{g}^3_P{ranks ** 3}_ppn64_8xf64",
            "grid": [g] * 3, "ranks": ranks ** 3, "ranks_per_node": 64, "elem_bytes": p.elem_size,
            "V": p.volume, "E": p.n_edges, "l2": "inputs larger than L2 (8.59 GB field), no flush"
            if full else "reduced size", "seed": pt.SEED + 5,
            "parallelism": "replicas" if world > 1 else "single"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("gbx_move.cu", "gbx_device.cuh"):
        with open(os.path.join(ROOT, "paper_2309_07337_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            d = json.load(f)
        e = d[kernel_key]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples during the timed region (read-only queries)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def ready(self, timeout_s=3.0):
        """Waits (at most timeout_s) until nvidia-smi has written its first sample, so that
        the samples cover the region timed next rather than the tool's start-up."""
        if self.p is None:
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < timeout_s:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
                power.append(float(c[3]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------ multi-rank glue
def max_over_ranks(ms_local, dist=None, device="cpu"):
    """The slowest rank's time (the job's time); identity without a process group."""
    if dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def all_ranks_agree(flag, dist=None, device="cpu"):
    """True only if `flag` holds on every rank (so all ranks take the same branch)."""
    if dist is None:
        return bool(flag)
    import torch
    t = torch.tensor([1.0 if flag else 0.0], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return t.item() > 0.5


def host_mem_available():
    """MemAvailable of this host in bytes (0 when unknown)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def whole_job_rate(bytes_per_rank_step, world, ms):
    """Aggregate GB/s of `world` replicas that each move bytes_per_rank_step per step."""
    return bytes_per_rank_step * world / (ms * 1e-3) / 1e9


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(p, x_bytes, grad_bytes, nrecv):
    """The oracle's three exchanges restricted to receivers 0..nrecv-1 (same buffers).
    Returns (seconds, user bytes)."""
    import oracle
    q = pt.restrict_to_receivers(p, np.arange(nrecv))
    t0 = time.perf_counter()
    oracle.standard(q, x_bytes)
    _, st = oracle.locality(q, x_bytes)
    g = oracle.backward(q, grad_bytes, form=0)
    dt = time.perf_counter() - t0
    V = q.volume
    rows = distinct_sources(q)
    del g, st
    user = 2 * 2 * V * q.elem_size + V * q.elem_size + rows * q.elem_size
    return dt, user, V


def distinct_sources(q):
    """Number of distinct source elements the pattern reads (rows of its backward)."""
    owner = np.repeat(np.arange(q.P), np.diff(q.out_ptr))
    cnt = q.sendcounts.astype(np.int64)
    slot = np.repeat(q.send_slot_ptr[owner] + q.sdispls, cnt) + \
        (np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt))
    el = q.send_idx[slot] if q.send_idx is not None else slot - np.repeat(q.send_slot_ptr[owner], cnt)
    off = np.repeat(q.send_base[owner], cnt) + el.astype(np.int64) * q.elem_size
    return int(len(sorted_unique(off)))


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle on the host's cores: each step runs the three exchanges of the whole
    workload, its receivers split over one oracle process per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload(args.edge, args.ranks)
    x = pt.stencil_field(p, pt.SEED + 5)
    g = np.random.default_rng(pt.SEED + 6).standard_normal(p.recvbuf_bytes // 8)
    pool = CpuPool(p, x, g, max(1, len(os.sched_getaffinity(0))))
    for _ in range(args.warmup):
        pool.run()
    ts = []
    n = 1
    for _ in range(args.steps):
        dt, n = pool.run()
        ts.append(dt)
    pool.close()
    t = sum(ts) / len(ts)
    V, s = p.volume, p.elem_size
    ub = 2 * 2 * V * s + V * s + distinct_sources(p) * s
    val = ub / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(p, args.edge, int(os.environ.get("WORLD_SIZE", "1")), args.ranks),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": f"the three exchanges over all {p.P} receivers each step, split into {n} "
                                       f"receiver slices, one oracle process per core"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------- ours
def _cpu_worker(conn, p, x, g, lo, hi):
    """One oracle process of the all-cores CPU baseline: the three exchanges into receivers
    lo..hi-1, once per "go" from the parent (which gets the seconds back), until "stop"."""
    import oracle
    q = pt.restrict_to_receivers(p, np.arange(lo, hi))
    conn.send("ready")
    while conn.recv() == "go":
        t0 = time.perf_counter()
        oracle.standard(q, x)
        oracle.locality(q, x)
        oracle.backward(q, g, form=0)
        conn.send(time.perf_counter() - t0)


class CpuPool:
    """The oracle, unchanged, on every host core: one process per core, each owning a slice of
    the receivers.  The processes are forked before this process makes its first CUDA call
    (and never touch the GPU), so they share the pattern and the field copy-on-write."""

    def __init__(self, p, x, g, n):
        import multiprocessing as mp
        import oracle  # noqa: F401  (loaded before the fork)
        ctx = mp.get_context("fork")
        bounds = np.linspace(0, p.P, n + 1).astype(int)
        self.conns, self.procs = [], []
        for k in range(n):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_cpu_worker, args=(b, p, x, g, int(bounds[k]), int(bounds[k + 1])), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)

        self.ready = False

    def run(self):
        """Seconds for one pass of every process over its slice, started together."""
        if not self.ready:
            for c in self.conns:
                c.recv()
            self.ready = True
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("go")
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0, len(self.procs)

    def close(self):
        for c in self.conns:
            c.send("stop")
        for pr in self.procs:
            pr.join()


def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    p = workload(args.edge, args.ranks)
    x = pt.stencil_field(p, pt.SEED + 5)                          # host fp64
    g_cpu = np.random.default_rng(pt.SEED + 6).standard_normal(p.recvbuf_bytes // 8)
    cpu_pool = None
    if rank == 0 and not args.no_cpu:   # before any CUDA call
        cpu_pool = CpuPool(p, x, g_cpu, max(1, len(os.sched_getaffinity(0))))

    import torch
    import paper_2309_07337_gb300 as gbx
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    s = p.elem_size
    field = torch.from_numpy(x).cuda()
    halo_std = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    halo_loc = torch.zeros_like(halo_std)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 6)
    grad_halo = torch.randn(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    grad_field = torch.zeros_like(field)
    dp = gbx.DevicePattern(p)
    # set-up, timed by part: the graph (edge matching), then each request (device maps and
    # descriptors, program validation, autotuning, graph capture)
    tb = [time.perf_counter()]
    graph = gbx.DistGraph(gbx.Comm(p.P, p.ppn), dp.in_ptr, dp.sources, dp.out_ptr, dp.dests)
    torch.cuda.synchronize()
    tb.append(time.perf_counter())
    ex_std = gbx.Exchange(p, field, halo_std, "standard", dp=dp, graph=graph, info=args.info)
    tb.append(time.perf_counter())
    ex_loc = gbx.Exchange(p, field, halo_loc, "locality", dp=dp, graph=graph, info=args.info)
    tb.append(time.perf_counter())
    bwd = gbx.backward_init(ex_std.request, grad_halo, grad_field, info=args.info)
    torch.cuda.synchronize()
    tb.append(time.perf_counter())
    t_init = tb[-1] - tb[0]
    init_parts = {k: tb[i + 1] - tb[i] for i, k in enumerate(("graph", "standard", "locality", "backward"))}
    reqs = [ex_std.request, ex_loc.request, bwd]
    infos = [r.info() for r in reqs]

    def step(ev=None):
        for i, r in enumerate(reqs):
            if ev is not None:
                ev[i].record()
            r.start()
        if ev is not None:
            ev[3].record()
        for r in reqs:
            r.wait()

    for _ in range(args.warmup):
        step()
    # the two forms must agree byte for byte
    assert torch.equal(halo_std.view(torch.uint8), halo_loc.view(torch.uint8)), "standard != locality"

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    clocks = Clocks(local)
    clocks.ready()
    barrier()
    torch.cuda.nvtx.range_push("timed")
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(K):
        step(evs[k])
    t1.record()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    per = [sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K)) / K for i in range(3)]
    ms = max_over_ranks(total_ms / K, dist, device="cuda")

    V = p.volume
    rows = infos[2]["rows"]
    user = [2 * V * s, 2 * V * s, V * s + rows * s]
    step_user = sum(user)
    value = whole_job_rate(step_user, world, ms)
    peak, peak_kind = measured_peaks()
    forms = {}
    for name, info, u, t in zip(("standard", "locality", "backward"), infos, user, per):
        forms[name] = {"ms": t, "user_GBps": u / (t * 1e-3) / 1e9,
                       "algo_bytes": info["algo_bytes"], "algo_GBps": info["algo_bytes"] / (t * 1e-3) / 1e9,
                       "frac_of_measured_hbm": info["algo_bytes"] / (t * 1e-3) / 1e9 / peak,
                       "frac_of_nominal_hbm": info["algo_bytes"] / (t * 1e-3) / 1e9 / NOMINAL_HBM_GBPS,
                       "launches": info["launches"], "vec": info["vec_bytes"], "block": info["block"]}
    forms["locality"].update({"U": infos[1]["U"], "node_pairs": infos[1]["node_pairs"],
                              "V_direct": infos[1]["V_direct"], "V_inter": infos[1]["V_inter"]})
    forms["backward"].update({"rows": rows, "terms": infos[2]["terms"]})
    lfl = locality_line_floor(p)
    if lfl is not None:
        forms["locality"].update({"line_floor_bytes": lfl["total"], "line_floor": lfl,
                                  "frac_of_line_floor": lfl["total"] / (per[1] * 1e-3) / 1e9 / peak})
    bfl = bwd_line_floor(p, infos[2])
    forms["backward"].update({"line_floor_bytes": bfl["total"], "line_floor": bfl,
                              "frac_of_line_floor": bfl["total"] / (per[2] * 1e-3) / 1e9 / peak,
                              "frac_of_two_pass_floor": bfl["total_two_pass"] / (per[2] * 1e-3) / 1e9 / peak})
    for name, info in zip(("standard", "locality", "backward"), infos):
        forms[name]["copy_forms"] = form_names(info)
    # dominant kernel: the standard exchange's single move kernel
    std_ms = per[0]
    achieved = infos[0]["algo_bytes"] / (std_ms * 1e-3) / 1e9
    fl = line_floor(p)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                # the committed counters are for the 512^3 launch: other workloads report none
                "traffic": profiled_traffic("gbx_copy_kernel_std_stencil512")
                if (args.edge, args.ranks) == (32, 16) else None,
                "kernel": f"the standard exchange's move kernel ({form_names(infos[0])}, one launch per start)",
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "line_floor_bytes": fl["total"], "frac_of_line_floor": fl["total"] / (std_ms * 1e-3) / 1e9 / peak,
                "traffic_note": "DRAM traffic above the algorithmic bytes is the 128-byte-line floor of the x-face "
                                "points (isolated 64-byte elements 2 KB apart, each fetched as a whole line): "
                                "line_floor_bytes counts the lines the exchange must touch"}
    launches = sum(i["launches"] for i in infos) * K

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(p, args.edge, world, args.ranks),
            "roofline": roofline, "gpu_launches": launches, "clocks": clk, "forms": forms,
            "init_s": t_init, "init_parts_s": init_parts}

    # ---------------------------------------------------------------- e2e
    # Steps end to end with the data on the host, through the library's C ABI, two ways.
    # (1) `e2e`: the three persistent requests are bound to pinned host buffers (the field,
    # both halos, the incoming halo gradient and the field gradient); the kernels read and
    # write them in place over the host link, so only the bytes the exchange touches cross
    # it.  (2) `e2e_staged`: requests bound to device buffers, driven by
    # gbx_start_host_async, which uploads the whole field and gradient and reads whole halos
    # and field gradient back (two device buffer sets, so a step's uploads overlap the
    # previous step's downloads).
    # Every rank on this host pins its own host buffers (22 GB at 512^3): the replicas of a
    # multi-GPU run measure end to end only where the host has room for all of them.
    local_world = int(os.environ.get("LOCAL_WORLD_SIZE", world))
    pinned_need = 2 * (p.sendbuf_bytes + 2 * p.recvbuf_bytes) * local_world
    e2e_fits = True
    if not args.no_e2e:
        barrier()
        e2e_fits = all_ranks_agree(host_mem_available() > 1.15 * pinned_need, dist, device="cuda")
        if not e2e_fits:
            line["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                           "skipped": f"the {local_world} replicas on this host need {pinned_need / 1e9:.0f} GB "
                                      f"of pinned host memory; {host_mem_available() / 1e9:.0f} GB available"}
    if not args.no_e2e and e2e_fits:
        hx = torch.empty(p.sendbuf_bytes, dtype=torch.uint8).pin_memory()
        hx.copy_(torch.from_numpy(x.view(np.uint8)))
        hg = torch.empty(p.recvbuf_bytes, dtype=torch.uint8).pin_memory()
        hg.copy_(grad_halo.view(torch.uint8).cpu())
        hres = [torch.zeros(p.recvbuf_bytes, dtype=torch.uint8).pin_memory(),
                torch.zeros(p.recvbuf_bytes, dtype=torch.uint8).pin_memory(),
                torch.zeros(p.sendbuf_bytes, dtype=torch.uint8).pin_memory()]
        eh_std = gbx.Exchange(p, hx, hres[0], "standard", dp=dp, graph=ex_std.graph)
        eh_loc = gbx.Exchange(p, hx, hres[1], "locality", dp=dp, graph=ex_std.graph)
        hreqs = [eh_std.request, eh_loc.request, gbx.backward_init(eh_std.request, hg, hres[2])]

        def host_step():
            for r in hreqs:
                r.start()
            for r in hreqs:
                r.wait()

        for _ in range(2):
            host_step()
        torch.cuda.synchronize()
        barrier()
        e0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            host_step()
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks((time.perf_counter() - e0) / args.e2e_steps * 1e3, dist, device="cuda")
        hi = [r.info() for r in hreqs]
        line["e2e"] = {"value": whole_job_rate(step_user, world, e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": s * (hi[0]["V"] + hi[1]["V_direct"] + hi[1]["U"] + hi[2]["terms"]),
                       "d2h_bytes_per_step": s * (hi[0]["V"] + hi[1]["V"] + hi[2]["rows"]),
                       "ms_per_step": e_ms, "steps": args.e2e_steps,
                       "api": "the three persistent requests bound to pinned host buffers (field, halos, "
                              "gradients); per step gbx_start + gbx_wait on each; the kernels read the field and "
                              "gradient and write the halos and field gradient in place over the host link"}
        assert torch.equal(hres[0], halo_std.view(torch.uint8).cpu()), "host-resident standard halo differs"
        assert torch.equal(hres[1], hres[0]), "host-resident locality halo differs"
        assert torch.equal(hres[2], grad_field.view(torch.uint8).cpu()), "host-resident field gradient differs"
        del eh_std, eh_loc, hreqs, hres

        # the staged comparison holds two more device buffer sets and 23.6 GB of pinned host
        # memory per rank, so replicas (N > 1) leave it out
        if world == 1:
            side = torch.cuda.Stream()           # completes the requests without ordering their stream
            sets = []
            for k in range(2):
                S = {"field": field if k == 0 else torch.empty_like(field),
                     "hs": halo_std if k == 0 else torch.empty_like(halo_std),
                     "hl": halo_loc if k == 0 else torch.empty_like(halo_loc),
                     "g": grad_halo if k == 0 else torch.empty_like(grad_halo),
                     "gf": grad_field if k == 0 else torch.empty_like(grad_field)}
                if k == 0:
                    S["reqs"] = reqs
                else:
                    a = gbx.Exchange(p, S["field"], S["hs"], "standard", dp=dp, graph=ex_std.graph)
                    b = gbx.Exchange(p, S["field"], S["hl"], "locality", dp=dp, graph=ex_std.graph)
                    S["keep"] = (a, b)
                    S["reqs"] = [a.request, b.request, gbx.backward_init(a.request, S["g"], S["gf"])]
                S["out"] = [torch.empty(p.recvbuf_bytes, dtype=torch.uint8).pin_memory(),
                            torch.empty(p.recvbuf_bytes, dtype=torch.uint8).pin_memory(),
                            torch.empty(p.sendbuf_bytes, dtype=torch.uint8).pin_memory()]
                sets.append(S)

            def staged_step(k):
                S = sets[k % 2]
                r_std, r_loc, r_bwd = S["reqs"]
                r_std.start_host_async(hx, S["out"][0])
                r_loc.start_host_async(None, S["out"][1])
                r_bwd.start_host_async(hg, S["out"][2])
                for r in (r_std, r_loc, r_bwd):
                    r.wait_stream(side)

            for k in range(2):
                staged_step(k)
            torch.cuda.synchronize()
            barrier()
            e0 = time.perf_counter()
            for k in range(args.e2e_steps):
                staged_step(k)
            torch.cuda.synchronize()
            barrier()
            e_ms = max_over_ranks((time.perf_counter() - e0) / args.e2e_steps * 1e3, dist, device="cuda")
            line["e2e_staged"] = {"value": whole_job_rate(step_user, world, e_ms), "unit": UNIT,
                                  "h2d_bytes_per_step": p.sendbuf_bytes + p.recvbuf_bytes,
                                  "d2h_bytes_per_step": 2 * p.recvbuf_bytes + p.sendbuf_bytes,
                                  "ms_per_step": e_ms, "steps": args.e2e_steps,
                                  "api": "gbx_start_host_async on device-bound requests: whole field + gradient "
                                         "uploaded, both halos + whole field gradient read back; two device buffer "
                                         "sets, so a step's uploads overlap the previous step's downloads"}
            for S in sets:
                assert torch.equal(S["out"][0], S["out"][1])
                assert torch.equal(S["out"][2].cuda(), sets[0]["gf"].view(torch.uint8))
            del sets
        del hx, hg

    # ---------------------------------------------------------- cpu baseline
    if rank == 0 and not args.no_cpu:
        dt, ub, Vs = oracle_sample(p, x, g_cpu, args.cpu_sample_ranks)
        line["cpu_baseline"] = {"value": ub / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "seconds": dt,
                                "sample": f"the three exchanges into receivers 0..{args.cpu_sample_ranks - 1} "
                                          f"of 4096 ({Vs} of {V} elements), full buffers, single thread"}
        if cpu_pool is not None:
            wall, n = cpu_pool.run()
            cpu_pool.close()
            line["cpu_baseline"]["all_cores"] = {
                "value": step_user / wall / 1e9, "unit": UNIT, "cores": n, "seconds": wall,
                "sample": f"the same three exchanges over all {p.P} receivers, split into {n} receiver slices, "
                          f"one oracle process per core"}

    # --------------------------------------------------------------- extras
    if not args.no_extras and rank == 0:
        line["extras"] = extras(gbx, torch, p, field, halo_std, grad_halo, grad_field, dp, ex_std, bwd)
    line["device_status"] = gbx.device_status()   # 0: no bounded wait of a move kernel gave up
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def paired(torch, fa, fb, reps=24, warm=3, flush=None):
    """Times two ways of doing the same work interleaved (a, b, a, b, ...), so that both see
    the same clocks and the same state: each repetition starts from an idle device (and a
    flushed L2 when `flush` is given) and is bracketed by CUDA events on the current stream,
    host waits included.  Returns the spread of a, of b and of the per-pair ratio a / b."""
    for _ in range(warm):
        fa()
        fb()
    ta, tb = [], []
    for _ in range(reps):
        for f, ts in ((fa, ta), (fb, tb)):
            if flush is not None:
                flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return spread(ta), spread(tb), spread([a / b for a, b in zip(ta, tb)])


def factor_entry(name_a, name_b, res):
    """JSON of a paired timing: both spreads and the factor a / b with its 10th-90th
    percentile band over the repetitions."""
    a, b, r = res
    return {f"{name_a}_ms": a, f"{name_b}_ms": b, "speedup": r["median"], "speedup_p10": r["p10"],
            "speedup_p90": r["p90"], "reps": r["n"]}


def _partitioned(gbx, torch, p, field, ex_std, n=8):
    pc = np.array([p.send_base[k * p.P // n] for k in range(n)] + [p.sendbuf_bytes], np.int64)
    rc = np.array([p.recv_base[k * p.P // n] for k in range(n)] + [p.recvbuf_bytes], np.int64)
    # the partitions' moves leave four SMs to the producer (a persistent move grid would
    # otherwise hold every SM until it ends, and the next slab's production would queue behind it)
    import torch as _t
    sms = _t.cuda.get_device_properties(0).multi_processor_count
    pr = gbx.partitioned_init(ex_std.request, pc, rc, info=f"max_ctas={2 * (sms - 4)}")
    base = field.clone()
    lo = [int(pc[k]) // 8 for k in range(n + 1)]
    prod, xch = torch.cuda.Stream(), torch.cuda.Stream()
    ga = torch.randn(8192, 4096, dtype=torch.bfloat16, device="cuda")
    gb = torch.randn(4096, 8192, dtype=torch.bfloat16, device="cuda")
    gc = torch.empty(8192, 8192, dtype=torch.bfloat16, device="cuda")
    kind = ["hbm"]

    def produce(k):
        if kind[0] == "hbm":        # the slab's blocks rewritten (memory-bound)
            torch.mul(base[lo[k]:lo[k + 1]], 1.0, out=field[lo[k]:lo[k + 1]])
        elif kind[0] == "compute":  # a compute-bound stage (bf16 GEMM) that the slab waits for
            torch.mm(ga, gb, out=gc)
        else:                       # a latency-bound stage that leaves most SMs idle
            torch.cuda._sleep(600_000)

    def sequential():
        with torch.cuda.stream(prod):
            for k in range(n):
                produce(k)
        torch.cuda.current_stream().wait_stream(prod)   # the request's stream
        ex_std.request.start()
        ex_std.request.wait()

    def early_bird():
        pr.start()
        for k in range(n):
            with torch.cuda.stream(prod):
                produce(k)
                # timing enabled: a stream waiting on a disable-timing event held back the work
                # behind the wait on this GPU (2.99 against 2.47 ms for the latency-bound case)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(prod)
            xch.wait_event(ev)
            pr.pready(k, xch)
        pr.wait()

    def produce_only():
        with torch.cuda.stream(prod):
            for k in range(n):
                produce(k)

    res = {"slabs": n, "launches_per_epoch": pr.info()["launches"], "move_grid_cap": 2 * (sms - 4),
           "timing": "interleaved pairs (sequential, early-bird), CUDA events, median and p10/p90 of 24"}
    what = {"hbm": "one elementwise kernel per slab rewriting 512 ranks' blocks (1.07 GB read + write)",
            "compute": "one 8192x4096x8192 bf16 GEMM per slab (0.55 TFLOP)",
            "latency": "one single-block kernel per slab busy for 600k cycles (~0.3 ms), most SMs idle"}
    for k_ in ("hbm", "compute", "latency"):
        kind[0] = k_
        r = factor_entry("sequential", "early_bird", paired(torch, sequential, early_bird, reps=24))
        ts = []
        for _ in range(12):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            produce_only()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        r["produce_only_ms"] = spread(ts)
        r["producer"] = what[k_]
        res[k_] = r
    del pr, base, ga, gb, gc
    torch.cuda.empty_cache()
    return res


def _dense_and_allgather(gbx, torch, p5, flush):
    res = {}
    P, ppn, c, s = 1024, 32, 4, 64
    r = np.arange(P, dtype=np.int64)
    sd = np.tile(r * c, P)                       # sdispls[r*P + d] = d*c
    rd = np.tile(r * c, P)                       # rdispls[d*P + src] = src*c
    cnt = np.full(P * P, c, np.int32)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    base = torch.from_numpy(r * P * c * s).cuda()
    comm = gbx.Comm(P, ppn)
    send = torch.randint(0, 256, (P * P * c * s,), dtype=torch.uint8, device="cuda")
    recvs = {}
    for alg in ("standard", "locality"):
        recvs[alg] = torch.zeros_like(send)
        req = gbx.alltoallv_init(comm, send, base, t32(cnt), t32(sd), recvs[alg], base, t32(cnt), t32(rd), s,
                                 gbx.BYTES, info=f"algorithm={alg}")
        ms = _cold_ms(torch, req, flush)
        info = req.info()
        res[alg] = {"ms": ms, "user_GBps": 2 * P * P * c * s / (ms * 1e-3) / 1e9,
                    "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9, "launches": info["launches"],
                    "U": info["U"], "node_pairs": info["node_pairs"]}
        del req
    res["identical"] = bool(torch.equal(recvs["standard"], recvs["locality"]))
    res["workload"] = f"P={P}, {ppn} per node, {c} points of {s} bytes per rank pair"
    del recvs, send
    # neighbourhood allgather on the stencil graph
    dq = gbx.DevicePattern(p5)
    g = gbx.DistGraph(gbx.Comm(p5.P, p5.ppn), dq.in_ptr, dq.sources, dq.out_ptr, dq.dests)
    n, es = 128, 64
    deg_in = np.diff(p5.in_ptr)
    sbase = torch.from_numpy(np.arange(p5.P, dtype=np.int64) * n * es).cuda()
    rbase = torch.from_numpy(np.concatenate([[0], np.cumsum(deg_in)[:-1]]).astype(np.int64) * n * es).cuda()
    send = torch.randint(0, 256, (p5.P * n * es,), dtype=torch.uint8, device="cuda")
    ag = {}
    outs = {}
    for alg in ("standard", "locality"):
        outs[alg] = torch.zeros(int(deg_in.sum()) * n * es, dtype=torch.uint8, device="cuda")
        req = gbx.neighbor_allgather_init(send, sbase, outs[alg], rbase, n, g, es, info=f"algorithm={alg}")
        ms = _cold_ms(torch, req, flush)
        info = req.info()
        ag[alg] = {"ms": ms, "user_GBps": 2 * info["V"] * es / (ms * 1e-3) / 1e9,
                   "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9, "V": info["V"], "V_inter": info["V_inter"],
                   "U": info["U"], "launches": info["launches"]}
        del req
    ag["identical"] = bool(torch.equal(outs["standard"], outs["locality"]))
    ag["workload"] = f"27-point stencil graph P={p5.P}, {p5.ppn} per node, {n} points of {es} bytes per rank"
    res["allgather_stencil"] = ag
    del outs, send, g, dq
    torch.cuda.empty_cache()
    return res


def extras(gbx, torch, p, field, halo, grad_halo, grad_field, dp, ex_std, bwd):
    out = {}
    # start -> wait latency on the L2-resident config 1 (2D 5-point halo, 3,072 elements)
    q1 = pt.config1()
    f1 = torch.from_numpy(pt.stencil_field(q1, pt.SEED + 1)).cuda()
    lat = {"V": q1.volume, "E": q1.n_edges}
    for name in ("standard", "locality"):
        for mode in ("graph=1", "graph=0"):
            h = torch.zeros(q1.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
            ex = gbx.Exchange(q1, f1, h, name, info=mode)
            wall, dev = [], []
            for i in range(220):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                t = time.perf_counter()
                e0.record()
                ex.request.start()
                e1.record()
                ex.request.wait()
                t = time.perf_counter() - t
                e1.synchronize()
                if i >= 20:
                    wall.append(t * 1e6)
                    dev.append(e0.elapsed_time(e1) * 1e3)
            lat[f"{name}_{'graph' if mode == 'graph=1' else 'eager'}"] = {
                "start_wait_us": statistics.median(wall), "device_us": statistics.median(dev),
                "launches": ex.info()["launches"]}
            del ex, h
    lat["note"] = "L2-resident: latency instead of a fraction of HBM bandwidth; median of 200"
    out["latency_cfg1"] = lat
    # fused forward + backward (one graph, fused level launches) vs plain
    plain_f = gbx.Exchange(p, field, halo, "standard", info="graph=0", dp=dp, graph=ex_std.graph)
    plain_b = gbx.backward_init(plain_f.request, grad_halo, grad_field, info="graph=0")

    def plain():
        plain_f.request.start()
        plain_f.request.wait()
        plain_b.start()
        plain_b.wait()

    def fused():
        gbx.startall([ex_std.request, bwd])
        gbx.waitall([ex_std.request, bwd])
    out["fwd_bwd_cfg5"] = dict(factor_entry("plain", "fused", paired(torch, plain, fused, reps=24)),
                               plain="eager launches, start+wait per exchange",
                               fused="startall of forward+backward: one CUDA graph, fused launches",
                               timing="interleaved pairs, CUDA events, median and p10/p90 of 24")
    del plain_f, plain_b
    # batched uneven patterns (config 3) vs plain
    out["batched_cfg3"] = _batched(gbx, torch, measured_peaks()[0], 24, nvtx=False)
    # fused forward + backward on the differentiable SpMV halo (config 4: 2^20 rows, fp32)
    q4 = pt.config4()
    dq4 = gbx.DevicePattern(q4)
    x4 = torch.randn(q4.meta["n"], device="cuda", dtype=torch.float32)
    h4 = torch.zeros(q4.recvbuf_bytes // 4, device="cuda", dtype=torch.float32)
    g4 = torch.randn(q4.recvbuf_bytes // 4, device="cuda", dtype=torch.float32)
    gx4 = torch.zeros_like(x4)
    f_graph = gbx.Exchange(q4, x4, h4, "standard", dp=dq4)
    b_graph = gbx.backward_init(f_graph.request, g4, gx4)
    f_plain = gbx.Exchange(q4, x4, h4, "standard", info="graph=0", dp=dq4, graph=f_graph.graph)
    b_plain = gbx.backward_init(f_plain.request, g4, gx4, info="graph=0")

    def plain4():
        f_plain.request.start()
        f_plain.request.wait()
        b_plain.start()
        b_plain.wait()

    def fused4():
        gbx.startall([f_graph.request, b_graph])
        gbx.waitall([f_graph.request, b_graph])
    out["fwd_bwd_cfg4"] = dict(factor_entry("plain", "fused", paired(torch, plain4, fused4, reps=48)), V=q4.volume,
                               plain="eager launches, start+wait per exchange",
                               fused="startall of forward+backward: one CUDA graph",
                               timing="interleaved pairs, CUDA events, median and p10/p90 of 48")
    del f_graph, b_graph, f_plain, b_plain
    # the same stencil exchange through per-edge datatypes (neighbourhood all-to-all-w) over the
    # point-major field and over a component-major copy of it, L2 flushed between repetitions
    flush = L2Flush(torch)
    wres = {"standard_v_ms": _cold_ms(torch, ex_std.request, flush)}
    for layout in ("aos", "soa"):
        w = pt.stencil_w(tuple(p.meta["grid"]), tuple(p.meta["ranks"]), p.ppn, comps=p.meta["comps"],
                         layout=layout)
        npts = int(np.prod(p.meta["blk"]))
        xs = field if layout == "aos" else \
            field.view(p.P, npts, p.meta["comps"]).transpose(1, 2).contiguous().view(-1)
        hw = torch.zeros_like(halo)
        ew = gbx.WExchange(w, xs, hw)
        ms = _cold_ms(torch, ew.request, flush)
        ew.start()
        ew.wait()
        ex_std.request.start()
        ex_std.request.wait()
        info = ew.info()
        wres[layout] = {"ms": ms, "user_GBps": w.user_bytes() / (ms * 1e-3) / 1e9,
                        "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9, "unit_bytes": info["elem_size"],
                        "units": info["V"], "launches": info["launches"],
                        "identical_to_index_list_exchange": bool(torch.equal(hw, halo))}
        del ew, hw, xs
        torch.cuda.empty_cache()
    wres["l2"] = L2Flush.L2_NOTE + "; median of 20"
    out["alltoallw_cfg5"] = wres
    # partitioned (early-bird) exchange: a producer rewrites the field in 8 slabs of 512 ranks;
    # sequential = produce all, then exchange; early-bird = each slab marked ready as soon as
    # it is produced, its moves overlapping the production of the next slab
    out["partitioned_cfg5"] = _partitioned(gbx, torch, p, field, ex_std)
    # dense all-to-all-v over the emulated communicator (P = 1024, 32 per node, 4 points of
    # 64 bytes per rank pair) and the neighbourhood allgather on the stencil graph (128 points
    # of 64 bytes per rank to each of its neighbours): standard vs locality-aware form, whose
    # values are named by their source elements (an allgathered point crosses a node pair once)
    out["alltoallv_dense"] = _dense_and_allgather(gbx, torch, p, flush)
    # SpMV halo (config 2), standard vs locality, L2 flushed between repetitions
    q = pt.config2()
    xs = torch.randn(q.meta["n"], device="cuda", dtype=torch.float64)
    r1 = torch.zeros(q.recvbuf_bytes // 8, device="cuda", dtype=torch.float64)
    r2 = torch.zeros_like(r1)
    dq = gbx.DevicePattern(q)
    a = gbx.Exchange(q, xs, r1, "standard", dp=dq)
    b = gbx.Exchange(q, xs, r2, "locality", dp=dq, graph=a.graph)
    res = {}
    peak = measured_peaks()[0]
    for name, ex in (("standard", a), ("locality", b)):
        st = spread(_cold_times(torch, ex.request.start, ex.request.wait, flush, reps=20))
        ms = st["median"]
        info = ex.info()
        res[name] = {"ms": st, "user_GBps": q.user_bytes() / (ms * 1e-3) / 1e9, "algo_bytes": info["algo_bytes"],
                     "frac_of_measured_hbm": info["algo_bytes"] / (ms * 1e-3) / 1e9 / peak,
                     "copy_forms": form_names(info)}
    res["identical"] = bool(torch.equal(r1, r2))
    res["V"] = q.volume
    res["E"] = q.n_edges
    res["U"] = b.info()["U"]
    res["node_pairs"] = b.info()["node_pairs"]
    res["l2"] = L2Flush.L2_NOTE
    out["spmv_cfg2"] = res
    return out


class L2Flush:
    """Leaves L2 holding none of the exchange's data before a timed repetition: a 256 MB write
    (twice L2), then a 256 MB read of a second buffer, so that the write's dirty lines are
    written back before the timed region instead of inside it (the read leaves clean lines)."""
    L2_NOTE = ("flushed before every repetition: a 256 MB write, then a 256 MB read of another "
               "buffer (no dirty flush lines are written back inside the timed region)")

    def __init__(self, torch):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
        self.acc = torch.zeros((), dtype=torch.float32, device="cuda")

    def fill_(self, v):
        self.w.fill_(v)
        self.acc += self.r.sum()   # the read; the result stays on the device


def _cold_times(torch, start, wait, flush, reps=20, warm=3):
    """CUDA-event times (ms) of `start()` over `reps` repetitions, L2 flushed (a 256 MB
    write) before each; `wait()` completes each one outside the timed interval."""
    for _ in range(warm):
        start()
        wait()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        start()
        e1.record()
        wait()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def _cold_ms(torch, req, flush, reps=20, warm=3):
    """Median CUDA-event time of start() with L2 flushed (L2Flush) before each rep."""
    return statistics.median(_cold_times(torch, req.start, req.wait, flush, reps, warm))


def spread(ts):
    """median, 10th and 90th percentile of a list of times."""
    q = np.percentile(np.asarray(ts, dtype=np.float64), [10, 50, 90])
    return {"median": float(q[1]), "p10": float(q[0]), "p90": float(q[2]), "n": len(ts)}


def run_spmv(args):
    """The SpMV halo exchange (2^20 rows, P = 1024 at 32 per node, 20 nnz per row, fp64 x),
    standard and locality forms, L2 flushed before each of 20 repetitions; then one more
    start of each inside an NVTX range (cfg2_standard, cfg2_locality) for ncu --nvtx-include."""
    import torch
    import paper_2309_07337_gb300 as gbx
    peak, peak_kind = measured_peaks()
    q = pt.config2()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 2)
    xs = torch.randn(q.meta["n"], device="cuda", dtype=torch.float64, generator=gen)
    flush = L2Flush(torch)
    dq = gbx.DevicePattern(q)
    outs = {}
    res = {"workload": "spmv_halo_2^20rows_P1024_ppn32_nnz20_f64", "V": q.volume, "E": q.n_edges,
           "l2": L2Flush.L2_NOTE, "peak_GBps": peak, "peak_kind": peak_kind}
    graph = None
    keep = []
    for name in ("standard", "locality"):
        outs[name] = torch.zeros(q.recvbuf_bytes // 8, device="cuda", dtype=torch.float64)
        ex = gbx.Exchange(q, xs, outs[name], name, dp=dq, graph=graph, info=args.info)
        graph = ex.graph
        st = spread(_cold_times(torch, ex.start, ex.wait, flush, reps=args.reps))
        info = ex.info()
        ms = st["median"]
        res[name] = {"ms": st, "user_GBps": q.user_bytes() / (ms * 1e-3) / 1e9, "algo_bytes": info["algo_bytes"],
                     "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9,
                     "frac_of_measured_hbm": info["algo_bytes"] / (ms * 1e-3) / 1e9 / peak,
                     "launches": info["launches"], "vec": info["vec_bytes"], "block": info["block"],
                     "copy_forms": [COPY_FORM_NAMES.get(f, str(f)) for f in range(16) if info["copy_forms"] >> f & 1],
                     "U": info["U"], "node_pairs": info["node_pairs"]}
        flush.fill_(1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(f"cfg2_{name}")
        ex.start()
        torch.cuda.nvtx.range_pop()
        ex.wait()
        keep.append(ex)   # the locality request shares the standard one's graph
    res["identical"] = bool(torch.equal(outs["standard"], outs["locality"]))
    print(json.dumps(res))


def run_batched(args):
    """The uneven batch (64 SpMV halo patterns, P 64..1024, 2^14..2^20 rows, 8..32 nnz per
    row, fp32 or fp64): one start+wait per pattern (eager launches) against gbx_startall of
    all 64 (one CUDA graph), each timed over `reps` repetitions; then one more batched start
    inside the NVTX range cfg3_batched for ncu --nvtx-include.  The batch's buffers exceed L2."""
    import torch
    import paper_2309_07337_gb300 as gbx
    peak, peak_kind = measured_peaks()
    out = _batched(gbx, torch, peak, args.reps, count=args.count, info=args.info)
    print(json.dumps(out))


def _batched(gbx, torch, peak, reps, nvtx=True, count=64, info=""):
    t = time.perf_counter()
    pats = pt.config3_torch(count, device="cuda")
    gen_s = time.perf_counter() - t
    bufs, g_reqs, p_reqs = [], [], []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 3)
    for q in pats:
        dt = torch.float64 if q.dtype == "f64" else torch.float32
        sb = torch.randn(q.sendbuf_bytes // (8 if q.dtype == "f64" else 4), device="cuda", dtype=dt, generator=gen)
        rb = torch.zeros(q.recvbuf_bytes // sb.element_size(), device="cuda", dtype=dt)
        rb2 = torch.zeros_like(rb)
        dq = gbx.DevicePattern(q)
        e1 = gbx.Exchange(q, sb, rb, "standard", dp=dq, info=info)
        e2 = gbx.Exchange(q, sb, rb2, "standard", info="graph=0" + (";" + info if info else ""), dp=dq,
                          graph=e1.graph)
        bufs.append((sb, rb, rb2, e1, e2))
        g_reqs.append(e1.request)
        p_reqs.append(e2.request)
    Vtot = sum(q.volume for q in pats)
    Btot = sum(q.user_bytes() for q in pats)
    algo = sum(r.info()["algo_bytes"] for r in g_reqs)

    def plain3():
        for r in p_reqs:
            r.start()
            r.wait()

    def batched3():
        gbx.startall(g_reqs)
        gbx.waitall(g_reqs)
    tp, tb, ratio = paired(torch, plain3, batched3, reps=reps)
    # the batch's device time alone: a bounded sleep kernel holds the stream while the host
    # enqueues the start, so the first event is stamped when the sleep ends and the batch's
    # graph begins right after it (no host latency inside the interval)
    td = []
    for _ in range(max(reps, 5)):
        torch.cuda.synchronize()
        torch.cuda._sleep(400_000)   # about 0.2 ms at 2 GHz
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        gbx.startall(g_reqs)
        e1.record()
        gbx.waitall(g_reqs)
        e1.synchronize()
        td.append(e0.elapsed_time(e1))
    td = spread(td)
    same = all(torch.equal(b[1], b[2]) for b in bufs)
    if nvtx:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cfg3_batched")
        gbx.startall(g_reqs)
        torch.cuda.nvtx.range_pop()
        gbx.waitall(g_reqs)
    ms = tb["median"]
    res = {"patterns": len(pats), "V_total": Vtot, "user_bytes": Btot, "algo_bytes": algo,
           "plain_ms": tp, "batched_ms": tb, "speedup": ratio["median"], "speedup_p10": ratio["p10"],
           "speedup_p90": ratio["p90"],
           "batched_user_GBps": Btot / (ms * 1e-3) / 1e9, "batched_algo_GBps": algo / (ms * 1e-3) / 1e9,
           "frac_of_measured_hbm": algo / (ms * 1e-3) / 1e9 / peak,
           "batched_device_ms": td, "device_algo_GBps": algo / (td["median"] * 1e-3) / 1e9,
           "device_frac_of_measured_hbm": algo / (td["median"] * 1e-3) / 1e9 / peak,
           "identical_results": same, "generation_s": gen_s,
           "dtypes": {d: sum(1 for q in pats if q.dtype == d) for d in ("f32", "f64")},
           "plain": "eager launches, start+wait per pattern (host wait each)",
           "batched": "startall of 64 requests: one CUDA graph, one fused launch per kernel class",
           "timing": "interleaved pairs (plain, batched), CUDA events around each including the host waits; "
                     "median and p10/p90; the batch's buffers exceed L2; batched_device_ms: the batch's graph "
                     "alone on the stream (events around startall behind a sleep kernel, no host latency)"}
    del bufs, g_reqs, p_reqs
    torch.cuda.empty_cache()
    return res


def run_sweep(args):
    """Message-size sweep of the 27-point stencil at P = 4096 (16^3 ranks, 64 per node):
    block edge 8, 16, 32 points and 1, 2, 4, 8, 16 fp64 components per point; standard and
    locality forms, cold L2, bytes of both forms compared."""
    import torch
    import paper_2309_07337_gb300 as gbx
    peak, peak_kind = measured_peaks()
    flush = L2Flush(torch)
    gen = torch.Generator(device="cuda")
    rows = []
    for edge in (8, 16, 32):
        for comps in (1, 2, 4, 8, 16):
            p = pt.config5(edge=edge, comps=comps)
            gen.manual_seed(pt.SEED + 5)
            field = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
            h1 = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
            h2 = torch.zeros_like(h1)
            dp = gbx.DevicePattern(p)
            a = gbx.Exchange(p, field, h1, "standard", dp=dp)
            b = gbx.Exchange(p, field, h2, "locality", dp=dp, graph=a.graph)
            row = {"edge": edge, "comps": comps, "elem_bytes": p.elem_size, "V": p.volume,
                   "field_bytes": p.sendbuf_bytes, "user_bytes": 2 * p.volume * p.elem_size}
            for name, ex in (("standard", a), ("locality", b)):
                ms = _cold_ms(torch, ex.request, flush)
                info = ex.info()
                row[name] = {"ms": ms, "user_GBps": row["user_bytes"] / (ms * 1e-3) / 1e9,
                             "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9,
                             "frac_of_measured_hbm": info["algo_bytes"] / (ms * 1e-3) / 1e9 / peak,
                             "vec": info["vec_bytes"], "block": info["block"], "launches": info["launches"]}
            row["identical"] = bool(torch.equal(h1.view(torch.uint8), h2.view(torch.uint8)))
            lf = line_floor(p)["total"]
            row["line_floor_bytes"] = lf
            row["standard"]["frac_of_line_floor"] = lf / (row["standard"]["ms"] * 1e-3) / 1e9 / peak
            rows.append(row)
            print(json.dumps(row), file=sys.stderr)
            del a, b, dp, field, h1, h2
            torch.cuda.empty_cache()
    print(json.dumps({"sweep": "stencil27_P4096_message_size", "peak_GBps": peak, "peak_kind": peak_kind,
                      "l2": L2Flush.L2_NOTE + "; median of 20", "rows": rows}))


def sorted_unique(a):
    """np.unique by a sort and a neighbour test (np.unique is far slower on 10^7 values)."""
    a = np.sort(np.asarray(a), kind="stable")
    return a[np.concatenate([[True], a[1:] != a[:-1]])] if len(a) else a


def line_floor(p):
    """DRAM bytes a standard exchange of `p` cannot avoid when memory moves in 128-byte
    lines: every 128-byte line holding a sent element is read once, the receive buffer is
    written once, and the 4-byte source index of every element is read."""
    sc = np.asarray(p.sendcounts, dtype=np.int64)
    owner = np.repeat(np.arange(p.P), np.diff(np.asarray(p.out_ptr)))
    V = int(sc.sum())
    first = np.cumsum(sc) - sc
    slot = np.repeat(np.asarray(p.sdispls, dtype=np.int64), sc) + (np.arange(V) - np.repeat(first, sc))
    r = np.repeat(owner, sc)
    el = slot if p.send_idx is None else np.asarray(p.send_idx)[np.asarray(p.send_slot_ptr)[r] + slot]
    off = np.asarray(p.send_base)[r] + el.astype(np.int64) * p.elem_size
    lines = sorted_unique(np.concatenate([off >> 7, (off + p.elem_size - 1) >> 7]))
    return {"read_lines_bytes": int(len(lines)) * 128, "index_bytes": 4 * V, "write_bytes": V * p.elem_size,
            "total": int(len(lines)) * 128 + 4 * V + V * p.elem_size}


def locality_line_floor(p):
    """The same floor for the locality form's three launches: (1) every 128-byte line of the
    send buffer holding a value some node pair carries is read once, 4 bytes of index per
    aggregate slot, the send aggregates written; (2) the aggregates read and written once
    (contiguous blocks); (3) every line holding a value sent within its node read once, the
    receive aggregates read, 4 bytes of index per receive slot, the receive buffer written.
    The aggregate slots are the distinct (sender node, receiver node, global index) triples.
    None for a pattern without global indices."""
    if p.global_sidx is None or p.send_slot_ptr is None:
        return None
    s = p.elem_size
    sc = np.asarray(p.sendcounts, dtype=np.int64)
    owner = np.repeat(np.arange(p.P), np.diff(np.asarray(p.out_ptr)))
    V = int(sc.sum())
    first = np.cumsum(sc) - sc
    slot = np.repeat(np.asarray(p.sdispls, dtype=np.int64), sc) + (np.arange(V) - np.repeat(first, sc))
    r = np.repeat(owner, sc)
    d = np.repeat(np.asarray(p.dests, dtype=np.int64), sc)
    sp = np.asarray(p.send_slot_ptr, dtype=np.int64)[r] + slot
    el = slot if p.send_idx is None else np.asarray(p.send_idx)[sp]
    off = np.asarray(p.send_base)[r] + el.astype(np.int64) * s
    g = np.asarray(p.global_sidx, dtype=np.int64)[sp]
    nn = (p.P + p.ppn - 1) // p.ppn
    inter = (r // p.ppn) != (d // p.ppn)
    gmax = int(g.max()) + 1 if V else 1
    if nn * nn * gmax >= (1 << 62):
        return None
    key = ((r // p.ppn) * nn + d // p.ppn)[inter] * gmax + g[inter]
    order = np.argsort(key, kind="stable")
    k = key[order]
    new = np.concatenate([[True], k[1:] != k[:-1]]) if len(k) else np.zeros(0, bool)
    U = int(new.sum())

    def lines(o):
        return 128 * len(sorted_unique(np.concatenate([o >> 7, (o + s - 1) >> 7])))
    st1 = lines(off[inter][order][new]) + 4 * U + s * U
    st2 = 2 * s * U
    st3 = lines(off[~inter]) + s * U + 4 * V + s * V
    return {"U": U, "V_direct": int((~inter).sum()), "step1": st1, "step2": st2, "step3": st3,
            "total": st1 + st2 + st3}


def _match_edges(p):
    """For every out-edge, the in-edge it pairs with under the multigraph rule (the t-th
    listing of d by r with the t-th listing of r by d): both edge lists sorted by (receiver,
    sender, occurrence)."""
    out_r = np.repeat(np.arange(p.P), np.diff(np.asarray(p.out_ptr)))
    in_d = np.repeat(np.arange(p.P), np.diff(np.asarray(p.in_ptr)))
    dests, srcs = np.asarray(p.dests, np.int64), np.asarray(p.sources, np.int64)

    def occurrence(a, b):   # running count of each (a, b) pair, in list order
        key = a * p.P + b
        order = np.argsort(key, kind="stable")
        k = key[order]
        start = np.concatenate([[True], k[1:] != k[:-1]]) if len(k) else np.zeros(0, bool)
        idx = np.arange(len(k))
        run0 = np.maximum.accumulate(np.where(start, idx, 0)) if len(k) else idx
        t = np.empty(len(k), np.int64)
        t[order] = idx - run0
        return t
    to = occurrence(out_r, dests)
    ti = occurrence(in_d, srcs)
    ko = np.lexsort((to, out_r, dests))
    ki = np.lexsort((ti, srcs, in_d))
    match = np.empty(len(dests), np.int64)
    match[ko] = ki
    return match


def bwd_line_floor(p, info):
    """DRAM bytes the standard-order reverse exchange of `p` cannot avoid when memory moves
    in 128-byte lines.  One pass: every incoming gradient line is read once, the program's
    index and record bytes are read, and every 128-byte line holding a written source
    element is written once (an isolated 64-byte x-face gradient costs a whole line, the
    mirror image of the forward's reads).  Two passes (the program the library runs: one
    copy for the source elements read by a single receive slot, one fold for the rest):
    each pass reads and writes its own lines, so a line shared by the two passes is read
    or written twice."""
    s = p.elem_size
    sc = np.asarray(p.sendcounts, dtype=np.int64)
    owner = np.repeat(np.arange(p.P), np.diff(np.asarray(p.out_ptr)))
    V = int(sc.sum())
    first = np.cumsum(sc) - sc
    k = np.arange(V) - np.repeat(first, sc)
    slot = np.repeat(np.asarray(p.sdispls, dtype=np.int64), sc) + k
    r = np.repeat(owner, sc)
    el = slot if p.send_idx is None else np.asarray(p.send_idx)[np.asarray(p.send_slot_ptr)[r] + slot]
    src = np.asarray(p.send_base)[r] + el.astype(np.int64) * s
    m = _match_edges(p)
    d = np.asarray(p.dests, np.int64)
    dst = np.repeat(np.asarray(p.recv_base)[d] + np.asarray(p.rdispls, np.int64)[m] * s, sc) + k * s

    def lines(off):
        return len(sorted_unique(np.concatenate([off >> 7, (off + s - 1) >> 7]))) * 128
    order = np.argsort(src, kind="stable")
    ss = src[order]
    new = np.concatenate([[True], ss[1:] != ss[:-1]]) if V else np.zeros(0, bool)
    rowid = np.cumsum(new) - 1
    single = np.empty(V, bool)
    single[order] = np.bincount(rowid)[rowid] == 1
    rows = ss[new]
    read, index = lines(dst), max(0, int(info["algo_bytes"]) - V * s - len(rows) * s)
    one = {"read_bytes": read, "index_bytes": index, "write_lines_bytes": lines(rows), "rows": int(len(rows))}
    one["total"] = read + index + one["write_lines_bytes"]
    two = {"read_bytes": lines(dst[single]) + lines(dst[~single]), "index_bytes": index,
           "write_lines_bytes": lines(sorted_unique(src[single])) + lines(sorted_unique(src[~single]))}
    two["total"] = two["read_bytes"] + index + two["write_lines_bytes"]
    return {"one_pass": one, "two_pass": two, "total": one["total"], "total_two_pass": two["total"]}


def form_names(info):
    """The copy forms a request's program runs in, by name."""
    return [COPY_FORM_NAMES.get(f, str(f)) for f in range(16) if info["copy_forms"] >> f & 1]


def run_faces(args):
    """The standard exchange of the 512^3 27-point stencil restricted to one direction class
    at a time (x faces: single 64-byte points 2 KB apart; y faces: rows of 32 points; z
    faces: whole 32x32 planes; edges and corners), so that DRAM counters of each launch can
    be set against its algorithmic bytes and its 128-byte-line floor."""
    import torch
    import paper_2309_07337_gb300 as gbx
    peak, peak_kind = measured_peaks()
    R = args.ranks
    g = R * args.edge
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 5)
    field = torch.rand(g ** 3 * 8, dtype=torch.float64, device="cuda", generator=gen)
    dirs_all = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]
    cases = [("all", None), ("x_faces", [(-1, 0, 0), (1, 0, 0)]), ("y_faces", [(0, -1, 0), (0, 1, 0)]),
             ("z_faces", [(0, 0, -1), (0, 0, 1)]),
             ("edges_corners", [d for d in dirs_all if sum(map(abs, d)) >= 2])]
    rows = []
    for name, dirs in cases:
        p = pt.stencil((g, g, g), (R, R, R), ppn=64, comps=8, dtype="f64", neighbors="all", directions=dirs)
        h = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
        ex = gbx.Exchange(p, field, h, "standard")
        for _ in range(3):
            ex.start()
            ex.wait()
        torch.cuda.synchronize()
        ts = []
        for _ in range(20):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ex.start()
            e1.record()
            ex.wait()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_push(f"face_{name}")   # one more start, for ncu --nvtx-include
        ex.start()
        torch.cuda.nvtx.range_pop()
        ex.wait()
        ms = statistics.median(ts)
        info = ex.info()
        fl = line_floor(p)
        row = {"case": name, "V": p.volume, "ms": ms, "algo_bytes": info["algo_bytes"],
               "algo_GBps": info["algo_bytes"] / (ms * 1e-3) / 1e9, "floor_bytes": fl,
               "floor_GBps": fl["total"] / (ms * 1e-3) / 1e9,
               "floor_frac_of_measured_hbm": fl["total"] / (ms * 1e-3) / 1e9 / peak}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr)
        del ex, h
        torch.cuda.empty_cache()
    print(json.dumps({"faces": f"stencil27_{g}cube_P{R ** 3}_c8_standard", "peak_GBps": peak, "peak_kind": peak_kind,
                      "rows": rows}))


COPY_FORM_NAMES = {0: "segments", 1: "gather", 3: "two-index", 5: "gather pipelined", 7: "two-index pipelined",
                   8: "bulk pieces", 9: "scatter windows", 10: "gather streamed", 11: "two-index streamed",
                   12: "fold streamed"}


def run_bwd_forms(args):
    """The backward of the 512^3 exchange in each program shape, CUDA-event timed (median of
    20 starts; the gradient buffers, 1.6 GB and 8.6 GB, exceed L2)."""
    import torch
    import paper_2309_07337_gb300 as gbx
    peak, peak_kind = measured_peaks()
    p = pt.config5(edge=args.edge)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(pt.SEED + 5)
    x = torch.rand(p.sendbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    h = torch.zeros(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda")
    g = torch.randn(p.recvbuf_bytes // 8, dtype=torch.float64, device="cuda", generator=gen)
    shapes = ["", "bulk=0", "bulk=2", "single_split=0", "split_order=dest", "stream=0", "stream=2;bulk=0",
              "stream=0;single_split=0", "stream=2;single_split=0"]
    rows = []
    for alg in ("standard", "locality"):
        ex = gbx.Exchange(p, x, h, alg)
        ref = None
        for info in shapes:
            gs = torch.zeros_like(x)
            b = gbx.backward_init(ex.request, g, gs, info=info)
            for _ in range(3):
                b.start()
                b.wait()
            ts = []
            tag = "bwdform_" + alg + "_" + ("".join(c if c.isalnum() else "_" for c in info) or "default")
            torch.cuda.nvtx.range_push(tag)   # for ncu --nvtx-include "<tag>/"
            for _ in range(20):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                b.start()
                e1.record()
                b.wait()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            torch.cuda.nvtx.range_pop()
            ms = statistics.median(ts)
            i = b.info()
            if ref is None:
                ref = gs
            forms = [COPY_FORM_NAMES.get(f, str(f)) for f in range(16) if i["copy_forms"] >> f & 1]
            row = {"order": alg, "info": info or "(default)", "ms": ms, "launches": i["launches"],
                   "copy_forms": forms, "block": i["block"], "algo_bytes": i["algo_bytes"],
                   "algo_GBps": i["algo_bytes"] / (ms * 1e-3) / 1e9,
                   "frac_of_measured_hbm": i["algo_bytes"] / (ms * 1e-3) / 1e9 / peak,
                   "device_bytes": i["device_bytes"],
                   "identical_to_default": bool(torch.equal(gs.view(torch.uint8), ref.view(torch.uint8)))}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr)
            del b
            if gs is not ref:
                del gs
            torch.cuda.empty_cache()
        del ex, ref
        torch.cuda.empty_cache()
    print(json.dumps({"bwd_forms": f"stencil27_{16 * args.edge}cube_P4096_c8", "peak_GBps": peak,
                      "peak_kind": peak_kind, "rows": rows}))


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.faces:
        run_faces(args)
    elif args.spmv:
        run_spmv(args)
    elif args.batched:
        run_batched(args)
    elif args.bwd_forms:
        run_bwd_forms(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
