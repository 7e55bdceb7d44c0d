"""Benchmark of the memory-sampling replay path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

A step is one pass of the whole path -- threshold sampler, attribution, high-water
crossings, leak membership test, leak scores, copy-volume sampler -- over one
trace resident in HBM (the trace's state is reset before each step).  The default
workload is the single 2^28-event trace (5 leaking lines, a +2 GiB ramp, 2^28/10
memcpys, T = 10,485,767); its 5.9 GB of input is far larger than the 129 MB L2,
so no flush is needed between steps.  Under torchrun each rank replays its own
trace (seed + rank): per-GPU work is fixed (weak scaling).

One JSON line is printed by rank 0.  `value` is alloc/free events per second over
all ranks, timed with CUDA events on the replay stream; `e2e` is the same metric
through scl_replay_batch_host with pinned host buffers (host-to-device copies and
the read-back of the per-line results inside the timed region); `roofline` is the
dominant kernel's algorithmic bytes per launch over its CUDA-event duration;
`cpu_baseline` times the sequential oracle on this host and also checks that the
last GPU step agrees with it exactly.  --impl reference times the oracle instead.
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

# algorithmic bytes each kernel must read per unit it processes
ALG_BYTES = {
    "sketch": 8.0,        # delta per event: the candidate counters (warm-up re-reads are overhead, not counted)
    "final": 17.0,        # delta (8) + addr (8) + is_python (1) per event: the exact replay
    "copy_apply": 13.0,   # size (8) + line (4) + is_python (1) per memcpy event
    "copy_sum": 8.0,      # size per memcpy event
}
EVENT_KERNELS = ("sketch", "final")
PATH_BYTES_PER_EVENT = 17.0        # delta + addr + is_python: every event field the path reads
PATH_BYTES_PER_COPY = 13.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="long_256m", choices=["long_256m", "plain_1m", "batched", "serving"])
    p.add_argument("--events", type=int, default=0, help="override the trace length (testing)")
    p.add_argument("--traces", type=int, default=0, help="batched: number of traces (default 4,096)")
    p.add_argument("--procs", type=int, default=0, help="serving: processes (default 512)")
    p.add_argument("--segs", type=int, default=0, help="serving: segments per process (default 16)")
    p.add_argument("--no-tune", action="store_true", help="batched: skip the autotuner")
    p.add_argument("--tune", action="store_true", help="long/plain: run the autotuner before timing")
    p.add_argument("--no-clocks", action="store_true", help="skip nvidia-smi clock sampling (profiler runs)")
    p.add_argument("--no-rate", action="store_true", help="long/plain: skip the rate-based sampling comparison")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(times_ms, events):
    """Whole-job throughput: all ranks' events over the slowest rank's time."""
    t = max(times_ms)
    return sum(events) / (t / 1e3), t


def job_throughput(ms, events, device="cpu"):
    """(events/s, slowest ms) of the whole job: under torch.distributed, the events of every
    rank (sum) over the slowest rank's time (max); alone, this rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return aggregate([ms], [events])
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    e = torch.tensor([float(events)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return aggregate([float(t.item())], [float(e.item())])


def make_trace(workload: str, rank: int, n_override: int = 0):
    from paper_2212_07597_gb300 import tracegen as tg
    if workload == "long_256m":
        n = n_override or (1 << 28)
        return tg.long_trace(n, seed=1 + rank), dict(workload=f"single long trace, {n:,} events", events=n,
                                                     memcpys=n // 10, threshold=tg.T_PLAIN, n_lines=256)
    n = n_override or 1_000_000
    return tg.plain_trace(n, seed=rank), dict(workload=f"plain trace, {n:,} events", events=n, memcpys=n // 10,
                                              threshold=tg.T_PLAIN, n_lines=256)


class Clocks:
    """nvidia-smi clock / throttle sampling (every 50 ms) around the timed region.

    Each sample carries nvidia-smi's own timestamp, so the samples inside the timed
    region are told apart from those of the warm-up just before it."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def _rows(self):
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        except OSError:
            pass
        return rows

    def warm(self, step, sync, max_s=3.0):
        """Run untimed steps until the sampler has produced samples (it starts slowly)."""
        t = time.time()
        while self.p is not None and len(self._rows()) < 2 and time.time() - t < max_s:
            step()
            sync()

    def start(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.06)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = self._rows()
        os.unlink(self.f.name)
        if not rows:
            return None
        import datetime

        def when(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None
        inside = [r for r in rows if self.t0 and when(r) is not None and self.t0 <= when(r) <= self.t1 + 0.05]
        use = inside or rows
        num = lambda x: x.replace(".", "", 1).isdigit()
        sm = [float(r[2]) for r in use if num(r[2])]
        mx = [float(r[3]) for r in rows if num(r[3])]
        reasons = sorted({self.NAMES[i] for r in use for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_in_timed_region": len(inside),
                "basis": "timed region" if inside else "warm-up just before the timed region (region shorter "
                                                        "than the sampling period)"}


def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("scl_sketch.cu", "scl_final.cu", "scl_post.cu", "scl_stage.cuh", "scl_internal.cuh", "scl_exact.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2212_07597_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, units: int, streamed: int = 0):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json), if it
    was taken on the current kernels: bytes per unit x units, where a unit is an event
    (exact replay), a memcpy (copy kernels), or for the sketch an event streamed through
    it (its unit plus its warm-up, `streamed`)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or d.get("source_hash") != source_hash():
        return None
    return k["dram_bytes_per_unit"] * (streamed if k.get("unit") == "streamed event" else units)


def oracle_replay(tr, meta):
    import oracle
    o = oracle.Oracle(meta["threshold"], n_lines=meta["n_lines"])
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    o.replay_copies(tr.csize, tr.cline, tr.cpy)
    return o


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("batched", "serving"):
        # a bounded sample of the workload's traces, replayed one after another
        from paper_2212_07597_gb300 import tracegen as tg
        if args.workload == "batched":
            lens = tg.batched_lengths(4096, seed=2)[:args.traces or 4096]
            pick = list(range(0, len(lens), max(1, len(lens) // 16)))[:16]
            trs = [tg.batched_trace(i, int(lens[i]), seed=2) for i in pick]
            meta = {"threshold": tg.T_PLAIN, "n_lines": 4096, "memcpys": sum(len(t.csize) for t in trs),
                    "workload": f"batched: sampled traces {pick}"}
        else:
            n_p = (args.segs or 16) * (args.events or 65536)
            pick = list(range(0, args.procs or 512, 64))
            trs = [tg.serving_process(p, n_p, seed=4, n_lines=1024) for p in pick]
            meta = {"threshold": tg.T_PLAIN, "n_lines": 1024, "memcpys": sum(len(t.csize) for t in trs),
                    "workload": f"serving: sampled processes {pick}"}
        n = sum(t.n for t in trs)
        meta["events"] = n
        run = lambda: [oracle_replay(t, meta) for t in trs]
    else:
        tr, meta = make_trace(args.workload, 0, args.events)
        n = meta["events"]
        run = lambda: oracle_replay(tr, meta)
    for _ in range(args.warmup):
        run()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run()
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    v = n * args.steps / tot
    line = {"impl": "reference", "metric": "alloc/free events replayed per second (bit-exact)", "value": v,
            "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": meta["workload"], "threshold": meta["threshold"], "n_lines": meta["n_lines"]},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n:,} events (+{meta['memcpys']:,} memcpys) per step, sequential"},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measured_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    if peaks.get("hbm_gbs"):
        return float(peaks["hbm_gbs"]), "of measured"
    return 6800.0, "of fallback"


def roofline_of(ktimes, n, m, traffic=True, sketch_n=None):
    """Dominant kernel of the path and its algorithmic GB/s over its CUDA-event time per launch.
    The sketch and the exact replay take the events of every unit but the traces' first ones
    (sketch_n; those are replayed by k_first).  The
    dominant kernel is taken on the event path's stream: the copy-volume kernels run on a
    lower-priority side stream beside it, so their event-timed spans include waits for SMs."""
    dom = max((k for k in ktimes if k in EVENT_KERNELS), key=lambda k: ktimes[k][0])
    d_ms, d_cnt = ktimes[dom]
    units = n if dom in EVENT_KERNELS else m
    if dom in EVENT_KERNELS and sketch_n is not None:
        units = sketch_n
    achieved = ALG_BYTES[dom] * units / (d_ms / d_cnt / 1e3) / 1e9
    peak, src = measured_peak()
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": src,
            "traffic": traffic_for(dom, units) if traffic else None, "alg_bytes_per_unit": ALG_BYTES[dom]}


def oracle_matches(ctx, tid, o, scl):
    gl, wl = scl.scl_line_stats(ctx, tid), o.lines()
    lk = scl.scl_leak_scores(ctx, tid)
    num, den = o.leak_scores()
    st, ost = scl.scl_trace_state(ctx, tid), o.state()
    ok = all(np.array_equal(gl[k], wl[k]) for k in ("n_growth", "n_shrink", "A", "F", "A_py", "F_py", "net",
                                                     "copy_samples", "copy_bytes"))
    ok = ok and np.array_equal(lk["mallocs"], wl["mallocs"]) and np.array_equal(lk["frees"], wl["frees"])
    ok = ok and np.array_equal(lk["num"], num) and np.array_equal(lk["den"], den)
    ok = ok and all(st[k] == ost[k] for k in ("c", "A", "F", "footprint", "hwm", "n_events", "copy_counter"))
    return ok and st["n_samples"] == len(o.samples())


def chunked(fn, items, workers):
    """fn over items on a thread pool (the generators release the GIL), results in order,
    a bounded number in flight."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(workers) as ex:
        for k in range(0, len(items), 2 * workers):
            yield from zip(items[k:k + 2 * workers], ex.map(fn, items[k:k + 2 * workers]))


def pad16(x):
    return (int(x) + 15) // 16 * 16


def run_batched(args):
    """4,096 independent traces (log-uniform 10k-4M events, 4,096 lines, leak injection in
    every 100th) replayed by one scl_replay_batch call per step, relaunched as a CUDA graph."""
    import torch
    from paper_2212_07597_gb300 import build as scl_build
    from paper_2212_07597_gb300 import tracegen as tg
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    scl_build.build()
    from paper_2212_07597_gb300 import scl
    ntr = args.traces or 4096
    lens = tg.batched_lengths(4096, seed=2 + rank)[:ntr].astype(np.int64)
    if args.events:
        lens = np.minimum(lens, args.events)
    mlen = lens // 10
    eo = np.concatenate([[0], np.cumsum([pad16(x) for x in lens])])
    co = np.concatenate([[0], np.cumsum([pad16(x) for x in mlen])])
    N, M = int(eo[-1]), int(co[-1])
    n_tot, m_tot = int(lens.sum()), int(mlen.sum())
    dev = torch.device("cuda", torch.cuda.current_device())
    cols = [torch.empty(N, dtype=torch.int64, device=dev), torch.empty(N, dtype=torch.int64, device=dev),
            torch.empty(N, dtype=torch.int32, device=dev), torch.empty(N, dtype=torch.uint8, device=dev),
            torch.empty(M, dtype=torch.int64, device=dev), torch.empty(M, dtype=torch.int32, device=dev),
            torch.empty(M, dtype=torch.uint8, device=dev)]
    views = (np.int64, np.int64, np.int32, np.uint8)
    t_gen = time.perf_counter()
    workers = min(32, os.cpu_count() or 4)
    for i, tr in chunked(lambda i: tg.batched_trace(i, int(lens[i]), seed=2 + rank), list(range(ntr)), workers):
        a, b = int(eo[i]), int(co[i])
        for c, x, v in zip(cols[:4], (tr.delta, tr.addr, tr.line, tr.is_python), views):
            c[a:a + len(x)].copy_(torch.from_numpy(x.view(v)))
        for c, x, v in zip(cols[4:], (tr.csize, tr.cline, tr.cpy), (np.int64, np.int32, np.uint8)):
            c[b:b + len(x)].copy_(torch.from_numpy(x.view(v)))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    ptr = [c.data_ptr() for c in cols]
    segs = []
    for i in range(ntr):
        a, b = int(eo[i]), int(co[i])
        segs.append(scl.segment(i, ptr[0] + 8 * a, ptr[1] + 8 * a, ptr[2] + 4 * a, ptr[3] + a,
                                ptr[4] + 8 * b, ptr[5] + 4 * b, ptr[6] + b, n=int(lens[i]), m=int(mlen[i])))
    ctx = scl.scl_replay_init(scl.config(threshold=tg.T_PLAIN, n_lines=4096, max_traces=ntr,
                                         sample_log_capacity=1 << 16))
    stream = torch.cuda.Stream()
    tuned = None
    if not args.no_tune:
        best, best_ms = scl.scl_autotune(ctx, segs, stream)
        tuned = {"unit_events": best.unit_events, "sketch_warps": best.warps_per_block,
                 "warmup_events": best.ext_events, "final_warps": best.final_warps, "ms": best_ms}
    scl.scl_graph_enable(ctx, True)

    def step():
        scl.scl_trace_reset(ctx, scl.SCL_ALL_TRACES, stream)
        scl.scl_replay_batch(ctx, segs, stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    scl.scl_sync(ctx)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 and not args.no_clocks else None
    if clocks:
        clocks.warm(step, torch.cuda.synchronize)
    barrier()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    if clocks:
        clocks.end()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    scl.scl_sync(ctx)
    value, tmax = job_throughput(ms, n_tot * args.steps, dev)
    bstats = scl.scl_batch_stats(ctx)

    # per-kernel times (profiling replaces the graph by plain launches) for the roofline
    scl.scl_profile_reset(ctx)
    scl.scl_profile_enable(ctx, True)
    psteps = 2
    for _ in range(psteps):
        step()
    scl.scl_profile_enable(ctx, False)
    ktimes = scl.scl_kernel_times(ctx)
    launches_per_step = sum(c for _, c in ktimes.values()) // psteps
    roof = roofline_of(ktimes, n_tot, m_tot, traffic=False, sketch_n=n_tot - bstats["first_events"])

    # the plain per-trace path looped over the same traces on the same GPU
    def loop_step():
        scl.scl_trace_reset(ctx, scl.SCL_ALL_TRACES, stream)
        for sg in segs:
            scl.scl_replay_batch(ctx, [sg], stream)

    scl.scl_graph_enable(ctx, False)
    loop_step()
    barrier()
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    loop_step()
    l1.record(stream)
    barrier()
    loop_ms = l0.elapsed_time(l1)

    # exactness and the oracle's pace on a sample of the traces (regenerated on the host)
    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        step()
        scl.scl_sync(ctx)
        pick = sorted({0, 100, int(np.argmax(lens)), int(np.argmin(lens)), 1, ntr // 2, ntr - 1, (7 * ntr) // 9})
        pick = [i for i in pick if i < ntr]
        oks, el, ev = [], 0.0, 0
        for i in pick:
            tr = tg.batched_trace(i, int(lens[i]), seed=2 + rank)
            t0 = time.perf_counter()
            o = oracle_replay(tr, {"threshold": tg.T_PLAIN, "n_lines": 4096})
            el += time.perf_counter() - t0
            ev += int(lens[i])
            oks.append(oracle_matches(ctx, i, o, scl))
        cpu = {"value": ev / el, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": f"traces {pick} ({ev:,} events), sequential, {el:.1f} s"}
        parity = f"bit-exact vs oracle on {len(pick)} sampled traces" if all(oks) else \
            f"MISMATCH vs oracle on traces {[i for i, k in zip(pick, oks) if not k]}"

    # end to end on a subset: pinned host arrays through scl_replay_batch_host
    e2e = None
    if not args.no_e2e:
        sub = list(range(min(ntr, 512)))
        hcols = [c[:int(eo[len(sub)])].cpu().pin_memory() for c in cols[:4]] + \
                [c[:int(co[len(sub)])].cpu().pin_memory() for c in cols[4:]]
        hp = [c.data_ptr() for c in hcols]
        hsegs = [scl.segment(i, hp[0] + 8 * int(eo[i]), hp[1] + 8 * int(eo[i]), hp[2] + 4 * int(eo[i]),
                             hp[3] + int(eo[i]), hp[4] + 8 * int(co[i]), hp[5] + 4 * int(co[i]), hp[6] + int(co[i]),
                             n=int(lens[i]), m=int(mlen[i])) for i in sub]
        sub_n = int(lens[:len(sub)].sum())
        h2d = sum(int(lens[i]) * 21 + int(mlen[i]) * 13 for i in sub)
        d2h = len(sub) * 4096 * (scl.LINE_STAT_DTYPE.itemsize + scl.LEAK_DTYPE.itemsize)

        def e2e_step():
            scl.scl_trace_reset(ctx, scl.SCL_ALL_TRACES, stream)
            scl.scl_replay_batch_host(ctx, hsegs, stream)
            for i in sub:
                scl.scl_line_stats(ctx, i)
                scl.scl_leak_scores(ctx, i)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        ks = 3
        for _ in range(ks):
            e2e_step()
        barrier()
        el = time.perf_counter() - t0
        e2e = {"value": sub_n * ks * ws / el, "unit": "events/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ks,
               "sample": f"first {len(sub)} traces ({sub_n:,} events): host-pinned arrays in, per-line "
                         f"stats and leak scores of every trace out"}

    if rank == 0:
        line = {"metric": "alloc/free events replayed per second (bit-exact)", "value": value, "unit": "events/s",
                "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": f"batched: {ntr:,} traces, {n_tot:,} events, {m_tot:,} memcpys, "
                                       f"log-uniform 10k-4M, 4,096 lines, leak injection every 100th trace",
                           "threshold": tg.T_PLAIN, "n_lines": 4096,
                           "l2": f"inputs larger than L2 ({(21 * N + 13 * M) / 1e9:.0f} GB), no flush",
                           "graph": "one scl_replay_batch per step, relaunched as a CUDA graph",
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
                "tuning": tuned,
                "per_trace_loop": {"value": n_tot / (loop_ms / 1e3), "unit": "events/s", "ms_per_step": loop_ms,
                                   "calls_per_step": ntr},
                "hbm_gbs_path": (PATH_BYTES_PER_EVENT * n_tot + PATH_BYTES_PER_COPY * m_tot) / (tmax / args.steps / 1e3) / 1e9,
                "roofline": dict(roof, measured="per-kernel CUDA events over 2 profiled steps after the timed region"),
                "kernels_ms_per_step": {k: v[0] / psteps for k, v in ktimes.items()},
                "gpu_launches": launches_per_step * args.steps, "batch": bstats,
                "generation_s": t_gen, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "parity": parity}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """512 processes pushing 64k-event segments, Poisson arrivals at 2M segments/min, served
    by scl_serve (continuous batching, copies overlapped with replay, state resident)."""
    import torch
    from paper_2212_07597_gb300 import build as scl_build
    from paper_2212_07597_gb300 import tracegen as tg
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    scl_build.build()
    from paper_2212_07597_gb300 import scl
    P, S, L = args.procs or 512, args.segs or 16, args.events or 65536
    NL = 1024
    n_p = S * L
    m_p = n_p // 10
    N, M = P * n_p, P * m_p
    hcols = [torch.empty(N, dtype=torch.int64, pin_memory=True), torch.empty(N, dtype=torch.int64, pin_memory=True),
             torch.empty(N, dtype=torch.int32, pin_memory=True), torch.empty(N, dtype=torch.uint8, pin_memory=True),
             torch.empty(M, dtype=torch.int64, pin_memory=True), torch.empty(M, dtype=torch.int32, pin_memory=True),
             torch.empty(M, dtype=torch.uint8, pin_memory=True)]
    hn = [c.numpy() for c in hcols]
    t_gen = time.perf_counter()
    seed = 4 + rank
    workers = min(32, os.cpu_count() or 4)
    for p, tr in chunked(lambda p: tg.serving_process(p, n_p, seed=seed, n_lines=NL), list(range(P)), workers):
        for h, x in zip(hn[:4], (tr.delta, tr.addr, tr.line, tr.is_python)):
            h[p * n_p:(p + 1) * n_p] = x.view(h.dtype)
        for h, x in zip(hn[4:], (tr.csize, tr.cline, tr.cpy)):
            h[p * m_p:(p + 1) * m_p] = x.view(h.dtype)
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng(seed)
    owner = rng.permutation(np.repeat(np.arange(P), S))
    gap_ns = 60e9 / 2e6
    arr = tg.arrivals_ns(len(owner), gap_ns, seed=seed)
    hp = [c.data_ptr() for c in hcols]
    nxt = np.zeros(P, np.int64)
    reqs = []
    for i, p in enumerate(owner):
        k = int(nxt[p])
        nxt[p] += 1
        p = int(p)
        a = p * n_p + k * L
        b0, b1 = p * m_p + k * L // 10, p * m_p + (k + 1) * L // 10
        r = scl.scl_request()
        r.trace_id, r.arrival_ns = int(p), int(arr[i])
        r.ev = scl.scl_events(hp[0] + 8 * a, hp[1] + 8 * a, hp[2] + 4 * a, hp[3] + a, L)
        r.cp = scl.scl_copies(hp[4] + 8 * b0, hp[5] + 4 * b0, hp[6] + b0, b1 - b0)
        reqs.append(r)
    ctx = scl.scl_replay_init(scl.config(threshold=tg.T_PLAIN, n_lines=NL, max_traces=P,
                                         sample_log_capacity=1 << 15))

    def serve(realtime):
        scl.scl_trace_reset(ctx, scl.SCL_ALL_TRACES, None)
        scl.scl_sync(ctx)
        return scl.scl_serve(ctx, reqs, realtime=realtime)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        serve(False)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 and not args.no_clocks else None
    if clocks:
        clocks.warm(lambda: serve(False), torch.cuda.synchronize)
    barrier()
    if clocks:
        clocks.start()
    # saturation: every request present at the start; host-to-device copies inside
    walls, batches = [], []
    for _ in range(args.steps):
        res, sm = serve(False)
        walls.append(sm["wall_s"])
        batches.append(sm["batches"])
    barrier()
    # offered load: Poisson arrivals at 2M segments/min, latency = completion - arrival
    lat, rt_walls, rt_batches = [], [], []
    for _ in range(max(1, args.steps // 2)):
        res, sm = serve(True)
        lat.append(res["latency_ns"].astype(np.float64))
        rt_walls.append(sm["wall_s"])
        rt_batches.append(sm["batches"])
    barrier()
    if clocks:
        clocks.end()
    clk = clocks.stop() if clocks else None
    lat = np.concatenate(lat) / 1e6
    wall = sum(walls)
    value, tmax = job_throughput(wall * 1e3, N * args.steps, "cuda")

    # per-kernel times of one saturated pass for the roofline (profiling on)
    scl.scl_profile_reset(ctx)
    scl.scl_profile_enable(ctx, True)
    serve(False)
    scl.scl_profile_enable(ctx, False)
    ktimes = scl.scl_kernel_times(ctx)
    nb = max(1, ktimes.get("final", (0, 1))[1])
    roof = roofline_of({k: v for k, v in ktimes.items()}, N // nb, M // nb, traffic=False)

    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        serve(False)
        pick = sorted({0, 1, 10, P // 2, P - 1, (3 * P) // 7})
        pick = [p for p in pick if p < P]
        oks, el = [], 0.0
        for p in pick:
            tr = tg.serving_process(p, n_p, seed=seed, n_lines=NL)
            t0 = time.perf_counter()
            o = oracle_replay(tr, {"threshold": tg.T_PLAIN, "n_lines": NL})
            el += time.perf_counter() - t0
            oks.append(oracle_matches(ctx, p, o, scl))
        cpu = {"value": len(pick) * n_p / el, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": f"processes {pick} ({len(pick) * n_p:,} events), sequential, {el:.1f} s"}
        parity = f"bit-exact vs oracle on {len(pick)} sampled processes" if all(oks) else \
            f"MISMATCH vs oracle on processes {[p for p, k in zip(pick, oks) if not k]}"

    if rank == 0:
        h2d = 17 * N + 13 * M   # the event line column is read in place (pinned), not moved
        line = {"metric": "alloc/free events replayed per second (bit-exact)", "value": value, "unit": "events/s",
                "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup),
                "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": f"serving: {P} processes x {S} segments of {L:,} events "
                                       f"({N:,} events, {M:,} memcpys), 1,024 lines, leak injection in 10%",
                           "threshold": tg.T_PLAIN, "n_lines": NL,
                           "arrivals": "Poisson, 2M segments/min (mean gap 30 us)",
                           "l2": "inputs copied from pinned host memory every step (larger than L2), no flush",
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "max": float(lat.max()), "requests": int(lat.size),
                               "offered_events_per_s": L * 2e6 / 60,
                               "served_events_per_s": N / (sum(rt_walls) / len(rt_walls)),
                               "batches_per_pass": float(np.mean(rt_batches))},
                "saturated_batches_per_pass": float(np.mean(batches)),
                "roofline": dict(roof, measured="per-kernel CUDA events over one profiled saturated pass",
                                 note="units = a batch's events on average; the traces' first units of each "
                                      "batch go to k_first instead, so this is an upper bound"),
                "kernels_ms_per_pass": {k: v[0] for k, v in ktimes.items()},
                "gpu_launches": int(sum(c for _, c in ktimes.values())) * args.steps,
                "generation_s": t_gen, "clocks": clk,
                "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 0,
                        "note": "value is already end to end: scl_serve copies every segment from pinned host "
                                "memory inside the timed region"},
                "cpu_baseline": cpu, "parity": parity}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2212_07597_gb300 import build as scl_build
    scl_build.build()
    from paper_2212_07597_gb300 import scl

    tr, meta = make_trace(args.workload, rank, args.events)
    n, m = meta["events"], len(tr.csize)
    dev = torch.device("cuda", torch.cuda.current_device())
    seg, keep = scl.trace_segment(0, tr, device=dev)
    ctx = scl.scl_replay_init(scl.config(threshold=meta["threshold"], n_lines=meta["n_lines"],
                                         sample_log_capacity=1 << 20))
    stream = torch.cuda.current_stream()
    tuned = None
    if args.tune:
        best, best_ms = scl.scl_autotune(ctx, [seg], stream)
        tuned = {"unit_events": best.unit_events, "sketch_warps": best.warps_per_block,
                 "warmup_events": best.ext_events, "final_warps": best.final_warps, "ms": best_ms}

    def step():
        scl.scl_trace_reset(ctx, 0, stream)
        scl.scl_replay_batch(ctx, [seg], stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    scl.scl_sync(ctx)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 and not args.no_clocks else None
    if clocks:
        clocks.warm(step, torch.cuda.synchronize)
    scl.scl_sync(ctx)
    scl.scl_profile_reset(ctx)
    scl.scl_profile_enable(ctx, True)
    barrier()
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    if clocks:
        clocks.end()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    scl.scl_profile_enable(ctx, False)
    ktimes = scl.scl_kernel_times(ctx)
    scl.scl_sync(ctx)
    bstats = scl.scl_batch_stats(ctx)

    value, tmax = job_throughput(ms, n * args.steps, dev)

    # dominant kernel and its roofline
    launches = sum(c for _, c in ktimes.values())
    dom = max((k for k in ktimes if k in EVENT_KERNELS), key=lambda k: ktimes[k][0])   # see roofline_of
    d_ms, d_cnt = ktimes[dom]
    per_launch_units = n if dom in EVENT_KERNELS else m
    if dom in EVENT_KERNELS:   # the trace's first unit is replayed exactly by k_first instead
        per_launch_units = n - bstats["first_events"]
    alg = ALG_BYTES[dom] * per_launch_units
    achieved = alg / (d_ms / d_cnt / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "of measured" if peak else "of fallback"
    peak = peak or 6800.0
    path_gbs = (PATH_BYTES_PER_EVENT * n + PATH_BYTES_PER_COPY * m) * args.steps / (ms / 1e3) / 1e9
    # both event-path kernels (the dominant one above, and the other), same arithmetic
    ev_roof = {}
    for k in EVENT_KERNELS:
        if k in ktimes and ktimes[k][1]:
            u = n - bstats["first_events"]
            a_k = ALG_BYTES[k] * u / (ktimes[k][0] / ktimes[k][1] / 1e3) / 1e9
            ev_roof[k] = {"ms": ktimes[k][0] / ktimes[k][1], "achieved": a_k, "frac": a_k / peak,
                          "traffic": traffic_for(k, u, bstats["sketch_events"])}

    # end to end through the host entry point
    e2e = None
    if not args.no_e2e:
        pins = [torch.from_numpy(a).pin_memory() for a in (tr.delta, tr.addr, tr.line, tr.is_python, tr.csize,
                                                          tr.cline, tr.cpy)]
        hseg = scl.segment(0, *[p.numpy() for p in pins])
        out_rows = np.zeros(meta["n_lines"], scl.LINE_STAT_DTYPE)
        # bytes the copies move: the event line column stays in (pinned) host memory and is
        # read in place at the sampled events only
        h2d = sum(p.numel() * p.element_size() for i, p in enumerate(pins) if i != 2)
        d2h = out_rows.nbytes + meta["n_lines"] * scl.LEAK_DTYPE.itemsize

        def e2e_step():
            scl.scl_trace_reset(ctx, 0, stream)
            scl.scl_replay_batch_host(ctx, [hseg], stream)
            scl.scl_line_stats(ctx, 0)
            scl.scl_leak_scores(ctx, 0)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 5))
        for _ in range(ksteps):
            e2e_step()
        barrier()
        el = time.perf_counter() - t0
        e2e = {"value": n * ksteps * ws / el, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": ksteps}

    # the Table 2 comparison: rate-based sampling (one sample per T bytes moved on average,
    # geometric gaps) over the same trace, against the threshold sampler's sample count
    rate = None
    if not args.no_rate:
        from paper_2212_07597_gb300 import tracegen as tg
        total_bytes = int(np.abs(tr.delta).sum(dtype=np.uint64))
        T = meta["threshold"]
        gaps = tg.gaps(int(total_bytes / T * 1.1) + 1024, T, seed=11 + rank)
        gd = torch.from_numpy(gaps.view(np.int64)).to(dev)
        d_delta, d_line, d_py = keep[0], keep[2], keep[3]
        scl.scl_rate_samples(ctx, d_delta, d_line, d_py, gd, 0, stream)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        r0.record(stream)
        for _ in range(reps):
            rc, rs = scl.scl_rate_samples(ctx, d_delta, d_line, d_py, gd, 0, stream)
        r1.record(stream)
        torch.cuda.synchronize()
        rms = r0.elapsed_time(r1) / reps
        step()
        scl.scl_sync(ctx)
        thr = scl.scl_trace_state(ctx, 0)["n_samples"]
        rate = {"rate_samples": int(rs[0]), "threshold_samples": int(thr),
                "ratio": int(rs[0]) / max(1, int(thr)), "gap_mean_bytes": T, "flags": int(rs[3]),
                "ms": rms, "events_per_s": n / (rms / 1e3),
                "note": "rate-based sampling (Section 3.2 baseline) on the same trace; ms includes "
                        "the synchronising read-back of the counts"}

    # oracle on this host: timed baseline and exact check of the last GPU step
    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        step()
        scl.scl_sync(ctx)
        t0 = time.perf_counter()
        o = oracle_replay(tr, meta)
        el = time.perf_counter() - t0
        cpu = {"value": n / el, "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": f"whole {n:,}-event trace (+{m:,} memcpys), one sequential pass, {el:.1f} s"}
        gl, wl = scl.scl_line_stats(ctx, 0), o.lines()
        lk = scl.scl_leak_scores(ctx, 0)
        num, den = o.leak_scores()
        st, ost = scl.scl_trace_state(ctx, 0), o.state()
        ok = all(np.array_equal(gl[k], wl[k]) for k in ("n_growth", "n_shrink", "A", "F", "A_py", "F_py", "net",
                                                         "copy_samples", "copy_bytes"))
        ok = ok and np.array_equal(lk["mallocs"], wl["mallocs"]) and np.array_equal(lk["frees"], wl["frees"])
        ok = ok and np.array_equal(lk["num"], num) and np.array_equal(lk["den"], den)
        ok = ok and all(st[k] == ost[k] for k in ("c", "A", "F", "footprint", "hwm", "n_events", "copy_counter"))
        ok = ok and st["n_samples"] == len(o.samples())
        parity = "bit-exact vs oracle" if ok else "MISMATCH vs oracle"

    if rank == 0:
        line = {"metric": "alloc/free events replayed per second (bit-exact)", "value": value, "unit": "events/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic",
                "config": {"workload": meta["workload"], "threshold": meta["threshold"], "n_lines": meta["n_lines"],
                           "memcpys": m,
                           "l2": f"inputs larger than L2 ({(PATH_BYTES_PER_EVENT * n + PATH_BYTES_PER_COPY * m) / 1e9:.1f} GB "
                                 "per step), no flush",
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
                "hbm_gbs_path": path_gbs,
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_src,
                             "traffic": traffic_for(dom, per_launch_units, bstats["sketch_events"]),
                             "alg_bytes_per_unit": ALG_BYTES[dom]},
                "roofline_event_kernels": ev_roof,
                "kernels_ms_per_step": {k: v[0] / max(1, v[1]) * (v[1] / args.steps) for k, v in ktimes.items()},
                "tuning": tuned,
                "gpu_launches": launches,
                "batch": bstats,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "parity": parity, "rate_based": rate}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
