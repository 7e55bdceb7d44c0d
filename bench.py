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
    "sketch": 9.0,        # delta (8) + is_python (1) per event: candidate counters and unit totals
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
    p.add_argument("--workload", default="long_256m", choices=["long_256m", "plain_1m"])
    p.add_argument("--events", type=int, default=0, help="override the trace length (testing)")
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
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("scl_sketch.cu", "scl_final.cu", "scl_post.cu", "scl_stage.cuh", "scl_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2212_07597_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, events: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernels."""
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
    return k["dram_bytes_per_event"] * events


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
    tr, meta = make_trace(args.workload, 0, args.events)
    n = meta["events"]
    for _ in range(args.warmup):
        oracle_replay(tr, meta)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_replay(tr, meta)
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    v = n * args.steps / tot
    line = {"impl": "reference", "metric": "alloc/free events replayed per second (bit-exact)", "value": v,
            "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": meta["workload"], "threshold": meta["threshold"], "n_lines": meta["n_lines"]},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"whole {n:,}-event trace (+{meta['memcpys']:,} memcpys) per step, sequential"},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
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

    def step():
        scl.scl_trace_reset(ctx, 0, stream)
        scl.scl_replay_batch(ctx, [seg], stream)

    for _ in range(args.warmup):
        step()
    scl.scl_sync(ctx)
    scl.scl_profile_reset(ctx)
    scl.scl_profile_enable(ctx, True)
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    scl.scl_profile_enable(ctx, False)
    ktimes = scl.scl_kernel_times(ctx)
    scl.scl_sync(ctx)
    bstats = scl.scl_batch_stats(ctx)

    times = [ms]
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        times = [float(t.item())]
    value, tmax = aggregate(times, [n * args.steps] * ws) if ws > 1 else (n * args.steps / (ms / 1e3), ms)

    # dominant kernel and its roofline
    launches = sum(c for _, c in ktimes.values())
    dom = max((k for k in ktimes if k in ALG_BYTES), key=lambda k: ktimes[k][0])
    d_ms, d_cnt = ktimes[dom]
    per_launch_units = n if dom in EVENT_KERNELS else m
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

    # end to end through the host entry point
    e2e = None
    if not args.no_e2e:
        pins = [torch.from_numpy(a).pin_memory() for a in (tr.delta, tr.addr, tr.line, tr.is_python, tr.csize,
                                                          tr.cline, tr.cpy)]
        hseg = scl.segment(0, *[p.numpy() for p in pins])
        out_rows = np.zeros(meta["n_lines"], scl.LINE_STAT_DTYPE)
        h2d = sum(p.numel() * p.element_size() for p in pins)
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
                           "memcpys": m, "l2": "inputs larger than L2 (5.9 GB per step), no flush",
                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
                "hbm_gbs_path": path_gbs,
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_src,
                             "traffic": traffic_for(dom, per_launch_units),
                             "alg_bytes_per_unit": ALG_BYTES[dom]},
                "kernels_ms_per_step": {k: v[0] / max(1, v[1]) * (v[1] / args.steps) for k, v in ktimes.items()},
                "gpu_launches": launches,
                "batch": bstats,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "parity": parity}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
