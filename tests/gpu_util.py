"""Helpers for the GPU parity tests: run traces through libscl (C ABI) and the oracle, compare exactly."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2212_07597_gb300 import scl

SAMPLE_FIELDS = ("idx", "A", "F", "A_py", "F_py", "footprint", "line", "kind", "is_python", "is_hwm")
LINE_FIELDS = ("n_growth", "n_shrink", "A", "F", "A_py", "F_py", "net", "copy_samples", "copy_bytes")
STATE_FIELDS = ("c", "A", "F", "A_py", "F_py", "footprint", "hwm", "tracked_valid", "n_events", "n_copies",
                "copy_counter")


def gpu_ctx(T, n_lines=256, max_traces=1, log_cap=1 << 20, shift=4, unit=None, warps=16, ext=0, final_warps=14, **kw):
    ctx = scl.scl_replay_init(scl.config(threshold=T, n_lines=n_lines, max_traces=max_traces,
                                         sample_log_capacity=log_cap, sample_budget_shift=shift, **kw))
    if unit is not None or ext:
        scl.scl_tuning_set(ctx, unit or 131072, warps, ext, final_warps)
    return ctx


def replay(ctx, items):
    """items: list of (trace_id, tracegen.Trace); one batch call; returns the device tensors (kept alive)."""
    segs, keep = [], []
    for tid, tr in items:
        s, ts = scl.trace_segment(tid, tr)
        segs.append(s)
        keep.append(ts)
    scl.scl_replay_batch(ctx, segs)
    scl.scl_sync(ctx)
    return keep


def oracle_of(tr, T, n_lines=256, **kw):
    o = oracle.Oracle(T, n_lines=n_lines, **kw)
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    o.replay_copies(tr.csize, tr.cline, tr.cpy)
    return o


def assert_same(ctx, tid, o: oracle.Oracle, samples=True):
    if samples:
        g = scl.scl_samples(ctx, tid)
        w = o.samples()
        assert len(g) == len(w), (len(g), len(w))
        for k in SAMPLE_FIELDS:
            if not np.array_equal(g[k], w[k]):
                bad = np.nonzero(g[k] != w[k])[0][:5]
                raise AssertionError(f"sample field {k} differs at {bad}: gpu {g[bad]} oracle {w[bad]}")
    gl = scl.scl_line_stats(ctx, tid)
    wl = o.lines()
    for k in LINE_FIELDS:
        assert np.array_equal(gl[k], wl[k]), (k, np.nonzero(np.any(np.atleast_2d((gl[k] != wl[k]).T).T, axis=-1)
                                                           if gl[k].ndim > 1 else gl[k] != wl[k])[0][:8])
    gk = scl.scl_leak_scores(ctx, tid)
    num, den = o.leak_scores()
    assert np.array_equal(gk["mallocs"], wl["mallocs"]), np.nonzero(gk["mallocs"] != wl["mallocs"])[0][:8]
    assert np.array_equal(gk["frees"], wl["frees"]), np.nonzero(gk["frees"] != wl["frees"])[0][:8]
    assert np.array_equal(gk["num"], num) and np.array_equal(gk["den"], den)
    gs = scl.scl_trace_state(ctx, tid)
    ws = o.state()
    for k in STATE_FIELDS:
        assert gs[k] == ws[k], (k, gs[k], ws[k])
    if ws["tracked_valid"]:
        for k in ("tracked_addr", "tracked_line", "tracked_idx", "tracked_reclaimed"):
            assert gs[k] == ws[k], (k, gs[k], ws[k])
    assert gs["n_samples"] == len(o.samples())
