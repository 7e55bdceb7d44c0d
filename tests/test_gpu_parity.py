"""GPU parity: libscl (through its C ABI) against the CPU oracle, bit-exact on every output.

Everything compared is integer: sample indices, kinds, window totals, footprints,
line ids, flags, high-water marks, per-line totals, leak pairs and their rational
scores, copy-volume counts and the resident trace state.  The tolerance is zero.
"""
import numpy as np
import pytest

import oracle
from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg
from tests.gpu_util import assert_same, gpu_ctx, oracle_of, replay

pytestmark = pytest.mark.gpu
T0 = tg.T_PLAIN


def test_plain_1m_default_tuning():
    tr = tg.plain_trace(1_000_000, seed=0)
    ctx = gpu_ctx(T0)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T0))


@pytest.mark.parametrize("unit", [1024, 4096, 32768, 131072])
def test_small_units_speculation_and_merge(unit):
    tr = tg.plain_trace(300_001, seed=1, leak_lines=(0, 3))
    ctx = gpu_ctx(T0, unit=unit)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T0))


@pytest.mark.parametrize("warmup", [512, 1024])
def test_short_warmup_forces_on_demand_walks(warmup):
    # a warm-up too short for the candidates to collapse leaves many units to the chain's own walk
    tr = tg.plain_trace(200_000, seed=15, leak_lines=(0,))
    ctx = gpu_ctx(1_048_573, unit=8192, ext=warmup)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


@pytest.mark.parametrize("T,shift", [(1, 0), (1_048_573, 2), (104_857_601, 4)])
def test_thresholds(T, shift):
    tr = tg.plain_trace(150_000 + 7, seed=2, big_count=3, big_size=4 * tg.GIB)
    ctx = gpu_ctx(T, shift=shift, unit=4096)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T))


@pytest.mark.parametrize("T", [1_048_573, 10_485_767])
def test_adversarial_never_merges(T):
    d, a, l, y = tg.adversarial(100_000, T, period=4099)
    tr = tg.Trace(d, a, l, y)
    ctx = gpu_ctx(T, unit=1024)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T))


@pytest.mark.parametrize("T", [1 << 30, (1 << 30) + 1, 1_048_573])
def test_candidate_counter_32bit_step_boundaries(T):
    # the candidate counters take a 32-bit form of a step when T <= 2^30 and every delta of
    # the step lies in [-2^22, 2^22): runs of the extreme deltas -2^22 and 2^22 - 1 (prefixes
    # reaching -2^30 within one step), counters near +-T, and steps holding one delta just
    # outside the range (2^22, -2^22 - 1, 2^40) mixed in
    rng = np.random.default_rng(31)
    parts = []
    while sum(len(x) for x in parts) < 250_000:
        n = int(rng.integers(1, 700))
        mode = int(rng.integers(0, 5))
        if mode == 0:
            parts.append(np.full(n, (1 << 22) - 1, np.int64))
        elif mode == 1:
            parts.append(np.full(n, -(1 << 22), np.int64))
        elif mode == 2:
            parts.append(rng.choice(np.array([-(1 << 22), (1 << 22) - 1], np.int64), n))
        elif mode == 3:
            parts.append(rng.integers(-4096, 4097, n).astype(np.int64))
        else:
            x = rng.integers(-(1 << 22), 1 << 22, n).astype(np.int64)
            x[int(rng.integers(0, n))] = int(rng.choice([1 << 22, -(1 << 22) - 1, 1 << 40, -(1 << 40)]))
            parts.append(x)
    d = np.concatenate(parts)
    n = len(d)
    tr = tg.Trace(d, np.arange(n, dtype=np.uint64) * 64, rng.integers(0, 64, n).astype(np.uint32),
                  rng.integers(0, 2, n).astype(np.uint8))
    ctx = gpu_ctx(T, n_lines=64, unit=8192, shift=0)   # up to one sample per event
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T, n_lines=64))


def test_constant_closed_form():
    T = 1_048_573
    d, a, l, y = tg.constant(65536 + 100, 4096, 256)
    ctx = gpu_ctx(T, unit=2048)
    keep = replay(ctx, [(0, tg.Trace(d, a, l, y))])
    s = scl.scl_samples(ctx, 0)
    assert np.array_equal(s["idx"], np.arange(1, len(d) // 256 + 1, dtype=np.uint64) * 256 - 1)
    assert s["is_hwm"].all()


def test_free_heavy_with_address_reuse():
    tr = tg.plain_trace(200_000, seed=5, p_malloc=0.3, addr_reuse=True)
    ctx = gpu_ctx(1_048_573, unit=8192)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


def test_segments_across_calls_equal_whole():
    tr = tg.plain_trace(250_000, seed=6, leak_lines=(1,))
    rng = np.random.default_rng(0)
    cuts = np.sort(rng.choice(np.arange(1, tr.n), 6, replace=False))
    ccuts = np.sort(rng.choice(np.arange(1, len(tr.csize)), 6, replace=False))
    pieces = [tr.slice(a, b, ca, cb) for a, b, ca, cb in zip(np.r_[0, cuts], np.r_[cuts, tr.n],
                                                            np.r_[0, ccuts], np.r_[ccuts, len(tr.csize)])]
    ctx = gpu_ctx(T0, unit=4096)
    keep = []
    keep += replay(ctx, [(0, pieces[0])])
    keep += replay(ctx, [(0, pieces[1]), (0, pieces[2])])       # two segments of one trace in one call
    keep += replay(ctx, [(0, p) for p in pieces[3:]])
    assert_same(ctx, 0, oracle_of(tr, T0))


def test_many_traces_one_batch():
    lens = [1, 31, 1000, 1024, 5000, 77_777, 300_000]
    trs = [tg.plain_trace(n, seed=7, trace=i, n_lines=64) for i, n in enumerate(lens)]
    ctx = gpu_ctx(1_048_573, n_lines=64, max_traces=len(lens), unit=8192)
    keep = replay(ctx, list(enumerate(trs)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, 1_048_573, n_lines=64))


@pytest.mark.parametrize("n_lines", [1024, 4096, 5000])
def test_wide_line_spaces_many_copy_tiles(n_lines):
    # more copy tiles than one wave of copy blocks, so blocks span several tiles and traces;
    # 4,096 lines is the largest shared-memory table, 5,000 takes the global-memory path
    lens = [1_700_000] * 10 + [3, 50_001]
    trs = [tg.plain_trace(n, seed=21, trace=i, n_lines=n_lines) for i, n in enumerate(lens)]
    ctx = gpu_ctx(T0, n_lines=n_lines, max_traces=len(lens), log_cap=1 << 16)
    keep = replay(ctx, list(enumerate(trs)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, T0, n_lines=n_lines))


def test_initial_footprint_rule1_and_phase():
    tr = tg.plain_trace(120_000, seed=8, p_malloc=0.5)
    kw = dict(initial_footprint=5 * tg.GIB, leak_rule=1, copy_phase=12345, copy_multiple=3)
    ctx = gpu_ctx(1_048_573, unit=4096, **kw)
    keep = replay(ctx, [(0, tr)])
    o = oracle.Oracle(1_048_573, copy_threshold=3 * 1_048_573, copy_phase=12345, initial_footprint=5 * tg.GIB,
                      leak_rule=1)
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    o.replay_copies(tr.csize, tr.cline, tr.cpy)
    assert_same(ctx, 0, o)


def test_copies_only_and_zero_deltas():
    tr = tg.plain_trace(50_000, seed=9)
    tr.delta[::3] = 0
    ctx = gpu_ctx(1_048_573, unit=2048)
    keep = replay(ctx, [(0, tg.Trace(tr.delta[:0], tr.addr[:0], tr.line[:0], tr.is_python[:0],
                                     tr.csize, tr.cline, tr.cpy))])
    keep += replay(ctx, [(0, tg.Trace(tr.delta, tr.addr, tr.line, tr.is_python))])
    o = oracle.Oracle(1_048_573)
    o.replay_copies(tr.csize, tr.cline, tr.cpy)
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    assert_same(ctx, 0, o)


def test_host_entry_point_matches_device_path():
    tr = tg.plain_trace(200_000, seed=10)
    ctx = gpu_ctx(T0, unit=16384)
    seg = scl.segment(0, tr.delta, tr.addr, tr.line, tr.is_python, tr.csize, tr.cline, tr.cpy)
    scl.scl_replay_batch_host(ctx, [seg])
    scl.scl_sync(ctx)
    assert_same(ctx, 0, oracle_of(tr, T0))


def test_state_export_import_resume():
    tr = tg.plain_trace(180_000, seed=11, leak_lines=(2,))
    a, b = tr.slice(0, 90_000, 0, 9000), tr.slice(90_000, tr.n, 9000, len(tr.csize))
    ctx1 = gpu_ctx(1_048_573, unit=4096)
    keep = replay(ctx1, [(0, a)])
    blob = scl.scl_state_export(ctx1, 0)
    ctx2 = gpu_ctx(1_048_573, unit=4096, max_traces=2)
    with pytest.raises(scl.SclError):
        bad = gpu_ctx(1_048_573, n_lines=128)
        scl.scl_state_import(bad, 0, blob)
    scl.scl_state_import(ctx2, 1, blob)
    keep += replay(ctx2, [(1, b)])
    assert_same(ctx2, 1, oracle_of(tr, 1_048_573), samples=False)


def test_reset_returns_to_initial_state():
    tr = tg.plain_trace(60_000, seed=12)
    ctx = gpu_ctx(1_048_573, unit=2048)
    keep = replay(ctx, [(0, tg.plain_trace(40_000, seed=99))])
    scl.scl_trace_reset(ctx, 0)
    keep += replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


# ---------------------------------------------------------------- errors are reported, never faulted

def test_line_out_of_range_at_sample_is_reported():
    tr = tg.constant(5000, 4096, 16)
    d, a, l, y = tr
    l = l.copy()
    l[255] = 999          # event 255 triggers the first sample at T = 1,048,573
    ctx = gpu_ctx(1_048_573, n_lines=16, unit=1024)
    with pytest.raises(scl.SclError) as e:
        replay(ctx, [(0, tg.Trace(d, a, l, y))])
    assert e.value.code == scl.SCL_ERANGE


def test_record_space_overflow_is_reported():
    tr = tg.plain_trace(20_000, seed=13)
    ctx = gpu_ctx(1, shift=6, unit=4096)   # T = 1 samples every event: (n >> 6) + 64 records cannot hold them
    with pytest.raises(scl.SclError) as e:
        replay(ctx, [(0, tr)])
    assert e.value.code == scl.SCL_EOVERFLOW


def test_bounded_wait_times_out_and_context_survives():
    ctx = gpu_ctx(1_048_573, unit=2048)
    assert scl.scl_selftest_wait(ctx, 1000) == scl.SCL_ETIMEOUT
    tr = tg.plain_trace(30_000, seed=14)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


def test_bad_descriptors_rejected_on_host():
    ctx = gpu_ctx(T0)
    with pytest.raises(scl.SclError) as e:
        scl.scl_replay_batch(ctx, [scl.segment(5, None, None, None, None, n=10)])
    assert e.value.code == scl.SCL_EINVAL
    import torch
    d = torch.zeros(4097, dtype=torch.int64, device="cuda")
    with pytest.raises(scl.SclError):
        scl.scl_replay_batch(ctx, [scl.segment(0, d[1:], d[1:], d[1:], d[1:], n=4096)])   # misaligned


def test_graph_replay_of_identical_batches():
    import torch
    tr = tg.plain_trace(200_000, seed=16, leak_lines=(1,))
    ctx = gpu_ctx(1_048_573, unit=16384)
    scl.scl_graph_enable(ctx, True)
    stream = torch.cuda.Stream()
    seg, keep = scl.trace_segment(0, tr)
    with torch.cuda.stream(stream):
        for _ in range(3):   # capture once, relaunch twice
            scl.scl_trace_reset(ctx, 0, stream)
            scl.scl_replay_batch(ctx, [seg], stream)
    scl.scl_sync(ctx)
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))
    # a different plan is captured anew
    tr2 = tg.plain_trace(50_000, seed=17)
    seg2, keep2 = scl.trace_segment(0, tr2)
    scl.scl_replay_batch(ctx, [seg2], stream)
    scl.scl_sync(ctx)
    o = oracle.Oracle(1_048_573)
    for t in (tr, tr2):
        o.replay_events(t.delta, t.addr, t.line, t.is_python)
    o.replay_copies(np.concatenate([tr.csize, tr2.csize]), np.concatenate([tr.cline, tr2.cline]),
                    np.concatenate([tr.cpy, tr2.cpy]))
    assert_same(ctx, 0, o)


def test_autotune_restores_state_and_keeps_results_exact():
    tr = tg.plain_trace(400_000, seed=18, leak_lines=(0,))
    a, b = tr.slice(0, 150_000, 0, 15_000), tr.slice(150_000, tr.n, 15_000, len(tr.csize))
    ctx = gpu_ctx(1_048_573)
    keep = replay(ctx, [(0, a)])
    before = scl.scl_state_export(ctx, 0)
    seg, kb = scl.trace_segment(0, b)
    best, ms = scl.scl_autotune(ctx, [seg])
    # every field within the documented search space (0: the default it starts from)
    assert ms > 0 and best.final_warps in (10, 12, 14) and best.ext_events in (16384, 32768)
    assert best.unit_events in (0, 32768, 65536, 131072, 262144, 524288, 1048576, 2097152) and best.fixup in (0, 1)
    assert best.first_events in (0, 524288, 786432, 1048576, 1310720, 1572864)
    assert best.warps_per_block in (8, 12, 16) and best.piece_events in (0, 32768, 65536, 131072, 1 << 22)
    assert scl.scl_state_export(ctx, 0) == before
    t = scl.scl_tuning_get(ctx)
    fields = ("unit_events", "final_warps", "warps_per_block", "ext_events", "first_events", "fixup", "piece_events")
    assert [getattr(t, f) for f in fields] == [getattr(best, f) for f in fields]
    scl.scl_replay_batch(ctx, [seg])
    scl.scl_sync(ctx)
    assert_same(ctx, 0, oracle_of(tr, 1_048_573), samples=False)


@pytest.mark.parametrize("T", tg.SWEEP_THRESHOLDS)
def test_sweep_families_one_batch(T):
    # the threshold sweep's four families (plain with 4 GiB mallocs, adversarial +-(T-1),
    # malloc-only 4 KiB, free-heavy with address reuse), two traces each, in one batch
    n = 120_000
    trs = [tg.sweep_trace(i, T, n=n) for i in range(8)]
    shift = 0 if T == 1 else 4
    ctx = gpu_ctx(T, max_traces=len(trs), shift=shift, log_cap=n + 1, unit=16384)
    keep = replay(ctx, list(enumerate(trs)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, T))


def test_long_trace_all_samples_exact():
    # the long-trace generators (five leaking lines, a ramp) at 2^25 events, default tuning
    tr = tg.long_trace(1 << 25)
    ctx = gpu_ctx(T0, log_cap=1 << 20)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T0))
    # the warm-up candidates carry the true counter into almost every unit
    st = scl.scl_batch_stats(ctx)
    assert st["walked"] <= max(4, st["units"] // 8), st


def test_edge_cases_tiny_traces_one_line_huge_threshold():
    # one line id only; traces of 0, 1 and 2 events; a threshold no trace reaches
    ctx = gpu_ctx(1000, n_lines=1, max_traces=4)
    d1 = np.array([5000], np.int64)                    # one malloc of 5 T: one growth sample
    d2 = np.array([999, -999], np.int64)               # never reaches T
    mk = lambda d: tg.Trace(d, np.arange(1, len(d) + 1, dtype=np.uint64) * 16, np.zeros(len(d), np.uint32),
                            np.ones(len(d), np.uint8))
    trs = [mk(d1), mk(d2), mk(np.zeros(0, np.int64))]
    keep = replay(ctx, [(0, trs[0]), (1, trs[1]), (2, trs[2])])
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, 1000, n_lines=1))
    assert len(scl.scl_samples(ctx, 0)) == 1 and len(scl.scl_samples(ctx, 1)) == 0
    scl.scl_replay_batch(ctx, [])                      # an empty batch is a no-op
    scl.scl_sync(ctx)
    big = gpu_ctx(1 << 61)   # T_c = 2 T must stay within int64
    tr = tg.plain_trace(40_000, seed=31)
    keep = replay(big, [(0, tr)])
    assert_same(big, 0, oracle_of(tr, 1 << 61))
    assert len(scl.scl_samples(big, 0)) == 0


@pytest.mark.parametrize("pinned", [False, True])
def test_host_entry_point_many_pieces_over_copy_streams(pinned):
    # host arrays larger than one 64 MiB staging piece go over several copy streams, for
    # two traces in one call; a pinned event line column is read in place
    trs = [tg.plain_trace(777_777, seed=34), tg.plain_trace(16_000_000, seed=33)]
    ctx = gpu_ctx(T0, log_cap=1 << 18, max_traces=2)
    segs, keep = [], []   # the host arrays must outlive the call's stream work
    for tid, tr in enumerate(trs):
        cols = [tr.delta, tr.addr, tr.line, tr.is_python, tr.csize, tr.cline, tr.cpy]
        if pinned:
            import torch
            cols = [torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else
                                     x.view(np.int32) if x.dtype == np.uint32 else x).pin_memory().numpy()
                    for x in cols]
        keep.append(cols)
        segs.append(scl.segment(tid, *cols))
    scl.scl_replay_batch_host(ctx, segs)
    scl.scl_sync(ctx)
    for tid, tr in enumerate(trs):
        assert_same(ctx, tid, oracle_of(tr, T0))


def test_leak_report_matches_oracle():
    tr = tg.long_trace(1 << 22)
    ctx = gpu_ctx(T0)
    keep = replay(ctx, [(0, tr)])
    g = scl.scl_leak_report(ctx, 0)
    o = oracle_of(tr, T0)
    w = o.leak_report()
    for k in ("reported", "likely", "growth", "mallocs", "frees", "num", "den", "rate_num", "rate_den"):
        assert [int(x) for x in g[k]] == [int(r[k]) for r in w], k
    assert all(int(g["growth"][l]) == 1 for l in range(256))          # the trace grows
    assert int(g["reported"].sum()) > 0


def test_line_timeline_matches_oracle_samples():
    tr = tg.plain_trace(600_000, seed=41, n_lines=64, leak_lines=(0, 2))
    ctx = gpu_ctx(1_048_573, n_lines=64, log_cap=1 << 18)
    keep = replay(ctx, [(0, tr)])
    w = oracle_of(tr, 1_048_573, n_lines=64).samples()
    for l in (0, 1, 2, 63):
        idx, fp = scl.scl_line_timeline(ctx, 0, l)
        sel = w[w["line"] == l]
        assert np.array_equal(idx, sel["idx"]) and np.array_equal(fp, sel["footprint"]), l
        assert len(idx) == len(sel)


def test_range_queries_equal_per_trace_queries():
    # one call for a span of traces returns, trace-major, the rows of the per-trace queries
    lens = [5000, 1, 77_777, 300_000, 20_000]
    trs = [tg.plain_trace(n, seed=31, trace=i, n_lines=64) for i, n in enumerate(lens)]
    ctx = gpu_ctx(1_048_573, n_lines=64, max_traces=8, unit=8192)
    keep = replay(ctx, [(i + 2, tr) for i, tr in enumerate(trs)])
    stats = scl.scl_line_stats_range(ctx, 1, 7)
    scores = scl.scl_leak_scores_range(ctx, 1, 7)
    assert stats.shape == (7, 64) and scores.shape == (7, 64)
    for k in range(7):
        assert stats[k].tobytes() == scl.scl_line_stats(ctx, 1 + k).tobytes()
        assert scores[k].tobytes() == scl.scl_leak_scores(ctx, 1 + k).tobytes()
    for i, tr in enumerate(trs):
        o = oracle_of(tr, 1_048_573, n_lines=64)
        assert np.array_equal(stats[i + 1]["net"], o.lines()["net"])
    assert scl.scl_line_stats_range(ctx, 0, 0).shape == (0, 64)
    with pytest.raises(scl.SclError):
        scl.scl_line_stats_range(ctx, 5, 4)   # passes max_traces


@pytest.mark.parametrize("T", [1, 7, 100, 4096])
def test_small_thresholds_dense_steps(T):
    # at small T most steps are dense (every event 0 or at least 2T - 1 from zero: each nonzero
    # event is a sample); at T = 100 and 4096 dense and ordinary steps alternate.  Frees with
    # LIFO address reuse hit tracked blocks inside a step, across lanes and across steps.
    tr = tg.plain_trace(200_003, seed=41, p_malloc=0.45, addr_reuse=True)
    ctx = gpu_ctx(T, shift=0, unit=16384, log_cap=tr.n + 1)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T))
