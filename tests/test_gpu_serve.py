"""Serving loop (scl_serve): many processes' segments arriving as a Poisson stream.

Each process's result must be the same when its segments are served alone and when
they are interleaved with every other process's (continuous batching, three staging
slots, copy/compute overlap) -- bit-exact, like the oracle's replay of the process.
"""
import numpy as np
import pytest

from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg
from tests.gpu_util import assert_same, gpu_ctx, oracle_of

pytestmark = pytest.mark.gpu
T0 = tg.T_PLAIN
NL = 1024


def _workload(n_proc, n_seg, seg_len, seed=7, mean_gap_ns=20_000, pinned=False):
    """Processes cut into seg_len-event requests; request order = Poisson arrival order,
    the process of each arrival drawn at random (seeded), its segments in order.  With
    pinned, the request arrays live in page-locked host memory (gathered by a kernel),
    else in pageable memory (copied by the copy engine)."""
    procs = [tg.serving_process(p, n_seg * seg_len, seed=seed, n_lines=NL) for p in range(n_proc)]
    rng = np.random.default_rng(seed)
    owner = rng.permutation(np.repeat(np.arange(n_proc), n_seg))
    arr = tg.arrivals_ns(len(owner), mean_gap_ns, seed=seed)   # cumulative, non-decreasing
    nxt = [0] * n_proc
    reqs, keep = [], []
    for i, p in enumerate(owner):
        k = nxt[p]
        nxt[p] += 1
        m0, m1 = k * seg_len // 10, (k + 1) * seg_len // 10
        s = procs[p].slice(k * seg_len, (k + 1) * seg_len, m0, m1)
        arrays = [np.ascontiguousarray(x) for x in (s.delta, s.addr, s.line, s.is_python, s.csize, s.cline, s.cpy)]
        if pinned:
            import torch
            arrays = [torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else
                                       x.view(np.int32) if x.dtype == np.uint32 else x).pin_memory().numpy()
                      for x in arrays]
        keep.append(arrays)
        reqs.append(scl.request(int(p), int(arr[i]), *arrays))
    return procs, reqs, keep, owner


@pytest.mark.parametrize("pinned", [False, True])
def test_alone_equals_in_the_mix_and_oracle(pinned):
    n_proc, n_seg, seg_len = 24, 4, 16384
    procs, reqs, keep, owner = _workload(n_proc, n_seg, seg_len, pinned=pinned)
    mix = gpu_ctx(T0, n_lines=NL, max_traces=n_proc, log_cap=1 << 16, unit=16384)
    res, summ = scl.scl_serve(mix, reqs, max_batch=8, realtime=True)
    assert summ["requests"] == len(reqs) and summ["events"] == n_proc * n_seg * seg_len
    assert summ["batches"] >= len(reqs) // 8
    assert np.all(res["latency_ns"] > 0) and np.all(res["done_ns"] > 0)
    # every process against the oracle
    for p in range(n_proc):
        assert_same(mix, p, oracle_of(procs[p], T0, n_lines=NL))
    # a few processes served alone, in their own context: identical to the mix
    for p in (0, 5, 13):
        alone = gpu_ctx(T0, n_lines=NL, max_traces=1, log_cap=1 << 16, unit=16384)
        mine = [scl.request(0, reqs[i].arrival_ns, *keep[i]) for i in np.nonzero(owner == p)[0]]
        scl.scl_serve(alone, mine, realtime=False)
        a, m = scl.scl_samples(alone, 0), scl.scl_samples(mix, p)
        assert len(a) == len(m) and all(np.array_equal(a[k], m[k]) for k in a.dtype.names)
        al, ml = scl.scl_line_stats(alone, 0), scl.scl_line_stats(mix, p)
        assert all(np.array_equal(al[k], ml[k]) for k in al.dtype.names)
        ak, mk = scl.scl_leak_scores(alone, 0), scl.scl_leak_scores(mix, p)
        assert all(np.array_equal(ak[k], mk[k]) for k in ("mallocs", "frees", "num", "den"))
        sa, sm = scl.scl_trace_state(alone, 0), scl.scl_trace_state(mix, p)
        assert sa == sm
        scl.scl_replay_free(alone)
    scl.scl_replay_free(mix)


def test_tiny_staging_budget_forces_one_request_per_slot():
    n_proc, n_seg, seg_len = 6, 3, 8192
    procs, reqs, keep, owner = _workload(n_proc, n_seg, seg_len, seed=9)
    per_req = 256 * 7 + 8 * seg_len * 2 + 4 * seg_len + seg_len + (8 + 4 + 1) * (seg_len // 10)
    ctx = gpu_ctx(T0, n_lines=NL, max_traces=n_proc, log_cap=1 << 16, unit=4096)
    res, summ = scl.scl_serve(ctx, reqs, hbm_budget=3 * (per_req + 4096), realtime=False)
    assert summ["batches"] == len(reqs)          # every slot holds exactly one request
    assert len(set(res["batch"].tolist())) == len(reqs)
    for p in range(n_proc):
        assert_same(ctx, p, oracle_of(procs[p], T0, n_lines=NL))
    scl.scl_replay_free(ctx)


def test_serve_rejects_bad_requests():
    _, reqs, keep, _ = _workload(2, 2, 4096, seed=11)
    ctx = gpu_ctx(T0, n_lines=NL, max_traces=1)
    with pytest.raises(scl.SclError) as e:     # process 1 has no trace slot
        scl.scl_serve(ctx, reqs)
    assert e.value.code == scl.SCL_EINVAL
    ctx2 = gpu_ctx(T0, n_lines=NL, max_traces=2)
    rev = [scl.request(r.trace_id, 10_000 - i, *keep[i]) for i, r in enumerate(reqs)]
    with pytest.raises(scl.SclError) as e:     # arrivals out of order
        scl.scl_serve(ctx2, rev, realtime=True)
    assert e.value.code == scl.SCL_EINVAL
    with pytest.raises(scl.SclError) as e:     # a slot smaller than one request
        scl.scl_serve(ctx2, reqs, hbm_budget=3 * 1024)
    assert e.value.code == scl.SCL_ENOMEM
    scl.scl_replay_free(ctx)
    scl.scl_replay_free(ctx2)
