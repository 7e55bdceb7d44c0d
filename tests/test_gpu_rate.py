"""Rate-based sampling (Section 3.2's baseline) on the GPU against the oracle, bit-exact.

The gaps between sampled bytes are inputs (geometric draws from the generator, or
constants), so both sides see the same draws.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg
from tests.gpu_util import gpu_ctx

pytestmark = pytest.mark.gpu
T0 = tg.T_PLAIN


def _dev(*xs):
    return [torch.from_numpy(np.ascontiguousarray(x.view(np.int64) if x.dtype == np.uint64 else
                                                  x.view(np.int32) if x.dtype == np.uint32 else x)).cuda() for x in xs]


def _gaps_for(tr, mean, seed=1, slack=1.2):
    total = int(np.abs(tr.delta).astype(object).sum())
    return tg.gaps(int(total / mean * slack) + 64, mean, seed=seed)


def _check(ctx, tr, gaps, consumed, n_lines):
    d, l, p, g = _dev(tr.delta, tr.line, tr.is_python, gaps)
    counts, st = scl.scl_rate_samples(ctx, d, l, p, g, consumed)
    wc, ws = oracle.rate_samples(tr.delta, tr.line, tr.is_python, gaps, consumed, n_lines=n_lines)
    assert np.array_equal(counts, wc), np.nonzero(counts != wc)
    assert st.tolist() == ws.tolist(), (st, ws)
    return counts, st


@pytest.mark.parametrize("n,mean", [(1_000_000, T0), (300_001, 1_048_573), (50_000, 4096)])
def test_geometric_gaps_match_oracle(n, mean):
    tr = tg.plain_trace(n, seed=3, n_lines=256, big_count=2, big_size=4 * tg.GIB)
    ctx = gpu_ctx(T0)
    _, st = _check(ctx, tr, _gaps_for(tr, mean), 0, 256)
    assert st[0] > 0 and st[3] == 0


def test_every_byte_and_constant_gaps():
    rng = np.random.default_rng(4)
    n = 20_000
    delta = rng.integers(-16, 17, n).astype(np.int64)
    tr = tg.Trace(delta, np.arange(n, dtype=np.uint64) * 16, rng.integers(0, 8, n).astype(np.uint32),
                  rng.integers(0, 2, n).astype(np.uint8))
    ctx = gpu_ctx(T0, n_lines=8)
    total = int(np.abs(delta).sum())
    counts, st = _check(ctx, tr, np.ones(total + 5, np.uint64), 0, 8)   # every byte
    assert int(st[0]) == total
    for c, consumed in ((7, 3), (1000, 999)):
        _, st = _check(ctx, tr, np.full(total // c + 5, c, np.uint64), consumed, 8)
        assert int(st[0]) == (consumed + total) // c


def test_segments_continue_and_exhaustion_flag():
    tr = tg.plain_trace(400_000, seed=6, n_lines=64)
    ctx = gpu_ctx(T0, n_lines=64)
    gaps = _gaps_for(tr, 1_048_573, seed=2)
    whole, sw = _check(ctx, tr, gaps, 0, 64)
    acc = np.zeros_like(whole)
    k, consumed = 0, 0
    for a, b in ((0, 99_999), (99_999, 250_000), (250_000, tr.n)):
        piece = tr.slice(a, b)
        c, st = _check(ctx, piece, gaps[k:], consumed, 64)
        acc += c
        k += int(st[1])
        consumed = int(st[2])
    assert np.array_equal(acc, whole) and k == int(sw[1]) and consumed == int(sw[2])
    _, st = _check(ctx, tr, gaps[:10], 0, 64)       # far too few gaps
    assert int(st[0]) == 10 and int(st[3]) & 1


def test_long_trace_rate_vs_threshold_counts():
    # the Table 2 comparison on the long-trace generators: rate-based sampling at mean T
    # takes many more samples than the threshold sampler at T
    tr = tg.long_trace(1 << 24)
    ctx = gpu_ctx(T0)
    _, st = _check(ctx, tr, _gaps_for(tr, T0, seed=7), 0, 256)
    o = oracle.Oracle(T0, n_lines=256)
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    assert int(st[0]) > 3 * len(o.samples())


@pytest.mark.parametrize("n", [1, 777, 1_000_003])
def test_cpu_attribution_matches_oracle(n):
    q = 10_000_000
    rng = np.random.default_rng(n)
    vt = (np.cumsum(rng.integers(q // 2, 4 * q, n)) + 123).astype(np.int64)
    ln = rng.integers(0, 256, n).astype(np.uint32)
    ctx = gpu_ctx(T0)
    py, nat, fl = scl.scl_cpu_attribution(ctx, torch.from_numpy(vt).cuda(), torch.from_numpy(ln.view(np.int32)).cuda(),
                                          q, 123)
    wpy, wnat, wfl = oracle.cpu_attribution(vt, ln, q, 123, n_lines=256)
    assert np.array_equal(py, wpy) and np.array_equal(nat, wnat) and fl == wfl == 0
