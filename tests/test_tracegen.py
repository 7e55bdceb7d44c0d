"""The seeded workloads have the shapes and distributions they claim (CPU only)."""
import math

import numpy as np

from paper_2212_07597_gb300 import tracegen as tg


def test_plain_mix_and_distributions():
    tr = tg.plain_trace(400_000, seed=0)
    assert abs((tr.delta > 0).mean() - 0.6) < 0.005
    assert abs(tr.is_python.mean() - 0.7) < 0.005
    # Zipf(1.1) over 256 ids: P(line 0) = 1 / H(256, 1.1)
    H = sum(k ** -1.1 for k in range(1, 257))
    assert abs((tr.line == 0).mean() - 1 / H) < 0.004 and abs(1 / H - 0.207) < 0.001
    # log-uniform 16 B - 1 MiB has mean (hi - lo) / ln(hi / lo)
    mean = (tg.MIB - 16) / math.log(tg.MIB / 16)
    m = tr.delta[tr.delta > 0].mean()
    assert abs(m / mean - 1) < 0.02 and abs(mean - 94_500) < 100
    assert tr.delta.min() >= -tg.MIB and tr.delta[tr.delta > 0].min() >= 16
    assert (tr.addr % 16 == 0).all()
    cm = (tg.MIB * 64 - tg.KIB) / math.log(64 * tg.MIB / tg.KIB)
    assert abs(tr.csize.mean() / cm - 1) < 0.03 and len(tr.csize) == 40_000


def test_frees_release_exact_live_sizes():
    tr = tg.plain_trace(50_000, seed=3, leak_lines=(0, 1))
    live = {}
    for d, a in zip(tr.delta.tolist(), tr.addr.tolist()):
        if d > 0:
            assert a not in live
            live[a] = d
        else:
            assert live.pop(a) == -d


def test_long_trace_ramp_and_leaks():
    n = 1 << 20
    tr = tg.long_trace(n)
    ramp = (tr.line == 255) & (tr.delta == tg.MIB)
    assert ramp.sum() >= 2048
    freed = set(tr.addr[tr.delta < 0].tolist())
    ramp_addrs = tr.addr[ramp]
    # the 2,048 ramp blocks at the evenly spaced positions are never freed
    pos = (np.arange(2048) * (n // 2048) + (n // 2048) // 2)
    assert (tr.delta[pos] == tg.MIB).all() and not any(a in freed for a in tr.addr[pos].tolist())
    leak = np.isin(tr.line, tg.LEAK_LINES) & (tr.delta > 0)
    unfreed = np.array([a not in freed for a in tr.addr[leak].tolist()])
    assert unfreed.mean() > 0.88


def test_determinism_and_seeds():
    a = tg.plain_trace(10_000, seed=5, trace=2)
    b = tg.plain_trace(10_000, seed=5, trace=2)
    c = tg.plain_trace(10_000, seed=5, trace=3)
    assert all(np.array_equal(x, y) for x, y in zip(
        (a.delta, a.addr, a.line, a.is_python, a.csize), (b.delta, b.addr, b.line, b.is_python, b.csize)))
    assert not np.array_equal(a.delta, c.delta)
    lib = tg._load()
    for y in (-3.0, -0.5, 0.0, 0.3, 1.0, 5.99, 12.5):
        assert abs(lib.tg_det_exp(y) / math.exp(y) - 1) < 1e-14
    for x in (1e-3, 0.5, 1.0, 2.0, 400.0, 1e9):
        assert abs(lib.tg_det_log(x) - math.log(x)) < 1e-13 * max(1, abs(math.log(x)))


def test_sweep_families_and_lengths():
    T = 1_048_573
    adv = tg.sweep_trace(1, T, n=4096)
    assert set(np.unique(np.abs(adv.delta)).tolist()) <= {1, T - 1}
    const = tg.sweep_trace(2, T, n=4096)
    assert (const.delta == 4096).all()
    heavy = tg.sweep_trace(3, T, n=100_000)
    assert abs((heavy.delta > 0).mean() - 0.5) < 0.1     # 30% mallocs, forced when nothing is live
    big = tg.sweep_trace(0, T, n=100_000)
    assert (big.delta == 4 * tg.GIB).sum() >= 4
    L = tg.batched_lengths(4096)
    assert L.min() >= 10_000 and L.max() < 4_000_000
    assert 2.3e9 < L.sum() < 3.0e9
