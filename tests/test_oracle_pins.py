"""Pins that tie the CPU oracle to the paper, not to itself (CPU only).

Each check comes from something the paper or plain mathematics fixes:
brute force on tiny traces (tests/brute.py, a search-based restatement),
T = 1, the constant-size closed form, the adversarial +-(T-1) trace, the
net-within-T bound, the worked scenarios of Section 6.3 (tests/golden/),
invariance under relabelling, and the closed form of the copy sampler.
test_mutants_are_caught plants plausible mistakes in a copy of the oracle
and checks that these pins reject every one.
"""
from __future__ import annotations

import itertools
import os
import random
import re
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import brute
from paper_2212_07597_gb300 import tracegen as tg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _arr(delta, addr, line, py):
    return (np.asarray(delta, np.int64), np.asarray(addr, np.uint64), np.asarray(line, np.uint32),
            np.asarray(py, np.uint8))


def _run(delta, addr, line, py, T, n_lines=8, F0=0, lib_path=None, **kw):
    o = oracle.Oracle(T, n_lines=n_lines, initial_footprint=F0, lib_path=lib_path, **kw)
    o.replay_events(*_arr(delta, addr, line, py))
    return o


# ------------------------------------------------------------------ brute force

def _check_against_brute(delta, addr, line, py, T, n_lines, F0, lib_path=None):
    o = _run(delta, addr, line, py, T, n_lines, F0, lib_path)
    want = brute.samples(delta, addr, line, py, T, F0)
    mallocs, frees = brute.leak_pairs(delta, addr, want, n_lines, F0)
    got = o.samples()
    assert len(got) == len(want)
    for g, w in zip(got, want):
        for k in ("idx", "kind", "A", "F", "A_py", "F_py", "footprint", "line", "is_python", "is_hwm"):
            assert int(g[k]) == w[k], (k, g, w)
    L = o.lines()
    rows = brute.line_stats(want, n_lines)
    for l in range(n_lines):
        for k, v in rows[l].items():
            assert int(L[k][l]) == v, (l, k)
        assert int(L["mallocs"][l]) == mallocs[l] and int(L["frees"][l]) == frees[l], l


def _small_cases(rng, count, nmax=12):
    for _ in range(count):
        n = rng.randint(0, nmax)
        k = rng.choice((1, 2, 5))
        delta = [rng.randint(-3, 3) * k for _ in range(n)]
        addr = [rng.randint(1, 3) for _ in range(n)]      # few addresses: frees often hit the tracked one
        line = [rng.randint(0, 3) for _ in range(n)]
        py = [rng.randint(0, 1) for _ in range(n)]
        T = rng.randint(1, 7)
        F0 = rng.choice((0, 0, 3, -4))
        yield delta, addr, line, py, T, F0


def test_bruteforce_random_small():
    rng = random.Random(1234)
    for delta, addr, line, py, T, F0 in _small_cases(rng, 4000):
        _check_against_brute(delta, addr, line, py, T, 4, F0)


def test_bruteforce_exhaustive_n4():
    # every delta sequence of length <= 4 over {-3..3}, every T in 1..7
    for n in range(0, 5):
        for delta in itertools.product(range(-3, 4), repeat=n):
            for T in (1, 2, 3, 4, 5, 7):
                addr = [1 + (i % 2) for i in range(n)]
                line = [i % 3 for i in range(n)]
                py = [(i * 7) % 2 for i in range(n)]
                _check_against_brute(list(delta), addr, line, py, T, 3, 0)


# ------------------------------------------------------------------ sampler closed forms

def test_T1_samples_every_nonzero_event():
    d, a, l, y = tg.events(5000, seed=7, n_lines=16)
    d[::17] = 0
    o = _run(d, a, l, y, 1, n_lines=16)
    s = o.samples()
    assert np.array_equal(s["idx"], np.nonzero(d)[0])
    assert np.array_equal(s["kind"], np.sign(d[d != 0]).astype(np.int8))


@pytest.mark.parametrize("T,period", [(1_048_573, 256), (10_485_767, 2_561), (104_857_601, 25_601)])
def test_constant_malloc_closed_form(T, period):
    s_ = 4096
    assert -(-T // s_) == period
    n = 3 * period + 17
    d, a, l, y = tg.constant(n, s_, 16)
    o = _run(d, a, l, y, T, n_lines=16)
    s = o.samples()
    want = np.arange(1, n // period + 1, dtype=np.uint64) * period - 1
    assert np.array_equal(s["idx"], want)
    assert (s["A"] == period * s_).all() and (s["F"] == 0).all() and (s["kind"] == 1).all()
    # every sample of a malloc-only trace is a new high-water mark
    assert s["is_hwm"].all()


@pytest.mark.parametrize("T", [2, 3, 1_048_573, 10_485_767])
def test_adversarial_never_samples_from_zero(T):
    d, a, l, y = tg.adversarial(20000, T, period=0)
    o = _run(d, a, l, y, T, n_lines=256)
    assert len(o.samples()) == 0
    assert o.state()["c"] in (0, T - 1)


def test_adversarial_shifted_entry_samples_once():
    # entering the same trace one event later (counter at -(T-1) then +(T-1)...) still never
    # samples; entering with +1 samples exactly at the next +(T-1) and then never again
    T = 1_048_573
    d, a, l, y = tg.adversarial(1000, T, period=0)
    d2 = np.concatenate([[1], d])
    a2 = np.concatenate([[8], a]).astype(np.uint64)
    l2 = np.concatenate([[0], l]).astype(np.uint32)
    y2 = np.concatenate([[0], y]).astype(np.uint8)
    s = _run(d2, a2, l2, y2, T, n_lines=256).samples()
    assert list(s["idx"]) == [1] and s["kind"][0] == 1


def test_net_within_T_and_footprints():
    tr = tg.plain_trace(200_000, seed=11, n_lines=64)
    for T in (1_048_573, 10_485_767):
        o = _run(tr.delta, tr.addr, tr.line, tr.is_python, T, n_lines=64, F0=12345)
        s = o.samples()
        st = o.state()
        P = np.cumsum(tr.delta.astype(object))
        net = sum(int(a) - int(f) for a, f in zip(s["A"], s["F"]))
        assert net + st["c"] == P[-1]
        assert abs(st["c"]) < T
        assert (np.abs(s["A"] - s["F"]) >= T).all()
        assert np.array_equal(np.sign(s["A"] - s["F"]).astype(np.int8), s["kind"])
        assert all(int(fp) == 12345 + P[int(i)] for fp, i in zip(s["footprint"], s["idx"]))
        # a growth sample is always triggered by a malloc, a shrink sample by a free
        trig = tr.delta[s["idx"].astype(np.int64)]
        assert ((trig > 0) == (s["kind"] > 0)).all() and (trig != 0).all()


# ------------------------------------------------------------------ attribution

def test_line_stats_sum_to_samples_and_relabel():
    tr = tg.plain_trace(100_000, seed=5, n_lines=32)
    T = 1_048_573
    o = _run(tr.delta, tr.addr, tr.line, tr.is_python, T, n_lines=32)
    s, L = o.samples(), o.lines()
    for k in ("A", "F", "A_py", "F_py"):
        assert int(L[k].sum()) == int(s[k].sum())
    assert int(L["n_growth"].sum()) == int((s["kind"] > 0).sum())
    assert int(L["n_shrink"].sum()) == int((s["kind"] < 0).sum())
    perm = np.random.default_rng(0).permutation(32).astype(np.uint32)
    o2 = _run(tr.delta, tr.addr, perm[tr.line], tr.is_python, T, n_lines=32)
    L2 = o2.lines()
    for k in ("n_growth", "n_shrink", "A", "F", "A_py", "F_py", "net", "mallocs", "frees"):
        assert np.array_equal(L2[k][perm], L[k]), k


# ------------------------------------------------------------------ worked scenarios (Section 6.3)

def _load_golden(name):
    cfg, ev, smp, leak = {}, [], [], []
    for raw in open(os.path.join(GOLDEN, name)):
        t = raw.split("#")[0].split()
        if not t:
            continue
        if t[0] in ("threshold", "initial_footprint"):
            cfg[t[0]] = int(t[1])
        elif t[0] == "event":
            ev.append([int(x) for x in t[1:]])
        elif t[0] == "sample":
            smp.append([int(x) for x in t[1:]])
        elif t[0] == "leak":
            leak.append([int(x) for x in t[1:]])
    return cfg, ev, smp, leak


@pytest.mark.parametrize("name", ["e3_peak_only.txt", "e2_single_array.txt"])
def test_golden_worked_scenarios(name, lib_path=None):
    cfg, ev, smp, leak = _load_golden(name)
    d, a, l, y = zip(*ev)
    o = _run(d, a, l, y, cfg["threshold"], n_lines=16, F0=cfg["initial_footprint"], lib_path=lib_path)
    s = o.samples()
    keys = ("idx", "kind", "A", "F", "A_py", "F_py", "footprint", "line", "is_python", "is_hwm")
    assert len(s) == len(smp)
    for g, w in zip(s, smp):
        assert [int(g[k]) for k in keys] == w
    L = o.lines()
    num, den = o.leak_scores()
    for line_, m, f, nu, de in leak:
        assert (int(L["mallocs"][line_]), int(L["frees"][line_]), int(num[line_]), int(den[line_])) == (m, f, nu, de)


# ------------------------------------------------------------------ leak detector

def test_leak_malloc_only():
    d, a, l, y = tg.constant(30_000, 4096, 8)
    T = 1_048_573
    o = _run(d, a, l, y, T, n_lines=8)
    s, L = o.samples(), o.lines()
    assert int(L["mallocs"].sum()) == int((s["kind"] > 0).sum()) == len(s)
    assert int(L["frees"].sum()) == 0
    num, den = o.leak_scores()
    m = L["mallocs"].astype(np.int64)
    assert np.array_equal(num, m + 1) and np.array_equal(den, m + 2)


def test_hwm_is_strict():
    T = 100
    # +T, -T, +T: footprints T, 0, T at the samples; the third does not beat the mark
    o = _run([T, -T, T], [16, 16, 32], [1, 2, 3], [0, 0, 0], T, n_lines=4)
    s = o.samples()
    assert list(s["is_hwm"]) == [1, 0, 0]
    assert list(o.lines()["mallocs"]) == [0, 1, 0, 0]
    # +T, -T, +(T+1): now it does, and the first block (freed at event 1) counts as reclaimed
    o = _run([T, -T, T + 1], [16, 16, 32], [1, 2, 3], [0, 0, 0], T, n_lines=4)
    L = o.lines()
    assert list(o.samples()["is_hwm"]) == [1, 0, 1]
    assert list(L["mallocs"]) == [0, 1, 0, 1] and list(L["frees"]) == [0, 1, 0, 0]


def test_leak_window_excludes_frees_after_next_crossing():
    T = 100
    # object 0 (addr 16) is freed only after crossing 1 -> not reclaimed in its window
    d = [T, T, -T]
    a = [16, 32, 16]
    o = _run(d, a, [1, 2, 3], [0, 0, 0], T, n_lines=4)
    L = o.lines()
    assert list(L["mallocs"]) == [0, 1, 1, 0] and list(L["frees"]) == [0, 0, 0, 0]
    # a malloc of the tracked address inside the window is not a reclamation
    d = [T, 5, T]
    a = [16, 16, 48]
    L = _run(d, a, [1, 2, 3], [0, 0, 0], T, n_lines=4).lines()
    assert list(L["frees"]) == [0, 0, 0, 0]


def test_leak_invariances_and_bounds():
    tr = tg.plain_trace(150_000, seed=9, n_lines=16, leak_lines=(1, 2), p_malloc=0.52)
    T = 1_048_573
    o = _run(tr.delta, tr.addr, tr.line, tr.is_python, T, n_lines=16)
    L, s = o.lines(), o.samples()
    K = int(s["is_hwm"].sum())
    assert int(L["mallocs"].sum()) == K
    assert int(L["frees"].sum()) <= K - 1
    assert (L["frees"] <= L["mallocs"]).all()
    assert int(L["frees"].sum()) > 0             # the workload does free tracked blocks
    # an address bijection changes nothing
    uniq, inv = np.unique(tr.addr, return_inverse=True)
    remap = np.random.default_rng(3).permutation(len(uniq)).astype(np.uint64) * 48 + 4096
    o2 = _run(tr.delta, remap[inv], tr.line, tr.is_python, T, n_lines=16)
    assert np.array_equal(o2.lines(), L)
    num, den = o.leak_scores()
    num2, den2 = o2.leak_scores()
    assert np.array_equal(num, num2) and np.array_equal(den, den2)


def test_leak_score_rules_match_section_3_4():
    o = oracle.Oracle(10, n_lines=1)
    o1 = oracle.Oracle(10, n_lines=1, leak_rule=1)
    # drive (mallocs, frees) through a sequence of crossings: each growth of T beats the mark;
    # on even steps free the tracked block inside its window (a -1 on its address, balanced
    # by a +1 elsewhere so the counter is back at 0 before the next +T)
    T = 10
    d, a = [], []
    for k in range(12):
        d.append(T); a.append(1000 + k)
        if k % 2 == 0:
            d += [-1, 1]; a += [1000 + k, 5000 + k]
    for x in (o, o1):
        x.replay_events(np.array(d, np.int64), np.array(a, np.uint64), np.zeros(len(d), np.uint32),
                        np.zeros(len(d), np.uint8))
    m, f = int(o.lines()["mallocs"][0]), int(o.lines()["frees"][0])
    assert m == 12 and f == 6
    num, den = o.leak_scores()
    assert Fraction(int(num[0]), int(den[0])) == 1 - Fraction(f + 1, m - f + 2)
    num, den = o1.leak_scores()
    assert Fraction(int(num[0]), int(den[0])) == 1 - Fraction(f + 1, m + 2)
    # Section 3.4's intuition for the textbook rule: many mallocs and no frees -> near 1
    assert Fraction(m + 1, m + 2) > Fraction(9, 10)


# ------------------------------------------------------------------ copy volume (Section 3.5)

@pytest.mark.parametrize("phase", [0, 12345])
def test_copy_sampler_closed_form(phase, lib_path=None):
    T = 1_048_573
    cs, cl, cy = tg.copies(20_000, seed=3, n_lines=16)
    o = oracle.Oracle(T, n_lines=16, copy_phase=phase, lib_path=lib_path)
    o.replay_copies(cs, cl, cy)
    L = o.lines()
    Tc = 2 * T
    S = int(cs.astype(object).sum())
    total = (phase + S) // Tc - phase // Tc
    assert int(L["copy_samples"].sum()) == total
    assert int(L["copy_bytes"].sum()) == total * Tc
    samp, byts = brute.copy_stats(cs, cl, cy, Tc, phase, 16)
    assert [list(map(int, r)) for r in L["copy_samples"]] == samp
    assert [list(map(int, r)) for r in L["copy_bytes"]] == byts
    assert o.state()["copy_counter"] == (phase + S) % Tc


# ------------------------------------------------------------------ resident state

def test_segmentation_invariance():
    tr = tg.plain_trace(60_000, seed=21, n_lines=32, leak_lines=(0,))
    T = 1_048_573
    whole = _run(tr.delta, tr.addr, tr.line, tr.is_python, T, n_lines=32)
    rng = np.random.default_rng(2)
    cuts = np.sort(rng.choice(np.arange(1, tr.n), 20, replace=False))
    o = oracle.Oracle(T, n_lines=32)
    for a_, b_ in zip(np.r_[0, cuts], np.r_[cuts, tr.n]):
        o.replay_events(tr.delta[a_:b_], tr.addr[a_:b_], tr.line[a_:b_], tr.is_python[a_:b_])
    assert np.array_equal(o.samples(), whole.samples())
    assert np.array_equal(o.lines(), whole.lines())
    assert o.state() == whole.state()


# ------------------------------------------------------------------ leak report (Section 3.4 filter)

def test_leak_report_thresholds():
    # m malloc-only 4 KiB objects... built directly: one line's crossings, no frees.  The
    # printed likelihood (m + 1) / (m + 2) first exceeds 95% at m = 19.
    T = 4096
    for m, want in ((18, False), (19, True)):
        d = np.full(m, 4096, np.int64)              # every event a new mark on line 0
        o = oracle.Oracle(T, n_lines=2)
        o.replay_events(d, np.arange(1, m + 1, dtype=np.uint64) * 4096, np.zeros(m, np.uint32),
                        np.ones(m, np.uint8))
        r = o.leak_report()
        assert r[0]["mallocs"] == m and r[0]["frees"] == 0 and r[0]["likely"] == want
        assert r[0]["growth"] and r[0]["reported"] == want         # footprint = mark: 100% growth
        assert r[0]["rate_num"] == m * 4096 and r[0]["rate_den"] == m
        assert not r[1]["likely"]                                   # no objects: 1/2


def test_leak_report_growth_rule():
    # growth: 100 (footprint - F0) >= mark.  Climb to a mark of 100 * 4096 bytes, then free
    # back down to exactly 1% of it (reported) or one block less (not)
    T = 4096
    for keep, want in ((1, True), (0, False)):
        up = np.full(100, 4096, np.int64)
        down = np.full(100 - keep, -4096, np.int64)
        d = np.concatenate([up, down])
        addr = np.concatenate([np.arange(1, 101, dtype=np.uint64), np.arange(100, keep, -1, dtype=np.uint64)]) * 4096
        o = oracle.Oracle(T, n_lines=1)
        o.replay_events(d, addr, np.zeros(len(d), np.uint32), np.zeros(len(d), np.uint8))
        st = o.state()
        assert st["hwm"] == 100 * 4096 and st["footprint"] == keep * 4096
        assert o.leak_report()[0]["growth"] == want


# ------------------------------------------------------------------ Python / native time (Section 2.2)

def test_cpu_attribution_rules():
    q = 10_000_000   # 10 ms quantum
    # interrupts exactly on time: all Python
    vt = np.arange(1, 101, dtype=np.int64) * q
    line = np.arange(100, dtype=np.uint32) % 4
    py, nat, fl = oracle.cpu_attribution(vt, line, q, 0, n_lines=4)
    assert py.tolist() == [25 * q] * 4 and nat.tolist() == [0] * 4 and fl == 0
    # a delayed interrupt: the delay is native time of the interrupted line
    vt2 = np.array([q, 2 * q, 5 * q], np.int64)
    py, nat, fl = oracle.cpu_attribution(vt2, np.array([0, 1, 1], np.uint32), q, 0, n_lines=2)
    assert py.tolist() == [q, 2 * q] and nat.tolist() == [0, 2 * q]
    # every interval attributed exactly once (with an early interrupt, T < q)
    rng = np.random.default_rng(1)
    vt3 = np.cumsum(rng.integers(0, 3 * q, 5000)).astype(np.int64) + 7
    ln = rng.integers(0, 16, 5000).astype(np.uint32)
    py, nat, fl = oracle.cpu_attribution(vt3, ln, q, 7, n_lines=16)
    assert int(py.sum() + nat.sum()) == int(vt3[-1] - 7) and fl == 0 and (nat >= 0).all()
    # brute force per interrupt
    bp, bn, prev = [0] * 16, [0] * 16, 7
    for t, l in zip(vt3.tolist(), ln.tolist()):
        T = t - prev
        bp[l] += min(T, q)
        bn[l] += T - min(T, q)
        prev = t
    assert py.tolist() == bp and nat.tolist() == bn
    # time going backwards is flagged and skipped
    _, _, fl = oracle.cpu_attribution(np.array([5, 3], np.int64), np.array([0, 0], np.uint32), q, 0, n_lines=1)
    assert fl & 1


# ------------------------------------------------------------------ rate-based sampling (Section 3.2)

def _rate_brute(delta, line, py, gaps, consumed, n_lines):
    """Byte by byte: expand every event into the bytes it moves and mark the bytes at the
    cumulative gap positions (an independent restatement of the Bernoulli-per-byte model)."""
    owner = []                                   # event index of every byte moved
    for i, d in enumerate(delta):
        owner += [i] * abs(int(d))
    counts = [[0, 0] for _ in range(n_lines)]
    pos, k, n = int(gaps[0]) - consumed if len(gaps) else None, 0, 0
    while k < len(gaps) and pos <= len(owner):
        i = owner[pos - 1]
        counts[int(line[i])][1 if py[i] else 0] += 1
        n += 1
        k += 1
        if k < len(gaps):
            pos += int(gaps[k])
    return counts, n, k


def test_rate_sampler_against_bytes(lib_path=None):
    rng = random.Random(5)
    for _ in range(300):
        n = rng.randint(0, 12)
        delta = np.array([rng.randint(-9, 9) for _ in range(n)], np.int64)
        line = np.array([rng.randint(0, 2) for _ in range(n)], np.uint32)
        py = np.array([rng.randint(0, 1) for _ in range(n)], np.uint8)
        total = int(np.abs(delta).sum())
        gaps = np.array([rng.randint(1, 6) for _ in range(total + 2)], np.uint64)
        consumed = rng.randint(0, int(gaps[0]) - 1)
        counts, st = oracle.rate_samples(delta, line, py, gaps, consumed, n_lines=3, lib_path=lib_path)
        want, nb, used = _rate_brute(delta, line, py, gaps, consumed, 3)
        assert counts.tolist() == want and int(st[0]) == nb and int(st[1]) == used and int(st[3]) == 0
        # bytes of the next gap consumed: total bytes minus the bytes up to the last sample
        upto = consumed + total
        done = int(gaps[:used].astype(object).sum()) if used else 0
        assert int(st[2]) == upto - done


@pytest.mark.parametrize("c,consumed", [(1, 0), (7, 3), (1_048_573, 12345)])
def test_rate_sampler_closed_forms(c, consumed, lib_path=None):
    # constant gaps c: one sample per c bytes, counted from `consumed` bytes into the first
    # gap -- floor((consumed + S) / c) samples (with c = 1: every byte)
    tr = tg.plain_trace(20_000, seed=9, n_lines=8)
    S = int(np.abs(tr.delta).astype(object).sum())
    K = (consumed + S) // c
    gaps = np.full(K + 1, c, np.uint64)
    counts, st = oracle.rate_samples(tr.delta, tr.line, tr.is_python, gaps, consumed, n_lines=8, lib_path=lib_path)
    assert int(st[0]) == K and int(counts.sum()) == K and int(st[3]) == 0
    assert int(st[2]) == (consumed + S) % c


def test_rate_sampler_segments_and_exhaustion():
    tr = tg.plain_trace(30_000, seed=11, n_lines=16)
    gaps = tg.gaps(100_000, 1_000_000, seed=3)
    whole, sw = oracle.rate_samples(tr.delta, tr.line, tr.is_python, gaps, 0, n_lines=16)
    acc = np.zeros_like(whole)
    k, used_bytes = 0, 0
    for a_, b_ in ((0, 7_001), (7_001, 19_999), (19_999, tr.n)):
        c_, st = oracle.rate_samples(tr.delta[a_:b_], tr.line[a_:b_], tr.is_python[a_:b_], gaps[k:], used_bytes,
                                     n_lines=16)
        acc += c_
        k += int(st[1])
        used_bytes = int(st[2])
    assert np.array_equal(acc, whole) and k == int(sw[1]) and used_bytes == int(sw[2])
    few, st = oracle.rate_samples(tr.delta, tr.line, tr.is_python, gaps[:3], 0, n_lines=16)
    assert int(st[0]) == 3 and int(st[3]) & 1   # ran out of gaps


# ------------------------------------------------------------------ mutants

_MUTANTS = {
    "gt_instead_of_ge": ("if (mag >= T) {", "if (mag > T) {"),
    "carry_excess": ("st->c = 0; st->A = 0;", "st->c = st->c > 0 ? st->c - T : st->c + T; st->A = 0;"),
    "hwm_non_strict": ("st->footprint > st->hwm", "st->footprint >= st->hwm"),
    # (testing the mark at shrink samples too would be an equivalent mutant: a shrink
    # sample's footprint is always below the previous sample's, so it never sets a mark)
    "hwm_never_raised": ("st->hwm = st->footprint;", ";"),
    "free_check_any_event": ("if (d < 0 && st->tracked_valid", "if (st->tracked_valid"),
    "free_credit_to_new_line": ("st->lines[st->tracked_line].frees", "st->lines[line[i]].frees"),
    "free_credit_at_last_object": ("if (st->tracked_valid) st->lines[st->tracked_line].frees", "if (0) st->lines[st->tracked_line].frees"),
    "no_reclaim_reset": ("st->tracked_reclaimed = 0;", ";"),
    "wrong_leak_den": ("*den = m - f + 2;", "*den = m + f + 2;"),
    "copy_bytes_raw": ("L->copy_bytes[f] += q * Tc;", "L->copy_bytes[f] += size[j];"),
    "copy_drop_remainder": ("st->copy_counter = total % Tc;", "st->copy_counter = 0;"),
    "py_swapped": ("if (is_python[i] && add_ovf(st->A_py, d, &st->A_py))", "if (!is_python[i] && add_ovf(st->A_py, d, &st->A_py))"),
    "footprint_before_event": ("s.footprint = st->footprint;", "s.footprint = st->footprint - d;"),
    "line_of_previous_event": ("s.line = line[i];", "s.line = line[i > 0 ? i - 1 : 0];"),
    "hwm_start_zero": ("st->hwm = cfg->initial_footprint;", "st->hwm = 0;"),
    "rate_sample_one_byte_late": ("if (b < left) { left -= b; b = 0; break; }", "if (b <= left) { left -= b; b = 0; break; }"),
    "rate_one_sample_per_event": ("left = k < n_gaps ? gap[k] : 0;", "left = k < n_gaps ? gap[k] : 0; b = 0;"),
    "rate_frees_not_counted": ("uint64_t b = d < 0 ? (uint64_t)0 - (uint64_t)d : (uint64_t)d;", "uint64_t b = d < 0 ? 0 : (uint64_t)d;"),
}


def _pins_pass(lib_path) -> bool:
    try:
        rng = random.Random(99)
        for delta, addr, line, py, T, F0 in _small_cases(rng, 400):
            _check_against_brute(delta, addr, line, py, T, 4, F0, lib_path)
        for name in ("e3_peak_only.txt", "e2_single_array.txt"):
            test_golden_worked_scenarios(name, lib_path)
        for phase in (0, 12345):
            test_copy_sampler_closed_form(phase, lib_path)
        test_rate_sampler_against_bytes(lib_path)
        for c, consumed in ((1, 0), (7, 3)):
            test_rate_sampler_closed_forms(c, consumed, lib_path)
    except AssertionError:
        return False
    return True


def test_mutants_are_caught():
    src = open(os.path.join(os.path.dirname(oracle.__file__), "scl_oracle.c")).read()
    assert _pins_pass(None)
    with tempfile.TemporaryDirectory() as td:
        for name, (old, new) in _MUTANTS.items():
            assert src.count(old) >= 1, name
            msrc = os.path.join(td, f"m_{name}.c")
            open(msrc, "w").write(src.replace(old, new, 1))
            so = oracle.compile_source(msrc, os.path.join(td, f"m_{name}.so"))
            assert not _pins_pass(so), f"mutant {name} survived the pins"
