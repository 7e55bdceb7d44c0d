"""What the leak report (Section 3.4, "Leak Report Filtering") flags on the leak-injected
workloads, from the oracle (CPU).

The filter's arithmetic is pinned algebraically: with likelihood num/den, "exceeds 95%"
is 20 num > 19 den; under the printed score num = m - 2f + 1, den = m - f + 2 this is
m > 21 f + 18, and under Laplace's rule (num = m - f + 1, den = m + 2) it is m > 20 f + 18,
for m tracked blocks of a line and f of them freed inside their trial.

The outcome on the long-trace generator: the ramp line (never freed) is reported, the five
injected leak lines are not.  Those lines are also the hottest of the Zipf line ids, so
nine in ten of their blocks never enter the free pool and frees drain an almost empty
pool, releasing blocks within a few events of their allocation: the leaking lines' freeable
tenth is caught inside its trial, so about 9% of their trials end freed, more than the 5%
the 95% cut tolerates, and every other line's tracked block is freed (f = m).
"""
import numpy as np
import pytest

import oracle
from paper_2212_07597_gb300 import tracegen as tg


def _report(tr, n_lines, rule=0):
    o = oracle.Oracle(tg.T_PLAIN, n_lines=n_lines, leak_rule=rule)
    o.replay_events(tr.delta, tr.addr, tr.line, tr.is_python)
    return o, o.leak_report()


@pytest.mark.parametrize("rule", [0, 1])
def test_filter_is_the_closed_form_inequality(rule):
    tr = tg.long_trace(1 << 21, seed=1)
    o, rows = _report(tr, 256, rule)
    for r in rows:
        m, f = r["mallocs"], r["frees"]
        assert r["likely"] == (m > (21 if rule == 0 else 20) * f + 18), r
        assert r["reported"] == (r["likely"] and r["growth"])
        assert 0 <= f <= m


def test_long_trace_reports_the_ramp_line_not_the_injected_leaks():
    tr = tg.long_trace(1 << 22, seed=1)
    o, rows = _report(tr, 256)
    lines = o.lines()
    assert rows[0]["growth"]
    assert [r["line"] for r in rows if r["reported"]] == [255]
    for l in tg.LEAK_LINES:
        m, f = int(lines["mallocs"][l]), int(lines["frees"][l])
        assert m > 100 and 0.05 < f / m < 0.15 and not rows[l]["likely"]
    # lines that do not leak: every tracked block is freed inside its trial
    for l in range(5, 9):
        assert lines["frees"][l] == lines["mallocs"][l] > 50


def test_batched_leaking_traces():
    lens = tg.batched_lengths(4096, seed=2)
    # trace 4,000 (476,938 events, 4,096 lines) reports its hottest leaking line only
    tr = tg.batched_trace(4000, int(lens[4000]), seed=2)
    o, rows = _report(tr, 4096)
    assert [r["line"] for r in rows if r["reported"]] == [0]
    # trace 100 (3,802,399 events): the five leaking lines are among the reported ones, and
    # so are lines whose few tracked blocks (at least 19) all outlived their trials
    tr = tg.batched_trace(100, int(lens[100]), seed=2)
    o, rows = _report(tr, 4096)
    rep = [r["line"] for r in rows if r["reported"]]
    assert set(tg.LEAK_LINES) <= set(rep)
    lines = o.lines()
    for l in rep:
        assert lines["mallocs"][l] > 21 * lines["frees"][l] + 18
