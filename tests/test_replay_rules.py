"""Two facts the GPU replay builds on, checked against the oracle's sequential replay (CPU).

1. A piece of the exact replay that starts after a sample needs only the samples before it
   (Section 3.2's reset, Section 3.4's high-water mark and tracked block): right after a
   sample the counter and the open window are zero, the mark is the initial footprint raised
   by every earlier growth sample's footprint, and the tracked block is that of the first
   sample attaining the mark (when it beats the initial footprint).
2. A dense stretch: when every event moves the counter by 0 or by at least 2T - 1, every
   nonzero event is a sample whose window holds just itself (from |c| < T it crosses and
   resets), so A = max(d, 0) and F = A - d.
"""
import numpy as np
import pytest

import oracle
from paper_2212_07597_gb300 import tracegen as tg


def _replay(tr, T, n=None, F0=0):
    o = oracle.Oracle(T, n_lines=256, initial_footprint=F0)
    n = tr.n if n is None else n
    o.replay_events(tr.delta[:n], tr.addr[:n], tr.line[:n], tr.is_python[:n])
    return o


@pytest.mark.parametrize("T,seed,F0,pm", [(1_048_573, 3, 0, 0.45), (10_485_767, 4, 0, 0.6), (1_048_573, 5, 1 << 30, 0.45)])
def test_state_after_a_sample_follows_from_the_samples_before_it(T, seed, F0, pm):
    tr = tg.plain_trace(60_000, seed=seed, p_malloc=pm, addr_reuse=True)
    s = _replay(tr, T, F0=F0).samples()
    assert len(s) > 40
    rng = np.random.default_rng(seed)
    for j in sorted(rng.choice(len(s), 12, replace=False)):
        st = _replay(tr, T, int(s["idx"][j]) + 1, F0=F0).state()
        assert st["c"] == 0 and st["A"] == 0 and st["F"] == 0 and st["A_py"] == 0 and st["F_py"] == 0
        growth = s[: j + 1][s["kind"][: j + 1] > 0]
        best = int(growth["footprint"].max()) if len(growth) else None
        mark = max(F0, best) if best is not None else F0
        assert st["hwm"] == mark
        if best is not None and best > F0:
            first = growth[growth["footprint"] == best][0]
            assert st["tracked_valid"] and st["tracked_idx"] == first["idx"]
            # and that sample is the last of the earlier samples flagged as setting the mark
            assert s["idx"][: j + 1][s["is_hwm"][: j + 1] == 1][-1] == first["idx"]


@pytest.mark.parametrize("T", [1, 7, 100, 4096])
def test_dense_events_are_samples_of_their_own(T):
    rng = np.random.default_rng(T)
    n = 20_000
    lim = 2 * T - 1
    mag = lim + rng.integers(0, 8 * lim + 64, n)
    d = np.where(rng.random(n) < 0.2, 0, np.where(rng.random(n) < 0.55, mag, -mag)).astype(np.int64)
    addr = (rng.integers(1, 1 << 20, n) * 16).astype(np.uint64)
    tr = tg.Trace(d, addr, rng.integers(0, 256, n).astype(np.uint32), (rng.random(n) < 0.5).astype(np.uint8))
    s = _replay(tr, T).samples()
    nz = np.nonzero(d)[0]
    assert np.array_equal(s["idx"], nz)
    dd = d[nz]
    assert np.array_equal(s["A"], np.maximum(dd, 0))
    assert np.array_equal(s["F"], np.maximum(dd, 0) - dd)
    assert np.array_equal(s["kind"], np.where(dd > 0, 1, -1))
    py = tr.is_python[nz] != 0
    assert np.array_equal(s["A_py"], np.where(py, np.maximum(dd, 0), 0))
    assert np.array_equal(s["F_py"], np.where(py, np.maximum(-dd, 0), 0))
