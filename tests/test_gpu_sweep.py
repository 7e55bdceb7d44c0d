"""GPU parity on the threshold sweep at full size and on mixed batches, with the default
configuration.

The sweep's four families (4 GiB mallocs, adversarial +-(T-1), malloc-only 4 KiB, 70%
frees with address reuse) run at 1M events each, at every threshold of the sweep, and
every sample record is compared with the oracle.  The default record budget is picked from
T, so T = 1 (every nonzero event samples) must replay without SCL_EOVERFLOW.  All outputs
are integers: the tolerance is zero.
"""
import numpy as np
import pytest

from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg
from tests.gpu_util import assert_same, oracle_of, replay

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T", tg.SWEEP_THRESHOLDS)
def test_sweep_families_full_size_default_config(T):
    n = 1_000_000
    trs = [tg.sweep_trace(i, T, n=n) for i in range(4)]
    ctx = scl.scl_replay_init(scl.config(threshold=T, n_lines=256, max_traces=4, sample_log_capacity=n + 1))
    keep = replay(ctx, list(enumerate(trs)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, T))


def test_crossing_search_fixup_strategy():
    # fix-up 1: the exact replay of every sketched unit searches its crossings instead of
    # following the reset list the sketch recorded
    T = 1_048_573
    tr = tg.plain_trace(600_001, seed=31, leak_lines=(0, 2))
    ctx = scl.scl_replay_init(scl.config(threshold=T, n_lines=256, sample_log_capacity=1 << 20))
    scl.scl_tuning_set(ctx, 32768, 16, 16384, 14, 0, 1)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T))
    assert scl.scl_batch_stats(ctx)["searched"] == scl.scl_batch_stats(ctx)["units"] - 1


@pytest.mark.parametrize("first", [0, 131072])
def test_mixed_batch_first_units_sketch_and_copy_tiles(first):
    # 96 traces of log-uniform lengths in one batch: whole short traces and long first units
    # replayed exactly, the rest sketched; memcpy tiles chained across each trace by look-back
    lens = tg.lengths(96, 3_000, 400_000, seed=5)
    trs = [tg.batched_trace(i, int(lens[i]), seed=6, n_lines=512, leak_every=7) for i in range(96)]
    ctx = scl.scl_replay_init(scl.config(threshold=1_048_573, n_lines=512, max_traces=96,
                                         sample_log_capacity=1 << 16))
    scl.scl_tuning_set(ctx, 16384, 12, 8192, 10, first, 0)
    keep = replay(ctx, list(enumerate(trs)))
    for i in (0, 1, 7, 14, int(np.argmax(lens)), int(np.argmin(lens)), 50, 95):
        assert_same(ctx, i, oracle_of(trs[i], 1_048_573, n_lines=512))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, 1_048_573, n_lines=512), samples=False)
    # the same batch again, continuing every trace (resident state carried over)
    keep2 = replay(ctx, list(enumerate(trs)))
    o = oracle_of(trs[3], 1_048_573, n_lines=512)
    o.replay_events(trs[3].delta, trs[3].addr, trs[3].line, trs[3].is_python)
    o.replay_copies(trs[3].csize, trs[3].cline, trs[3].cpy)
    assert_same(ctx, 3, o)
