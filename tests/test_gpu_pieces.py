"""GPU parity of the exact replay cut into pieces (k_final), against the CPU oracle, bit-exact.

A sketched unit whose true run has a reset list is replayed as pieces that start after a
listed reset (counter 0, window empty) and end at the first listed reset past the next
multiple of piece_events.  A piece derives its mark and tracked block from the listed growth
samples before it, and leaves to a later pass the frees it sees of blocks tracked by an
earlier piece's sample or of the block tracked entering the unit.  Small pieces put many cuts
in every unit, so each of those paths runs many times here.
"""
import pytest

from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg
from tests.gpu_util import assert_same, gpu_ctx, oracle_of, replay

pytestmark = pytest.mark.gpu
T0 = tg.T_PLAIN


def _ctx(T, unit, piece, fixup=0, **kw):
    ctx = gpu_ctx(T, **kw)
    scl.scl_tuning_set(ctx, unit, 16, 0, 14, 0, fixup, piece)
    assert scl.scl_tuning_get(ctx).piece_events == piece
    return ctx


@pytest.mark.parametrize("piece", [256, 1024, 8192])
def test_plain_trace_cut_into_pieces(piece):
    tr = tg.plain_trace(400_003, seed=21, leak_lines=(0, 2))
    ctx = _ctx(1_048_573, 65536, piece)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


@pytest.mark.parametrize("piece", [256, 2048])
def test_free_heavy_address_reuse_in_pieces(piece):
    # frees of tracked blocks in later pieces (LIFO reuse puts the same address back often)
    tr = tg.plain_trace(300_000, seed=22, p_malloc=0.3, addr_reuse=True)
    ctx = _ctx(1_048_573, 32768, piece)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, 1_048_573))


def test_long_trace_pieces_at_the_default_threshold():
    tr = tg.long_trace(1 << 22, seed=3)
    ctx = _ctx(T0, 262144, 4096, log_cap=1 << 18)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T0))


@pytest.mark.parametrize("T", tg.SWEEP_THRESHOLDS)
def test_sweep_families_in_pieces(T):
    n = 120_000
    trs = [tg.sweep_trace(i, T, n=n) for i in range(8)]
    shift = 0 if T == 1 else 4
    ctx = _ctx(T, 16384, 512, max_traces=len(trs), shift=shift, log_cap=n + 1)
    keep = replay(ctx, list(enumerate(trs)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, T))


def test_many_traces_pieces_and_segments_across_calls():
    lens = [1, 700, 5000, 77_777, 300_000, 500_001]
    trs = [tg.plain_trace(n, seed=23, trace=i, n_lines=64) for i, n in enumerate(lens)]
    ctx = _ctx(1_048_573, 32768, 1024, n_lines=64, max_traces=len(lens))
    keep = []
    half = [tr.slice(0, tr.n // 2, 0, len(tr.csize) // 2) for tr in trs]
    rest = [tr.slice(tr.n // 2, tr.n, len(tr.csize) // 2, len(tr.csize)) for tr in trs]
    keep += replay(ctx, list(enumerate(half)))
    keep += replay(ctx, list(enumerate(rest)))
    for i, tr in enumerate(trs):
        assert_same(ctx, i, oracle_of(tr, 1_048_573, n_lines=64))


def test_search_fixup_ignores_the_piece_length():
    # without reset lists every unit is replayed whole by its first piece
    tr = tg.plain_trace(250_000, seed=24, leak_lines=(1,))
    ctx = _ctx(T0, 32768, 256, fixup=1)
    keep = replay(ctx, [(0, tr)])
    assert_same(ctx, 0, oracle_of(tr, T0))
