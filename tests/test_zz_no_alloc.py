"""The allocation-free copy-volume entry point agrees with the regular replay entry point
and with the oracle.

scl_copy_volume_noalloc serves callers that must not allocate device memory (code
inside an allocation hook, processes whose device memory belongs to a caching
allocator or a quota, latency-bound callers).  It keeps its only scratch in a static
device array shared by every call, so the first test makes two calls in a row on
different memcpy streams, each checked against scl_replay_batch on a trace holding
only those memcpys.  The others check it against the sequential oracle (Section 3.5),
including memcpys whose line id is out of range and byte counts that pass 2^64.  All
values are integers: every comparison is exact.
"""
import numpy as np
import pytest

import oracle
from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg

pytestmark = pytest.mark.gpu

U64 = np.uint64


def _regular(cs, cl, cy, T, L, phase):
    ctx = scl.scl_replay_init(scl.config(threshold=T, n_lines=L, copy_phase=phase))
    seg, keep = scl.trace_segment(0, tg.Trace(np.zeros(0, np.int64), np.zeros(0, np.uint64),
                                              np.zeros(0, np.uint32), np.zeros(0, np.uint8), cs, cl, cy))
    scl.scl_replay_batch(ctx, [seg])
    rows = scl.scl_line_stats(ctx, 0)
    st = scl.scl_trace_state(ctx, 0)
    return rows["copy_samples"], rows["copy_bytes"], st["copy_counter"]


def _noalloc(cs, cl, cy, Tc, counter_in, L):
    """One call; returns (samples [L, 2], bytes [L, 2], state [3]) as uint64."""
    import torch
    samples = torch.full((2 * L,), -1, dtype=torch.int64, device="cuda")   # the call must clear them
    byts = torch.full((2 * L,), -1, dtype=torch.int64, device="cuda")
    state = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    d_cs, d_cl, d_cy = scl.to_device(cs, cl, cy)
    rc = scl.scl_copy_volume_noalloc(d_cs, d_cl, d_cy, Tc, counter_in, L, samples, byts, state)
    assert rc == scl.SCL_OK
    torch.cuda.synchronize()
    return (samples.cpu().numpy().view(U64).reshape(L, 2), byts.cpu().numpy().view(U64).reshape(L, 2),
            state.cpu().numpy().view(U64))


def _oracle(cs, cl, cy, Tc, counter_in, L):
    o = oracle.Oracle(Tc, copy_threshold=Tc, copy_phase=counter_in, n_lines=L)
    o.replay_copies(cs, cl, cy)
    rows = o.lines()
    return rows["copy_samples"], rows["copy_bytes"], o.state()["copy_counter"]


def test_noalloc_matches_replay_batch_on_two_calls_in_a_row():
    T, L = 1_048_573, 64
    Tc = 2 * T
    cases = [(300_017, 31, 0), (123_457, 32, 777_777)]   # different sizes, seeds and starting counters
    for m, seed, phase in cases:
        cs, cl, cy = tg.copies(m, seed=seed, n_lines=L)
        got_s, got_b, got_st = _noalloc(cs, cl, cy, Tc, phase, L)
        want_s, want_b, want_counter = _regular(cs, cl, cy, T, L, phase)
        assert np.array_equal(got_s, want_s)
        assert np.array_equal(got_b, want_b)
        assert int(got_st[0]) == want_counter and int(got_st[1]) == 0 and int(got_st[2]) == 0
        assert int(got_s.sum()) > 0


@pytest.mark.parametrize("m,Tc,phase", [(1, 7, 3), (4095, 1, 0), (4097, 2_097_146, 5), (50_000, 123_456_789, 0),
                                        (70_001, 2_097_146, 2_097_145)])
def test_noalloc_matches_oracle(m, Tc, phase):
    L = 100
    cs, cl, cy = tg.copies(m, seed=m, n_lines=L)
    got_s, got_b, got_st = _noalloc(cs, cl, cy, Tc, phase, L)
    want_s, want_b, want_counter = _oracle(cs, cl, cy, Tc, phase, L)
    assert np.array_equal(got_s, want_s) and np.array_equal(got_b, want_b)
    assert int(got_st[0]) == want_counter and int(got_st[1]) == 0 and int(got_st[2]) == 0


def test_noalloc_counts_and_skips_out_of_range_lines():
    """Memcpys with line >= n_lines still move the counter; the ones that take a sample are
    counted in state[1] and their samples are dropped.  The oracle replays the same stream
    with those memcpys on a spare line L, one memcpy at a time."""
    L, Tc, m = 40, 3_000_017, 9_001
    cs, cl, cy = tg.copies(m, seed=5, n_lines=L)
    bad = np.arange(m) % 17 == 3
    cl_bad = cl.copy()
    cl_bad[bad] = L + 7 + (np.arange(m)[bad] % 5)
    got_s, got_b, got_st = _noalloc(cs, cl_bad, cy, Tc, 0, L)
    o = oracle.Oracle(Tc, copy_threshold=Tc, n_lines=L + 1)
    spare = cl.copy()
    spare[bad] = L
    skipped = 0
    for j in range(m):
        before = int(o.lines()["copy_samples"][L].sum())
        o.replay_copies(cs[j:j + 1], spare[j:j + 1], cy[j:j + 1])
        skipped += int(o.lines()["copy_samples"][L].sum()) > before
    rows = o.lines()
    assert skipped > 0
    assert np.array_equal(got_s, rows["copy_samples"][:L]) and np.array_equal(got_b, rows["copy_bytes"][:L])
    assert int(got_st[0]) == o.state()["copy_counter"]
    assert int(got_st[1]) == skipped and int(got_st[2]) == 0


def test_noalloc_flags_a_byte_count_past_2_64():
    """Two 2^63-byte memcpys on neighbouring threads of one tile, and four 2^62-byte ones in
    four tiles (the carry then happens in the scan over tiles): the flag is set and the
    outputs stay cleared.  A stream that ends exactly at 2^64 - 1 bytes is not flagged and
    matches the oracle."""
    L, Tc = 8, 2_097_146
    for sizes, positions in (([1 << 63, 1 << 63], [0, 1]),
                             ([1 << 62] * 4, [0, 4096, 8192, 3 * 4096 + 17])):
        m = 4 * 4096 + 100
        cs = np.full(m, 1000, U64)
        for s, p in zip(sizes, positions):
            cs[p] = U64(s)
        cl = (np.arange(m) % L).astype(np.uint32)
        cy = (np.arange(m) % 2).astype(np.uint8)
        got_s, got_b, got_st = _noalloc(cs, cl, cy, Tc, 0, L)
        assert int(got_st[2]) == 1
        assert not got_s.any() and not got_b.any()
    cs = np.array([1 << 63, (1 << 63) - 1 - 3000, 1000, 2000], U64)
    cl = np.array([1, 2, 3, 1], np.uint32)
    cy = np.array([0, 1, 1, 0], np.uint8)
    got_s, got_b, got_st = _noalloc(cs, cl, cy, Tc, 0, L)
    want_s, want_b, want_counter = _oracle(cs, cl, cy, Tc, 0, L)
    assert int(got_st[2]) == 0 and int(got_st[0]) == want_counter
    assert np.array_equal(got_s, want_s) and np.array_equal(got_b, want_b)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    too_many = 16384 * 4096 + 1
    rc = scl.scl_copy_volume_noalloc(dummy, dummy, dummy, 2_097_146, 0, 4, dummy, dummy, dummy, m=too_many)
    assert rc == scl.SCL_EINVAL
