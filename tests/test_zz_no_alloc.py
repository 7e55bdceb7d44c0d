"""The allocation-free copy-volume entry point agrees with the regular replay entry point.

scl_copy_volume_noalloc serves callers that must not allocate device memory (code
inside an allocation hook, processes whose device memory belongs to a caching
allocator or a quota, latency-bound callers).  It keeps its only scratch in a static
device array shared by every call, so this test makes two calls in a row on
different memcpy streams, each checked against scl_replay_batch on a trace holding
only those memcpys.  All values are integers: the comparison is exact.
"""
import numpy as np
import pytest

from paper_2212_07597_gb300 import scl
from paper_2212_07597_gb300 import tracegen as tg

pytestmark = pytest.mark.gpu


def _regular(cs, cl, cy, T, L, phase):
    ctx = scl.scl_replay_init(scl.config(threshold=T, n_lines=L, copy_phase=phase))
    seg, keep = scl.trace_segment(0, tg.Trace(np.zeros(0, np.int64), np.zeros(0, np.uint64),
                                              np.zeros(0, np.uint32), np.zeros(0, np.uint8), cs, cl, cy))
    scl.scl_replay_batch(ctx, [seg])
    rows = scl.scl_line_stats(ctx, 0)
    st = scl.scl_trace_state(ctx, 0)
    return rows["copy_samples"], rows["copy_bytes"], st["copy_counter"]


def test_noalloc_matches_replay_batch_on_two_calls_in_a_row():
    import torch
    T, L = 1_048_573, 64
    Tc = 2 * T
    cases = [(300_017, 31, 0), (123_457, 32, 777_777)]   # different sizes, seeds and starting counters
    samples = torch.empty(2 * L, dtype=torch.int64, device="cuda")
    byts = torch.empty(2 * L, dtype=torch.int64, device="cuda")
    state = torch.empty(3, dtype=torch.int64, device="cuda")
    for m, seed, phase in cases:
        cs, cl, cy = tg.copies(m, seed=seed, n_lines=L)
        d_cs, d_cl, d_cy = scl.to_device(cs, cl, cy)
        rc = scl.scl_copy_volume_noalloc(d_cs, d_cl, d_cy, Tc, phase, L, samples, byts, state)
        assert rc == scl.SCL_OK
        torch.cuda.synchronize()
        got_s = samples.cpu().numpy().view(np.uint64).reshape(L, 2)
        got_b = byts.cpu().numpy().view(np.uint64).reshape(L, 2)
        got_st = state.cpu().numpy().view(np.uint64)
        want_s, want_b, want_counter = _regular(cs, cl, cy, T, L, phase)
        assert np.array_equal(got_s, want_s)
        assert np.array_equal(got_b, want_b)
        assert int(got_st[0]) == want_counter and int(got_st[1]) == 0 and int(got_st[2]) == 0
        assert int(got_s.sum()) > 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    too_many = 16384 * 4096 + 1
    rc = scl.scl_copy_volume_noalloc(dummy, dummy, dummy, 2_097_146, 0, 4, dummy, dummy, dummy, m=too_many)
    assert rc == scl.SCL_EINVAL
