"""Seeded synthetic trace workloads (Python side of tracegen.c).

The five workloads below stand in for the allocator activity of the profiled
programs of the paper's evaluation (Section 6; its pyperformance traces are not
available).  Sizes, mixes and distributions are those listed for each workload;
none of this module does sampler, footprint or leak arithmetic.

  plain_1m     1,000,000 events, 60% mallocs of 16 B-1 MiB (log-uniform), frees of a
               uniformly chosen live block, Zipf(1.1) lines over 256 ids, python p=0.7,
               100,000 memcpys of 1 KiB-64 MiB.  T = 10,485,767.
  long_256m    2^28 events, same generators, plus 5 leaking lines (ids 0-4; their mallocs
               are 4-256 KiB and stay live with p=0.9) and a +2 GiB ramp of 2,048 never
               freed 1 MiB mallocs on line 255; 2^28/10 memcpys.
  batched      4,096 traces of log-uniform 10k-4M events, 4,096 lines; 41 traces leak.
  sweep        1,024 traces x 1M events in four families (big 4 GiB allocations,
               adversarial +-(T-1), malloc-only 4 KiB, 70% frees) at T in
               {1; 1,048,573; 10,485,767; 104,857,601}.
  serving      512 processes, 64k-event segments, 1,024 lines, 10% leak, Poisson arrivals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtracegen.so")
_lock = threading.Lock()
_lib = None

T_PLAIN = 10_485_767                      # prime just above 10 MiB (Section 3.2)
SWEEP_THRESHOLDS = (1, 1_048_573, 10_485_767, 104_857_601)
KIB, MIB, GIB = 1 << 10, 1 << 20, 1 << 30


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("n_lines", ctypes.c_uint32), ("addr_reuse", ctypes.c_uint32),
                ("p_malloc", ctypes.c_double), ("p_python", ctypes.c_double), ("zipf_s", ctypes.c_double),
                ("size_lo", ctypes.c_uint64), ("size_hi", ctypes.c_uint64),
                ("n_leak_lines", ctypes.c_uint32), ("leak_lines", ctypes.c_uint32 * 16),
                ("p_leak_unfreed", ctypes.c_double), ("leak_lo", ctypes.c_uint64), ("leak_hi", ctypes.c_uint64),
                ("ramp_count", ctypes.c_uint64), ("ramp_size", ctypes.c_uint64), ("ramp_line", ctypes.c_uint32),
                ("big_count", ctypes.c_uint64), ("big_size", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "tracegen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-Wall", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P, U64, U32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
            lib.tg_events.argtypes = [ctypes.POINTER(_Params), U64, U64, P, P, P, P]
            lib.tg_copies.argtypes = [U64, U32, ctypes.c_double, ctypes.c_double, U64, U64, U64, U64, P, P, P]
            lib.tg_adversarial.argtypes = [U64, ctypes.c_int64, U64, U32, U64, U64, P, P, P, P]
            lib.tg_constant.argtypes = [U64, ctypes.c_int64, U32, U64, U64, P, P, P, P]
            lib.tg_lengths.argtypes = [U64, U64, U64, U64, P]
            lib.tg_arrivals.argtypes = [U64, ctypes.c_double, U64, P]
            lib.tg_gaps.argtypes = [U64, ctypes.c_double, U64, P]
            lib.tg_det_exp.argtypes = [ctypes.c_double]
            lib.tg_det_exp.restype = ctypes.c_double
            lib.tg_det_log.argtypes = [ctypes.c_double]
            lib.tg_det_log.restype = ctypes.c_double
            for f in ("tg_events", "tg_copies", "tg_adversarial", "tg_constant", "tg_lengths", "tg_arrivals",
                      "tg_gaps"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Trace:
    """One trace in SoA form (host numpy arrays), plus its memcpy stream."""
    delta: np.ndarray
    addr: np.ndarray
    line: np.ndarray
    is_python: np.ndarray
    csize: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint64))
    cline: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint32))
    cpy: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))

    @property
    def n(self) -> int:
        return len(self.delta)

    def slice(self, a: int, b: int, ca: int = 0, cb: int = 0) -> "Trace":
        return Trace(self.delta[a:b], self.addr[a:b], self.line[a:b], self.is_python[a:b],
                     self.csize[ca:cb], self.cline[ca:cb], self.cpy[ca:cb])


def _alloc(n):
    return (np.empty(n, np.int64), np.empty(n, np.uint64), np.empty(n, np.uint32), np.empty(n, np.uint8))


def events(n: int, seed: int = 0, trace: int = 0, n_lines: int = 256, p_malloc: float = 0.6,
           p_python: float = 0.7, zipf_s: float = 1.1, size_lo: int = 16, size_hi: int = MIB,
           leak_lines=(), p_leak_unfreed: float = 0.9, leak_lo: int = 4 * KIB, leak_hi: int = 256 * KIB,
           ramp_count: int = 0, ramp_size: int = MIB, ramp_line: int = 255,
           big_count: int = 0, big_size: int = 4 * GIB, addr_reuse: bool = False):
    p = _Params()
    p.n, p.n_lines, p.addr_reuse = n, n_lines, int(addr_reuse)
    p.p_malloc, p.p_python, p.zipf_s = p_malloc, p_python, zipf_s
    p.size_lo, p.size_hi = size_lo, size_hi
    p.n_leak_lines = len(leak_lines)
    for i, l in enumerate(leak_lines):
        p.leak_lines[i] = l
    p.p_leak_unfreed, p.leak_lo, p.leak_hi = p_leak_unfreed, leak_lo, leak_hi
    p.ramp_count, p.ramp_size, p.ramp_line = ramp_count, ramp_size, ramp_line
    p.big_count, p.big_size = big_count, big_size
    d, a, l, y = _alloc(n)
    rc = _load().tg_events(ctypes.byref(p), seed, trace, d.ctypes.data, a.ctypes.data, l.ctypes.data, y.ctypes.data)
    if rc:
        raise RuntimeError("tg_events failed")
    return d, a, l, y


def copies(m: int, seed: int = 0, trace: int = 0, n_lines: int = 256, zipf_s: float = 1.1,
           p_python: float = 0.7, lo: int = KIB, hi: int = 64 * MIB):
    s, l, y = np.empty(m, np.uint64), np.empty(m, np.uint32), np.empty(m, np.uint8)
    rc = _load().tg_copies(m, n_lines, zipf_s, p_python, lo, hi, seed, trace, s.ctypes.data, l.ctypes.data,
                           y.ctypes.data)
    if rc:
        raise RuntimeError("tg_copies failed")
    return s, l, y


def adversarial(n: int, T: int, period: int = 65536, n_lines: int = 256, seed: int = 0, trace: int = 0):
    d, a, l, y = _alloc(n)
    rc = _load().tg_adversarial(n, T, period, n_lines, seed, trace, d.ctypes.data, a.ctypes.data,
                                l.ctypes.data, y.ctypes.data)
    if rc:
        raise RuntimeError("tg_adversarial failed")
    return d, a, l, y


def constant(n: int, size: int, n_lines: int = 256, seed: int = 0, trace: int = 0):
    d, a, l, y = _alloc(n)
    rc = _load().tg_constant(n, size, n_lines, seed, trace, d.ctypes.data, a.ctypes.data, l.ctypes.data,
                             y.ctypes.data)
    if rc:
        raise RuntimeError("tg_constant failed")
    return d, a, l, y


def lengths(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    out = np.empty(count, np.uint64)
    if _load().tg_lengths(count, lo, hi, seed, out.ctypes.data):
        raise RuntimeError("tg_lengths failed")
    return out


def arrivals_ns(count: int, mean_gap_ns: float, seed: int = 0) -> np.ndarray:
    out = np.empty(count, np.uint64)
    _load().tg_arrivals(count, mean_gap_ns, seed, out.ctypes.data)
    return out


def gaps(count: int, mean: float, seed: int = 0) -> np.ndarray:
    """Geometric gaps (>= 1) between the sampled bytes of a rate-based sampler, mean `mean`."""
    out = np.empty(count, np.uint64)
    if _load().tg_gaps(count, float(mean), seed, out.ctypes.data):
        raise ValueError("mean must be >= 1")
    return out


# ---------------------------------------------------------------- workloads

def plain_trace(n: int = 1_000_000, m: int | None = None, seed: int = 0, trace: int = 0,
                n_lines: int = 256, **kw) -> Trace:
    """The 1M-event plain workload (and its shape at any n): memcpys are n/10 by default."""
    if m is None:
        m = n // 10
    d, a, l, y = events(n, seed=seed, trace=trace, n_lines=n_lines, **kw)
    cs, cl, cy = copies(m, seed=seed, trace=trace, n_lines=n_lines)
    return Trace(d, a, l, y, cs, cl, cy)


LEAK_LINES = (0, 1, 2, 3, 4)


def long_trace(n: int = 1 << 28, m: int | None = None, seed: int = 1, trace: int = 0,
               n_lines: int = 256) -> Trace:
    """The single long trace: plain generators + 5 leaking lines + a 2 GiB ramp on line 255."""
    return plain_trace(n, m, seed=seed, trace=trace, n_lines=n_lines, leak_lines=LEAK_LINES,
                       ramp_count=2048, ramp_size=MIB, ramp_line=n_lines - 1)


def batched_lengths(count: int = 4096, lo: int = 10_000, hi: int = 4_000_000, seed: int = 2) -> np.ndarray:
    return lengths(count, lo, hi, seed)


def batched_trace(i: int, n: int, seed: int = 2, n_lines: int = 4096, leak_every: int = 100) -> Trace:
    """Trace i of the batched workload; every leak_every-th trace carries leak injection."""
    kw = {}
    if leak_every and i % leak_every == 0:
        kw = dict(leak_lines=LEAK_LINES, ramp_count=max(1, n // 131072), ramp_size=MIB, ramp_line=n_lines - 1)
    return plain_trace(n, seed=seed, trace=i, n_lines=n_lines, **kw)


def sweep_trace(i: int, T: int, n: int = 1_000_000, seed: int = 3, n_lines: int = 256) -> Trace:
    """Trace i of the threshold sweep: family = i % 4."""
    fam = i % 4
    if fam == 0:
        tr = plain_trace(n, seed=seed, trace=i, n_lines=n_lines, big_count=4, big_size=4 * GIB)
    elif fam == 1:
        if T < 2:
            d, a, l, y = constant(n, 1, n_lines, seed, i)
            d[1::2] = -1
        else:
            d, a, l, y = adversarial(n, T, 65536, n_lines, seed, i)
        cs, cl, cy = copies(n // 10, seed=seed, trace=i, n_lines=n_lines)
        tr = Trace(d, a, l, y, cs, cl, cy)
    elif fam == 2:
        d, a, l, y = constant(n, 4 * KIB, n_lines, seed, i)
        cs, cl, cy = copies(n // 10, seed=seed, trace=i, n_lines=n_lines)
        tr = Trace(d, a, l, y, cs, cl, cy)
    else:
        tr = plain_trace(n, seed=seed, trace=i, n_lines=n_lines, p_malloc=0.3, addr_reuse=True)
    return tr


def serving_segment(process: int, k: int, seg_len: int = 65536, seed: int = 4, n_lines: int = 1024,
                    leak_every: int = 10) -> Trace:
    """Segment k of process `process`.  Each process is one long trace cut into seg_len pieces;
    generating piece k regenerates the prefix, so callers should use serving_process()."""
    tr = serving_process(process, (k + 1) * seg_len, seed, n_lines, leak_every)
    return tr.slice(k * seg_len, (k + 1) * seg_len, k * seg_len // 10, (k + 1) * seg_len // 10)


def serving_process(process: int, n: int, seed: int = 4, n_lines: int = 1024, leak_every: int = 10) -> Trace:
    kw = {}
    if leak_every and process % leak_every == 0:
        kw = dict(leak_lines=LEAK_LINES)
    return plain_trace(n, seed=seed, trace=process, n_lines=n_lines, **kw)
