"""CPU oracle for Scalene's memory-sampling path (arXiv 2212.07597, Section 3).

TEST INFRASTRUCTURE ONLY: this package is the plain sequential reference that
the CUDA library is checked against.  Only tests/, ``__graft_entry__.smoke()``
and bench.py's cpu_baseline / reference leg may import it; the library itself
never does, and this package imports nothing from the library.

Every function of the C core (scl_oracle.c) follows the steps of Sections
3.2 (threshold sampler), 3.3 (samples, attribution, footprint), 3.4 (leak
detector and score) and 3.5 (copy volume) in the paper's order.  The pins
that tie it to the paper live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SAMPLE_DTYPE = np.dtype([
    ("idx", "<u8"), ("A", "<i8"), ("F", "<i8"), ("A_py", "<i8"), ("F_py", "<i8"),
    ("footprint", "<i8"), ("line", "<u4"), ("kind", "i1"), ("is_python", "u1"),
    ("is_hwm", "u1"), ("pad", "u1"),
])
LINE_DTYPE = np.dtype([
    ("n_growth", "<u8"), ("n_shrink", "<u8"), ("A", "<i8"), ("F", "<i8"),
    ("A_py", "<i8"), ("F_py", "<i8"), ("net", "<i8"), ("mallocs", "<u8"), ("frees", "<u8"),
    ("copy_samples", "<u8", (2,)), ("copy_bytes", "<u8", (2,)),
])


class _Config(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_int64), ("copy_threshold", ctypes.c_uint64),
                ("copy_phase", ctypes.c_uint64), ("initial_footprint", ctypes.c_int64),
                ("n_lines", ctypes.c_uint32), ("leak_rule", ctypes.c_uint32)]


class _State(ctypes.Structure):
    _fields_ = [("cfg", _Config),
                ("c", ctypes.c_int64), ("A", ctypes.c_int64), ("F", ctypes.c_int64),
                ("A_py", ctypes.c_int64), ("F_py", ctypes.c_int64),
                ("footprint", ctypes.c_int64), ("hwm", ctypes.c_int64),
                ("tracked_valid", ctypes.c_int32), ("tracked_reclaimed", ctypes.c_int32),
                ("tracked_addr", ctypes.c_uint64), ("tracked_idx", ctypes.c_uint64),
                ("tracked_line", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("n_events", ctypes.c_uint64), ("n_copies", ctypes.c_uint64),
                ("copy_counter", ctypes.c_uint64),
                ("lines", ctypes.c_void_p), ("samples", ctypes.c_void_p),
                ("n_samples", ctypes.c_uint64), ("cap_samples", ctypes.c_uint64)]


assert SAMPLE_DTYPE.itemsize == 56 and LINE_DTYPE.itemsize == 104


def compile_source(src: str, out: str) -> str:
    """gcc a single oracle C source (with scl_oracle.h beside this file) into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-I", _HERE, "-o", tmp, src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile scl_oracle.c into liboracle.so next to it (plain C, gcc -O2)."""
    src = os.path.join(_HERE, "scl_oracle.c")
    hdr = os.path.join(_HERE, "scl_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    return compile_source(src, _SO)


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.orc_init.argtypes = [ctypes.POINTER(_State), ctypes.POINTER(_Config)]
    lib.orc_init.restype = ctypes.c_int
    lib.orc_free.argtypes = [ctypes.POINTER(_State)]
    lib.orc_replay_events.argtypes = [ctypes.POINTER(_State), P, P, P, P, ctypes.c_uint64]
    lib.orc_replay_events.restype = ctypes.c_int
    lib.orc_replay_copies.argtypes = [ctypes.POINTER(_State), P, P, P, ctypes.c_uint64]
    lib.orc_replay_copies.restype = ctypes.c_int
    lib.orc_leak_score.argtypes = [ctypes.POINTER(_State), ctypes.c_uint32,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.orc_rate_samples.argtypes = [P, P, P, ctypes.c_uint64, P, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_uint32, P, P]
    lib.orc_rate_samples.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = _bind(_SO)
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, dtype) -> int:
    assert a.dtype == np.dtype(dtype) and a.flags.c_contiguous, (a.dtype, dtype)
    return a.ctypes.data


class Oracle:
    """Resident per-trace state of the sequential replay; events may be fed in pieces."""

    def __init__(self, threshold: int, copy_threshold: int | None = None, copy_phase: int = 0,
                 initial_footprint: int = 0, n_lines: int = 256, leak_rule: int = 0, lib_path: str | None = None):
        self._lib = _load() if lib_path is None else _bind(lib_path)
        if copy_threshold is None:
            copy_threshold = 2 * threshold
        cfg = _Config(threshold, copy_threshold, copy_phase, initial_footprint, n_lines, leak_rule)
        self._st = _State()
        rc = self._lib.orc_init(ctypes.byref(self._st), ctypes.byref(cfg))
        if rc:
            raise ValueError(f"orc_init failed ({rc})")
        self.n_lines = n_lines
        self.initial_footprint = initial_footprint

    def __del__(self):
        lib = getattr(self, "_lib", None)
        if lib is not None and getattr(self, "_st", None) is not None:
            lib.orc_free(ctypes.byref(self._st))
            self._st = None

    def replay_events(self, delta, addr, line, is_python) -> None:
        delta = np.ascontiguousarray(delta, dtype=np.int64)
        addr = np.ascontiguousarray(addr, dtype=np.uint64)
        line = np.ascontiguousarray(line, dtype=np.uint32)
        is_python = np.ascontiguousarray(is_python, dtype=np.uint8)
        n = len(delta)
        assert len(addr) == n and len(line) == n and len(is_python) == n
        rc = self._lib.orc_replay_events(ctypes.byref(self._st), _ptr(delta, np.int64), _ptr(addr, np.uint64),
                                         _ptr(line, np.uint32), _ptr(is_python, np.uint8), n)
        if rc:
            raise ValueError({-1: "line id out of range", -2: "out of memory", -3: "int64 overflow"}.get(rc, rc))

    def replay_copies(self, size, line, is_python) -> None:
        size = np.ascontiguousarray(size, dtype=np.uint64)
        line = np.ascontiguousarray(line, dtype=np.uint32)
        is_python = np.ascontiguousarray(is_python, dtype=np.uint8)
        rc = self._lib.orc_replay_copies(ctypes.byref(self._st), _ptr(size, np.uint64), _ptr(line, np.uint32),
                                         _ptr(is_python, np.uint8), len(size))
        if rc:
            raise ValueError({-1: "line id out of range", -3: "uint64 overflow"}.get(rc, rc))

    def samples(self) -> np.ndarray:
        n = self._st.n_samples
        if n == 0:
            return np.zeros(0, SAMPLE_DTYPE)
        buf = (ctypes.c_char * (n * SAMPLE_DTYPE.itemsize)).from_address(self._st.samples)
        return np.frombuffer(buf, dtype=SAMPLE_DTYPE).copy()

    def lines(self) -> np.ndarray:
        buf = (ctypes.c_char * (self.n_lines * LINE_DTYPE.itemsize)).from_address(self._st.lines)
        return np.frombuffer(buf, dtype=LINE_DTYPE).copy()

    def leak_scores(self) -> tuple[np.ndarray, np.ndarray]:
        num = np.zeros(self.n_lines, np.int64)
        den = np.zeros(self.n_lines, np.int64)
        a, b = ctypes.c_int64(), ctypes.c_int64()
        for l in range(self.n_lines):
            self._lib.orc_leak_score(ctypes.byref(self._st), l, ctypes.byref(a), ctypes.byref(b))
            num[l], den[l] = a.value, b.value
        return num, den

    def leak_report(self) -> list[dict]:
        """Section 3.4's report filter, per line: reported when the leak likelihood exceeds
        95% and the trace's memory grew by at least 1%; leak rate = bytes allocated in the
        line's sample windows per elapsed event (readings: growth = footprint - F0 against
        the high-water mark; time = events)."""
        lines = self.lines()
        num, den = self.leak_scores()
        st = self.state()
        hwm, fp, n_ev = int(st["hwm"]), int(st["footprint"]), int(st["n_events"])
        growth = hwm > 0 and 100 * (fp - self.initial_footprint) >= hwm
        rows = []
        for l in range(self.n_lines):
            likely = 20 * int(num[l]) > 19 * int(den[l])        # likelihood = num / den > 0.95
            rows.append(dict(line=l, likely=likely, growth=growth, reported=likely and growth,
                             mallocs=int(lines["mallocs"][l]), frees=int(lines["frees"][l]), num=int(num[l]),
                             den=int(den[l]), rate_num=int(lines["A"][l]), rate_den=n_ev))
        return rows

    def state(self) -> dict:
        s = self._st
        return dict(c=s.c, A=s.A, F=s.F, A_py=s.A_py, F_py=s.F_py, footprint=s.footprint, hwm=s.hwm,
                    tracked_valid=s.tracked_valid, tracked_reclaimed=s.tracked_reclaimed,
                    tracked_addr=s.tracked_addr, tracked_line=s.tracked_line, tracked_idx=s.tracked_idx,
                    n_events=s.n_events, n_copies=s.n_copies, copy_counter=s.copy_counter)


def rate_samples(delta, line, is_python, gaps, consumed=0, n_lines=256, lib_path=None):
    """Rate-based sampling (Section 3.2's baseline) over one event stream: returns the
    per-(line, flag) sample counts [n_lines, 2] and the state (samples, gaps used,
    bytes of the next gap consumed, flags)."""
    lib = _bind(lib_path) if lib_path else _load()
    delta = np.ascontiguousarray(delta, dtype=np.int64)
    line = np.ascontiguousarray(line, dtype=np.uint32)
    is_python = np.ascontiguousarray(is_python, dtype=np.uint8)
    gaps = np.ascontiguousarray(gaps, dtype=np.uint64)
    counts = np.zeros(2 * n_lines, np.uint64)
    state = np.zeros(4, np.uint64)
    lib.orc_rate_samples(_ptr(delta, np.int64), _ptr(line, np.uint32), _ptr(is_python, np.uint8), len(delta),
                         _ptr(gaps, np.uint64), len(gaps), int(consumed), n_lines, counts.ctypes.data,
                         state.ctypes.data)
    return counts.reshape(n_lines, 2), state


def cpu_attribution(vtime, line, quantum, t_prev=0, n_lines=256):
    """Section 2.2: each CPU-timer interrupt adds the quantum q of the elapsed virtual time
    T to the interrupted line's Python time and the delay T - q to its native time
    (reading: python += min(T, q), native += T - min(T, q)).  Returns (python, native,
    flags) as in the library (1: time went backwards, 2: line id >= n_lines)."""
    vtime = np.asarray(vtime, dtype=np.int64)
    line = np.asarray(line, dtype=np.uint32)
    prev = np.concatenate([[t_prev], vtime[:-1]]).astype(np.int64) if len(vtime) else np.zeros(0, np.int64)
    T = vtime - prev
    bad_t = T < 0
    bad_l = line >= n_lines
    ok = ~bad_t & ~bad_l
    p = np.minimum(T, quantum)
    py = np.zeros(n_lines, np.int64)
    nat = np.zeros(n_lines, np.int64)
    np.add.at(py, line[ok], p[ok])
    np.add.at(nat, line[ok], (T - p)[ok])
    flags = (1 if bad_t.any() else 0) | (2 if bad_l.any() else 0)
    return py, nat, flags


def replay(delta, addr, line, is_python, threshold, n_lines=256, copies=None, **kw) -> Oracle:
    """One-shot helper: replay a whole trace (and optionally its memcpy stream)."""
    o = Oracle(threshold, n_lines=n_lines, **kw)
    o.replay_events(delta, addr, line, is_python)
    if copies is not None:
        o.replay_copies(*copies)
    return o
