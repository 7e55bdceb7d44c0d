"""Python binding of libscl (include/scl.h): argument marshalling only.

Every computation runs in the CUDA kernels of libscl.so; this module only turns
torch tensors / numpy arrays into the pointers and descriptors of the C ABI.
There is no CPU fallback: if libscl.so is missing or no CUDA device is present,
loading raises.

    from paper_2212_07597_gb300 import scl
    ctx = scl.scl_replay_init(scl.config(threshold=10_485_767, n_lines=256))
    scl.scl_replay_batch(ctx, [scl.segment(0, delta, addr, line, py, csize, cline, cpy)])
    stats = scl.scl_line_stats(ctx, 0)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libscl.so")

SCL_OK, SCL_EINVAL, SCL_ENOMEM, SCL_ECUDA, SCL_ETIMEOUT, SCL_EOVERFLOW, SCL_ERANGE = 0, -1, -2, -3, -4, -5, -6
SCL_ALL_TRACES = 0xFFFFFFFF
SCL_BUDGET_AUTO = 0xFFFFFFFF
_NAMES = {-1: "SCL_EINVAL", -2: "SCL_ENOMEM", -3: "SCL_ECUDA", -4: "SCL_ETIMEOUT", -5: "SCL_EOVERFLOW",
          -6: "SCL_ERANGE", -7: "SCL_EINTERNAL"}

# every symbol include/scl.h declares
EXPORTS = ("scl_config_default", "scl_replay_init", "scl_replay_free", "scl_last_error", "scl_replay_batch",
           "scl_replay_batch_host", "scl_sync", "scl_samples", "scl_line_stats", "scl_leak_scores",
           "scl_line_stats_range", "scl_leak_scores_range",
           "scl_trace_state", "scl_state_export", "scl_state_import", "scl_trace_reset", "scl_tuning_get",
           "scl_tuning_set", "scl_autotune", "scl_profile_enable", "scl_kernel_times", "scl_profile_reset",
           "scl_selftest_wait", "scl_copy_volume_noalloc", "scl_batch_stats", "scl_graph_enable", "scl_serve", "scl_rate_samples",
           "scl_leak_report", "scl_line_timeline", "scl_cpu_attribution")


class SclError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class scl_events(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_void_p), ("addr", ctypes.c_void_p), ("line", ctypes.c_void_p),
                ("is_python", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class scl_copies(ctypes.Structure):
    _fields_ = [("size", ctypes.c_void_p), ("line", ctypes.c_void_p), ("is_python", ctypes.c_void_p),
                ("n", ctypes.c_uint64)]


class scl_config(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_int64), ("copy_multiple", ctypes.c_uint32), ("n_lines", ctypes.c_uint32),
                ("copy_phase", ctypes.c_uint64), ("initial_footprint", ctypes.c_int64),
                ("max_traces", ctypes.c_uint32), ("leak_rule", ctypes.c_uint32), ("spin_limit", ctypes.c_uint64),
                ("sample_log_capacity", ctypes.c_uint64), ("sample_budget_shift", ctypes.c_uint32),
                ("unit_events", ctypes.c_uint32)]


class scl_segment(ctypes.Structure):
    _fields_ = [("trace_id", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("ev", scl_events),
                ("cp", scl_copies)]


class scl_request(ctypes.Structure):
    _fields_ = [("trace_id", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("arrival_ns", ctypes.c_uint64),
                ("ev", scl_events), ("cp", scl_copies)]


class scl_serve_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32), ("realtime", ctypes.c_uint32)]


class scl_serve_summary(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("events", ctypes.c_uint64),
                ("staging_bytes", ctypes.c_uint64), ("wall_s", ctypes.c_double)]


REQUEST_RESULT_DTYPE = np.dtype([("done_ns", "<u8"), ("latency_ns", "<u8"), ("batch", "<u4"),
                                 ("reserved", "<u4")])


class scl_tuning(ctypes.Structure):
    _fields_ = [("unit_events", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("ext_events", ctypes.c_uint32), ("final_warps", ctypes.c_uint32),
                ("first_events", ctypes.c_uint32), ("fixup", ctypes.c_uint32), ("piece_events", ctypes.c_uint32)]


SAMPLE_DTYPE = np.dtype([
    ("idx", "<u8"), ("A", "<i8"), ("F", "<i8"), ("A_py", "<i8"), ("F_py", "<i8"), ("footprint", "<i8"),
    ("line", "<u4"), ("kind", "i1"), ("is_python", "u1"), ("is_hwm", "u1"), ("reserved", "u1")])
LINE_STAT_DTYPE = np.dtype([
    ("n_growth", "<u8"), ("n_shrink", "<u8"), ("A", "<i8"), ("F", "<i8"), ("A_py", "<i8"), ("F_py", "<i8"),
    ("net", "<i8"), ("copy_samples", "<u8", (2,)), ("copy_bytes", "<u8", (2,))])
LEAK_DTYPE = np.dtype([("line", "<u4"), ("reserved", "<u4"), ("mallocs", "<u8"), ("frees", "<u8"),
                       ("num", "<i8"), ("den", "<i8")])
LEAK_REPORT_DTYPE = np.dtype([("line", "<u4"), ("reported", "u1"), ("likely", "u1"), ("growth", "u1"),
                              ("reserved", "u1"), ("mallocs", "<u8"), ("frees", "<u8"), ("num", "<i8"),
                              ("den", "<i8"), ("rate_num", "<i8"), ("rate_den", "<u8")])
TRACE_INFO_DTYPE = np.dtype([
    ("n_events", "<u8"), ("n_copies", "<u8"), ("n_samples", "<u8"), ("c", "<i8"), ("A", "<i8"), ("F", "<i8"),
    ("A_py", "<i8"), ("F_py", "<i8"), ("footprint", "<i8"), ("hwm", "<i8"), ("tracked_addr", "<u8"),
    ("tracked_idx", "<u8"), ("tracked_line", "<u4"), ("tracked_valid", "u1"), ("tracked_reclaimed", "u1"),
    ("reserved", "u1", (2,)), ("copy_counter", "<u8")])
assert SAMPLE_DTYPE.itemsize == 56 and LEAK_DTYPE.itemsize == 40 and LINE_STAT_DTYPE.itemsize == 88

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libscl.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2212_07597_gb300.build` "
                               "(the replay path has no CPU fallback)")
        lib = ctypes.CDLL(path)
        P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        sig = {
            "scl_config_default": ([ctypes.POINTER(scl_config)], I),
            "scl_replay_init": ([ctypes.POINTER(P), ctypes.POINTER(scl_config)], I),
            "scl_replay_free": ([P], None),
            "scl_last_error": ([P], ctypes.c_char_p),
            "scl_replay_batch": ([P, ctypes.POINTER(scl_segment), U32, P], I),
            "scl_replay_batch_host": ([P, ctypes.POINTER(scl_segment), U32, P], I),
            "scl_sync": ([P], I),
            "scl_samples": ([P, U32, P, U64, ctypes.POINTER(U64)], I),
            "scl_line_stats": ([P, U32, P, U32, ctypes.POINTER(U32)], I),
            "scl_leak_scores": ([P, U32, P, U32, ctypes.POINTER(U32)], I),
            "scl_line_stats_range": ([P, U32, U32, P, U64, ctypes.POINTER(U64)], I),
            "scl_leak_scores_range": ([P, U32, U32, P, U64, ctypes.POINTER(U64)], I),
            "scl_trace_state": ([P, U32, P], I),
            "scl_state_export": ([P, U32, P, U64, ctypes.POINTER(U64)], I),
            "scl_state_import": ([P, U32, P, U64], I),
            "scl_trace_reset": ([P, U32, P], I),
            "scl_tuning_get": ([P, ctypes.POINTER(scl_tuning)], I),
            "scl_tuning_set": ([P, ctypes.POINTER(scl_tuning)], I),
            "scl_autotune": ([P, ctypes.POINTER(scl_segment), U32, P, ctypes.POINTER(scl_tuning),
                              ctypes.POINTER(ctypes.c_double)], I),
            "scl_profile_enable": ([P, I], I),
            "scl_kernel_times": ([P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(U64), U32, ctypes.POINTER(U32)], I),
            "scl_profile_reset": ([P], I),
            "scl_selftest_wait": ([P, U64, P], I),
            "scl_batch_stats": ([P, P], I),
            "scl_graph_enable": ([P, I], I),
            "scl_serve": ([P, P, U32, P, P, P], I),
            "scl_rate_samples": ([P, P, P, P, U64, P, U64, U64, P, P, P], I),
            "scl_leak_report": ([P, U32, P, U32, P], I),
            "scl_line_timeline": ([P, U32, U32, P, P, U64, P], I),
            "scl_cpu_attribution": ([P, P, P, U64, ctypes.c_int64, ctypes.c_int64, P, P, P, P], I),
            "scl_copy_volume_noalloc": ([P, P, P, U64, U64, U64, U32, P, P, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


class Context:
    """Owns an scl_ctx*; freed with scl_replay_free."""

    def __init__(self, handle: int, cfg: scl_config):
        self.handle = handle
        self.cfg = cfg
        self._keep = []          # arrays referenced by in-flight asynchronous calls

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.scl_replay_free(self.handle)
            self.handle = None

    @property
    def as_parameter(self):
        return self.handle


def _check(ctx, rc: int):
    if rc != SCL_OK:
        msg = load().scl_last_error(ctx.handle if ctx is not None else None)
        raise SclError(rc, msg.decode() if msg else "")


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags.c_contiguous, "array must be C-contiguous"
    return x.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def config(**kw) -> scl_config:
    cfg = scl_config()
    load().scl_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


def segment(trace_id: int, delta=None, addr=None, line=None, is_python=None, csize=None, cline=None, cpy=None,
            n: int | None = None, m: int | None = None) -> scl_segment:
    """Descriptor of one segment; arrays are torch CUDA tensors (device) or numpy (host calls)."""
    s = scl_segment()
    s.trace_id = trace_id
    n = n if n is not None else (0 if delta is None else len(delta))
    m = m if m is not None else (0 if csize is None else len(csize))
    s.ev = scl_events(_ptr(delta), _ptr(addr), _ptr(line), _ptr(is_python), n)
    s.cp = scl_copies(_ptr(csize), _ptr(cline), _ptr(cpy), m)
    return s


def scl_replay_init(cfg: scl_config) -> Context:
    lib = load()
    h = ctypes.c_void_p()
    rc = lib.scl_replay_init(ctypes.byref(h), ctypes.byref(cfg))
    if rc != SCL_OK:
        raise SclError(rc, "scl_replay_init failed (invalid config or CUDA unavailable)")
    return Context(h.value, cfg)


def scl_replay_free(ctx: Context) -> None:
    if ctx.handle:
        load().scl_replay_free(ctx.handle)
        ctx.handle = None


def _segs(segs):
    arr = (scl_segment * max(1, len(segs)))(*segs)
    return arr


def scl_replay_batch(ctx: Context, segs, stream=None) -> None:
    arr = _segs(segs)
    _check(ctx, load().scl_replay_batch(ctx.handle, arr, len(segs), _stream(stream)))


def scl_replay_batch_host(ctx: Context, segs, stream=None) -> None:
    arr = _segs(segs)
    _check(ctx, load().scl_replay_batch_host(ctx.handle, arr, len(segs), _stream(stream)))


def scl_sync(ctx: Context) -> None:
    _check(ctx, load().scl_sync(ctx.handle))


def scl_samples(ctx: Context, trace: int, allow_truncated: bool = False) -> np.ndarray:
    lib = load()
    n = ctypes.c_uint64()
    rc = lib.scl_samples(ctx.handle, trace, None, 0, ctypes.byref(n))
    have = min(n.value, ctx.cfg.sample_log_capacity)
    if rc not in (SCL_OK, SCL_ERANGE, SCL_EOVERFLOW):
        _check(ctx, rc)
    out = np.zeros(have, SAMPLE_DTYPE)
    rc = lib.scl_samples(ctx.handle, trace, out.ctypes.data if have else None, have, ctypes.byref(n))
    if rc == SCL_EOVERFLOW and allow_truncated:
        return out
    _check(ctx, rc)
    return out


def scl_line_stats(ctx: Context, trace: int) -> np.ndarray:
    out = np.zeros(ctx.cfg.n_lines, LINE_STAT_DTYPE)
    n = ctypes.c_uint32()
    _check(ctx, load().scl_line_stats(ctx.handle, trace, out.ctypes.data, len(out), ctypes.byref(n)))
    return out


def scl_leak_scores(ctx: Context, trace: int) -> np.ndarray:
    out = np.zeros(ctx.cfg.n_lines, LEAK_DTYPE)
    n = ctypes.c_uint32()
    _check(ctx, load().scl_leak_scores(ctx.handle, trace, out.ctypes.data, len(out), ctypes.byref(n)))
    return out


def scl_line_stats_range(ctx: Context, trace0: int, ntr: int, out: np.ndarray | None = None) -> np.ndarray:
    """Line stats of traces trace0 .. trace0 + ntr - 1 in one call, shape (ntr, n_lines); `out` may be
    a preallocated (for instance pinned) array of that shape and dtype."""
    if out is None:
        out = np.zeros((ntr, ctx.cfg.n_lines), LINE_STAT_DTYPE)
    n = ctypes.c_uint64()
    _check(ctx, load().scl_line_stats_range(ctx.handle, trace0, ntr, out.ctypes.data, out.size, ctypes.byref(n)))
    return out


def scl_leak_scores_range(ctx: Context, trace0: int, ntr: int, out: np.ndarray | None = None) -> np.ndarray:
    """Leak scores of traces trace0 .. trace0 + ntr - 1 in one call, shape (ntr, n_lines)."""
    if out is None:
        out = np.zeros((ntr, ctx.cfg.n_lines), LEAK_DTYPE)
    n = ctypes.c_uint64()
    _check(ctx, load().scl_leak_scores_range(ctx.handle, trace0, ntr, out.ctypes.data, out.size, ctypes.byref(n)))
    return out


def scl_line_timeline(ctx: Context, trace: int, line: int) -> tuple[np.ndarray, np.ndarray]:
    """(event indices, footprints) of the retained samples of one line, in trace order."""
    lib = load()
    n = ctypes.c_uint64()
    rc = lib.scl_line_timeline(ctx.handle, trace, line, None, None, 0, ctypes.byref(n))
    if rc not in (SCL_OK, SCL_ERANGE):
        _check(ctx, rc)
    idx = np.zeros(max(1, n.value), np.uint64)
    fp = np.zeros(max(1, n.value), np.int64)
    _check(ctx, lib.scl_line_timeline(ctx.handle, trace, line, idx.ctypes.data, fp.ctypes.data, n.value,
                                      ctypes.byref(n)))
    return idx[:n.value], fp[:n.value]


def scl_leak_report(ctx: Context, trace: int) -> np.ndarray:
    out = np.zeros(ctx.cfg.n_lines, LEAK_REPORT_DTYPE)
    n = ctypes.c_uint32()
    _check(ctx, load().scl_leak_report(ctx.handle, trace, out.ctypes.data, len(out), ctypes.byref(n)))
    return out


def scl_trace_state(ctx: Context, trace: int) -> dict:
    out = np.zeros(1, TRACE_INFO_DTYPE)
    _check(ctx, load().scl_trace_state(ctx.handle, trace, out.ctypes.data))
    r = out[0]
    return {k: (int(r[k]) if k != "reserved" else None) for k in TRACE_INFO_DTYPE.names if k != "reserved"}


def scl_state_export(ctx: Context, trace: int) -> bytes:
    lib = load()
    n = ctypes.c_uint64()
    _check(ctx, lib.scl_state_export(ctx.handle, trace, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib.scl_state_export(ctx.handle, trace, buf, n.value, ctypes.byref(n)))
    return buf.raw


def scl_state_import(ctx: Context, trace: int, blob: bytes) -> None:
    _check(ctx, load().scl_state_import(ctx.handle, trace, blob, len(blob)))


def scl_trace_reset(ctx: Context, trace: int, stream=None) -> None:
    _check(ctx, load().scl_trace_reset(ctx.handle, trace, _stream(stream)))


def scl_tuning_get(ctx: Context) -> scl_tuning:
    t = scl_tuning()
    _check(ctx, load().scl_tuning_get(ctx.handle, ctypes.byref(t)))
    return t


def scl_tuning_set(ctx: Context, unit_events: int, warps_per_block: int = 16, ext_events: int = 0,
                   final_warps: int = 14, first_events: int = 0, fixup: int = 0, piece_events: int = 0) -> None:
    t = scl_tuning(unit_events, warps_per_block, ext_events, final_warps, first_events, fixup, piece_events)
    _check(ctx, load().scl_tuning_set(ctx.handle, ctypes.byref(t)))


def scl_autotune(ctx: Context, segs, stream=None) -> tuple[scl_tuning, float]:
    arr = _segs(segs)
    best = scl_tuning()
    ms = ctypes.c_double()
    _check(ctx, load().scl_autotune(ctx.handle, arr, len(segs), _stream(stream), ctypes.byref(best),
                                    ctypes.byref(ms)))
    return best, ms.value


def scl_graph_enable(ctx: Context, on: bool = True) -> None:
    _check(ctx, load().scl_graph_enable(ctx.handle, int(on)))


def request(trace_id: int, arrival_ns: int, delta, addr, line, is_python, csize=None, cline=None,
            cpy=None) -> scl_request:
    """Descriptor of one serving request; arrays are host numpy arrays (kept alive by the caller)."""
    r = scl_request()
    r.trace_id = trace_id
    r.arrival_ns = int(arrival_ns)
    r.ev = scl_events(_ptr(delta), _ptr(addr), _ptr(line), _ptr(is_python), 0 if delta is None else len(delta))
    r.cp = scl_copies(_ptr(csize), _ptr(cline), _ptr(cpy), 0 if csize is None else len(csize))
    return r


def scl_serve(ctx: Context, reqs, hbm_budget: int = 0, max_batch: int = 0, realtime: bool = False):
    """Serve the requests; returns (per-request results as REQUEST_RESULT_DTYPE, summary dict)."""
    arr = (scl_request * max(1, len(reqs)))(*reqs)
    opts = scl_serve_opts(hbm_budget, max_batch, int(realtime))
    out = np.zeros(max(1, len(reqs)), REQUEST_RESULT_DTYPE)
    sm = scl_serve_summary()
    _check(ctx, load().scl_serve(ctx.handle, arr, len(reqs), ctypes.byref(opts), out.ctypes.data,
                                 ctypes.byref(sm)))
    return out[:len(reqs)], {k: getattr(sm, k) for k, _ in scl_serve_summary._fields_}


def scl_rate_samples(ctx: Context, delta, line, is_python, gap, consumed: int = 0, stream=None):
    """Rate-based sampling over device arrays (torch CUDA tensors); returns
    (counts [n_lines, 2], state [4]) as numpy arrays after synchronising the stream."""
    import torch
    dev = gap.device
    counts = torch.empty(2 * ctx.cfg.n_lines, dtype=torch.int64, device=dev)
    state = torch.empty(4, dtype=torch.int64, device=dev)
    _check(ctx, load().scl_rate_samples(ctx.handle, _ptr(delta), _ptr(line), _ptr(is_python), len(delta), _ptr(gap),
                                        len(gap), int(consumed), _ptr(counts), _ptr(state), _stream(stream)))
    torch.cuda.synchronize(dev)
    return counts.cpu().numpy().view(np.uint64).reshape(-1, 2), state.cpu().numpy().view(np.uint64)


def scl_cpu_attribution(ctx: Context, vtime, line, quantum: int, t_prev: int = 0, stream=None):
    """Python / native time per line from CPU-timer interrupts (torch CUDA tensors);
    returns (python [n_lines], native [n_lines], flags) as numpy after synchronising."""
    import torch
    dev = vtime.device
    py = torch.empty(ctx.cfg.n_lines, dtype=torch.int64, device=dev)
    nat = torch.empty(ctx.cfg.n_lines, dtype=torch.int64, device=dev)
    fl = torch.empty(1, dtype=torch.int64, device=dev)
    _check(ctx, load().scl_cpu_attribution(ctx.handle, _ptr(vtime), _ptr(line), len(vtime), int(quantum), int(t_prev),
                                           _ptr(py), _ptr(nat), _ptr(fl), _stream(stream)))
    torch.cuda.synchronize(dev)
    return py.cpu().numpy(), nat.cpu().numpy(), int(fl.cpu().item())


def scl_profile_enable(ctx: Context, on: bool = True) -> None:
    _check(ctx, load().scl_profile_enable(ctx.handle, int(on)))


def scl_profile_reset(ctx: Context) -> None:
    _check(ctx, load().scl_profile_reset(ctx.handle))


def scl_kernel_times(ctx: Context) -> dict:
    lib = load()
    n = ctypes.c_uint32()
    lib.scl_kernel_times(ctx.handle, None, None, None, 0, ctypes.byref(n))
    k = n.value
    names = (ctypes.c_char_p * max(1, k))()
    ms = (ctypes.c_double * max(1, k))()
    cnt = (ctypes.c_uint64 * max(1, k))()
    _check(ctx, lib.scl_kernel_times(ctx.handle, names, ms, cnt, k, ctypes.byref(n)))
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(k)}


BATCH_INFO_DTYPE = np.dtype([("units", "<u8"), ("walked", "<u8"), ("walked_merged", "<u8"),
                             ("explicit_entries", "<u8"), ("transparent", "<u8"), ("unit_events", "<u8"),
                             ("walked_events", "<u8"), ("searched", "<u8"), ("first_events", "<u8"),
                             ("sketch_events", "<u8")])


def scl_batch_stats(ctx: Context) -> dict:
    out = np.zeros(1, BATCH_INFO_DTYPE)
    _check(ctx, load().scl_batch_stats(ctx.handle, out.ctypes.data))
    return {k: int(out[0][k]) for k in BATCH_INFO_DTYPE.names}


def scl_selftest_wait(ctx: Context, limit: int, stream=None) -> int:
    """Returns the status code of the bounded-wait self test (SCL_ETIMEOUT expected)."""
    return load().scl_selftest_wait(ctx.handle, limit, _stream(stream))


def scl_copy_volume_noalloc(size, line, is_python, copy_threshold: int, counter_in: int, n_lines: int,
                            samples_out, bytes_out, state_out, stream=None, m: int | None = None) -> int:
    """Allocation-free copy-volume sampler (see include/scl.h); returns the status code.
    Outputs are caller-owned device buffers of 2*n_lines, 2*n_lines and 3 64-bit words."""
    m = len(size) if m is None else m
    return load().scl_copy_volume_noalloc(_ptr(size), _ptr(line), _ptr(is_python), m, copy_threshold, counter_in,
                                          n_lines, _ptr(samples_out), _ptr(bytes_out), _ptr(state_out),
                                          _stream(stream))


# ------------------------------------------------------------------ convenience

def to_device(*arrays, device="cuda"):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in arrays]


def trace_segment(trace_id: int, tr, device="cuda"):
    """(descriptor, tensors) for a tracegen.Trace moved to the device; keep the tensors alive."""
    ts = to_device(tr.delta, tr.addr, tr.line, tr.is_python, tr.csize, tr.cline, tr.cpy, device=device)
    return segment(trace_id, *ts), ts
