"""The C-ABI library builds, loads without a GPU and exports every symbol include/scl.h declares (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2212_07597_gb300 import build as scl_build
from paper_2212_07597_gb300 import scl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "scl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(scl_[a-z_]+)\s*\(", src)))


def test_builds_and_exports_every_declared_symbol():
    path = scl_build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(scl.EXPORTS)


def test_struct_layouts_match_header():
    assert ctypes.sizeof(scl.scl_config) == 64
    assert ctypes.sizeof(scl.scl_segment) == 8 + 40 + 32
    assert scl.SAMPLE_DTYPE.itemsize == 56
    assert scl.LINE_STAT_DTYPE.itemsize == 88
    assert scl.LEAK_DTYPE.itemsize == 40
    assert scl.TRACE_INFO_DTYPE.itemsize == 112


def test_struct_layouts_match_c_compiler(tmp_path):
    """sizeof of every ABI struct as gcc lays it out from include/scl.h == the binding's."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    pairs = {"scl_config": ctypes.sizeof(scl.scl_config), "scl_segment": ctypes.sizeof(scl.scl_segment),
             "scl_events": ctypes.sizeof(scl.scl_events), "scl_copies": ctypes.sizeof(scl.scl_copies),
             "scl_tuning": ctypes.sizeof(scl.scl_tuning), "scl_request": ctypes.sizeof(scl.scl_request),
             "scl_serve_opts": ctypes.sizeof(scl.scl_serve_opts),
             "scl_serve_summary": ctypes.sizeof(scl.scl_serve_summary),
             "scl_request_result": scl.REQUEST_RESULT_DTYPE.itemsize,
             "scl_sample": scl.SAMPLE_DTYPE.itemsize, "scl_line_stat": scl.LINE_STAT_DTYPE.itemsize,
             "scl_leak_score": scl.LEAK_DTYPE.itemsize, "scl_trace_info": scl.TRACE_INFO_DTYPE.itemsize,
             "scl_batch_info": scl.BATCH_INFO_DTYPE.itemsize,
             "scl_leak_report_row": scl.LEAK_REPORT_DTYPE.itemsize}
    inc = os.path.join(ROOT, "include")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "scl.h"\nint main(void){\n' +
                   "".join(f'printf("{k} %zu\\n", sizeof({k}));\n' for k in pairs) + "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for k, v in pairs.items():
        assert int(got[k]) == v, (k, got[k], v)


def test_config_defaults_without_gpu():
    cfg = scl.config()
    assert cfg.threshold == 10_485_767 and cfg.copy_multiple == 2 and cfg.n_lines == 256
    assert cfg.sample_budget_shift == scl.SCL_BUDGET_AUTO and cfg.leak_rule == 0


def test_init_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(scl.SclError):
        scl.scl_replay_init(scl.config())
