"""The C-ABI library builds, loads and exports what include/esi.h declares.

These run without a GPU: no call here reaches a kernel.
"""
import ctypes
import os
import re

import pytest

from paper_2508_02238_gb300 import esi
from paper_2508_02238_gb300 import build as esi_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(esi_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    lib_path = esi_build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers every declared function
    assert not (names - set(esi.SIGNATURES)), names - set(esi.SIGNATURES)


def test_strerror_codes():
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert esi.esi_strerror(code) != "unknown error"
    assert esi.esi_strerror(-99) == "unknown error"


GOOD = dict(C=0.2, k_per_s=10.0, b=2.0, s_min=-1.0, s_max=1.0)


@pytest.mark.parametrize("W,H,over", [
    (0, 10, {}), (10, 0, {}), (70000, 10, {}), (10, 70000, {}),
    (10, 10, {"C": 0.0}), (10, 10, {"C": -1.0}), (10, 10, {"C": float("nan")}),
    (10, 10, {"k_per_s": -1.0}), (10, 10, {"k_per_s": float("inf")}),
    (10, 10, {"b": 0.0}), (10, 10, {"s_min": 1.0, "s_max": 1.0}),
    (10, 10, {"s_min": 2.0, "s_max": 1.0}), (10, 10, {"s_max": float("inf")}),
    (10, 10, {"k_per_s": 2e12}), (10, 10, {"method": 3}), (10, 10, {"method": -1}),
    (10, 10, {"b": 0.0, "method": 1}), (10, 10, {"s_min": 1.0, "s_max": 1.0, "method": 2}),
])
def test_create_rejects_bad_arguments_before_touching_cuda(W, H, over):
    kw = dict(GOOD)
    kw.update(over)
    p = esi.make_params(**kw)
    rc, h = esi.esi_create(W, H, p)
    assert rc == esi.ESI_EINVAL and not h.value


def test_create_bad_render_mode():
    p = esi.make_params(**GOOD, render_decay=2)
    rc, _ = esi.esi_create(8, 8, p)
    assert rc == esi.ESI_EINVAL


def test_null_handle_calls_are_rejected():
    assert esi.esi_push_events(None, None, 0, 0) == esi.ESI_EINVAL
    assert esi.esi_render_frame(None, 0, None, 0) == esi.ESI_EINVAL
    assert esi.esi_synchronize(None) == esi.ESI_EINVAL
    assert esi.esi_autotune(None, None, 0, None, 0)[0] == esi.ESI_EINVAL
    assert esi.esi_noise_map(None, None, 0) == esi.ESI_EINVAL
    assert esi.esi_count_events(None, None, 0, 0, None, 0) == esi.ESI_EINVAL
    assert esi.esi_push_packed(None, None, 0, 0, 0) == esi.ESI_EINVAL
    assert esi.esi_event_states(None, None, 0, 0)[0] == esi.ESI_EINVAL
    esi.esi_destroy(None)  # no-op


def test_method_constants_match_the_header():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "esi.h")).read()
    for name in ("ESI_METHOD_ALG2", "ESI_METHOD_ALG1", "ESI_METHOD_EQ3_EXP",
                 "ESI_APPLY_EVERY_TICK", "ESI_APPLY_AT_FRAMES", "ESI_PACK_T_SHIFT"):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, hdr)
        assert m and int(m.group(1)) == getattr(esi, name), name


def test_pack_macro_layout(tmp_path):
    # the header's packing macro, compiled as plain C, against the bit layout
    # its comment states (x: bits 0-15, y: 16-31, polarity: 32, dt: 33-63)
    import os
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        import pytest
        pytest.skip("no gcc")
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    src = tmp_path / "pack.c"
    src.write_text('#include <stdio.h>\n#include "esi.h"\nint main(void) {\n'
                   '  printf("%llu %llu %llu\\n",\n'
                   '    (unsigned long long)ESI_PACK_EVENT(5, 7, 1, 123),\n'
                   '    (unsigned long long)ESI_PACK_EVENT(65535, 65535, 0, 2147483647),\n'
                   '    (unsigned long long)ESI_PACK_EVENT(0, 1, -1, 0));\n  return 0;\n}\n')
    exe = tmp_path / "pack"
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got[0] == 5 + 7 * 2**16 + 2**32 + 123 * 2**33
    assert got[1] == (2**16 - 1) + (2**16 - 1) * 2**16 + (2**31 - 1) * 2**33
    assert got[2] == 2**16 + 2**32     # any non-zero polarity argument is +1
    assert got[1] < 2**64


def test_server_options_are_checked_before_touching_cuda():
    for field, bad in (("apply_mode", 3), ("apply_mode", -1), ("copy_threads", 17),
                       ("copy_threads", -1), ("host_pool_bytes", 4096), ("scan_chain", 34),
                       ("fuse_tick", 3), ("fuse_tick", -1), ("_reserved", 1),
                       ("frame_slots", 1), ("tile_h", 5)):
        opts = esi.esi_server_opts()
        setattr(opts, field, bad)
        rc, srv = esi.esi_server_create(1 << 20, opts, 0)
        assert rc == esi.ESI_EINVAL and not srv, field


def test_server_trace_and_last_error_reject_null_servers():
    assert esi.esi_server_trace(None)[0] == esi.ESI_EINVAL
    assert esi.esi_server_last_error(None) == ""


def test_bin_events_checks_its_arguments_before_touching_cuda():
    # every refusal happens on the host; without a CUDA device a valid call
    # gets as far as the runtime and fails there (never ESI_EINVAL)
    import torch
    sh = esi.esi_tuning()
    good = dict(width=346, height=260, ring_capacity=1 << 12, first=0, n=100)

    def call(ring=16 * 4096, **kw):
        a = dict(good, **kw)
        return esi.esi_bin_events(a["width"], a["height"], sh, ring, a["ring_capacity"],
                                  a["first"], a["n"], 0, 1 << 20, 1 << 21)[0]

    assert call(width=0) == esi.ESI_EINVAL
    assert call(height=70000) == esi.ESI_EINVAL
    assert call(ring_capacity=3000) == esi.ESI_EINVAL
    assert call(n=5000) == esi.ESI_EINVAL              # more than the ring holds
    assert call(ring=16 * 4096 + 8) == esi.ESI_EINVAL  # not 16-byte aligned
    sh.tile_h = 5
    assert call() == esi.ESI_EINVAL
    sh.tile_h = 0
    assert esi.esi_bin_events(346, 260, sh, 0, 1 << 12, 0, 0, 0, 0, 0)[0] == esi.ESI_OK  # n = 0
    if not torch.cuda.is_available():
        assert call() == esi.ESI_ECUDA
