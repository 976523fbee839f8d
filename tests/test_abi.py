"""The C-ABI library builds, loads without a GPU, exports every function that
include/*.h declares, and validates arguments on the host (no CUDA calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(fft_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_00567_b300 import build
    build.build()
    import paper_2604_00567_b300 as dsfft
    return dsfft.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fft_plan_create", "fft_exec", "fft_plan_destroy", "fft_plan_get_table",
                     "fft_plan_get_info", "fft_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_00567_b300 import LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    for n in _declared_functions():
        assert hasattr(lib, n)


def test_opts_defaults(lib):
    import paper_2604_00567_b300 as dsfft
    o = dsfft.PlanOpts()
    assert lib.fft_plan_opts_init(1, ctypes.byref(o)) == 0
    assert o.lf_eps == 1e-7 and o.scale_forward == 1 and o.scale_inverse == 0 and o.device == -1
    assert o.autotune == 0 and o.variant == 0 and o.radix == 0 and o.sweep_passes == 0
    assert lib.fft_plan_opts_init(0, ctypes.byref(o)) == 0
    assert o.scale_forward == 0
    assert lib.fft_plan_opts_init(7, ctypes.byref(o)) == 1
    assert lib.fft_plan_opts_init(0, None) == 1


def test_host_side_validation_without_gpu(lib):
    """Errors detected before any CUDA call: bad sizes, enums, options, null
    handles."""
    import paper_2604_00567_b300 as dsfft
    h = ctypes.c_void_p()
    for n in (0, 1, 3, 6, 1000, 1 << 25, -4):
        assert lib.fft_plan_create(ctypes.byref(h), n, 0, 2, None) == 2
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 9, 2, None) == 1
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 9, None) == 1
    assert lib.fft_plan_create(None, 1024, 0, 2, None) == 1
    o = dsfft.PlanOpts()
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.lf_eps = 0.0
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 0, ctypes.byref(o)) == 1
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.reserved[0] = 5
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 1
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.sweep_passes = 6
    assert lib.fft_plan_create(ctypes.byref(h), 1 << 18, 0, 2, ctypes.byref(o)) == 1   # outside 7..12
    o.sweep_passes = 9
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 3      # no sweeps at 2^10
    assert lib.fft_plan_create(ctypes.byref(h), 1 << 22, 0, 2, ctypes.byref(o)) == 3   # 9 + 13 passes
    o.variant = 3
    assert lib.fft_plan_create(ctypes.byref(h), 1 << 16, 0, 2, ctypes.byref(o)) == 3   # cluster has no sweeps
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.radix = 3
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 1
    o.radix = 4
    o.variant = 3
    assert lib.fft_plan_create(ctypes.byref(h), 1 << 15, 0, 2, ctypes.byref(o)) == 3   # radix-4 above 2^14: sweeps
    o.variant = 2
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 3      # radix-4: fused wide only
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.scale_forward = 3
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 1
    lib.fft_plan_opts_init(0, ctypes.byref(o))
    o.variant = 9
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 1
    o.variant = 0
    o.autotune = 2
    assert lib.fft_plan_create(ctypes.byref(h), 1024, 0, 2, ctypes.byref(o)) == 1
    o.autotune = 0
    for n, variant in ((1024, 3), (1024, 4), (1 << 20, 1), (1 << 20, 2), (1 << 18, 3), (1 << 17, 3), (8, 2),
                       (128, 5), (1 << 14, 5), (1 << 15, 5)):
        o.variant = variant   # a variant the size does not have (FP32)
        assert lib.fft_plan_create(ctypes.byref(h), n, 0, 2, ctypes.byref(o)) == 3, (n, variant)
    assert lib.fft_exec(None, None, None, 1, -1, None) == 1
    assert lib.fft_plan_destroy(None) == 0
    assert lib.fft_plan_get_info(None, None) == 1
    assert lib.fft_plan_device_status(None) == 1
    assert lib.fft_plan_get_table(None, -1, None, 0) == 1
    assert lib.fft_plan_get_table4(None, -1, None, 0) == 1
    assert lib.fft_status_string(2).decode().startswith("invalid size")
    assert lib.fft_status_string(99).decode() == "unknown status"


def test_status_codes_match_binding():
    import paper_2604_00567_b300 as dsfft
    hdr = open(os.path.join(ROOT, "include", "dsfft.h")).read()
    for code, name in dsfft.STATUS.items():
        assert re.search(rf"\b{name}\s*=\s*{code}\b", hdr), name


def test_batch_validation_without_gpu(lib):
    """fft_batch_create rejects bad items before any CUDA call."""
    import paper_2604_00567_b300 as dsfft
    h = ctypes.c_void_p()
    arr = (dsfft.BatchItemC * 2)()
    for a in arr:
        a.n, a.precision, a.factorization, a.direction = 1024, 0, 2, -1
        a.in_, a.out = 0x1000, 0x2000
    arr[1].n = 1000
    assert lib.fft_batch_create(ctypes.byref(h), arr, 2, None) == 2
    arr[1].n = 1024
    arr[1].direction = 0
    assert lib.fft_batch_create(ctypes.byref(h), arr, 2, None) == 1
    arr[1].direction = 1
    arr[1].in_ = None
    assert lib.fft_batch_create(ctypes.byref(h), arr, 2, None) == 1
    arr[1].in_ = 0x1004    # not 8-byte aligned for complex64
    assert lib.fft_batch_create(ctypes.byref(h), arr, 2, None) == 1
    assert lib.fft_batch_create(None, arr, 2, None) == 1
    assert lib.fft_batch_create(ctypes.byref(h), None, 2, None) == 1
    assert lib.fft_batch_create(ctypes.byref(h), arr, -1, None) == 1
    assert lib.fft_batch_exec(None, None) == 1
    assert lib.fft_batch_destroy(None) == 0


def test_server_validation_without_gpu(lib):
    """fft_server_* argument checks that precede any CUDA call."""
    import paper_2604_00567_b300 as dsfft
    o = dsfft.ServerOptsC()
    assert lib.fft_server_opts_init(ctypes.byref(o)) == 0
    assert o.device == -1 and o.max_ticks_in_flight == 2 and o.memory_budget == 40_000_000_000
    assert o.max_tick_transforms == 1 << 20 and o.autotune == 0 and o.release_on_complete == 0
    assert o.max_tick_bytes == 0
    assert lib.fft_server_opts_init(None) == 1
    h = ctypes.c_void_p()
    assert lib.fft_server_create(None, ctypes.byref(o)) == 1
    for field, bad in (("max_ticks_in_flight", 0), ("max_ticks_in_flight", 9), ("memory_budget", 0),
                       ("max_tick_transforms", 0), ("autotune", 2), ("release_on_complete", 3),
                       ("max_tick_bytes", -1)):
        lib.fft_server_opts_init(ctypes.byref(o))
        setattr(o, field, bad)
        assert lib.fft_server_create(ctypes.byref(h), ctypes.byref(o)) == 1, field
    lib.fft_server_opts_init(ctypes.byref(o))
    o.reserved[1] = 1
    assert lib.fft_server_create(ctypes.byref(h), ctypes.byref(o)) == 1
    assert lib.fft_server_submit(None, None, None) == 1
    assert lib.fft_server_poll(None, None, 0, None) == 1
    assert lib.fft_server_release(None, 1) == 1
    assert lib.fft_server_drain(None, 1.0) == 1
    assert lib.fft_server_destroy(None) == 0
