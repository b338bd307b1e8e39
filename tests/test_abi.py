"""CPU-only checks of the C ABI library: it builds, loads without a GPU and
exports every function include/pcv.h declares; host-only entry points
behave (no compute calls without a GPU)."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "pcv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pcv_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpcv():
    from paper_2310_07002_b300.build import build
    path = build()
    from paper_2310_07002_b300 import pcv
    return pcv.load(), path


def test_exports_every_declared_symbol(libpcv):
    L, path = libpcv
    declared = header_functions()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pcv_\w+)", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        getattr(L, f)


def test_binding_covers_header():
    from paper_2310_07002_b300 import pcv
    assert set(pcv.exported_symbols()) <= set(header_functions())


def test_built_for_sm103a(libpcv):
    _, path = libpcv
    # the fatbin's target list as printed by the CUDA tool (no disassembly)
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_default_options_host_only(libpcv):
    L, _ = libpcv
    from paper_2310_07002_b300.pcv import Options
    o = Options()
    L.pcv_default_options(ct.byref(o))
    assert o.leapfrog_steps == 16 and o.batch_size == 50 and o.step_size < 0
    assert o.acov_max_lag == 64 and o.use_graphs == 1 and o.max_batches == 1024
    assert o.trajectory_length == -1.0 and o.step_jitter == -1.0     # defaults: auto
    assert o.fused_trajectory == -1 and o.tc_steps_per_launch == 0 and o.tc_grid == 0


def test_create_rejects_bad_arguments_before_any_cuda_call(libpcv):
    L, _ = libpcv
    from paper_2310_07002_b300.pcv import Model, Options, E_INVALID_ARG
    o = Options()
    L.pcv_default_options(ct.byref(o))
    m = Model(0, 10.0, 1.0, 1.0, 1.0, None, 0)
    h = ct.c_void_p()
    # null data pointers; the message stays with the thread for pcv_last_error(NULL)
    assert L.pcv_create(ct.byref(m), None, None, None, 10, 2, 4, ct.byref(o), ct.byref(h)) == E_INVALID_ARG
    assert b"NULL" in L.pcv_last_error(None)
    import numpy as np
    X = np.zeros((10, 2), np.float32)
    y = np.zeros(10, np.float32)
    f = np.zeros(10, np.int32)
    # L < 2 (R-hat needs two chains), p < 1, N < 1
    for N, p, Lc in [(10, 2, 1), (10, 0, 4), (0, 2, 4)]:
        assert L.pcv_create(ct.byref(m), X.ctypes.data, y.ctypes.data, f.ctypes.data, N, p, Lc,
                            ct.byref(o), ct.byref(h)) == E_INVALID_ARG
        assert b"chains_per_fold" in L.pcv_last_error(None)
    # bad options
    o.batch_size = 0
    assert L.pcv_create(ct.byref(m), X.ctypes.data, y.ctypes.data, f.ctypes.data, 10, 2, 4,
                        ct.byref(o), ct.byref(h)) == E_INVALID_ARG
    assert L.pcv_last_error(None) == b"an option is out of range"
    L.pcv_default_options(ct.byref(o))
    o.step_jitter = 1.0                      # a step size of zero would be possible
    assert L.pcv_create(ct.byref(m), X.ctypes.data, y.ctypes.data, f.ctypes.data, 10, 2, 4,
                        ct.byref(o), ct.byref(h)) == E_INVALID_ARG
    assert not h.value
    assert L.pcv_num_folds(None) == -1
    assert L.pcv_last_error(None) == b"an option is out of range"
    # the launch-shape options take only their listed values
    for field, bad in [("fused_trajectory", 3), ("tc_steps_per_launch", 2), ("tc_steps_per_launch", -1),
                       ("tc_grid", 3), ("tc_grid", -1)]:
        L.pcv_default_options(ct.byref(o))
        setattr(o, field, bad)
        assert L.pcv_create(ct.byref(m), X.ctypes.data, y.ctypes.data, f.ctypes.data, 10, 2, 4,
                            ct.byref(o), ct.byref(h)) == E_INVALID_ARG, (field, bad)
        assert L.pcv_last_error(None) == b"an option is out of range"
    # a model kind the library does not know
    L.pcv_default_options(ct.byref(o))
    m.kind = 99
    assert L.pcv_create(ct.byref(m), X.ctypes.data, y.ctypes.data, f.ctypes.data, 10, 2, 4,
                        ct.byref(o), ct.byref(h)) == E_INVALID_ARG
    assert L.pcv_last_error(None) == b"unknown model kind"
    L.pcv_destroy(None)
