"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute call is made here (no GPU needed).
"""
import ctypes
import os
import re

from paper_1212_3032_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "bem.h")).read()
    return re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(bem_\w+)\s*\(", text, re.M)


def test_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.EXPORTED)


def test_struct_layouts_match_header():
    # bem_opts: 11 fields with natural alignment; bem_freq_stats likewise
    assert ctypes.sizeof(binding.Opts) == 64
    assert ctypes.sizeof(binding.FreqStats) == 16 + 7 * 8 + 2 * 8 + 8 + 8 + 8
    assert ctypes.sizeof(binding.Profile) == 9 * 8
    assert ctypes.sizeof(binding.FarStorage) == 4 + 4 + 3 * 8 + 4 + 4
    o = binding.default_opts()
    assert o.tol == 1e-5 and o.restart == 50 and o.leaf_size == 64 and o.sem_k == 4
    assert o.precision == binding.PREC_C64_MIXED and o.guess == binding.GUESS_SEM
    assert o.precond == binding.PRECOND_BLOCK3


def test_create_without_device_fails_cleanly():
    # on a host without a GPU the context cannot be created; the call must
    # return an error code, not crash
    lib = binding.load_library()
    h = ctypes.c_void_p()
    rc = lib.bem_create(ctypes.byref(h), 99, None)
    assert rc != 0 and not h.value
