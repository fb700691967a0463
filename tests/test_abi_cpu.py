"""CPU checks of the C ABI library: it builds, loads, exports every symbol
declared in include/psl1.h, and refuses to run without a GPU (no fallback)."""
import ctypes
import os
import re

import pytest

from paper_2510_11023_gb300 import psl1, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(psl1_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = psl1.load()
    declared = _declared()
    assert "psl1_solve_parareal" in declared and "psl1_create" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(psl1.SIGNATURES), declared - set(psl1.SIGNATURES)


def test_invalid_arguments_rejected_before_device_use():
    L = psl1.load()
    h = ctypes.c_void_p()
    st = L.psl1_create(ctypes.byref(h), 0, None, 4, 0, None)
    assert st == -1
    wl = workloads.cfg1()
    arr = (psl1.Instance * 1)(psl1.to_instance(wl.specs[0]))
    assert L.psl1_create(ctypes.byref(h), 1, arr, 7, 0, None) == -1   # 7 does not divide 256
    assert b"multiple" in L.psl1_last_error(None)
    bad = psl1.to_instance(wl.specs[0])
    bad.alpha = 1.5
    arr = (psl1.Instance * 1)(bad)
    assert L.psl1_create(ctypes.byref(h), 1, arr, 8, 0, None) == -1
    assert L.psl1_set_inexact_fine(None, 1e-4) == -1


def test_invalid_2d_arguments_rejected_before_device_use():
    L = psl1.load()
    h = ctypes.c_void_p()
    wl = workloads.small_batch_2d()

    def create(*insts):
        arr = (psl1.Instance * len(insts))(*insts)
        return L.psl1_create(ctypes.byref(h), len(insts), arr, wl.P, 0, None)

    ok = psl1.to_instance(wl.specs[0])
    bad = psl1.to_instance(wl.specs[0])
    bad.dim = 3
    assert create(bad) == -1
    bad = psl1.to_instance(wl.specs[0])
    bad.modes[1] = 65                      # more than 64 modes per axis in 2D
    assert create(bad) == -1
    assert b"modes[1]" in L.psl1_last_error(None)
    bad = psl1.to_instance(wl.specs[0])
    bad.qnodes[1] = 15                     # odd node count
    assert create(bad) == -1
    bad = psl1.to_instance(wl.specs[0])
    bad.hi[1] = bad.lo[1]                  # empty y interval
    assert create(bad) == -1
    one_d = psl1.to_instance(workloads.cfg1(N=wl.P * 4, P=wl.P).specs[0])
    assert create(ok, one_d) == -1        # 1D and 2D instances in one handle
    assert b"same dim" in L.psl1_last_error(None)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(psl1.PSL1Error) as ei:
        psl1.Problem(workloads.cfg1())
    assert ei.value.status == -4


def test_invalid_collocation_arguments_rejected_before_device_use():
    L = psl1.load()
    h = ctypes.c_void_p()
    spec = workloads.e1_collocation(P=4, m=2).specs[0]

    def create(inst, prec=0):
        arr = (psl1.Instance * 1)(inst)
        return L.psl1_create(ctypes.byref(h), 1, arr, 4, prec, None)

    bad = psl1.to_instance(spec)
    bad.modes[0] = 65                      # more than 64 collocation intervals
    assert create(bad) == -1 and b"collocation" in L.psl1_last_error(None)
    bad = psl1.to_instance(spec)
    bad.dim = 2                            # collocation is 1D
    bad.modes[1] = 4
    assert create(bad) == -1
    bad = psl1.to_instance(spec)
    bad.basis = 7                          # unknown scheme
    assert create(bad) == -1 and b"basis" in L.psl1_last_error(None)
    assert create(psl1.to_instance(spec), prec=1) == -1   # collocation runs in FP64 only
    assert b"FP64" in L.psl1_last_error(None)
