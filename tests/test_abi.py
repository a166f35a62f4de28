"""CPU checks of the C ABI: the library loads, exports every declared symbol, and
validates arguments on the host (no device calls)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from paper_2406_16238_b300 import _lib
from synthetic_inputs import config_small

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "afqmc.h")) as f:
        text = f.read()
    decl = r"^\s*(?:afqmc_status|void|uint64_t|const char\s*\*)\s*(afqmc_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    names = declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_params_struct_layout():
    assert ctypes.sizeof(_lib.Params) == 56
    assert _lib.Params.stream.offset == 48
    assert ctypes.sizeof(_lib.Info) == 72


def _ws(prob, **kw):
    lib = pkg.load()
    p = _lib.Params(kw.get("dt", 0.005), kw.get("nwalkers", 64), kw.get("taylor", 6), 1.0, 1, kw.get("prec", 0),
                    kw.get("reserved", 0), math.nan, None)
    psiT = np.ascontiguousarray(prob.psiT)
    n = ctypes.c_size_t()
    st = lib.afqmc_workspace_size(prob.norb, prob.naux, kw.get("na", prob.nalpha), kw.get("nb", prob.nbeta),
                                  psiT.ctypes.data_as(_lib._dp), ctypes.byref(p), ctypes.byref(n))
    return st, n.value, lib.afqmc_last_error().decode()


def test_workspace_size_and_validation():
    prob = config_small()
    st, n64, _ = _ws(prob)
    assert st == 0 and n64 > 0
    st, n32, _ = _ws(prob, prec=1)
    assert st == 0 and 0 < n32 < n64
    st, n2, _ = _ws(prob, nwalkers=128)
    assert n2 > n64
    for kw, msg in [(dict(dt=0.0), "dt"), (dict(nwalkers=0), "nwalkers"), (dict(taylor=0), "taylor"),
                    (dict(prec=9), "prec"), (dict(reserved=1), "reserved"), (dict(na=0), "nalpha"),
                    (dict(na=65), "nalpha")]:
        st, _, err = _ws(prob, **kw)
        assert st == 1 and msg in err, (kw, err)


def test_create_rejects_bad_host_inputs_before_touching_the_device():
    lib = pkg.load()
    prob = config_small()
    p = _lib.Params(0.005, 4, 6, 1.0, 1, 0, 0, math.nan, None)
    ctx = ctypes.c_void_p()
    psiT = np.ascontiguousarray(prob.psiT)
    # no workspace
    st = lib.afqmc_create(prob.h1e.ctypes.data_as(_lib._dp), prob.chol.ctypes.data_as(_lib._dp), 0.0, prob.norb,
                          prob.naux, 2, 2, psiT.ctypes.data_as(_lib._dp), ctypes.byref(p), None, 0, ctypes.byref(ctx))
    assert st == 1 and "workspace" in lib.afqmc_last_error().decode()
    # workspace too small (a fake aligned address; never dereferenced because the size check fails first)
    st = lib.afqmc_create(prob.h1e.ctypes.data_as(_lib._dp), prob.chol.ctypes.data_as(_lib._dp), 0.0, prob.norb,
                          prob.naux, 2, 2, psiT.ctypes.data_as(_lib._dp), ctypes.byref(p), ctypes.c_void_p(256), 1024,
                          ctypes.byref(ctx))
    assert st == 2
    _, need, _ = _ws(prob, nwalkers=4)
    bad = prob.chol.copy()
    bad[3, 0, 1] += 1.0
    st = lib.afqmc_create(prob.h1e.ctypes.data_as(_lib._dp), bad.ctypes.data_as(_lib._dp), 0.0, prob.norb,
                          prob.naux, 2, 2, psiT.ctypes.data_as(_lib._dp), ctypes.byref(p), ctypes.c_void_p(256), need,
                          ctypes.byref(ctx))
    assert st == 1 and "symmetric" in lib.afqmc_last_error().decode()
    nanh = prob.h1e.copy()
    nanh[1, 1] = np.nan
    st = lib.afqmc_create(nanh.ctypes.data_as(_lib._dp), prob.chol.ctypes.data_as(_lib._dp), 0.0, prob.norb,
                          prob.naux, 2, 2, psiT.ctypes.data_as(_lib._dp), ctypes.byref(p), ctypes.c_void_p(256), need,
                          ctypes.byref(ctx))
    assert st == 1 and "non-finite" in lib.afqmc_last_error().decode()


def test_null_context_is_rejected():
    lib = pkg.load()
    assert lib.afqmc_propagate(None, 1) == 1
    assert lib.afqmc_reortho(None) == 1
    assert lib.afqmc_launch_count(None) == 0


def test_noalloc_binding_rejects_bad_tensors_before_any_call():
    """The allocation-free comb plan's binding checks dtype, device, contiguity and sizes itself."""
    import torch
    w = torch.ones(4, dtype=torch.float64)
    src = torch.zeros(4, dtype=torch.int32)
    neww = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        pkg._lib.comb_plan_noalloc(w, 1, 0, src, neww)
