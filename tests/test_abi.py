"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/sg.h declares, and its host-side argument validation
rejects bad input before touching a GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2606_22984_gb300 import build, inputs, sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sg.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_param_count_agrees_with_blob_layouts(lib):
    for wl in inputs.workloads().values():
        m = wl.model
        n = sg.param_count(m)
        assert n == inputs.param_count(m) == oracle.param_count(oracle.ModelCfg(**vars(m)))


def test_grouped_param_count(lib):
    m = inputs.workloads()["ea2d64"].model
    one = lib.sg_param_count(ctypes.byref(sg.config(m)))
    assert lib.sg_param_count(ctypes.byref(sg.config(m, n_models=8))) == 8 * one
    assert lib.sg_param_count(ctypes.byref(sg.config(m, n_models=0))) == one
    assert inputs.make_group_weights(m, 5, 2).size == 2 * one
    assert lib.sg_param_count(ctypes.byref(sg.config(m, n_models=65))) == -1
    assert lib.sg_param_count(ctypes.byref(sg.config(m, n_models=-1))) == -1


@pytest.mark.parametrize("bad", [dict(N=0), dict(n_heads=5), dict(d_token=32), dict(n_layers=17),
                                 dict(mask_kind=3)])
def test_invalid_config_rejected(lib, bad):
    kw = dict(N=20, n_layers=2, d=32, n_heads=4)
    kw.update({k: v for k, v in bad.items() if k in kw})
    m = inputs.ModelShape(**kw)
    for k, v in bad.items():
        setattr(m, k, v)
    assert lib.sg_param_count(ctypes.byref(sg.config(m))) == -1
    h = ctypes.c_void_p()
    w = np.zeros(10, np.float32)
    rc = lib.sg_model_create(ctypes.byref(sg.config(m)), w.ctypes.data_as(ctypes.c_void_p), 10,
                             ctypes.byref(h))
    assert rc == 1 and not h.value
    assert lib.sg_last_error()


def test_blob_size_and_nan_rejected_on_host(lib):
    m = inputs.ModelShape(20, 2, 32, 4)
    cfg = sg.config(m)
    h = ctypes.c_void_p()
    w = inputs.make_weights(m, 1)
    rc = lib.sg_model_create(ctypes.byref(cfg), w.ctypes.data_as(ctypes.c_void_p), w.size - 1,
                             ctypes.byref(h))
    assert rc == 1
    w[5] = np.inf
    rc = lib.sg_model_create(ctypes.byref(cfg), w.ctypes.data_as(ctypes.c_void_p), w.size,
                             ctypes.byref(h))
    assert rc == 4 and b"non-finite" in lib.sg_last_error()


def test_instance_validation_on_host(lib):
    h = ctypes.c_void_p()
    J = np.ones((4, 4), np.float32)  # non-zero diagonal
    assert lib.sg_instance_create(0, 4, 0, 0, 0, J.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(h)) == 1
    J = np.triu(np.ones((4, 4), np.float32), 1)  # not symmetric
    assert lib.sg_instance_create(0, 4, 0, 0, 0, J.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(h)) == 1
    bonds = np.ones((10, 2), np.float32)  # N != L^D
    assert lib.sg_instance_create(1, 10, 2, 3, 1, bonds.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(h)) == 1


def test_call_argument_validation_on_host(lib):
    P = ctypes.c_void_p
    assert lib.sg_sample(None, 10, 1.0, 1, 0, 0.0, P(1), P(1), None, None) == 1
    assert lib.sg_free_energy(P(1), P(1), 10, -1.0, P(1), None, None) == 1
    assert lib.sg_mh_step(P(1), P(1), P(1), 10, 4, 3, 1.0, 1, P(1), P(1), P(1), P(1), None,
                          None) == 1
    assert lib.sg_adam_step(P(1), P(1), P(1), P(1), 5, 1e-3, 0.9, 0.999, 1e-8, 0, None) == 1


def test_patched_param_count_and_validation(lib):
    m = inputs.ModelShape(64, 2, 32, 4, d_token=16, patch=4, lat_D=2, lat_L=8)
    assert lib.sg_param_count(ctypes.byref(sg.config(m))) == inputs.param_count(m) == \
        oracle.param_count(oracle.ModelCfg(**vars(m)))
    for bad in (dict(patch=3), dict(patch=4, lat_D=3), dict(patch=4, lat_L=7),
                dict(patch=16), dict(patch=4, lat_D=2, lat_L=6)):
        b = inputs.ModelShape(64, 2, 32, 4, d_token=16, patch=4, lat_D=2, lat_L=8)
        for k, v in bad.items():
            setattr(b, k, v)
        assert lib.sg_param_count(ctypes.byref(sg.config(b))) == -1
