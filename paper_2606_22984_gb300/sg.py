"""Python binding of libsg (include/sg.h): argument marshalling only.

Every function here checks tensor devices, dtypes and shapes, passes raw
pointers through ctypes to the C ABI of the same name, and raises
``SgError`` with the library's message on failure.  No step of the method
runs in Python.  The library must have been built (``build.build()`` or
``__graft_entry__.build()``); loading raises if ``libsg.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsg.so")

SG_FP32, SG_BF16 = 0, 1
SG_MASK_DENSE, SG_MASK_BAND_SINK = 0, 1
SG_SK_DENSE, SG_EA_LATTICE = 0, 1
_STATUS = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ENOMEM", 3: "SG_ECUDA", 4: "SG_ENUMERIC",
           5: "SG_EUNSUPPORTED"}


class SgError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn}: {_STATUS.get(code, code)}: {msg}")
        self.code = code


class SgConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("N", "n_layers", "d", "n_heads", "d_token", "d_ff",
                                              "mask_kind", "W", "S", "precision", "n_models",
                                              "patch", "lat_D", "lat_L")]


_P, _I64, _I32, _U32, _U64, _D, _F = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.c_float)
_SIGS = {
    "sg_param_count": ([ctypes.POINTER(SgConfig)], _I64),
    "sg_model_create": ([ctypes.POINTER(SgConfig), _P, _I64, ctypes.POINTER(_P)], _I32),
    "sg_model_destroy": ([_P], _I32),
    "sg_model_weights": ([_P], _P),
    "sg_model_refresh": ([_P, _P], _I32),
    "sg_model_check": ([_P, _P], _I32),
    "sg_model_reserve": ([_P, _I64], _I32),
    "sg_model_set_max_chunk": ([_P, _I64], _I32),
    "sg_sample": ([_P, _I64, _D, _U64, _U32, _F, _P, _P, _P, _P], _I32),
    "sg_logprob": ([_P, _P, _I64, _P, _P], _I32),
    "sg_grad": ([_P, _P, _P, _I64, _P, _P, _P], _I32),
    "sg_instance_create": ([_I32, _I32, _I32, _I32, _I32, _P, ctypes.POINTER(_P)], _I32),
    "sg_instance_destroy": ([_P], _I32),
    "sg_energy": ([_P, _P, _I64, _I32, _P, _P, _P], _I32),
    "sg_free_energy": ([_P, _P, _I64, _D, _P, _P, _P], _I32),
    "sg_loss_coeff": ([_P, _P, _I64, _D, _D, _D, _P, _P, _P], _I32),
    "sg_muon_step": ([_P, _P, _P, _P, _P, _P, _D, _D, _D, _I32, _I64, _P], _I32),
    "sg_gelu_selfcheck": ([_I64, _P, _P], _I32),
    "sg_mh_step": ([_P, _P, _P, _I64, _I32, _I32, _D, _U64, _P, _P, _P, _P, _P, _P], _I32),
    "sg_metropolis": ([_P, _P, _I64, _I32, _D, _U64, _P, _P, _P], _I32),
    "sg_overlap_hist": ([_P, _I64, _I32, _P, _P], _I32),
    "sg_adam_step": ([_P, _P, _P, _P, _I64, _F, _F, _F, _F, _I64, _P], _I32),
    "sg_last_error": ([], ctypes.c_char_p),
    "sg_launch_count": ([], _I64),
    "sg_sample_noalloc": ([ctypes.POINTER(SgConfig), _P, _I64, _D, _U64, _U32, _F, _P, _P, _P,
                           _P], _I32),
}
_lib = None


def lib():
    """Load libsg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsg.so not found at {LIB_PATH}; build it with "
                               "paper_2606_22984_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(fn, code):
    if code != 0:
        raise SgError(fn, code, lib().sg_last_error().decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def launch_count() -> int:
    """Kernels libsg has launched in this process."""
    return int(lib().sg_launch_count())


def config(shape: _inputs.ModelShape, precision: int = SG_FP32, n_models: int = 1) -> SgConfig:
    return SgConfig(shape.N, shape.n_layers, shape.d, shape.n_heads, shape.d_token, shape.d_ff,
                    shape.mask_kind, shape.W, shape.S, precision, n_models,
                    getattr(shape, "patch", 1), getattr(shape, "lat_D", 0), getattr(shape, "lat_L", 0))


def param_count(shape: _inputs.ModelShape, precision: int = SG_FP32) -> int:
    return int(lib().sg_param_count(ctypes.byref(config(shape, precision))))


class Model:
    """Owns an sg_model.  ``weights`` is the float32 blob (host numpy array);
    for a group of ``n_models`` models, their blobs concatenated."""

    def __init__(self, shape: _inputs.ModelShape, weights: np.ndarray, precision: int = SG_FP32,
                 n_models: int = 1):
        self.shape = shape
        self.precision = precision
        self.n_models = n_models
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self._cfg = config(shape, precision, n_models)
        h = ctypes.c_void_p()
        _check("sg_model_create",
               lib().sg_model_create(ctypes.byref(self._cfg), w.ctypes.data_as(_P), w.size,
                                     ctypes.byref(h)))
        self.handle = h
        self.n_params = w.size

    def close(self):
        if getattr(self, "handle", None):
            lib().sg_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self) -> torch.Tensor:
        """The model's device FP32 master blob as a tensor view (shares memory)."""
        ptr = lib().sg_model_weights(self.handle)
        return _wrap_device_ptr(ptr, self.n_params)

    def refresh(self, stream=None):
        _check("sg_model_refresh", lib().sg_model_refresh(self.handle, _stream(stream)))

    def reserve(self, B):
        """Size the sampling workspace for B configurations (sg_model_reserve)."""
        _check("sg_model_reserve", lib().sg_model_reserve(self.handle, B))

    def set_max_chunk(self, max_samples):
        """Cap the samples per chunk of sg_logprob / sg_grad (0: automatic)."""
        _check("sg_model_set_max_chunk", lib().sg_model_set_max_chunk(self.handle, max_samples))

    def check(self, stream=None):
        """Synchronise and raise if a kernel recorded a bounded-wait timeout or NaN."""
        _check("sg_model_check", lib().sg_model_check(self.handle, _stream(stream)))

    def sample(self, B, seed, stream_id=0, beta=1.0, flag_band=0.0, with_flags=False,
               spins=None, logq=None, stream=None):
        N = self.shape.N
        dev = torch.device("cuda")
        spins = torch.empty((B, N), dtype=torch.int8, device=dev) if spins is None else spins
        logq = torch.empty(B, dtype=torch.float32, device=dev) if logq is None else logq
        T = N // max(1, getattr(self.shape, "patch", 1))  # flags: one bit per token position
        flags = (torch.empty((B, (T + 31) // 32), dtype=torch.int32, device=dev)
                 if with_flags else None)
        _check("sg_sample", lib().sg_sample(
            self.handle, B, beta, seed, stream_id, flag_band, _dev(spins, torch.int8, (B, N)),
            _dev(logq, torch.float32, (B,)), _dev(flags, torch.int32), _stream(stream)))
        return (spins, logq, flags) if with_flags else (spins, logq)

    def muon_step(self, grad, momentum, adam_m, adam_v, lr, step, mu=0.95, weight_decay=0.0,
                  ns_steps=5, stream=None):
        """Muon on the weight matrices, AdamW on the rest, in place on weights()."""
        n = self.n_params
        _check("sg_muon_step", lib().sg_muon_step(
            self.handle, _dev(self.weights(), torch.float32, (n,)), _dev(grad, torch.float32, (n,)),
            _dev(momentum, torch.float32, (n,)), _dev(adam_m, torch.float32, (n,)),
            _dev(adam_v, torch.float32, (n,)), lr, mu, weight_decay, ns_steps, step,
            _stream(stream)))

    def logprob(self, spins, logq=None, stream=None):
        B = spins.shape[0]
        logq = torch.empty(B, dtype=torch.float32, device=spins.device) if logq is None else logq
        _check("sg_logprob", lib().sg_logprob(
            self.handle, _dev(spins, torch.int8, (B, self.shape.N)), B,
            _dev(logq, torch.float32, (B,)), _stream(stream)))
        return logq

    def grad(self, spins, coeff, grad=None, logq=None, stream=None):
        B = spins.shape[0]
        grad = (torch.empty(self.n_params, dtype=torch.float32, device=spins.device)
                if grad is None else grad)
        _check("sg_grad", lib().sg_grad(
            self.handle, _dev(spins, torch.int8, (B, self.shape.N)),
            _dev(coeff, torch.float32, (B,)), B, _dev(grad, torch.float32, (self.n_params,)),
            _dev(logq, torch.float32, (B,)), _stream(stream)))
        return grad


def _wrap_device_ptr(ptr, n):
    """A float32 CUDA tensor aliasing n floats at a device pointer owned by libsg."""
    class _Holder:
        pass
    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False),
                                  "version": 3, "strides": None}
    return torch.as_tensor(h, device="cuda")


class Instance:
    """Owns an sg_instance built from an ``inputs.Instance``."""

    def __init__(self, inst: _inputs.Instance):
        self.src = inst
        self.N = inst.N
        J = np.ascontiguousarray(inst.J, dtype=np.float32)
        kind = SG_SK_DENSE if inst.kind == "sk" else SG_EA_LATTICE
        h = ctypes.c_void_p()
        _check("sg_instance_create", lib().sg_instance_create(
            kind, inst.N, inst.D, inst.L, int(inst.periodic), J.ctypes.data_as(_P),
            ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().sg_instance_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, spins, precision=SG_FP32, E=None, E_int=None, want_int=False, stream=None):
        B = spins.shape[0]
        E = torch.empty(B, dtype=torch.float32, device=spins.device) if E is None else E
        if want_int and E_int is None:
            E_int = torch.empty(B, dtype=torch.int32, device=spins.device)
        _check("sg_energy", lib().sg_energy(
            self.handle, _dev(spins, torch.int8, (B, self.N)), B, precision,
            _dev(E, torch.float32, (B,)), _dev(E_int, torch.int32, (B,)), _stream(stream)))
        return (E, E_int) if want_int else E

    def metropolis(self, spins, sweeps, beta, seed, E=None, trace=False, stream=None):
        """In place on ``spins`` [R][N] int8; returns (E float64 [R], trace or None)."""
        R = spins.shape[0]
        if E is None:
            E = self.energy(spins).to(torch.float64)
        tr = (torch.empty((sweeps, R), dtype=torch.float32, device=spins.device)
              if trace else None)
        _check("sg_metropolis", lib().sg_metropolis(
            self.handle, _dev(spins, torch.int8, (R, self.N)), R, sweeps, beta, seed,
            _dev(E, torch.float64, (R,)), _dev(tr, torch.float32), _stream(stream)))
        return E, tr


def free_energy(E, logq, beta, out=None, coeff=None, want_coeff=False, stream=None):
    """Returns the device tensor [F_q, F_IS, ESS] (float64) and optionally coeff."""
    B = E.shape[0]
    out = torch.empty(3, dtype=torch.float64, device=E.device) if out is None else out
    if want_coeff and coeff is None:
        coeff = torch.empty(B, dtype=torch.float32, device=E.device)
    _check("sg_free_energy", lib().sg_free_energy(
        _dev(E, torch.float32, (B,)), _dev(logq, torch.float32, (B,)), B, beta,
        _dev(out, torch.float64, (3,)), _dev(coeff, torch.float32, (B,)), _stream(stream)))
    return (out, coeff) if want_coeff else out


def loss_coeff(E, logq, a, c, w=0.0, coeff=None, mean=None, stream=None):
    """REINFORCE weights (a E + c ln q - mean - w) / B; returns (coeff, mean[2])."""
    B = E.shape[0]
    coeff = torch.empty(B, dtype=torch.float32, device=E.device) if coeff is None else coeff
    mean = torch.empty(2, dtype=torch.float64, device=E.device) if mean is None else mean
    _check("sg_loss_coeff", lib().sg_loss_coeff(
        _dev(E, torch.float32, (B,)), _dev(logq, torch.float32, (B,)), B, a, c, w,
        _dev(mean, torch.float64, (2,)), _dev(coeff, torch.float32, (B,)), _stream(stream)))
    return coeff, mean


def gelu_selfcheck(n=1 << 20):
    """Largest errors of the BF16 path's GELU and GELU' against erff / expf
    over n points of [-12, 12] (sg_gelu_selfcheck)."""
    eg, ed = ctypes.c_double(), ctypes.c_double()
    _check("sg_gelu_selfcheck", lib().sg_gelu_selfcheck(n, ctypes.byref(eg), ctypes.byref(ed)))
    return eg.value, ed.value


def mh_step(prop_spins, E, logq, C, beta, seed, chain_spins, chain_E, chain_lq, accepts=None,
            trace=False, stream=None):
    B, N = prop_spins.shape
    accepts = (torch.empty(C, dtype=torch.int64, device=E.device) if accepts is None
               else accepts)
    tr = torch.empty((B // C, C), dtype=torch.float32, device=E.device) if trace else None
    _check("sg_mh_step", lib().sg_mh_step(
        _dev(prop_spins, torch.int8, (B, N)), _dev(E, torch.float32, (B,)),
        _dev(logq, torch.float32, (B,)), B, N, C, beta, seed,
        _dev(chain_spins, torch.int8, (C, N)), _dev(chain_E, torch.float64, (C,)),
        _dev(chain_lq, torch.float64, (C,)), _dev(accepts, torch.int64, (C,)),
        _dev(tr, torch.float32), _stream(stream)))
    return accepts, tr


def overlap_hist(spins, hist=None, stream=None):
    B, N = spins.shape
    hist = torch.empty(N + 1, dtype=torch.int64, device=spins.device) if hist is None else hist
    _check("sg_overlap_hist", lib().sg_overlap_hist(
        _dev(spins, torch.int8, (B, N)), B, N, _dev(hist, torch.int64, (N + 1,)),
        _stream(stream)))
    return hist


def adam_step(w, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    n = w.numel()
    _check("sg_adam_step", lib().sg_adam_step(
        _dev(w, torch.float32, (n,)), _dev(g, torch.float32, (n,)), _dev(m, torch.float32, (n,)),
        _dev(v, torch.float32, (n,)), n, lr, beta1, beta2, eps, step, _stream(stream)))
