"""FP64 CPU oracle for the FlashVAN hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2606_22984_gb300``) never imports it and fails loudly when its
CUDA library is missing.

The arithmetic lives in ``sg_oracle.c`` (plain C, double precision, one
function per paper passage).  This module only compiles it with gcc and
marshals numpy arrays through ctypes.

Every function is pinned by tests/test_oracle_pins.py against something other
than itself: closed forms, enumeration, an independent composition from
PyTorch routines, finite differences, exact Boltzmann laws and, for
Philox4x32-10, PyTorch's independent header-only engine word for word.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsg_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile sg_oracle.c into a shared library with gcc (OpenMP if present)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrCfg(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("N", "n_layers", "d", "n_heads", "d_token", "d_ff", "mask_kind", "W", "S",
                 "patch", "lat_D", "lat_L")]


@dataclass
class ModelCfg:
    """Model shape as the paper's hyper-parameter tables name it."""
    N: int
    n_layers: int
    d: int
    n_heads: int
    d_token: int = 2
    d_ff: int = 0          # 0 -> 4 d
    mask_kind: int = 0     # 0 dense causal, 1 band + sink (W, S in tokens)
    W: int = 0
    S: int = 0
    patch: int = 1         # spins per token (2^D for a lattice of dimension D)
    lat_D: int = 0         # lattice of the patch map (0: consecutive spins)
    lat_L: int = 0

    def __post_init__(self):
        if self.d_ff == 0:
            self.d_ff = 4 * self.d

    def c(self) -> OrCfg:
        return OrCfg(self.N, self.n_layers, self.d, self.n_heads, self.d_token, self.d_ff,
                     self.mask_kind, self.W, self.S, self.patch, self.lat_D, self.lat_L)


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_I32 = ctypes.c_int32
_I = ctypes.c_int


def lib():
    """The compiled oracle.  ``SG_ORACLE_LIB`` names another build of the same
    source to load instead; the mutation tests use it to run the pins against
    copies of the oracle with a planted mistake."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("SG_ORACLE_LIB") or build())
        L.or_param_count.argtypes = [ctypes.POINTER(OrCfg)]
        L.or_param_count.restype = _I64
        L.or_philox.argtypes = [_P, _P, _P]
        L.or_uniform.argtypes = [_U64, _U32, _U32, _U32, _U32]
        L.or_uniform.restype = _D
        L.or_sample.argtypes = [ctypes.POINTER(OrCfg), _P, _I64, _P, _U64, _U32, _D, _P, _P, _P,
                                _P, _P, _P, _I, _P]
        L.or_logprob.argtypes = [ctypes.POINTER(OrCfg), _P, _I64, _P, _P, _P, _I]
        L.or_grad.argtypes = [ctypes.POINTER(OrCfg), _P, _I64, _P, _P, _P, _P, _I]
        L.or_energy_sk.argtypes = [_I, _P, _I64, _P, _P]
        L.or_energy_ea.argtypes = [_I, _I, _I, _P, _I64, _P, _P]
        L.or_free_energy.argtypes = [_I64, _P, _P, _D, _P]
        L.or_loss_coeff.argtypes = [_I64, _P, _P, _D, _D, _D, _P, _P]
        L.or_newton_schulz.argtypes = [_P, _I32, _I32, _I32, _P]
        L.or_muon_step.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _D, _I32, _I64]
        L.or_enumerate.argtypes = [ctypes.POINTER(OrCfg), _P, _I, _I, _I, _I, _P, _D, _P, _I]
        L.or_mh.argtypes = [_I64, _I, _P, _P, _D, _U64, _D, _P, _P, _P, _P, _P, _P, _P]
        L.or_metropolis.argtypes = [_I, _I, _I, _I, _I, _P, _I64, _I, _D, _U64, _P, _P, _P, _P]
        L.or_overlap_hist.argtypes = [_I, _I64, _P, _P]
        L.or_num_threads.restype = _I
        for fn in ("or_sample", "or_logprob", "or_grad", "or_enumerate", "or_mh", "or_metropolis"):
            getattr(L, fn).restype = _I
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def param_count(cfg: ModelCfg) -> int:
    return int(lib().or_param_count(ctypes.byref(cfg.c())))


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed, a, b, stream, e=0):
    return lib().or_uniform(seed, a, b, stream, e)


def num_threads() -> int:
    return int(lib().or_num_threads())


def sample(cfg: ModelCfg, weights, B, seed, stream=0, flag_band=1e-5, override_mask=None,
           override_spins=None, n_threads=0, rows=None, with_cdf=False):
    """Ancestral sampling (Algorithm 2).  Returns spins, logq, pplus, flags.
    ``rows`` (optional) lists the sample index of each output row; then B is
    its length.  ``with_cdf`` (patched models) also returns cdf_lo [B][N]: the
    cumulative probability of the classes before each drawn class, whose
    interval is then [cdf_lo, cdf_lo + pplus)."""
    w = _f64(weights)
    N = cfg.N
    rid = None
    if rows is not None:
        rid = np.ascontiguousarray(rows, dtype=np.int64)
        B = rid.shape[0]
    spins = np.zeros((B, N), np.int8)
    logq = np.zeros(B, np.float64)
    pplus = np.zeros((B, N), np.float64)
    flags = np.zeros((B, N), np.uint8)
    cdf_lo = np.zeros((B, N), np.float64) if with_cdf else None
    om = None if override_mask is None else np.ascontiguousarray(override_mask, dtype=np.uint8)
    os_ = None if override_spins is None else _i8(override_spins)
    rc = lib().or_sample(ctypes.byref(cfg.c()), _ptr(w), B, _ptr(rid), seed, stream, flag_band, _ptr(om),
                         _ptr(os_), _ptr(spins), _ptr(logq), _ptr(pplus), _ptr(flags), n_threads,
                         _ptr(cdf_lo))
    assert rc == 0
    return (spins, logq, pplus, flags, cdf_lo) if with_cdf else (spins, logq, pplus, flags)


def logprob(cfg: ModelCfg, weights, spins, n_threads=0, with_pplus=False):
    """Teacher-forced log q (Algorithm 1)."""
    w = _f64(weights)
    s = _i8(spins)
    B = s.shape[0]
    logq = np.zeros(B, np.float64)
    pplus = np.zeros((B, cfg.N), np.float64) if with_pplus else None
    rc = lib().or_logprob(ctypes.byref(cfg.c()), _ptr(w), B, _ptr(s), _ptr(logq), _ptr(pplus),
                          n_threads)
    assert rc == 0
    return (logq, pplus) if with_pplus else logq


def grad(cfg: ModelCfg, weights, spins, coeff, n_threads=0):
    """sum_b coeff_b * grad log q(sigma_b) in blob layout; also returns log q."""
    w = _f64(weights)
    s = _i8(spins)
    c = _f64(coeff)
    B = s.shape[0]
    g = np.zeros(param_count(cfg), np.float64)
    lq = np.zeros(B, np.float64)
    rc = lib().or_grad(ctypes.byref(cfg.c()), _ptr(w), B, _ptr(s), _ptr(c), _ptr(g), _ptr(lq),
                       n_threads)
    assert rc == 0
    return g, lq


def energy_sk(J, spins):
    J = _f32(J)
    s = _i8(spins)
    E = np.zeros(s.shape[0], np.float64)
    lib().or_energy_sk(J.shape[0], _ptr(J), s.shape[0], _ptr(s), _ptr(E))
    return E


def energy_ea(D, L, bonds, spins, periodic=True):
    b = _f32(bonds)
    s = _i8(spins)
    E = np.zeros(s.shape[0], np.float64)
    lib().or_energy_ea(D, L, int(periodic), _ptr(b), s.shape[0], _ptr(s), _ptr(E))
    return E


def energy(inst, spins):
    if inst.kind == "sk":
        return energy_sk(inst.J, spins)
    return energy_ea(inst.D, inst.L, inst.J, spins, inst.periodic)


def free_energy(E, logq, beta):
    """(F_q, F_IS, Kish ESS) of Eqs. (KL_div), (free_energy)."""
    E = _f64(E)
    lq = _f64(logq)
    out = np.zeros(3, np.float64)
    lib().or_free_energy(E.shape[0], _ptr(E), _ptr(lq), beta, _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def loss_coeff(E, logq, a, c, w=0.0):
    """REINFORCE weights (a E + c ln q - mean - w) / B of Eqs. loss1 / loss2;
    returns (coeff, mean L, mean E)."""
    E = _f64(E)
    lq = _f64(logq)
    coeff = np.zeros(E.shape[0], np.float64)
    mean = np.zeros(2, np.float64)
    lib().or_loss_coeff(E.shape[0], _ptr(E), _ptr(lq), a, c, w, _ptr(mean), _ptr(coeff))
    return coeff, float(mean[0]), float(mean[1])


def newton_schulz(M, steps=5):
    """The quintic Newton-Schulz orthogonalisation of Muon (FP64)."""
    M = _f64(M)
    O = np.zeros_like(M)
    lib().or_newton_schulz(_ptr(M), M.shape[0], M.shape[1], steps, _ptr(O))
    return O


def muon_step(cfg: ModelCfg, w, g, mom, am, av, lr, mu, wd, ns_steps, step):
    """One Muon step on the blob (matrices) with AdamW on the rest; arrays
    updated in place (float64)."""
    for a in (w, mom, am, av):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().or_muon_step(ctypes.byref(cfg.c()), _ptr(w), _ptr(g), _ptr(mom), _ptr(am), _ptr(av), lr, mu,
                       wd, ns_steps, step)


def enumerate_exact(cfg: ModelCfg, weights, inst, beta, n_threads=0):
    """Exhaustive enumeration: dict(sum_q, lnZ, F, Fq, Emin)."""
    w = _f64(weights)
    J = _f32(inst.J)
    out = np.zeros(5, np.float64)
    kind = 0 if inst.kind == "sk" else 1
    D = getattr(inst, "D", 0)
    L = getattr(inst, "L", 0)
    per = int(getattr(inst, "periodic", True))
    rc = lib().or_enumerate(ctypes.byref(cfg.c()), _ptr(w), kind, D, L, per, _ptr(J), beta,
                            _ptr(out), n_threads)
    assert rc == 0
    return dict(sum_q=out[0], lnZ=out[1], F=out[2], Fq=out[3], Emin=out[4])


def mh(E, logq, C, beta, seed, chain_E, chain_lq, chain_idx=None, flag_band=1e-9,
       override_acc=None):
    """Chain-ordered independence MH.  Returns (chain_E, chain_lq, chain_idx, trace, accepts, flags)."""
    E = _f64(E)
    lq = _f64(logq)
    B = E.shape[0]
    cE = _f64(chain_E).copy()
    cL = _f64(chain_lq).copy()
    ci = (np.full(C, -1, np.int64) if chain_idx is None
          else np.ascontiguousarray(chain_idx, dtype=np.int64).copy())
    trace = np.zeros((B // C, C), np.float64)
    acc = np.zeros(C, np.int64)
    flags = np.zeros(B, np.uint8)
    ov = None if override_acc is None else _i8(override_acc)
    rc = lib().or_mh(B, C, _ptr(E), _ptr(lq), beta, seed, flag_band, _ptr(ov), _ptr(cE), _ptr(cL),
                     _ptr(ci), _ptr(trace), _ptr(acc), _ptr(flags))
    assert rc == 0
    return cE, cL, ci, trace, acc, flags


def metropolis(inst, spins, sweeps, beta, seed):
    """Single-spin-flip Metropolis.  Returns (spins, E, trace[sweeps][R], n_flagged)."""
    s = _i8(spins).copy()
    R = s.shape[0]
    E = energy(inst, s).astype(np.float64)
    trace = np.zeros((sweeps, R), np.float64)
    nflag = np.zeros(1, np.int64)
    kind = 0 if inst.kind == "sk" else 1
    J = _f32(inst.J)
    rc = lib().or_metropolis(kind, inst.N, getattr(inst, "D", 0), getattr(inst, "L", 0),
                             int(getattr(inst, "periodic", True)), _ptr(J), R, sweeps, beta, seed,
                             _ptr(s), _ptr(E), _ptr(trace), _ptr(nflag))
    assert rc == 0
    return s, E, trace, int(nflag[0])


def overlap_hist(spins):
    s = _i8(spins)
    B, N = s.shape
    h = np.zeros(N + 1, np.int64)
    lib().or_overlap_hist(N, B, _ptr(s), _ptr(h))
    return h
