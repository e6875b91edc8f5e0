"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
of the documented shapes and lays them out.  Both the CUDA library and the
CPU oracle consume what it produces, so neither depends on the other.

* Weight blob: one flat float32 array in the documented order
  (tok, pos, per layer [ln1_g, ln1_b, Wqkv, bqkv, ln2_g, ln2_b, W1, b1, W2,
  b2], lnf_g, lnf_b, Wh, bh).  Random init: embeddings N(0, 1); linear maps
  and biases U(-1/sqrt(fan_in), 1/sqrt(fan_in)); LayerNorm gain 1, bias 0.
* SK couplings: J_ij ~ N(0, 1/N) for i < j, symmetric, zero diagonal (the
  paper's N(0,1) with the 1/sqrt(N) prefactor folded in, Eq. SKHam).
* EA bonds: bonds[i, mu] couples raster site i = x0 + L x1 + L^2 x2 to its
  +mu neighbour; +-1 with p = 0.5 or N(0, 1) (Eq. EAHam).

numpy's Philox bit generator keyed by the seed makes every array
reproducible on any host.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ModelShape:
    """Transformer shape (paper's Supplementary Table of symbols)."""
    N: int
    n_layers: int
    d: int
    n_heads: int
    d_token: int = 2
    d_ff: int = 0
    mask_kind: int = 0     # 0 dense causal, 1 band + sink (W, S counted in tokens)
    W: int = 0
    S: int = 0
    patch: int = 1         # spins per token P (patching: 2^D spins of a lattice cell)
    lat_D: int = 0         # lattice of the patch map (0: token t holds spins tP..tP+P-1)
    lat_L: int = 0

    def __post_init__(self):
        if self.d_ff == 0:
            self.d_ff = 4 * self.d

    @property
    def n_tokens(self) -> int:
        return self.N // max(1, self.patch)

    @property
    def n_classes(self) -> int:
        return 1 << max(1, self.patch)


@dataclass
class Instance:
    """A spin-glass instance: kind 'sk' (dense J[N][N]) or 'ea' (bonds[N][D])."""
    kind: str
    N: int
    J: np.ndarray
    D: int = 0
    L: int = 0
    periodic: bool = True
    pm: bool = False       # +-1 couplings (integer energies)


def _rng(seed: int, salt: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, salt]))


def segments(m: ModelShape):
    """(name, shape, init) for every tensor of the blob, in blob order."""
    d, f, K = m.d, m.d_ff, m.n_classes
    segs = [("tok", (K, m.d_token), "normal"), ("pos", (m.n_tokens, d - m.d_token), "normal")]
    for l in range(m.n_layers):
        segs += [
            (f"l{l}.ln1_g", (d,), "ones"), (f"l{l}.ln1_b", (d,), "zeros"),
            (f"l{l}.Wqkv", (3 * d, d), ("unif", d)), (f"l{l}.bqkv", (3 * d,), ("unif", d)),
            (f"l{l}.ln2_g", (d,), "ones"), (f"l{l}.ln2_b", (d,), "zeros"),
            (f"l{l}.W1", (f, d), ("unif", d)), (f"l{l}.b1", (f,), ("unif", d)),
            (f"l{l}.W2", (d, f), ("unif", f)), (f"l{l}.b2", (d,), ("unif", f)),
        ]
    segs += [("lnf_g", (d,), "ones"), ("lnf_b", (d,), "zeros"),
             ("Wh", (K, d), ("unif", d)), ("bh", (K,), ("unif", d))]
    return segs


def param_count(m: ModelShape) -> int:
    return int(sum(np.prod(s) for _, s, _ in segments(m)))


def offsets(m: ModelShape) -> dict:
    """name -> (offset, shape) inside the blob."""
    out, o = {}, 0
    for name, shape, _ in segments(m):
        out[name] = (o, shape)
        o += int(np.prod(shape))
    return out


def make_weights(m: ModelShape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded random-init float32 weight blob.  ``scale`` multiplies every
    random (non-LayerNorm) tensor, e.g. to make a sharper or flatter model."""
    rng = _rng(seed, 3)
    parts = []
    for _, shape, init in segments(m):
        n = int(np.prod(shape))
        if init == "ones":
            parts.append(np.ones(n))
        elif init == "zeros":
            parts.append(np.zeros(n))
        elif init == "normal":
            parts.append(scale * rng.standard_normal(n))
        else:
            bound = 1.0 / np.sqrt(init[1])
            parts.append(scale * rng.uniform(-bound, bound, n))
    return np.concatenate(parts).astype(np.float32)


def make_sk(N: int, seed: int) -> Instance:
    rng = _rng(seed, 1)
    g = rng.standard_normal((N, N)) / np.sqrt(N)
    J = np.triu(g, 1)
    J = (J + J.T).astype(np.float32)
    return Instance("sk", N, J)


def make_ea(D: int, L: int, seed: int, pm: bool = True, periodic: bool = True) -> Instance:
    rng = _rng(seed, 2)
    N = L ** D
    if pm:
        J = np.where(rng.random((N, D)) < 0.5, 1.0, -1.0)
    else:
        J = rng.standard_normal((N, D))
    return Instance("ea", N, J.astype(np.float32), D=D, L=L, periodic=periodic, pm=pm)


def make_ferro(D: int, L: int, periodic: bool = True) -> Instance:
    N = L ** D
    return Instance("ea", N, np.ones((N, D), np.float32), D=D, L=L, periodic=periodic, pm=True)


def make_group_weights(m: ModelShape, seed: int, n: int, scale: float = 1.0) -> np.ndarray:
    """Blobs of a group of n models of one shape, concatenated; model i
    draws its weights from seed + 7919 i."""
    return np.concatenate([make_weights(m, seed + 7919 * i, scale) for i in range(n)])


def random_spins(B: int, N: int, seed: int) -> np.ndarray:
    rng = _rng(seed, 4)
    return np.where(rng.random((B, N)) < 0.5, 1, -1).astype(np.int8)


@dataclass
class Workload:
    """One of the five synthetic workloads (sizes of the paper's experiments)."""
    name: str
    model: ModelShape
    make_instance: object
    betas: list
    B: int
    seed: int
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def instance(self) -> Instance:
        return self.make_instance()

    def weights(self, scale: float = 1.0) -> np.ndarray:
        return make_weights(self.model, self.seed, scale)

    def group_weights(self, scale: float = 1.0) -> np.ndarray:
        """One model per beta, blobs concatenated (model i seeded seed + 7919 i)."""
        return make_group_weights(self.model, self.seed, len(self.betas), scale)


def lattice_mask(D: int, L: int):
    """(W, S) of the band + sink reading for a D-dim lattice of side L:
    band W = L^(D-1) >= d_max (SI Sec. I.A); sink S = L^(D-1) + 1 keys
    (start token plus the first row / plane, reached through the periodic
    wrap)."""
    w = L ** (D - 1)
    return w, w + 1


def workloads() -> dict:
    W2, S2 = lattice_mask(2, 16)
    W3, S3 = lattice_mask(3, 10)
    W5, S5 = lattice_mask(2, 64)
    return {
        "sk20": Workload("SK N=20 beta=1.0, 2L d32 h4, B=4096, dense",
                         ModelShape(20, 2, 32, 4), lambda: make_sk(20, 1), [1.0], 4096, 1),
        "ea2d16": Workload("2D EA L=16 +-J periodic, 4L d64 h4, band W=16 S=17, B=16384",
                           ModelShape(256, 4, 64, 4, mask_kind=1, W=W2, S=S2),
                           lambda: make_ea(2, 16, 2, pm=True), [0.5, 1.0, 2.0], 16384, 2),
        "sk1024": Workload("SK N=1024 beta=1.5, 6L d128 h8, dense, B=8192",
                           ModelShape(1024, 6, 128, 8), lambda: make_sk(1024, 3), [1.5], 8192, 3),
        "ea3d10": Workload("3D EA L=10 +-J periodic, 6L d128 h8, band W=100 S=101, B=32768",
                           ModelShape(1000, 6, 128, 8, mask_kind=1, W=W3, S=S3),
                           lambda: make_ea(3, 10, 4, pm=True), [0.9], 32768, 4),
        "ea2d64": Workload("2D EA L=64 Gaussian periodic, 8L d256 h8, band W=64 S=65, 8 betas x B=1024",
                           ModelShape(4096, 8, 256, 8, mask_kind=1, W=W5, S=S5),
                           lambda: make_ea(2, 64, 5, pm=False), list(np.linspace(0.2, 3.0, 8)),
                           1024, 5),
    }
