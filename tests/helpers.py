"""Shared helpers for the parity tests (test code only)."""
import numpy as np

import oracle
from paper_2606_22984_gb300 import inputs


def ocfg(m: inputs.ModelShape) -> oracle.ModelCfg:
    return oracle.ModelCfg(**vars(m))


def unpack_flags(flags: np.ndarray, N: int) -> np.ndarray:
    """uint32 words [B][ceil(N/32)] -> bool [B][N] (bit t of word t/32)."""
    f = np.ascontiguousarray(flags).view(np.uint32)
    B = f.shape[0]
    bits = (f[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1
    return bits.reshape(B, -1)[:, :N].astype(bool)


def oracle_replay(m, w, seed, gpu_spins, gpu_flags, rows=None, stream=0, n_threads=0):
    """Oracle ancestral samples of the given sample indices, replaying the
    GPU's decision at every draw the GPU flagged (the protocol for draws with
    |p+ - u| inside the flag band).  Returns spins, logq, pplus, oracle flags."""
    rows = np.arange(gpu_spins.shape[0]) if rows is None else np.asarray(rows, np.int64)
    T = m.N // max(1, getattr(m, "patch", 1))  # flags are per token position
    fl = unpack_flags(gpu_flags[rows], T)
    if T < m.N:
        fl = np.pad(fl, ((0, 0), (0, m.N - T)))
    return oracle.sample(ocfg(m), w, len(rows), seed, stream, override_mask=fl,
                         override_spins=gpu_spins[rows], n_threads=n_threads, rows=rows)
