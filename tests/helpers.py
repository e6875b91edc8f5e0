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


def oracle_replay(m, w, seed, gpu_spins, gpu_flags, band, rows=None, stream=0, n_threads=0):
    """Oracle ancestral samples of the given sample indices, replaying the
    GPU's decision at every draw the GPU flagged (the protocol for draws with
    |p+ - u| inside the flag band).  Returns spins, logq, pplus, oracle flags.

    ``band`` is the GPU's flag band.  A flag only excuses a draw the oracle
    also finds close: at every GPU-flagged draw of an unpatched model, the
    oracle's own p+ (computed from the same prefix) must lie within 2 band of
    the draw's uniform u, so a wrong GPU logit cannot hide behind its flag.  For
    a patched model, u must lie within 2 band of the oracle's cumulative
    probability interval of the class the GPU drew."""
    rows = np.arange(gpu_spins.shape[0]) if rows is None else np.asarray(rows, np.int64)
    T = m.N // max(1, getattr(m, "patch", 1))  # flags are per token position
    fl = unpack_flags(gpu_flags[rows], T)
    if T < m.N:
        fl = np.pad(fl, ((0, 0), (0, m.N - T)))
    patched = T < m.N
    res = oracle.sample(ocfg(m), w, len(rows), seed, stream, override_mask=fl,
                        override_spins=gpu_spins[rows], n_threads=n_threads, rows=rows,
                        with_cdf=patched)
    pp = res[2]
    for i, t in zip(*np.nonzero(fl)):
        u = oracle.uniform(seed, int(rows[i]), int(t), stream)
        if not patched:
            assert abs(pp[i, t] - u) < 2 * band, (
                f"GPU flagged draw (row {rows[i]}, t {t}) but the oracle's p+ {pp[i, t]:.6g} "
                f"is {abs(pp[i, t] - u):.3g} from u {u:.6g} (band {band})")
        else:
            # the GPU's class: u inside the oracle's interval of that class,
            # widened by 2 band
            lo = res[4][i, t]
            assert lo - 2 * band < u < lo + pp[i, t] + 2 * band, (
                f"GPU flagged draw (row {rows[i]}, token {t}) took a class whose oracle "
                f"interval [{lo:.6g}, {lo + pp[i, t]:.6g}) is more than 2 band from u {u:.6g}")
    return res[:4]


def grad_block_errors(m, g, go):
    """Per blob tensor (inputs.segments order): name, |g - go|, |go| and the
    norm the tensor would have if |go| were spread evenly over the blob."""
    n_tot = go.size
    tot = float(np.linalg.norm(go))
    out = []
    for name, (off, shape) in inputs.offsets(m).items():
        n = int(np.prod(shape))
        d = float(np.linalg.norm(g[off:off + n] - go[off:off + n]))
        r = float(np.linalg.norm(go[off:off + n]))
        out.append((name, d, r, tot * np.sqrt(n / n_tot)))
    return out


def assert_grad_blocks(m, g, go, rel, floor=0.1):
    """Every weight tensor's gradient within ``rel`` of the oracle's, relative
    to its own norm, or to ``floor`` times its even-spread share of the total
    norm for tensors whose true gradient is that small.  A wrong block (a
    dropped bias or LayerNorm gradient, a swapped head) fails it even when the
    whole blob's relative error is small."""
    bad = [(n, d, r, e) for n, d, r, e in grad_block_errors(m, g, go)
           if d > rel * max(r, floor * e)]
    assert not bad, "gradient blocks off: " + ", ".join(
        f"{n} (|d| {d:.3g}, |g| {r:.3g})" for n, d, r, _ in bad[:8])
