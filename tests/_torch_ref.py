"""An independent composition of the FlashVAN forward from PyTorch library
routines (layer_norm, linear, scaled_dot_product_attention, gelu, logsigmoid)
in float64 on the CPU.  Used only to pin the C oracle: a mistake in the
oracle's own loops (an index, a dropped term, a transposed operand) makes the
two disagree, and autograd through it checks the oracle's hand-written
backward.
"""
import numpy as np
import torch
import torch.nn.functional as F

from paper_2606_22984_gb300 import inputs


def patch_sites(m: inputs.ModelShape) -> np.ndarray:
    """[T, P] raster site of bit j of token t: patches of 2^D sites of a
    periodic lattice in raster order of the patch grid, bit j at offset
    (j & 1, (j >> 1) & 1, ...) from the even corner; consecutive spins when
    there is no lattice."""
    P = max(1, m.patch)
    T = m.N // P
    if P == 1 or m.lat_D == 0:
        return np.arange(T * P).reshape(T, P)
    D, L = m.lat_D, m.lat_L
    M = L // 2
    grid = np.stack(np.unravel_index(np.arange(T), (M,) * D, order="F"), -1)   # [T, D] patch coords
    offs = np.array([[(j >> k) & 1 for k in range(D)] for j in range(P)])       # [P, D]
    coords = 2 * grid[:, None, :] + offs[None, :, :]                            # [T, P, D]
    return np.ravel_multi_index(tuple(coords[..., k] for k in range(D)), (L,) * D, order="F")


def allowed_mask(m: inputs.ModelShape) -> torch.Tensor:
    T = m.N // max(1, m.patch)
    t = torch.arange(T)[:, None]
    k = torch.arange(T)[None, :]
    causal = k <= t
    if m.mask_kind == 0:
        return causal
    return causal & ((t - k <= m.W) | (k < m.S))


def logq(m: inputs.ModelShape, w: torch.Tensor, spins: np.ndarray) -> torch.Tensor:
    off = inputs.offsets(m)

    def P(name):
        o, shape = off[name]
        return w[o:o + int(np.prod(shape))].view(*shape)

    s = torch.as_tensor(np.asarray(spins, dtype=np.int64))
    B = s.shape[0]
    d, nh = m.d, m.n_heads
    dh = d // nh
    sites = torch.as_tensor(patch_sites(m))                       # [T, P]
    N = sites.shape[0]
    bits = (s[:, sites] + 1) // 2                                 # [B, T, P]
    tok = (bits * (2 ** torch.arange(sites.shape[1]))).sum(-1)    # [B, T]
    tok_in = torch.zeros(B, N, dtype=torch.int64)
    tok_in[:, 1:] = tok[:, :-1]
    h = torch.cat([P("tok")[tok_in], P("pos")[None].expand(B, N, d - m.d_token)], dim=-1)
    mask = allowed_mask(m)
    for l in range(m.n_layers):
        a = F.layer_norm(h, (d,), P(f"l{l}.ln1_g"), P(f"l{l}.ln1_b"), eps=1e-5)
        qkv = F.linear(a, P(f"l{l}.Wqkv"), P(f"l{l}.bqkv"))
        q, k, v = (qkv[..., i * d:(i + 1) * d].reshape(B, N, nh, dh).transpose(1, 2)
                   for i in range(3))
        o = F.scaled_dot_product_attention(q, k, v, attn_mask=mask)
        h = h + o.transpose(1, 2).reshape(B, N, d)
        a2 = F.layer_norm(h, (d,), P(f"l{l}.ln2_g"), P(f"l{l}.ln2_b"), eps=1e-5)
        h = h + F.linear(F.gelu(F.linear(a2, P(f"l{l}.W1"), P(f"l{l}.b1"))), P(f"l{l}.W2"),
                         P(f"l{l}.b2"))
    y = F.layer_norm(h, (d,), P("lnf_g"), P("lnf_b"), eps=1e-5)
    z = F.linear(y, P("Wh"), P("bh"))
    if max(1, m.patch) > 1:
        return torch.log_softmax(z, -1).gather(-1, tok[..., None])[..., 0].sum(-1)
    ell = z[..., 1] - z[..., 0]
    return F.logsigmoid(s.to(torch.float64) * ell).sum(-1)
