"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

Each test ties an oracle function to something other than itself: a value the
paper prints, a closed form, an invariant, brute force over all states, or an
independent composition from PyTorch library routines.  None of these needs a
GPU and none reads the CUDA path.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.special
import torch

import oracle
from paper_2606_22984_gb300 import inputs

import _torch_ref

HERE = os.path.dirname(os.path.abspath(__file__))


def ocfg(m: inputs.ModelShape) -> oracle.ModelCfg:
    return oracle.ModelCfg(**vars(m))


def all_states(N):
    """Every configuration of N spins, +-1, as int8 [2^N, N]."""
    idx = np.arange(2 ** N)[:, None]
    bits = (idx >> np.arange(N)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


# --------------------------------------------------------------------------
# Philox4x32-10: word for word against PyTorch's independent header-only
# engine, plus the uniform's definition and its statistics
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def torch_philox():
    """PyTorch's at::philox_engine (ATen/core/PhiloxRNGEngine.h, source only)
    compiled into a small helper library with g++."""
    import ctypes
    import os
    import shutil
    import subprocess
    import tempfile

    import torch

    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(hdr):
        pytest.skip("g++ or PyTorch's PhiloxRNGEngine.h not available")
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "philox_torch_ref.cpp")
    out = os.path.join(tempfile.mkdtemp(prefix="philox_ref_"), "libphilox_ref.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", inc, src, "-o", out],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.torch_philox_blocks.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64]

    def blocks(ctr, key):
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
        key = np.ascontiguousarray(key, dtype=np.uint32)
        res = np.zeros((ctr.shape[0], 4), np.uint32)
        lib.torch_philox_blocks(ctr.ctypes.data, key.ctypes.data, res.ctypes.data, ctr.shape[0])
        return res

    return blocks


def test_philox_matches_pytorch_engine_word_for_word(torch_philox):
    """The oracle's Philox4x32-10 against PyTorch's engine on 4096 random
    (counter, key) pairs and on the edge words (all zeros, all ones, single
    high bits): every one of the four output words equal."""
    rng = np.random.default_rng(20260604)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    edge = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
    ec = np.array([[a, b, c, d] for a in edge for b in (0, 0xFFFFFFFF) for c in edge
                   for d in (0, 0xFFFFFFFF)], np.uint32)
    ek = np.array([[a, b] for a in (0, 0xFFFFFFFF) for b in (0, 0xFFFFFFFF)], np.uint32)
    ctr = np.concatenate([ctr, np.repeat(ec, len(ek), 0)])
    key = np.concatenate([key, np.tile(ek, (len(ec), 1))])
    ref = torch_philox(ctr, key)
    ours = np.array([oracle.philox(c, k) for c, k in zip(ctr, key)], np.uint32)
    assert np.array_equal(ours, ref)


def test_philox_uniform_counter_layout_matches_pytorch_engine(torch_philox):
    """u(seed, a, b, stream, e) reads word 0 of the block with counter
    (a, b, stream, e) and key (seed lo, seed hi), for 64-bit seeds."""
    rng = np.random.default_rng(7)
    for seed in (0, 1, 12345, 2 ** 32 + 17, 2 ** 64 - 1):
        abse = rng.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64).astype(np.uint32)
        abse[:, 2] %= 4   # stream ids in use
        key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32), (200, 1))
        x0 = torch_philox(abse, key)[:, 0]
        u = np.array([oracle.uniform(seed, *map(int, r)) for r in abse])
        assert np.array_equal(u, ((x0 >> 8).astype(np.float64) + 0.5) / 2 ** 24)


def test_philox_uniform_definition_and_statistics():
    seed = 12345
    us = np.array([oracle.uniform(seed, b, t, 0) for b in range(64) for t in range(256)])
    # u = ((x0 >> 8) + 0.5) 2^-24: a half-integer multiple of 2^-24 inside (0, 1)
    k = us * 2 ** 24 - 0.5
    assert np.all(k == np.round(k)) and k.min() >= 0 and k.max() < 2 ** 24
    x0 = oracle.philox([3, 7, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[0]
    assert oracle.uniform(seed, 3, 7, 0) == ((int(x0) >> 8) + 0.5) / 2 ** 24
    # uniformity: chi^2 over 64 bins, mean, lag-1 correlation
    counts, _ = np.histogram(us, bins=64, range=(0, 1))
    chi2 = ((counts - len(us) / 64) ** 2 / (len(us) / 64)).sum()
    assert scipy_chi2_sf(chi2, 63) > 1e-4
    assert abs(us.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(us))
    assert abs(np.corrcoef(us[:-1], us[1:])[0, 1]) < 4 / math.sqrt(len(us))


def scipy_chi2_sf(x, dof):
    import scipy.stats
    return scipy.stats.chi2.sf(x, dof)


def test_philox_avalanche():
    """Flipping any single counter or key bit changes about half the 128 output bits."""
    base_c, base_k = np.array([1, 2, 3, 4], np.uint32), np.array([5, 6], np.uint32)
    ref = oracle.philox(base_c, base_k)
    dists = []
    for word in range(6):
        for bit in range(32):
            c, k = base_c.copy(), base_k.copy()
            if word < 4:
                c[word] ^= np.uint32(1 << bit)
            else:
                k[word - 4] ^= np.uint32(1 << bit)
            out = oracle.philox(c, k)
            dists.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(ref, out)))
    dists = np.array(dists)
    assert abs(dists.mean() - 64) < 2.0
    assert dists.min() > 32


# --------------------------------------------------------------------------
# Model: special cases with closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mask_kind", [0, 1])
def test_zero_model_is_uniform(mask_kind):
    m = inputs.ModelShape(17, 2, 16, 4, mask_kind=mask_kind, W=3, S=4)
    w = np.zeros(inputs.param_count(m), np.float32)
    spins, lq, pp, _ = oracle.sample(ocfg(m), w, 9, seed=77)
    assert np.all(pp == 0.5)
    assert np.allclose(lq, -m.N * math.log(2), atol=1e-12, rtol=0)
    u = np.array([[oracle.uniform(77, b, t, 0) for t in range(m.N)] for b in range(9)])
    assert np.array_equal(spins, np.where(u < 0.5, 1, -1))


def test_head_bias_alone_sets_the_conditional():
    """With every weight zero but the head bias, l_t = bh1 - bh0 for all t
    (softmax over two logits, index 1 = spin +1)."""
    m = inputs.ModelShape(11, 1, 8, 2)
    w = np.zeros(inputs.param_count(m), np.float32)
    o, _ = inputs.offsets(m)["bh"]
    w[o], w[o + 1] = -0.3, 0.9
    ell = 0.9 - (-0.3)
    spins, lq, pp, _ = oracle.sample(ocfg(m), w.astype(np.float64), 40, seed=3)
    p = 1 / (1 + math.exp(-ell))
    assert np.allclose(pp, p, rtol=1e-7)
    n_up = (spins == 1).sum(1)
    expect = n_up * math.log(p) + (m.N - n_up) * math.log(1 - p)
    assert np.allclose(lq, expect, rtol=1e-6)
    u = np.array([[oracle.uniform(3, b, t, 0) for t in range(m.N)] for b in range(40)])
    assert np.array_equal(spins, np.where(u < np.float32(p), 1, -1))


# --------------------------------------------------------------------------
# Model: independent composition from PyTorch library routines
# --------------------------------------------------------------------------

MODELS = [
    inputs.ModelShape(12, 2, 16, 2),
    inputs.ModelShape(13, 3, 16, 4, mask_kind=1, W=3, S=4),
    inputs.ModelShape(16, 2, 24, 3, d_token=2, mask_kind=1, W=4, S=5),
]


@pytest.mark.parametrize("m", MODELS)
def test_teacher_forced_logq_matches_torch_composition(m):
    w = inputs.make_weights(m, 11, scale=1.5)
    spins = inputs.random_spins(7, m.N, 5)
    lq = oracle.logprob(ocfg(m), w, spins)
    ref = _torch_ref.logq(m, torch.tensor(w, dtype=torch.float64), spins).numpy()
    assert np.allclose(lq, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m", MODELS)
def test_sampled_logq_equals_teacher_forced(m):
    """Algorithm 2 (KV-cache decode) and Algorithm 1 (full sequence) give the
    same log q and the same conditionals on the sampled configurations."""
    w = inputs.make_weights(m, 12)
    spins, lq, pp, _ = oracle.sample(ocfg(m), w, 16, seed=9)
    lq_tf, pp_tf = oracle.logprob(ocfg(m), w, spins, with_pplus=True)
    assert np.allclose(lq, lq_tf, rtol=1e-12, atol=1e-12)
    assert np.allclose(pp, pp_tf, rtol=1e-12, atol=1e-13)
    ref = _torch_ref.logq(m, torch.tensor(w, dtype=torch.float64), spins).numpy()
    assert np.allclose(lq, ref, rtol=1e-12, atol=1e-12)


def test_band_at_least_N_is_dense():
    dense = inputs.ModelShape(14, 2, 16, 2)
    band = inputs.ModelShape(14, 2, 16, 2, mask_kind=1, W=13, S=0)
    w = inputs.make_weights(dense, 3)
    s = inputs.random_spins(5, 14, 1)
    assert np.array_equal(oracle.logprob(ocfg(dense), w, s), oracle.logprob(ocfg(band), w, s))
    narrow = inputs.ModelShape(14, 2, 16, 2, mask_kind=1, W=12, S=0)
    assert not np.allclose(oracle.logprob(ocfg(dense), w, s), oracle.logprob(ocfg(narrow), w, s))


def test_one_layer_receptive_field_is_band_plus_sink():
    """SI Sec. I.A: A_tk = 0 for t - k > W.  With one layer, the conditional of
    query t sees the token of spin j (key j+1) iff t-(j+1) <= W or j+1 < S."""
    W, S, N, t = 3, 2, 12, 10
    m = inputs.ModelShape(N, 1, 16, 2, mask_kind=1, W=W, S=S)
    w = inputs.make_weights(m, 21, scale=2.0)
    base = inputs.random_spins(1, N, 8)
    _, p0 = oracle.logprob(ocfg(m), w, base, with_pplus=True)
    for j in range(t):
        s = base.copy()
        s[0, j] *= -1
        _, p1 = oracle.logprob(ocfg(m), w, s, with_pplus=True)
        seen = (t - (j + 1) <= W) or (j + 1 < S)
        if seen:
            assert abs(p1[0, t] - p0[0, t]) > 1e-9, j
        else:
            assert p1[0, t] == p0[0, t], j


# --------------------------------------------------------------------------
# Enumeration: normalisation, exact Z, F <= F_q
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [inputs.ModelShape(12, 2, 16, 2),
                               inputs.ModelShape(12, 2, 16, 4, mask_kind=1, W=3, S=4)])
def test_enumeration_normalisation_Z_and_variational_bound(m):
    inst = inputs.make_sk(m.N, 4)
    w = inputs.make_weights(m, 5)
    beta = 1.3
    ex = oracle.enumerate_exact(ocfg(m), w, inst, beta)
    assert abs(ex["sum_q"] - 1.0) < 1e-12
    states = all_states(m.N)
    E = -0.5 * np.einsum("bi,ij,bj->b", states.astype(np.float64), inst.J.astype(np.float64),
                         states.astype(np.float64))
    lnZ = scipy.special.logsumexp(-beta * E)
    assert abs(ex["lnZ"] - lnZ) < 1e-10 * abs(lnZ)
    assert abs(ex["Emin"] - E.min()) < 1e-10
    lq = oracle.logprob(ocfg(m), w, states)
    q = np.exp(lq)
    assert abs(q.sum() - 1.0) < 1e-12
    Fq = (q * (beta * E + lq)).sum() / beta
    assert abs(ex["Fq"] - Fq) < 1e-10 * abs(Fq)
    # Eq. (KL_div): D_KL = beta (F_q - F) >= 0
    assert ex["Fq"] >= ex["F"]
    kl = (q * (lq - (-beta * E - lnZ))).sum()
    assert abs(kl - beta * (ex["Fq"] - ex["F"])) < 1e-9


def test_sk_annealed_partition_function_and_paper_value():
    """E_J[Z] = 2^N exp(beta^2 (N-1)/4) for J_ij ~ N(0, 1/N), i<j, which pins the
    coupling normalisation; its N -> inf free energy per spin,
    -ln2/beta - beta/4, is the paper's printed F_inf at beta = 0.5."""
    beta, F_printed, tol = np.loadtxt(os.path.join(HERE, "golden",
                                                   "sk_paramagnetic_free_energy.txt"))
    f_inf = -math.log(2) / beta - beta / 4
    assert abs(f_inf - F_printed) < tol
    N = 10
    m = inputs.ModelShape(N, 1, 4, 1)
    w = inputs.make_weights(m, 1)
    Z = []
    for seed in range(300):
        ex = oracle.enumerate_exact(ocfg(m), w, inputs.make_sk(N, 1000 + seed), beta)
        Z.append(math.exp(ex["lnZ"]))
    Z = np.array(Z)
    expect = 2 ** N * math.exp(beta ** 2 * (N - 1) / 4)
    assert abs(Z.mean() - expect) < 4 * Z.std(ddof=1) / math.sqrt(len(Z))
    # the wrong normalisation (J ~ N(0,1)) would give a far larger mean
    wrong = 2 ** N * math.exp(beta ** 2 * N * (N - 1) / 4)
    assert abs(Z.mean() - wrong) > 20 * Z.std(ddof=1) / math.sqrt(len(Z))


# --------------------------------------------------------------------------
# Energies
# --------------------------------------------------------------------------

def test_sk_energy_is_half_quadratic_form():
    inst = inputs.make_sk(30, 2)
    s = inputs.random_spins(50, 30, 3)
    E = oracle.energy(inst, s)
    ref = -0.5 * np.einsum("bi,ij,bj->b", s.astype(np.float64), inst.J.astype(np.float64),
                           s.astype(np.float64))
    assert np.allclose(E, ref, rtol=1e-12, atol=1e-12)
    assert np.array_equal(E, oracle.energy(inst, -s))


@pytest.mark.parametrize("D,L", [(2, 4), (2, 5), (3, 4)])
def test_ea_ferromagnet_closed_forms(D, L):
    inst = inputs.make_ferro(D, L)
    N = L ** D
    up = np.ones((1, N), np.int8)
    assert oracle.energy(inst, up)[0] == -D * N
    if L % 2 == 0:
        coords = np.indices((L,) * D).reshape(D, -1)[::-1]  # x0 fastest
        cb = np.where(coords.sum(0) % 2 == 0, 1, -1).astype(np.int8)[None]
        assert oracle.energy(inst, cb)[0] == D * N
    open_inst = inputs.make_ferro(D, L, periodic=False)
    assert oracle.energy(open_inst, up)[0] == -D * L ** (D - 1) * (L - 1)


def test_ea_pm_energies_are_integers_and_flip_invariant():
    inst = inputs.make_ea(3, 5, 7, pm=True)
    s = inputs.random_spins(40, inst.N, 2)
    E = oracle.energy(inst, s)
    assert np.all(E == np.round(E))
    assert np.array_equal(E, oracle.energy(inst, -s))
    # brute-force pair list: each nearest-neighbour pair once
    L, D = inst.L, inst.D
    coords = np.indices((L,) * D).reshape(D, -1)[::-1].T
    ref = np.zeros(40)
    for i, x in enumerate(coords):
        for mu in range(D):
            y = x.copy()
            y[mu] = (y[mu] + 1) % L
            j = int(sum(y[k] * L ** k for k in range(D)))
            ref -= inst.J[i, mu] * s[:, i] * s[:, j]
    assert np.array_equal(E, ref)


# --------------------------------------------------------------------------
# Free energies from a batch
# --------------------------------------------------------------------------

def test_importance_weighted_free_energy_is_exact_on_full_uniform_batch():
    """With q uniform and every state in the batch once, F_IS = -ln Z / beta."""
    N, beta = 12, 0.8
    inst = inputs.make_sk(N, 9)
    states = all_states(N)
    E = oracle.energy(inst, states)
    lq = np.full(len(states), -N * math.log(2))
    Fq, Fis, ess = oracle.free_energy(E, lq, beta)
    assert abs(Fis - (-scipy.special.logsumexp(-beta * E) / beta)) < 1e-12
    assert abs(Fq - (beta * E + lq).mean() / beta) < 1e-12
    # Kish ESS of equal weights is B
    _, _, ess_eq = oracle.free_energy(np.zeros(100), np.zeros(100), beta)
    assert abs(ess_eq - 100) < 1e-9


def test_importance_weighted_free_energy_below_batch_fq():
    m = inputs.ModelShape(10, 2, 16, 2)
    w = inputs.make_weights(m, 2)
    inst = inputs.make_sk(10, 2)
    s, lq, _, _ = oracle.sample(ocfg(m), w, 500, seed=1)
    E = oracle.energy(inst, s)
    Fq, Fis, ess = oracle.free_energy(E, lq, 1.0)
    assert Fis <= Fq  # Jensen
    assert 1.0 <= ess <= 500


# --------------------------------------------------------------------------
# Backward: finite differences, autograd, exact enumerated gradient
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [inputs.ModelShape(6, 2, 8, 2, d_ff=16),
                               inputs.ModelShape(7, 2, 8, 2, d_ff=12, mask_kind=1, W=2, S=2)])
def test_grad_matches_central_finite_differences(m):
    w = inputs.make_weights(m, 4, scale=1.3).astype(np.float64)
    s = inputs.random_spins(3, m.N, 6)
    c = np.array([0.7, -1.1, 0.4])
    g, _ = oracle.grad(ocfg(m), w, s, c)
    h = 1e-6
    fd = np.zeros_like(w)
    for i in range(len(w)):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd[i] = (c @ oracle.logprob(ocfg(m), wp, s) - c @ oracle.logprob(ocfg(m), wm, s)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-7)


def test_grad_matches_torch_autograd():
    m = inputs.ModelShape(10, 2, 16, 4, mask_kind=1, W=3, S=3)
    w = inputs.make_weights(m, 8, scale=1.2)
    s = inputs.random_spins(5, m.N, 2)
    c = np.linspace(-1, 1, 5)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    (torch.tensor(c) * _torch_ref.logq(m, wt, s)).sum().backward()
    g, _ = oracle.grad(ocfg(m), w, s, c)
    assert np.allclose(g, wt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_reinforce_estimate_matches_exact_enumerated_gradient():
    """Eq. (loss1): (1/M) sum (L - Lbar) grad ln q estimates
    beta grad F_q = sum_sigma q grad ln q (beta E + ln q)."""
    N, beta = 8, 1.0
    m = inputs.ModelShape(N, 1, 8, 2, d_ff=16)
    w = inputs.make_weights(m, 3)
    inst = inputs.make_sk(N, 3)
    states = all_states(N)
    lq = oracle.logprob(ocfg(m), w, states)
    E = oracle.energy(inst, states)
    exact, _ = oracle.grad(ocfg(m), w, states, np.exp(lq) * (beta * E + lq))
    K, M = 16, 4000
    ests = []
    for k in range(K):
        s, lqs, _, _ = oracle.sample(ocfg(m), w, M, seed=100 + k)
        Lb = beta * oracle.energy(inst, s) + lqs
        g, _ = oracle.grad(ocfg(m), w, s, (Lb - Lb.mean()) / M)
        ests.append(g)
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(K)
    big = np.abs(exact) > 1e-8
    z = np.abs(mean - exact)[big] / np.maximum(se[big], 1e-12)
    assert np.mean(z < 4) > 0.98
    assert np.linalg.norm(mean - exact) < 0.1 * np.linalg.norm(exact)


# --------------------------------------------------------------------------
# Markov chains: stationary distributions against exact Boltzmann weights
# --------------------------------------------------------------------------

def _level_tv(E_samples, E_states, beta):
    """Total variation between the energy-level histogram of samples and the
    Boltzmann law over all states (levels merged to 1e-9)."""
    levels = np.unique(np.round(E_states, 9))
    p = np.exp(-beta * E_states - scipy.special.logsumexp(-beta * E_states))
    pl = np.array([p[np.round(E_states, 9) == v].sum() for v in levels])
    el = np.array([(np.round(E_samples, 9) == v).mean() for v in levels])
    return 0.5 * np.abs(pl - el).sum()


def test_independence_mh_targets_boltzmann():
    N, beta, C, per = 6, 1.0, 64, 1500
    m = inputs.ModelShape(N, 1, 8, 2, d_ff=16)
    w = inputs.make_weights(m, 6)
    inst = inputs.make_sk(N, 6)
    s, lq, _, _ = oracle.sample(ocfg(m), w, C * per, seed=5)
    E = oracle.energy(inst, s)
    s0, lq0, _, _ = oracle.sample(ocfg(m), w, C, seed=6)
    cE, cL, ci, trace, acc, _ = oracle.mh(E, lq, C, beta, 99, oracle.energy(inst, s0), lq0)
    E_states = oracle.energy(inst, all_states(N))
    tv = _level_tv(trace[100:].ravel(), E_states, beta)
    assert tv < 0.02
    assert _level_tv(E, E_states, beta) > 2 * tv  # raw proposals are off target
    # chain_idx points at the proposal whose energy the chain holds
    moved = ci >= 0
    assert np.array_equal(cE[moved], E[ci[moved]])


@pytest.mark.parametrize("kind", ["sk", "ea"])
def test_metropolis_targets_boltzmann(kind):
    beta = 0.9
    inst = inputs.make_sk(8, 2) if kind == "sk" else inputs.make_ea(2, 3, 5, pm=True)
    s0 = inputs.random_spins(256, inst.N, 1)
    _, _, trace, nflag = oracle.metropolis(inst, s0, 300, beta, 4)
    assert nflag == 0
    tv = _level_tv(trace[50:].ravel(), oracle.energy(inst, all_states(inst.N)), beta)
    assert tv < 0.02


@pytest.mark.parametrize("kind", ["sk", "ea"])
def test_metropolis_tracked_energy_equals_recomputed(kind):
    """dE = 2 s_i h_i must be the exact energy change of every single flip:
    the energy tracked by summing dE equals the recomputed energy, and at
    beta = 0 a sweep flips every spin (E(-s) = E(s))."""
    inst = inputs.make_sk(12, 3) if kind == "sk" else inputs.make_ea(3, 3, 2, pm=True)
    s0 = inputs.random_spins(20, inst.N, 4)
    s1, E1, trace, _ = oracle.metropolis(inst, s0, 1, 0.0, 1)
    assert np.array_equal(s1, -s0)
    assert np.allclose(E1, oracle.energy(inst, s0), atol=1e-9)
    s2, E2, _, _ = oracle.metropolis(inst, s0, 5, 0.7, 2)
    assert np.allclose(E2, oracle.energy(inst, s2), atol=1e-9)


def test_overlap_histogram():
    s = inputs.random_spins(10, 16, 1)
    same = np.repeat(s, 2, axis=0)
    h = oracle.overlap_hist(same)
    assert h[16] == 10 and h.sum() == 10
    opp = np.stack([s, -s], 1).reshape(20, 16)
    assert oracle.overlap_hist(opp)[0] == 10
    pairs = inputs.random_spins(2000, 16, 2)
    h = oracle.overlap_hist(pairs)
    q = (np.arange(17) * 2 - 16) / 16
    assert h.sum() == 1000 and abs((h * q).sum() / 1000) < 0.05


# --------------------------------------------------------------------------
# Loss weights of Eq. loss1 / loss2 and the ground-state form (Methods)
# --------------------------------------------------------------------------

def test_ground_state_form_weights_estimate_exact_gradient():
    """L = E + T ln q (Methods "Variational annealing"): the REINFORCE estimate
    with the oracle's weights matches sum_sigma q grad ln q (E + T ln q) by
    enumeration, and the likelihood term (w > 0) adds a zero-mean term under q."""
    N, T = 8, 0.7
    m = inputs.ModelShape(N, 1, 8, 2, d_ff=16)
    w = inputs.make_weights(m, 4)
    inst = inputs.make_sk(N, 5)
    states = all_states(N)
    lq = oracle.logprob(ocfg(m), w, states)
    E = oracle.energy(inst, states)
    exact, _ = oracle.grad(ocfg(m), w, states, np.exp(lq) * (E + T * lq))
    K, M = 12, 3000
    ests = []
    for k in range(K):
        s, lqs, _, _ = oracle.sample(ocfg(m), w, M, seed=300 + k)
        coeff, mL, mE = oracle.loss_coeff(oracle.energy(inst, s), lqs, 1.0, T, 0.5)
        assert abs(coeff.sum() + 0.5) < 1e-12          # sum of the weights is -w
        assert abs(mE - oracle.energy(inst, s).mean()) < 1e-12
        g, _ = oracle.grad(ocfg(m), w, s, coeff)
        ests.append(g)
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(K)
    big = np.abs(exact) > 1e-8
    z = np.abs(mean - exact)[big] / np.maximum(se[big], 1e-12)
    assert np.mean(z < 4) > 0.97
    assert np.linalg.norm(mean - exact) < 0.15 * np.linalg.norm(exact)


def test_loss_weights_scale_and_shift():
    """The ground-state weights at temperature T are T times the free-energy
    weights at beta = 1/T; a constant energy shift leaves the weights unchanged."""
    rng = np.random.default_rng(3)
    E = rng.normal(0, 5, 257)
    lq = -np.abs(rng.normal(10, 2, 257))
    T = 0.37
    c_gs, _, _ = oracle.loss_coeff(E, lq, 1.0, T, 0.0)
    c_fe, _, _ = oracle.loss_coeff(E, lq, 1.0 / T, 1.0, 0.0)
    assert np.allclose(c_gs, T * c_fe, rtol=1e-12, atol=1e-15)
    c_sh, _, _ = oracle.loss_coeff(E + 123.0, lq, 1.0, T, 0.2)
    c_0, _, _ = oracle.loss_coeff(E, lq, 1.0, T, 0.2)
    assert np.allclose(c_sh, c_0, rtol=1e-9, atol=1e-12)


def test_likelihood_term_ascends_the_batch_log_likelihood():
    """Eq. loss2's extra term alone (a = c = 0, w = 1): the weights -1/B make
    sg_grad's sum equal minus the gradient of the mean log-likelihood of the
    batch, checked against central finite differences of the oracle's log q."""
    m = inputs.ModelShape(6, 1, 8, 2, d_ff=16)
    w = inputs.make_weights(m, 6)
    s = inputs.random_spins(5, m.N, 7)
    coeff, _, _ = oracle.loss_coeff(np.zeros(5), np.zeros(5), 0.0, 0.0, 1.0)
    g, _ = oracle.grad(ocfg(m), w, s, coeff)
    rng = np.random.default_rng(1)
    for idx in rng.choice(w.size, 12, replace=False):
        h = 1e-6
        wp, wm = w.astype(np.float64).copy(), w.astype(np.float64).copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (oracle.logprob(ocfg(m), wp, s).mean() - oracle.logprob(ocfg(m), wm, s).mean()) / (2 * h)
        assert abs(g[idx] + fd) < 1e-6 + 1e-5 * abs(fd)


# --------------------------------------------------------------------------
# Muon (Methods "Comparison on optimizers")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(48, 16), (16, 40), (24, 24)])
def test_newton_schulz_acts_on_singular_values_only(shape):
    """Each quintic step maps every singular value s of X to a s + b s^3 + c s^5
    and keeps the singular vectors: NS_k(M) = U phi^k(S / |M|_F) V^T, checked
    against numpy's SVD for both orientations."""
    rng = np.random.default_rng(sum(shape))
    M = rng.normal(size=shape)
    a, b, c = 3.4445, -4.7750, 2.0315
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    s = S / (np.linalg.norm(M) + 1e-7)
    for _ in range(5):
        s = a * s + b * s ** 3 + c * s ** 5
    O = oracle.newton_schulz(M, 5)
    assert np.allclose(O, (U * s) @ Vt, atol=1e-10)
    sv = np.linalg.svd(O, compute_uv=False)
    assert sv.min() > 0.6 and sv.max() < 1.2  # approximately orthogonal


def test_muon_step_matrices_and_adamw_rest():
    """One step from zero state: every weight matrix moves by
    -lr (0.2 sqrt(max(r, c)) NS(G) + wd W); every other parameter takes the
    torch.optim.AdamW step; momentum holds G on the matrices."""
    m = inputs.ModelShape(10, 1, 16, 2, d_ff=32)
    cfg = ocfg(m)
    w0 = inputs.make_weights(m, 2).astype(np.float64)
    g = np.random.default_rng(5).normal(0, 1e-2, w0.size)
    w, mom, am, av = w0.copy(), np.zeros_like(w0), np.zeros_like(w0), np.zeros_like(w0)
    lr, mu, wd = 2e-3, 0.95, 0.1
    oracle.muon_step(cfg, w, g, mom, am, av, lr, mu, wd, 5, 1)
    d, f = m.d, m.d_ff
    off = 2 * m.d_token + m.N * (d - m.d_token)
    mats = []
    off += 2 * d
    mats.append((off, 3 * d, d)); off += 3 * d * d + 3 * d + 2 * d
    mats.append((off, f, d)); off += f * d + f
    mats.append((off, d, f)); off += d * f + d
    is_mat = np.zeros(w0.size, bool)
    for o, r, cc in mats:
        n = r * cc
        is_mat[o:o + n] = True
        G = g[o:o + n].reshape(r, cc)
        exp = w0[o:o + n] - lr * (0.2 * np.sqrt(max(r, cc)) * oracle.newton_schulz(G, 5).ravel()
                                   + wd * w0[o:o + n])
        assert np.allclose(w[o:o + n], exp, atol=1e-12)
        assert np.allclose(mom[o:o + n], g[o:o + n])
    p = torch.nn.Parameter(torch.tensor(w0[~is_mat]))
    opt = torch.optim.AdamW([p], lr=lr, betas=(0.9, 0.999), eps=1e-8, weight_decay=wd)
    p.grad = torch.tensor(g[~is_mat])
    opt.step()
    # torch applies the decay as w (1 - lr wd) before the Adam step: the same to O(lr^2 wd)
    assert np.allclose(w[~is_mat], p.detach().numpy(), atol=1e-7)
    assert np.all(mom[~is_mat] == 0)


# --------------------------------------------------------------------------
# Patching: 2^D spins per token, softmax over 2^(2^D) classes
# --------------------------------------------------------------------------

PATCHED = [
    inputs.ModelShape(16, 2, 16, 2, d_ff=32, mask_kind=1, W=2, S=3, patch=4, lat_D=2, lat_L=4),
    inputs.ModelShape(8, 1, 8, 2, d_ff=16, patch=2),                       # chain, 4 classes
    inputs.ModelShape(8, 1, 8, 2, d_ff=16, patch=8, lat_D=3, lat_L=2),     # one 2x2x2 patch
]


@pytest.mark.parametrize("m", PATCHED)
def test_patched_model_matches_torch_and_is_normalised(m):
    """Teacher-forced log q against the torch composition (tokens from the
    patch map, K-way head); sampled = teacher-forced; sum over all 2^N
    configurations of q = 1 by enumeration; F_q >= F."""
    w = inputs.make_weights(m, 13, scale=1.3)
    spins = inputs.random_spins(6, m.N, 3)
    lq = oracle.logprob(ocfg(m), w, spins)
    ref = _torch_ref.logq(m, torch.tensor(w, dtype=torch.float64), spins).numpy()
    assert np.allclose(lq, ref, rtol=1e-12, atol=1e-12)
    s, lqs, _, _ = oracle.sample(ocfg(m), w, 20, seed=4)
    assert np.allclose(oracle.logprob(ocfg(m), w, s), lqs, rtol=1e-12, atol=1e-12)
    inst = inputs.make_ea(2, 4, 1, pm=True) if m.N == 16 else inputs.make_sk(m.N, 2)
    ex = oracle.enumerate_exact(ocfg(m), w, inst, 0.8)
    assert abs(ex["sum_q"] - 1.0) < 1e-12
    assert ex["Fq"] >= ex["F"] - 1e-12


def test_patched_zero_model_is_uniform():
    m = PATCHED[0]
    w = inputs.make_weights(m, 1) * 0.0
    o = inputs.offsets(m)
    for name in o:
        if name.endswith("_g"):
            off, shape = o[name]
            w[off:off + int(np.prod(shape))] = 1.0
    s, lq, _, _ = oracle.sample(ocfg(m), w, 5, seed=2)
    assert np.allclose(lq, -m.N * math.log(2), rtol=0, atol=1e-12)


@pytest.mark.parametrize("m", PATCHED)
def test_patched_draw_lies_in_its_class_interval(m):
    """The inverse-CDF draw: every token's uniform u lies in the interval
    [cdf_lo, cdf_lo + p) of the class drawn (the oracle's cdf_lo output, used
    to check the GPU's classes at flagged draws)."""
    w = inputs.make_weights(m, 5, scale=1.3)
    B, T = 30, m.N // m.patch
    _, _, pp, _, lo = oracle.sample(ocfg(m), w, B, seed=12, with_cdf=True)
    for b in range(B):
        for t in range(T):
            u = oracle.uniform(12, b, t, 0)
            assert lo[b, t] - 1e-12 <= u < lo[b, t] + pp[b, t] + 1e-12


def test_patched_uniform_model_class_intervals():
    """All classes equally likely (zero weights, unit LayerNorm gains): the
    class drawn, read back from the spins through the torch patch map, is k
    with cdf_lo = k / K and p = 1 / K."""
    m = PATCHED[2]
    w = inputs.make_weights(m, 1) * 0.0
    o = inputs.offsets(m)
    for name in o:
        if name.endswith("_g"):
            off, shape = o[name]
            w[off:off + int(np.prod(shape))] = 1.0
    K = 1 << m.patch
    s, _, pp, _, lo = oracle.sample(ocfg(m), w, 64, seed=3, with_cdf=True)
    sites = _torch_ref.patch_sites(m)
    for b in range(64):
        for t in range(sites.shape[0]):
            k = sum(1 << j for j in range(m.patch) if s[b, sites[t, j]] > 0)
            assert abs(lo[b, t] - k / K) < 1e-12
            assert abs(pp[b, t] - 1 / K) < 1e-12


def test_patch_bits_land_on_the_patch_map():
    """A head bias that is a sum over bits, everything else zero: the classes
    factorise, bit j is +1 with probability sigmoid(a_j), and every site
    carries the marginal of its bit under the patch map (2D lattice L=4)."""
    m = PATCHED[0]
    w = np.zeros(inputs.param_count(m), np.float32)
    o = inputs.offsets(m)
    for name in o:
        if name.endswith("_g"):
            off, shape = o[name]
            w[off:off + int(np.prod(shape))] = 1.0
    a = np.array([1.2, -0.7, 0.3, -1.6])
    off, _ = o["bh"]
    w[off:off + 16] = [sum(a[j] for j in range(4) if (k >> j) & 1) for k in range(16)]
    s, _, _, _ = oracle.sample(ocfg(m), w, 40000, seed=8)
    sites = _torch_ref.patch_sites(m)
    p1 = 1 / (1 + np.exp(-a))
    mean = s.mean(0)
    for t in range(sites.shape[0]):
        for j in range(4):
            assert abs(mean[sites[t, j]] - (2 * p1[j] - 1)) < 0.02
    # the four bits of a patch are one 2x2 cell of the lattice
    x, y = sites % 4, sites // 4
    assert np.all(x.max(1) - x.min(1) == 1) and np.all(y.max(1) - y.min(1) == 1)


@pytest.mark.parametrize("m", PATCHED[:2])
def test_patched_grad_matches_torch_autograd(m):
    w = inputs.make_weights(m, 21)
    s = inputs.random_spins(4, m.N, 6)
    c = np.array([0.3, -1.1, 0.7, 0.25])
    g, _ = oracle.grad(ocfg(m), w, s, c)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    (torch.tensor(c) * _torch_ref.logq(m, wt, s)).sum().backward()
    assert np.allclose(g, wt.grad.numpy(), rtol=1e-9, atol=1e-11)
