"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: spins and +-J energies bit-exact (flagged draws replayed), per-sample
|delta log q| <= 1e-4 N for FP32 and <= 2e-2 N for BF16, FP64 reductions to
rounding, gradients to FP32 accumulation error.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2606_22984_gb300 import inputs, sg

from helpers import assert_grad_blocks, grad_block_errors, ocfg, oracle_replay, unpack_flags

pytestmark = pytest.mark.gpu

FP32_LOGQ_TOL = 1e-4     # per spin, FP32 path (per-sample bound 1e-4 * N)
BF16_LOGQ_TOL = 2e-2     # per spin, BF16 path
BF16_GRAD_BLOCK_TOL = 5e-2  # per weight tensor, BF16 gradient (relative, see assert_grad_blocks)
FP32_BAND = 1e-5         # flag bands the library uses by default
BF16_BAND = 1e-2


def _band(precision):
    return BF16_BAND if precision == sg.SG_BF16 else FP32_BAND


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_22984_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _np(t):
    return t.detach().cpu().numpy()


SAMPLE_CASES = {
    # name: (shape, B, weight scale)
    "sk20_dense": (inputs.ModelShape(20, 2, 32, 4), 300, 1.0),
    "ea6_ring": (inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7), 200, 1.0),
    "dense_d128_h8": (inputs.ModelShape(40, 2, 128, 8), 70, 1.0),
    "band_d128_h4": (inputs.ModelShape(30, 1, 128, 4, mask_kind=1, W=5, S=3), 65, 1.5),
    "single_spin": (inputs.ModelShape(1, 1, 32, 4), 5, 1.0),
    "band_W0_S0": (inputs.ModelShape(17, 2, 64, 8, mask_kind=1, W=0, S=0), 33, 1.0),
    "d64_h8_ring": (inputs.ModelShape(50, 3, 64, 8, mask_kind=1, W=4, S=6), 97, 1.0),
}


def _sample_and_check(m, w, B, seed, precision, tol):
    model = sg.Model(m, w, precision)
    spins, logq, flags = model.sample(B, seed=seed, with_flags=True)
    torch.cuda.synchronize()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    so, lqo, ppo, flo = oracle_replay(m, w, seed, s, fl, _band(precision))
    assert np.array_equal(so, s), "spins differ from the oracle outside flagged draws"
    assert np.all(np.isin(s, (-1, 1)))
    dl = np.abs(lqo - lq)
    assert dl.max() <= tol * m.N, f"max |dlogq| {dl.max()} > {tol * m.N}"
    frac = unpack_flags(fl, m.N).mean()
    return model, spins, logq, frac, dl


@pytest.mark.parametrize("name", list(SAMPLE_CASES))
def test_fp32_sampling_matches_oracle(name):
    m, B, scale = SAMPLE_CASES[name]
    w = inputs.make_weights(m, 7, scale)
    _, _, _, frac, _ = _sample_and_check(m, w, B, 1234, sg.SG_FP32, FP32_LOGQ_TOL)
    assert frac < 0.01


BF16_CASES = {
    "ea6_ring": (inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7), 200, 1.0),
    "dense_n40": (inputs.ModelShape(40, 3, 64, 4), 300, 1.0),
    "single_spin": (inputs.ModelShape(1, 1, 64, 4), 5, 1.0),
    "band_W0_S0": (inputs.ModelShape(17, 2, 64, 4, mask_kind=1, W=0, S=0), 129, 1.0),
    "short_sink": (inputs.ModelShape(20, 2, 64, 4, mask_kind=1, W=3, S=30), 64, 1.0),
    "dense_d128": (inputs.ModelShape(40, 2, 128, 8), 200, 1.0),
    "ring_d128": (inputs.ModelShape(64, 3, 128, 8, mask_kind=1, W=6, S=9), 300, 1.0),
    "tiny_d128": (inputs.ModelShape(3, 1, 128, 8), 7, 1.0),
    "ring_d256": (inputs.ModelShape(40, 2, 256, 8, mask_kind=1, W=5, S=3), 200, 1.0),
    "dense_d256": (inputs.ModelShape(24, 1, 256, 8), 130, 1.0),
    "tiny_d256": (inputs.ModelShape(2, 1, 256, 8), 3, 1.0),
    "one_spin_d128": (inputs.ModelShape(1, 1, 128, 8), 1, 1.0),
    "one_spin_d256": (inputs.ModelShape(1, 2, 256, 8), 2, 1.0),
    "one_sample_d64": (inputs.ModelShape(45, 2, 64, 4, mask_kind=1, W=5, S=6), 1, 1.0),
    # N beyond the three-stage shared-memory budget: the two-stage d = 64 kernel
    "two_stage_d64": (inputs.ModelShape(5000, 1, 64, 4, mask_kind=1, W=8, S=9), 24, 1.0),
}


@pytest.mark.parametrize("name,precision,rows", [("sk1024", "bf16", [0, 4321, 8191]),
                                                 ("ea3d10", "bf16", [0, 127, 128, 32767]),
                                                 ("sk1024", "fp32", [1, 8190])])
def test_full_size_d128_sampled_rows(name, precision, rows):
    """Full-size SK N=1024 (dense) and 3D EA L=10 (band + sink) workloads in
    the benchmark's launch configuration: sampled rows against the oracle,
    every energy against the oracle (bit-exact for +-J)."""
    wl = inputs.workloads()[name]
    m, inst = wl.model, wl.instance()
    w = wl.weights()
    prec = sg.SG_BF16 if precision == "bf16" else sg.SG_FP32
    tol = BF16_LOGQ_TOL if precision == "bf16" else FP32_LOGQ_TOL
    model = sg.Model(m, w, prec)
    spins, logq, flags = model.sample(wl.B, seed=2025, with_flags=True)
    model.check()
    gi = sg.Instance(inst)
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    rows = np.array(rows)
    so, lqo, _, _ = oracle_replay(m, w, 2025, s, fl, _band(prec), rows=rows)
    assert np.array_equal(so, s[rows])
    assert np.abs(lqo - lq[rows]).max() <= tol * m.N
    assert unpack_flags(fl, m.N).mean() < (0.05 if precision == "bf16" else 0.01)
    if precision == "bf16":
        # the teacher-forced BF16 pass (tcgen05 GEMMs) scores the same spins
        tf = _np(model.logprob(spins[:256]))
        assert np.abs(tf - lq[:256]).max() <= tol * m.N
    if inst.pm:
        _, Ei = gi.energy(spins, want_int=True)
        assert np.array_equal(_np(Ei).astype(np.float64), oracle.energy(inst, s))
    else:
        E = _np(gi.energy(spins[:256]))
        assert np.allclose(E, oracle.energy(inst, s[:256]), rtol=1e-5, atol=1e-3)
    del model


def test_full_size_patched_3d_rows():
    """The 3D EA L=10 model with (2, 2, 2) cells (125 tokens of 8 spins, 256
    classes, 6L d128 h8, band and sink over the token lattice of side 5) at
    the benchmark's batch, B = 32768, BF16: sampled rows against the oracle
    (each flagged draw inside the oracle's interval for the drawn class), and
    the teacher-forced log q of the same spins."""
    W, S = inputs.lattice_mask(3, 5)
    m = inputs.ModelShape(1000, 6, 128, 8, d_token=16, mask_kind=1, W=W, S=S, patch=8, lat_D=3,
                          lat_L=10)
    w = inputs.make_weights(m, 4)
    model = sg.Model(m, w, sg.SG_BF16)
    spins, logq, flags = model.sample(32768, seed=77, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    assert np.all(np.isin(s, (-1, 1)))
    rows = np.array([0, 127, 128, 32767])
    so, lqo, _, _ = oracle_replay(m, w, 77, s, fl, BF16_BAND, rows=rows)
    assert np.array_equal(so, s[rows])
    assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N
    tf = _np(model.logprob(spins[:256]))
    assert np.abs(tf - lq[:256]).max() <= BF16_LOGQ_TOL * m.N
    del model

def test_bf16_gelu_approximation_within_its_bound():
    """The GELU of the BF16 path (erf by Abramowitz & Stegun 7.1.26, |error|
    <= 1.5e-7) against CUDA's erff / expf over [-12, 12]: within that bound
    plus FP32 rounding, far below the BF16 step (2^-8) its results get."""
    eg, ed = sg.gelu_selfcheck(1 << 20)
    print(f"gelu max err {eg:.2e}, gelu' max err {ed:.2e}")
    assert eg <= 4e-7
    assert ed <= 4e-7


@pytest.mark.parametrize("name", list(BF16_CASES))
def test_bf16_sampling_matches_oracle(name):
    """BF16 decode on tcgen05: spins equal to the oracle once the draws inside
    the BF16 flag band (|p+ - u| < 1e-2) replay the GPU's decision; per-sample
    |delta log q| <= 2e-2 N."""
    m, B, scale = BF16_CASES[name]
    w = inputs.make_weights(m, 7, scale)
    model, _, _, frac, dl = _sample_and_check(m, w, B, 4321, sg.SG_BF16, BF16_LOGQ_TOL)
    model.check()
    assert frac < 0.05
    print(f"{name}: flagged {frac:.4f} of draws, max |dlogq|/N {dl.max() / m.N:.2e}")


@pytest.mark.parametrize("n_models,per_model", [(3, 100), (2, 1000)])
def test_bf16_grouped_models_match_oracle(n_models, per_model):
    """A group of d = 256 models in one launch: sample b uses model
    b // per_model (its own weights), Philox counters keep the global row."""
    m = inputs.ModelShape(30, 2, 256, 8, mask_kind=1, W=4, S=5)
    w = inputs.make_group_weights(m, 11, n_models)
    P1 = w.size // n_models
    B = n_models * per_model
    model = sg.Model(m, w, sg.SG_BF16, n_models=n_models)
    spins, logq, flags = model.sample(B, seed=99, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    assert unpack_flags(fl, m.N).mean() < 0.05
    for i in range(n_models):
        rows = np.arange(i * per_model, (i + 1) * per_model)
        rows = rows if per_model <= 100 else rows[[0, 1, per_model // 2, per_model - 1]]
        so, lqo, _, _ = oracle_replay(m, w[i * P1:(i + 1) * P1], 99, s, fl, BF16_BAND, rows=rows)
        assert np.array_equal(so, s[rows]), f"model {i}: spins differ"
        assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N
    # rows of model 0 are bit-identical to a single-model launch of model 0
    # (per-row arithmetic does not depend on how rows are grouped into CTAs)
    single = sg.Model(m, w[:P1], sg.SG_BF16)
    s1, l1 = single.sample(per_model, seed=99)
    assert np.array_equal(s[:per_model], _np(s1))
    assert np.array_equal(lq[:per_model], _np(l1))


def test_d256_rows_do_not_depend_on_rows_per_cta():
    """The d = 256 decode pairs each row with a mirror thread when a CTA
    serves at most 64 rows and runs both key halves in one thread otherwise;
    the two schedules give bit-identical rows (and match the oracle)."""
    m = inputs.ModelShape(7, 1, 256, 8, mask_kind=1, W=3, S=2)
    w = inputs.make_weights(m, 31)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    B = 64 * sms + 1  # 65 rows per CTA: the single-thread schedule
    model = sg.Model(m, w, sg.SG_BF16)
    s_big, l_big, f_big = model.sample(B, seed=4, with_flags=True)
    s_small, l_small = model.sample(100, seed=4)  # one row per CTA: mirrored
    model.check()
    assert np.array_equal(_np(s_big[:100]), _np(s_small))
    assert np.array_equal(_np(l_big[:100]), _np(l_small))
    s, lq, fl = _np(s_big), _np(l_big), _np(f_big)
    rows = [0, 64, B - 1]
    so, lqo, _, _ = oracle_replay(m, w, 4, s, fl, BF16_BAND, rows=rows)
    assert np.array_equal(so, s[rows])
    assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N


def test_bf16_grouped_models_at_the_group_limit():
    """64 models (the limit) of one sample each, and 65 rejected."""
    m = inputs.ModelShape(6, 1, 256, 8, mask_kind=1, W=2, S=1)
    w = inputs.make_group_weights(m, 21, 64)
    P1 = w.size // 64
    model = sg.Model(m, w, sg.SG_BF16, n_models=64)
    spins, logq, flags = model.sample(64, seed=5, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    for i in (0, 31, 63):
        so, lqo, _, _ = oracle_replay(m, w[i * P1:(i + 1) * P1], 5, s, fl, BF16_BAND, rows=[i])
        assert np.array_equal(so, s[[i]])
        assert abs(lqo[0] - lq[i]) <= BF16_LOGQ_TOL * m.N
    with pytest.raises(sg.SgError):
        sg.Model(m, inputs.make_group_weights(m, 21, 65), sg.SG_BF16, n_models=65)


PATCHED_CASES = {
    # name: (shape, B, precision)
    "lat2d_p4_fp32": (inputs.ModelShape(64, 2, 32, 4, d_token=16, mask_kind=1, W=4, S=5,
                                        patch=4, lat_D=2, lat_L=8), 200, sg.SG_FP32),
    "chain_p2_fp32": (inputs.ModelShape(40, 1, 32, 4, patch=2), 130, sg.SG_FP32),
    "lat3d_p8_fp32": (inputs.ModelShape(64, 1, 32, 4, d_token=8, patch=8, lat_D=3, lat_L=4), 70,
                      sg.SG_FP32),
    "lat2d_p4_bf16": (inputs.ModelShape(256, 2, 64, 4, d_token=16, mask_kind=1, W=8, S=9,
                                        patch=4, lat_D=2, lat_L=16), 300, sg.SG_BF16),
    "lat2d_p4_bf16_d128": (inputs.ModelShape(256, 2, 128, 8, d_token=16, mask_kind=1, W=8, S=9,
                                             patch=4, lat_D=2, lat_L=16), 300, sg.SG_BF16),
    "lat2d_p4_bf16_d256": (inputs.ModelShape(144, 2, 256, 8, d_token=16, mask_kind=1, W=6, S=7,
                                             patch=4, lat_D=2, lat_L=12), 200, sg.SG_BF16),
    "chain_p2_bf16_d128": (inputs.ModelShape(60, 1, 128, 8, d_token=8, patch=2), 130, sg.SG_BF16),
    # 3D cells of (2, 2, 2) spins: 256 classes through the decodes' chunked head
    "lat3d_p8_bf16": (inputs.ModelShape(512, 2, 64, 4, d_token=16, mask_kind=1, W=16, S=17,
                                        patch=8, lat_D=3, lat_L=8), 200, sg.SG_BF16),
    "lat3d_p8_bf16_d128": (inputs.ModelShape(512, 2, 128, 8, d_token=16, mask_kind=1, W=16, S=17,
                                             patch=8, lat_D=3, lat_L=8), 200, sg.SG_BF16),
    "lat3d_p8_bf16_d256": (inputs.ModelShape(216, 2, 256, 8, d_token=16, mask_kind=1, W=9, S=10,
                                             patch=8, lat_D=3, lat_L=6), 130, sg.SG_BF16),
}


@pytest.mark.parametrize("name", list(PATCHED_CASES))
def test_patched_sampling_and_scoring_match_oracle(name):
    """Patching: spins of every token cell equal to the oracle outside flagged
    draws, sampled log q within the per-token bound, teacher-forced log q and
    the REINFORCE gradient against the oracle."""
    m, B, prec = PATCHED_CASES[name]
    w = inputs.make_weights(m, 17)
    tol = BF16_LOGQ_TOL if prec == sg.SG_BF16 else FP32_LOGQ_TOL
    model = sg.Model(m, w, prec)
    spins, logq, flags = model.sample(B, seed=31, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    assert np.all(np.isin(s, (-1, 1)))
    so, lqo, _, _ = oracle_replay(m, w, 31, s, fl, _band(prec))
    assert np.array_equal(so, s), "spins differ from the oracle outside flagged draws"
    assert np.abs(lqo - lq).max() <= tol * m.N
    tf = _np(model.logprob(spins))
    assert np.abs(tf - lqo).max() <= tol * m.N
    c = np.random.default_rng(1).normal(0, 1, B).astype(np.float32) / B
    g = _np(model.grad(spins, torch.tensor(c, device="cuda")))
    go, _ = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"{name}: flagged {unpack_flags(fl, m.N // m.patch).mean():.4f}, grad rel err {rel:.2e}")
    assert rel < (2e-2 if prec == sg.SG_BF16 else 1e-4)


def test_patched_bf16_rejected_where_not_built():
    """The d = 64 decode keeps the token columns in one quarter of a row
    (d_token <= 16); a wider token embedding is served by the FP32 decode."""
    m = inputs.ModelShape(64, 1, 64, 4, d_token=32, patch=8, lat_D=3, lat_L=4)
    model = sg.Model(m, inputs.make_weights(m, 1), sg.SG_BF16)
    with pytest.raises(sg.SgError):
        model.sample(8, seed=1)


def test_patched_bf16_d256_grouped_models_match_oracle():
    """Two patched d = 256 models in one grouped launch: each model's rows
    against the oracle with that model's weights."""
    m = inputs.ModelShape(144, 1, 256, 8, d_token=16, mask_kind=1, W=6, S=7, patch=4, lat_D=2,
                          lat_L=12)
    n, per = 2, 100
    w = inputs.make_group_weights(m, 23, n)
    P1 = w.size // n
    model = sg.Model(m, w, sg.SG_BF16, n_models=n)
    spins, logq, flags = model.sample(n * per, seed=41, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    for i in range(n):
        rows = np.arange(i * per, (i + 1) * per)
        so, lqo, _, _ = oracle_replay(m, w[i * P1:(i + 1) * P1], 41, s, fl, BF16_BAND, rows=rows)
        assert np.array_equal(so, s[rows]), f"model {i}: spins differ outside flagged draws"
        assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N


def test_grouped_models_rejected_outside_d256():
    m = inputs.ModelShape(20, 1, 64, 4)
    w = inputs.make_group_weights(m, 1, 2)
    with pytest.raises(sg.SgError):
        sg.Model(m, w, sg.SG_FP32, n_models=2).sample(8, seed=1)
    g = sg.Model(inputs.ModelShape(8, 1, 256, 8), inputs.make_group_weights(
        inputs.ModelShape(8, 1, 256, 8), 1, 2), sg.SG_BF16, n_models=2)
    with pytest.raises(sg.SgError):
        g.sample(7, seed=1)  # B not a multiple of n_models
    with pytest.raises(sg.SgError):
        g.logprob(torch.ones(3, 8, dtype=torch.int8, device="cuda"))
    with pytest.raises(sg.SgError):
        g.grad(torch.ones(3, 8, dtype=torch.int8, device="cuda"),
               torch.zeros(3, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_grouped_logprob_and_grad_equal_per_model_calls(precision):
    """A group of 3 models in one sg_logprob / sg_grad call: model i scores
    samples [i B/3, (i+1) B/3) and fills its own gradient block, equal to a
    single-model call on the same samples (up to FP32 summation order), and
    to the oracle."""
    m = inputs.ModelShape(30, 2, 64, 4, mask_kind=1, W=4, S=5)
    prec = sg.SG_BF16 if precision == "bf16" else sg.SG_FP32
    n, per = 3, 40
    w = inputs.make_group_weights(m, 11, n)
    P1 = w.size // n
    B = n * per
    s = inputs.random_spins(B, m.N, 6)
    c = np.random.default_rng(8).normal(0, 1, B).astype(np.float32)
    group = sg.Model(m, w, prec, n_models=n)
    ts, tc = torch.tensor(s, device="cuda"), torch.tensor(c, device="cuda")
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    g = _np(group.grad(ts, tc, logq=lq))
    lp = _np(group.logprob(ts))
    group.check()
    assert np.array_equal(lp, _np(lq))
    for i in range(n):
        one = sg.Model(m, w[i * P1:(i + 1) * P1], prec)
        sl = slice(i * per, (i + 1) * per)
        gi = _np(one.grad(ts[sl].contiguous(), tc[sl].contiguous()))
        assert np.abs(g[i * P1:(i + 1) * P1] - gi).max() <= 1e-5 * np.abs(gi).max()
        assert np.array_equal(_np(one.logprob(ts[sl].contiguous())), lp[sl])
    go, lqo = oracle.grad(ocfg(m), w[:P1], s[:per], c[:per].astype(np.float64))
    tol = BF16_LOGQ_TOL if prec == sg.SG_BF16 else FP32_LOGQ_TOL
    assert np.abs(lp[:per] - lqo).max() <= tol * m.N
    rel = np.linalg.norm(g[:P1] - go) / np.linalg.norm(go)
    assert rel < (2e-2 if prec == sg.SG_BF16 else 1e-4), rel


def test_full_size_ea2d64_grouped_training_step():
    """One REINFORCE step of the 2D EA L=64 workload at full size (N = 4096,
    8 layers d = 256, 8 models = 8 betas x 1024 samples, BF16): grouped
    sampling, Gaussian energies, per-beta loss weights (Eq. loss1), one
    grouped sg_grad (chunked by free memory), Adam.  Checks: weight blocks of
    models whose coefficients are all zero get exactly zero gradient; models 0
    and 7 equal single-model gradients of their samples under a different
    chunking; log q of the teacher-forced pass agrees with the sampler's.
    Prints the time and the device memory the step needed."""
    import time
    wl = inputs.workloads()["ea2d64"]
    m, betas = wl.model, [float(b) for b in wl.betas]
    nb, per = len(betas), wl.B
    B = nb * per
    w = wl.group_weights()
    P1 = w.size // nb
    free0 = torch.cuda.mem_get_info()[0]
    group = sg.Model(m, w, sg.SG_BF16, n_models=nb)
    inst = sg.Instance(wl.instance())
    t0 = time.perf_counter()
    spins, logq = group.sample(B, seed=31)
    E = inst.energy(spins)
    coeff = torch.empty(B, dtype=torch.float32, device="cuda")
    for i, beta in enumerate(betas):
        sl = slice(i * per, (i + 1) * per)
        cf, _ = sg.loss_coeff(E[sl].contiguous(), logq[sl].contiguous(), beta, 1.0)
        coeff[sl] = cf
    # zero every model's weights except those of models 0 and 7
    keep = torch.zeros(B, dtype=torch.bool, device="cuda")
    keep[:per] = True
    keep[(nb - 1) * per:] = True
    coeff = torch.where(keep, coeff, torch.zeros_like(coeff))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    tf = torch.empty(B, dtype=torch.float32, device="cuda")
    g = group.grad(spins, coeff, logq=tf)
    group.check()
    t2 = time.perf_counter()
    free1 = torch.cuda.mem_get_info()[0]
    mv, vv = torch.zeros_like(g), torch.zeros_like(g)
    sg.adam_step(group.weights(), g, mv, vv, 1e-3, 1)
    group.refresh()
    group.check()
    gn = _np(g)
    print(f"ea2d64 grouped step: sample + energy {t1 - t0:.2f} s, grouped grad (B={B}) "
          f"{t2 - t1:.2f} s, device memory in use by the step {(free0 - free1) / 2**30:.1f} GiB")
    assert np.all(np.isfinite(gn))
    for i in range(1, nb - 1):
        assert not gn[i * P1:(i + 1) * P1].any(), f"model {i} has no weight but got a gradient"
    assert np.abs(_np(tf) - _np(logq)).max() <= BF16_LOGQ_TOL * m.N
    for i in (0, nb - 1):
        one = sg.Model(m, w[i * P1:(i + 1) * P1], sg.SG_BF16)
        one.set_max_chunk(96)
        sl = slice(i * per, (i + 1) * per)
        gi = _np(one.grad(spins[sl].contiguous(), coeff[sl].contiguous()))
        one.check()
        assert np.abs(gn[i * P1:(i + 1) * P1] - gi).max() <= 1e-4 * np.abs(gi).max()
        del one


def test_full_size_ea2d64_grouped_bf16_sampled_rows():
    """2D EA L=64 (N=4096), 8 layers d=256, one model per beta (8 betas x
    B=1024) in one launch: sampled rows of three models against the oracle,
    and the Gaussian energies of the samples."""
    import time
    wl = inputs.workloads()["ea2d64"]
    m, nb = wl.model, len(wl.betas)
    w = wl.group_weights()
    P1 = w.size // nb
    B = nb * wl.B
    model = sg.Model(m, w, sg.SG_BF16, n_models=nb)
    model.sample(256 * nb, seed=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    spins, logq, flags = model.sample(B, seed=2026, with_flags=True)
    model.check()
    dt = time.perf_counter() - t0
    print(f"ea2d64 grouped BF16 decode: {B} samples x {m.N} spins in {dt:.2f} s "
          f"({B / dt:.0f} configs/s)")
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    assert np.all(np.isin(s, (-1, 1)))
    assert unpack_flags(fl, m.N).mean() < 0.05
    for i, rows in ((0, [0, 1023]), (3, [3 * 1024 + 17]), (7, [B - 1])):
        so, lqo, _, _ = oracle_replay(m, w[i * P1:(i + 1) * P1], 2026, s, fl, BF16_BAND, rows=rows)
        assert np.array_equal(so, s[rows]), f"model {i}: spins differ"
        assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N
    inst = wl.instance()
    E = _np(sg.Instance(inst).energy(spins[:64]))
    assert np.allclose(E, oracle.energy(inst, s[:64]), rtol=1e-5, atol=1e-2)


def test_full_size_ea2d16_bf16_sampled_rows():
    wl = inputs.workloads()["ea2d16"]
    m = wl.model
    w = wl.weights()
    model = sg.Model(m, w, sg.SG_BF16)
    spins, logq, flags = model.sample(wl.B, seed=77, with_flags=True)
    model.check()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    rows = np.array([0, 107, 108, 5000, 9999, wl.B - 1])
    so, lqo, _, _ = oracle_replay(m, w, 77, s, fl, BF16_BAND, rows=rows)
    assert np.array_equal(so, s[rows])
    assert np.abs(lqo - lq[rows]).max() <= BF16_LOGQ_TOL * m.N
    assert unpack_flags(fl, m.N).mean() < 0.05
    # BF16 sampled log q against the FP32 teacher-forced log q of the same spins
    m32 = sg.Model(m, w, sg.SG_FP32)
    tf = _np(m32.logprob(spins[:512]))
    assert np.abs(tf - lq[:512]).max() <= BF16_LOGQ_TOL * m.N


@pytest.mark.parametrize("name", ["sk20_dense", "ea6_ring", "dense_d128_h8", "d64_h8_ring"])
def test_fp32_teacher_forced_logq_matches_oracle_and_sampler(name):
    m, B, scale = SAMPLE_CASES[name]
    w = inputs.make_weights(m, 8, scale)
    model = sg.Model(m, w, sg.SG_FP32)
    rs = inputs.random_spins(B, m.N, 3)
    lq = _np(model.logprob(torch.tensor(rs, device="cuda")))
    lqo = oracle.logprob(ocfg(m), w, rs)
    assert np.abs(lq - lqo).max() <= FP32_LOGQ_TOL * m.N
    spins, logq = model.sample(B, seed=99)
    tf = model.logprob(spins)
    assert (tf - logq).abs().max().item() <= FP32_LOGQ_TOL * m.N


def test_fp32_logprob_beyond_65535_row_tiles():
    """FP32 teacher-forced pass over 70000 samples of N = 64 in one call:
    4.48 million rows, so a row-tiled launch needs more than 65535 tiles of
    64 rows (past the limit of a grid's y dimension).  Sampled rows against
    the oracle."""
    m = inputs.ModelShape(64, 2, 32, 4)
    w = inputs.make_weights(m, 4)
    B = 70000
    model = sg.Model(m, w, sg.SG_FP32)
    rs = inputs.random_spins(B, m.N, 21)
    lq = _np(model.logprob(torch.tensor(rs, device="cuda")))
    model.check()
    rows = np.array([0, 33333, 65536, B - 1])
    lqo = oracle.logprob(ocfg(m), w, rs[rows])
    assert np.abs(lq[rows] - lqo).max() <= FP32_LOGQ_TOL * m.N


def test_sampling_is_deterministic_and_seeded():
    m, B, _ = SAMPLE_CASES["ea6_ring"]
    model = sg.Model(m, inputs.make_weights(m, 1), sg.SG_FP32)
    a, la = model.sample(B, seed=5)
    b, lb = model.sample(B, seed=5)
    c, _ = model.sample(B, seed=6)
    assert torch.equal(a, b) and torch.equal(la, lb)
    assert not torch.equal(a, c)


def test_invalid_arguments_raise():
    m, _, _ = SAMPLE_CASES["sk20_dense"]
    model = sg.Model(m, inputs.make_weights(m, 1), sg.SG_FP32)
    with pytest.raises(sg.SgError):
        model.sample(0, seed=1)
    with pytest.raises(sg.SgError):
        sg.Model(m, np.zeros(10, np.float32), sg.SG_FP32)
    bad = inputs.make_weights(m, 1)
    bad[3] = np.nan
    with pytest.raises(sg.SgError):
        sg.Model(m, bad, sg.SG_FP32)


# --------------------------------------------------------------------------
# Energies
# --------------------------------------------------------------------------

@pytest.mark.parametrize("D,L", [(2, 16), (3, 10), (2, 5)])
def test_pm_ea_energies_bit_exact(D, L):
    inst = inputs.make_ea(D, L, 3, pm=True)
    gi = sg.Instance(inst)
    for B in (1, 1000):
        s = inputs.random_spins(B, inst.N, B)
        E, Ei = gi.energy(torch.tensor(s, device="cuda"), want_int=True)
        Eo = oracle.energy(inst, s)
        assert np.array_equal(_np(Ei).astype(np.float64), Eo)
        assert np.array_equal(_np(E).astype(np.float64), Eo)


def test_gaussian_ea_energy():
    inst = inputs.make_ea(2, 12, 4, pm=False)
    s = inputs.random_spins(333, inst.N, 1)
    E = _np(sg.Instance(inst).energy(torch.tensor(s, device="cuda")))
    Eo = oracle.energy(inst, s)
    assert np.allclose(E, Eo, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("N,B", [(20, 1), (50, 65), (1024, 130)])
def test_sk_energy_fp32(N, B):
    inst = inputs.make_sk(N, N)
    s = inputs.random_spins(B, N, 2)
    E = _np(sg.Instance(inst).energy(torch.tensor(s, device="cuda")))
    Eo = oracle.energy(inst, s)
    assert np.allclose(E, Eo, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("N,B,offset", [(256, 1, 0), (256, 130, 0), (256, 130, 1), (1024, 8192, 0)])
def test_sk_energy_bf16_tensor_cores(N, B, offset):
    """s.J.s on tcgen05 with J split into two BF16 terms: FP32-level accuracy.
    offset 1 places the spins one byte past an aligned address (the epilogue's
    byte-wise spin loads instead of its 16-byte loads)."""
    inst = inputs.make_sk(N, N + 1)
    s = inputs.random_spins(B, N, 5)
    gi = sg.Instance(inst)
    buf = torch.empty(B * N + offset, dtype=torch.int8, device="cuda")
    ts = buf[offset:].view(B, N)
    ts.copy_(torch.tensor(s))
    assert ts.data_ptr() % 16 == offset
    E = _np(gi.energy(ts, precision=sg.SG_BF16))
    E32 = _np(gi.energy(ts, precision=sg.SG_FP32))
    rows = np.arange(B) if B <= 256 else np.linspace(0, B - 1, 256).astype(int)
    Eo = oracle.energy(inst, s[rows])
    assert np.allclose(E[rows], Eo, rtol=1e-5, atol=1e-3)
    assert np.allclose(E, E32, rtol=1e-5, atol=1e-3)


# --------------------------------------------------------------------------
# Free energies (FP64 on the device)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("B", [1, 7, 5000])
def test_free_energy_fp64(B):
    rng = np.random.default_rng(B)
    E = rng.normal(-30, 5, B).astype(np.float32)
    lq = rng.normal(-20, 3, B).astype(np.float32)
    beta = 0.7
    out, coeff = sg.free_energy(torch.tensor(E, device="cuda"), torch.tensor(lq, device="cuda"),
                                beta, want_coeff=True)
    Fq, Fis, ess = oracle.free_energy(E.astype(np.float64), lq.astype(np.float64), beta)
    o = _np(out)
    assert abs(o[0] - Fq) <= 1e-12 * abs(Fq)
    assert abs(o[1] - Fis) <= 1e-12 * abs(Fis)
    assert abs(o[2] - ess) <= 1e-10 * ess
    L = beta * E.astype(np.float64) + lq.astype(np.float64)
    assert np.allclose(_np(coeff), ((L - L.mean()) / B).astype(np.float32), rtol=1e-6, atol=1e-12)


# --------------------------------------------------------------------------
# REINFORCE backward
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [inputs.ModelShape(12, 2, 32, 4),
                               inputs.ModelShape(20, 2, 64, 4, mask_kind=1, W=4, S=5),
                               inputs.ModelShape(33, 1, 32, 2, mask_kind=1, W=3, S=2)])
def test_fp32_grad_matches_oracle(m):
    w = inputs.make_weights(m, 5)
    B = 37
    s = inputs.random_spins(B, m.N, 9)
    c = np.random.default_rng(1).normal(0, 1, B).astype(np.float32)
    model = sg.Model(m, w, sg.SG_FP32)
    logq = torch.empty(B, dtype=torch.float32, device="cuda")
    g = _np(model.grad(torch.tensor(s, device="cuda"), torch.tensor(c, device="cuda"), logq=logq))
    go, lqo = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    assert rel < 1e-4, rel
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max() + 1e-6
    assert np.abs(_np(logq) - lqo).max() <= FP32_LOGQ_TOL * m.N


BF16_TF_MODELS = [inputs.ModelShape(20, 2, 32, 4), inputs.ModelShape(40, 2, 64, 4),
                  inputs.ModelShape(70, 3, 64, 4, mask_kind=1, W=8, S=9),
                  inputs.ModelShape(33, 1, 64, 4, mask_kind=1, W=3, S=2),
                  # weights beyond 256 x 256: column-blocked tile GEMM, split wgrad
                  inputs.ModelShape(24, 2, 128, 8),
                  inputs.ModelShape(30, 1, 96, 6, mask_kind=1, W=5, S=4),
                  inputs.ModelShape(20, 1, 256, 8, mask_kind=1, W=6, S=3),
                  # dense causal at d_h = 16 from 128 positions (the tcgen05
                  # attention): several 128-row tiles with a ragged tail, one
                  # row past a tile, the SK widths (d 128, 8 heads)
                  inputs.ModelShape(160, 2, 64, 4),
                  inputs.ModelShape(129, 1, 64, 4),
                  inputs.ModelShape(300, 2, 128, 8),
                  # warp-level MMA attention with many keys per query: a band
                  # crossing tile edges with its sink, the 3D EA widths with a
                  # sink that ends inside a 16-key block, d_h = 32
                  inputs.ModelShape(300, 1, 64, 4, mask_kind=1, W=70, S=9),
                  inputs.ModelShape(333, 1, 128, 8, mask_kind=1, W=100, S=37),
                  inputs.ModelShape(140, 1, 256, 8),
                  # sequences beyond the MMA kernels' shared memory (d_h = 32): a
                  # band (the per-tile tcgen05 kernels) and a dense one (the
                  # tcgen05 flash attention)
                  inputs.ModelShape(650, 1, 64, 2, mask_kind=1, W=70, S=9),
                  inputs.ModelShape(650, 1, 64, 2)]


@pytest.mark.parametrize("m", BF16_TF_MODELS)
def test_bf16_teacher_forced_logq_and_grad(m):
    """BF16 teacher-forced pass and REINFORCE backward with the GEMMs on
    tcgen05 (tiled BF16 operands, FP32 accumulation): log q within the BF16
    bound of the oracle, gradient within BF16 rounding of the oracle's."""
    w = inputs.make_weights(m, 5)
    B = 300  # several row blocks of 128 and a ragged tail
    s = inputs.random_spins(B, m.N, 9)
    c = np.random.default_rng(2).normal(0, 1, B).astype(np.float32)
    model = sg.Model(m, w, sg.SG_BF16)
    ts = torch.tensor(s, device="cuda")
    lq = _np(model.logprob(ts))
    lqo = oracle.logprob(ocfg(m), w, s)
    assert np.abs(lq - lqo).max() <= BF16_LOGQ_TOL * m.N
    logq = torch.empty(B, dtype=torch.float32, device="cuda")
    g = _np(model.grad(ts, torch.tensor(c, device="cuda"), logq=logq))
    model.check()
    go, _ = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    worst = max(grad_block_errors(m, g, go), key=lambda x: x[1] / max(x[2], 0.1 * x[3]))
    print(f"N={m.N} d={m.d}: max|dlogq|/N {np.abs(lq - lqo).max() / m.N:.2e}, grad rel err "
          f"{rel:.2e}, worst block {worst[0]} {worst[1] / max(worst[2], 0.1 * worst[3]):.2e}")
    assert rel < 2e-2
    assert_grad_blocks(m, g, go, BF16_GRAD_BLOCK_TOL)
    assert np.abs(_np(logq) - lqo).max() <= BF16_LOGQ_TOL * m.N


LONG_BAND_MODELS = [
    # d_h = 16 past the MMA kernels' 1200 positions, a ragged last tile
    inputs.ModelShape(1300, 1, 64, 4, mask_kind=1, W=60, S=33),
    # d_h = 32: two sink tiles (S = 150), two layers
    inputs.ModelShape(700, 2, 64, 2, mask_kind=1, W=60, S=150),
    # no sink
    inputs.ModelShape(640, 1, 64, 2, mask_kind=1, W=50, S=0),
    # the 2D EA L=64 widths and mask (d 256 is d_h 32 as here), 900 positions
    inputs.ModelShape(900, 1, 128, 4, mask_kind=1, W=64, S=65),
]


@pytest.mark.parametrize("m", LONG_BAND_MODELS)
def test_bf16_long_band_attention_logq_and_grad(m):
    """Band sequences too long to stage whole run on the per-tile tcgen05
    kernels (a CTA per sample, head and 128-query tile; sink keys' gradients
    gathered over the query tiles): log q and the REINFORCE gradient against
    the oracle within the BF16 bounds, the gradient also per weight tensor."""
    w = inputs.make_weights(m, 6)
    B = 40
    s = inputs.random_spins(B, m.N, 13)
    c = np.random.default_rng(5).normal(0, 1, B).astype(np.float32)
    model = sg.Model(m, w, sg.SG_BF16)
    ts = torch.tensor(s, device="cuda")
    lq = _np(model.logprob(ts))
    lqo = oracle.logprob(ocfg(m), w, s)
    assert np.abs(lq - lqo).max() <= BF16_LOGQ_TOL * m.N
    logq = torch.empty(B, dtype=torch.float32, device="cuda")
    g = _np(model.grad(ts, torch.tensor(c, device="cuda"), logq=logq))
    model.check()
    go, _ = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"N={m.N} d={m.d} h={m.n_heads} W={m.W} S={m.S}: max|dlogq|/N "
          f"{np.abs(lq - lqo).max() / m.N:.2e}, grad rel err {rel:.2e}")
    assert rel < 2e-2
    assert_grad_blocks(m, g, go, BF16_GRAD_BLOCK_TOL)
    assert np.array_equal(_np(logq), lq)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_grad_chunking_matches_one_chunk_and_oracle(precision):
    """sg_grad over several chunks of samples (a chunk cap of 64 samples on
    B = 300: five chunks, the last ragged) equals one chunk up to FP32
    summation order, and the oracle within the precision's bound."""
    m = inputs.ModelShape(40, 2, 64, 4, mask_kind=1, W=8, S=9)
    prec = sg.SG_BF16 if precision == "bf16" else sg.SG_FP32
    w = inputs.make_weights(m, 5)
    B = 300
    s = inputs.random_spins(B, m.N, 19)
    c = np.random.default_rng(4).normal(0, 1, B).astype(np.float32)
    model = sg.Model(m, w, prec)
    ts, tc = torch.tensor(s, device="cuda"), torch.tensor(c, device="cuda")
    lq1 = torch.empty(B, dtype=torch.float32, device="cuda")
    g1 = _np(model.grad(ts, tc, logq=lq1))
    model.set_max_chunk(64)
    lq5 = torch.empty(B, dtype=torch.float32, device="cuda")
    g5 = _np(model.grad(ts, tc, logq=lq5))
    lp5 = _np(model.logprob(ts))
    model.set_max_chunk(0)
    model.check()
    assert np.array_equal(_np(lq1), _np(lq5))  # log q is per sample: chunking cannot change it
    assert np.array_equal(lp5, _np(lq1))
    assert np.abs(g5 - g1).max() <= 1e-5 * np.abs(g1).max()
    go, lqo = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    rel = np.linalg.norm(g5 - go) / np.linalg.norm(go)
    assert rel < (2e-2 if prec == sg.SG_BF16 else 1e-4), rel
    if prec == sg.SG_BF16:
        assert_grad_blocks(m, g5, go, BF16_GRAD_BLOCK_TOL)


@pytest.mark.parametrize("name,precision,cap", [("ea2d16", "bf16", 0), ("ea2d16", "bf16", 4096),
                                                ("ea2d16", "fp32", 0), ("sk1024", "bf16", 0),
                                                ("ea3d10", "bf16", 0)])
def test_full_size_grad_on_isolated_samples(name, precision, cap):
    """The gradient call at full size (2D EA L=16, B = 16384, one chunk of
    16384 for BF16 or several under a chunk cap; SK N=1024, B = 8192, on the
    tcgen05 attention; 3D EA L=10, B = 32768): coefficients zero except on
    a few samples spread over the batch, so the oracle's gradient of those
    samples is the whole expected gradient.  Log q of those samples against
    the oracle too."""
    wl = inputs.workloads()[name]
    m = wl.model
    w = wl.weights()
    prec = sg.SG_BF16 if precision == "bf16" else sg.SG_FP32
    model = sg.Model(m, w, prec)
    if cap:
        model.set_max_chunk(cap)
    B = wl.B
    spins, _ = model.sample(B, seed=404)
    rows = np.array([0, 5000, 12345, B - 1]) if m.N <= 256 else np.array([0, B // 2 + 77, B - 1])
    c = np.zeros(B, np.float32)
    c[rows] = [0.7, -1.1, 0.4, 0.9][: len(rows)]
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    g = _np(model.grad(spins, torch.tensor(c, device="cuda"), logq=lq))
    model.check()
    s = _np(spins)
    go, lqo = oracle.grad(ocfg(m), w, s[rows], c[rows].astype(np.float64))
    tol = BF16_LOGQ_TOL if prec == sg.SG_BF16 else FP32_LOGQ_TOL
    assert np.abs(_np(lq)[rows] - lqo).max() <= tol * m.N
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"{name} {precision} cap {cap}: full-size grad rel err {rel:.2e}")
    assert rel < (2e-2 if prec == sg.SG_BF16 else 1e-4), rel
    if prec == sg.SG_BF16:
        assert_grad_blocks(m, g, go, BF16_GRAD_BLOCK_TOL)


# --------------------------------------------------------------------------
# MH, Metropolis, overlap, Adam
# --------------------------------------------------------------------------

def test_mh_step_matches_oracle():
    m = inputs.ModelShape(16, 1, 32, 4)
    inst = inputs.make_sk(16, 3)
    model = sg.Model(m, inputs.make_weights(m, 3), sg.SG_FP32)
    gi = sg.Instance(inst)
    C, per, beta = 64, 50, 1.0
    prop, lq = model.sample(C * per, seed=11)
    E = gi.energy(prop)
    cs, clq = model.sample(C, seed=12)
    cE = gi.energy(cs).double()
    clq = clq.double()
    cE0, clq0 = _np(cE).copy(), _np(clq).copy()
    acc, trace = sg.mh_step(prop, E, lq, C, beta, 77, cs, cE, clq, trace=True)
    torch.cuda.synchronize()
    oE, oL, oi, otr, oacc, ofl = oracle.mh(_np(E).astype(np.float64), _np(lq).astype(np.float64),
                                           C, beta, 77, cE0, clq0)
    flagged_chains = np.unique(np.nonzero(ofl.reshape(per, C))[1])
    ok = np.setdiff1d(np.arange(C), flagged_chains)
    assert np.array_equal(_np(acc)[ok], oacc[ok])
    assert np.array_equal(_np(cE)[ok], oE[ok])
    assert np.array_equal(_np(trace)[:, ok], otr[:, ok].astype(np.float32))
    moved = ok[oi[ok] >= 0]
    assert np.array_equal(_np(cs)[moved], _np(prop)[oi[moved]])


@pytest.mark.parametrize("kind", ["ea2", "ea3", "sk"])
def test_metropolis_matches_oracle(kind):
    inst = {"ea2": inputs.make_ea(2, 8, 1, pm=True), "ea3": inputs.make_ea(3, 4, 2, pm=True),
            "sk": inputs.make_sk(30, 5)}[kind]
    R, sweeps, beta = 100, 20, 1.0
    s0 = inputs.random_spins(R, inst.N, 3)
    gi = sg.Instance(inst)
    st = torch.tensor(s0, device="cuda")
    E0 = torch.tensor(oracle.energy(inst, s0), device="cuda")
    E, tr = gi.metropolis(st, sweeps, beta, 42, E=E0, trace=True)
    so, Eo, tro, nflag = oracle.metropolis(inst, s0, sweeps, beta, 42)
    assert nflag == 0
    assert np.array_equal(_np(st), so)
    if kind == "sk":
        assert np.allclose(_np(E), Eo, rtol=0, atol=1e-9)
    else:
        assert np.array_equal(_np(E), Eo)
        assert np.array_equal(_np(tr), tro.astype(np.float32))


def test_overlap_hist_matches_oracle():
    s = inputs.random_spins(101, 37, 4)
    h = _np(sg.overlap_hist(torch.tensor(s, device="cuda")))
    assert np.array_equal(h, oracle.overlap_hist(s))


def test_adam_step_matches_torch_reference():
    n = 1000
    rng = np.random.default_rng(0)
    w, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = rng.normal(size=n).astype(np.float32) * 0.1, rng.random(n).astype(np.float32) * 0.1
    tw, tg, tm, tv = (torch.tensor(x, device="cuda") for x in (w, g, m, v))
    sg.adam_step(tw, tg, tm, tv, lr=1e-3, step=3)
    b1, b2 = 0.9, 0.999
    m2 = b1 * torch.tensor(m) + (1 - b1) * torch.tensor(g)
    v2 = b2 * torch.tensor(v) + (1 - b2) * torch.tensor(g) ** 2
    w2 = torch.tensor(w) - 1e-3 * (m2 / (1 - b1 ** 3)) / ((v2 / (1 - b2 ** 3)).sqrt() + 1e-8)
    assert torch.allclose(tw.cpu(), w2, rtol=1e-6, atol=1e-7)


# --------------------------------------------------------------------------
# Full-size workloads in the benchmark's launch configuration
# --------------------------------------------------------------------------

def test_full_size_sk20_fp32_all_rows():
    wl = inputs.workloads()["sk20"]
    m, inst = wl.model, wl.instance()
    w = wl.weights()
    model, spins, logq, frac, dl = _sample_and_check(m, w, wl.B, 2024, sg.SG_FP32, FP32_LOGQ_TOL)
    assert frac < 0.01
    E = sg.Instance(inst).energy(spins)
    Eo = oracle.energy(inst, _np(spins))
    assert np.allclose(_np(E), Eo, rtol=1e-5, atol=1e-5)


def test_full_size_ea2d16_fp32_sampled_rows():
    wl = inputs.workloads()["ea2d16"]
    m, inst = wl.model, wl.instance()
    w = wl.weights()
    model = sg.Model(m, w, sg.SG_FP32)
    spins, logq, flags = model.sample(wl.B, seed=31, with_flags=True)
    E, Ei = sg.Instance(inst).energy(spins, want_int=True)
    torch.cuda.synchronize()
    s, lq, fl = _np(spins), _np(logq), _np(flags)
    rows = np.array([0, 1, 4095, 8191, 12345, wl.B - 1])
    so, lqo, _, _ = oracle_replay(m, w, 31, s, fl, FP32_BAND, rows=rows)
    assert np.array_equal(so, s[rows])
    assert np.abs(lqo - lq[rows]).max() <= FP32_LOGQ_TOL * m.N
    assert np.array_equal(_np(Ei).astype(np.float64), oracle.energy(inst, s))
    tf = _np(model.logprob(spins[:64]))
    assert np.abs(tf - oracle.logprob(ocfg(m), w, s[:64])).max() <= FP32_LOGQ_TOL * m.N
