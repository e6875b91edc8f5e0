"""End-to-end training on the GPU: REINFORCE (Eq. loss1) with the hand-written
backward and Adam, then the free energy of the trained model against exact
enumeration of all 2^N states by the oracle (Eqs. KL_div, free_energy)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_22984_gb300 import inputs, sg

from helpers import ocfg

pytestmark = pytest.mark.gpu

# Muon on a BF16 model: the Newton-Schulz iterate and its products' operands
# are BF16 (unit roundoff 2^-8); five steps of rounding X, A and Bm give update
# errors of 1.0e-2 to 1.9e-2 relative on GB300 (d = 64, 96, 128); the bound
# leaves a factor of about 2.5
MUON_BF16_TOL = 5e-2


def _train(model, inst, B, beta, steps, lr, seed0=100):
    w = model.weights()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    grad = torch.empty_like(w)
    hist = []
    for i in range(steps):
        spins, logq = model.sample(B, seed=seed0 + i)
        E = inst.energy(spins)
        out, coeff = sg.free_energy(E, logq, beta, want_coeff=True)
        model.grad(spins, coeff, grad=grad)
        sg.adam_step(w, grad, m, v, lr, i + 1)
        model.refresh()
        if i % 50 == 0 or i == steps - 1:
            hist.append(out.cpu().numpy().copy())
    model.check()
    return np.array(hist)


@pytest.mark.parametrize("precision", [sg.SG_FP32, sg.SG_BF16])
def test_sk20_training_reaches_exact_free_energy(precision):
    """SK N=20, beta=1: after REINFORCE training the importance-weighted
    free energy per spin is within 1e-3 of the exact F/N, and the exact
    variational F_q of the trained model lies above F (Eq. KL_div)."""
    wl = inputs.workloads()["sk20"]
    m = wl.model if precision == sg.SG_FP32 else inputs.ModelShape(20, 2, 64, 4)
    inst = wl.instance()
    beta = 1.0
    model = sg.Model(m, inputs.make_weights(m, 1), precision)
    gi = sg.Instance(inst)
    hist = _train(model, gi, 4096, beta, 400, 2e-3)
    assert hist[-1][0] < hist[0][0]  # F_q decreased
    w_trained = model.weights().cpu().numpy().astype(np.float64)
    ex = oracle.enumerate_exact(ocfg(m), w_trained, inst, beta)
    assert abs(ex["sum_q"] - 1) < 1e-10
    assert ex["Fq"] >= ex["F"]
    # fresh large batch from the trained model
    spins, logq = model.sample(65536, seed=999)
    E = gi.energy(spins)
    out = sg.free_energy(E, logq, beta).cpu().numpy()
    N = m.N
    print(f"prec={precision} F/N exact {ex['F'] / N:.6f}  F_IS/N {out[1] / N:.6f}  "
          f"F_q/N {out[0] / N:.6f} (exact F_q/N {ex['Fq'] / N:.6f})  ESS {out[2]:.0f}")
    assert abs(out[1] - ex["F"]) / N <= 1e-3
    # the batch estimate of F_q agrees with the exact F_q of the trained model
    assert abs(out[0] - ex["Fq"]) / N <= 2e-3


def test_loss_coeff_matches_oracle():
    rng = np.random.default_rng(4)
    B = 5000
    E = rng.normal(-10, 3, B).astype(np.float32)
    lq = (-np.abs(rng.normal(12, 2, B))).astype(np.float32)
    for a, c, w in ((1.3, 1.0, 0.0), (1.0, 0.25, 0.0), (1.0, 0.1, 0.3), (0.0, 0.0, 1.0)):
        co, mean = sg.loss_coeff(torch.tensor(E, device="cuda"), torch.tensor(lq, device="cuda"), a, c, w)
        ref, mL, mE = oracle.loss_coeff(E, lq, a, c, w)
        assert np.allclose(co.cpu().numpy(), ref, rtol=1e-5, atol=1e-9)
        mv = mean.cpu().numpy()
        assert abs(mv[0] - mL) < 1e-9 * max(1.0, abs(mL)) and abs(mv[1] - mE) < 1e-9 * max(1.0, abs(mE))
    with pytest.raises(sg.SgError):
        sg.loss_coeff(torch.tensor(E, device="cuda"), torch.tensor(lq, device="cuda"), float("nan"), 1.0)


def test_annealing_reaches_the_sk20_ground_state():
    """Methods "Variational annealing": training on L = E + T ln q while T is
    lowered to 0 concentrates q on the ground state of SK N=20, whose energy
    the oracle finds by enumerating all 2^20 states."""
    from paper_2606_22984_gb300.train import TrainConfig, Trainer, anneal_temperature
    wl = inputs.workloads()["sk20"]
    m, inst = wl.model, wl.instance()
    model = sg.Model(m, inputs.make_weights(m, 2), sg.SG_FP32)
    gi = sg.Instance(inst)
    sched = lambda i: anneal_temperature(i, 1.0, 100, 20, 15)
    tr = Trainer(model, gi, TrainConfig(B=2048, steps=401, lr=3e-3, schedule=sched, log_every=100))
    log = tr.run()
    assert log.T[-1] == 0.0
    ex = oracle.enumerate_exact(ocfg(m), model.weights().cpu().numpy().astype(np.float64), inst, 1.0)
    spins, _ = model.sample(8192, seed=77)
    E = gi.energy(spins).cpu().numpy()
    print(f"E_min exact {ex['Emin']:.4f}  sampled min {E.min():.4f}  mean {E.mean():.4f}")
    assert abs(E.min() - ex["Emin"]) < 1e-3
    assert E.mean() < 0.9 * ex["Emin"]


def test_lmc_refinement_with_self_distillation_trains_toward_ground_state():
    """Eq. loss2: samples refined by local Monte Carlo before scoring, plus the
    likelihood term w, on a 2D EA L=4 +-J instance (N=16, band + sink mask);
    the refinement lowers the batch energy at low T, and the annealed training
    reaches the exact ground state (enumeration of 2^16 states)."""
    from paper_2606_22984_gb300.train import TrainConfig, Trainer, anneal_temperature
    inst = inputs.make_ea(2, 4, 9, pm=True)
    W, S = inputs.lattice_mask(2, 4)
    m = inputs.ModelShape(16, 2, 64, 4, mask_kind=1, W=W, S=S)
    model = sg.Model(m, inputs.make_weights(m, 3), sg.SG_FP32)
    gi = sg.Instance(inst)
    # one refinement at low temperature lowers the mean energy of raw samples
    spins, _ = model.sample(4096, seed=5)
    E0 = gi.energy(spins).cpu().numpy().mean()
    gi.metropolis(spins, 2, 1.0 / 0.2, 6)
    E1 = gi.energy(spins).cpu().numpy().mean()
    assert E1 < E0
    sched = lambda i: anneal_temperature(i, 1.5, 80, 20, 10)
    cfg = TrainConfig(B=1024, steps=300, lr=2e-3, schedule=sched, lmc_sweeps=2, w=0.05,
                      log_every=100)
    log = Trainer(model, gi, cfg).run()
    ex = oracle.enumerate_exact(ocfg(m), model.weights().cpu().numpy().astype(np.float64), inst, 1.0)
    spins, _ = model.sample(8192, seed=78)
    E = gi.energy(spins).cpu().numpy()
    print(f"E_min exact {ex['Emin']:.1f}  sampled min {E.min():.1f}  mean {E.mean():.2f}  "
          f"log mean_E {log.mean_E}")
    assert abs(E.min() - ex["Emin"]) < 1e-3
    assert E.mean() < 0.8 * ex["Emin"]


@pytest.mark.parametrize("shape", [inputs.ModelShape(12, 2, 32, 4),
                                   inputs.ModelShape(20, 1, 64, 4, d_ff=96),
                                   inputs.ModelShape(8, 1, 128, 8)])
def test_muon_step_matches_oracle(shape):
    """Three Muon steps (Newton-Schulz in FP32 on the GPU, FP64 in the oracle):
    the weight updates agree to 1e-3 relative, matrices and AdamW parameters."""
    m = shape
    w0 = inputs.make_weights(m, 8)
    model = sg.Model(m, w0, sg.SG_FP32)
    n = model.n_params
    dev = torch.device("cuda")
    mom, am, av = (torch.zeros(n, device=dev) for _ in range(3))
    w, mo, amo, avo = (w0.astype(np.float64).copy(), np.zeros(n), np.zeros(n), np.zeros(n))
    rng = np.random.default_rng(9)
    for step in range(1, 4):
        g = rng.normal(0, 1e-2, n).astype(np.float32)
        model.muon_step(torch.tensor(g, device=dev), mom, am, av, 2e-3, step, mu=0.95,
                        weight_decay=0.1)
        oracle.muon_step(ocfg(m), w, g, mo, amo, avo, 2e-3, 0.95, 0.1, 5, step)
    model.check()
    wg = model.weights().cpu().numpy().astype(np.float64)
    dg, do = wg - w0, w - w0
    rel = np.linalg.norm(dg - do) / np.linalg.norm(do)
    print(f"d={m.d}: Muon update rel err {rel:.2e}")
    assert rel < 1e-3
    assert np.allclose(mom.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)


def test_sk20_training_with_muon_reaches_exact_free_energy():
    """The paper's optimiser: REINFORCE (Eq. loss1) with Muon on the weight
    matrices, SK N=20 at beta = 1; F_IS/N within 1e-3 of the enumerated F/N."""
    from paper_2606_22984_gb300.train import TrainConfig, Trainer
    wl = inputs.workloads()["sk20"]
    m, inst = wl.model, wl.instance()
    model = sg.Model(m, inputs.make_weights(m, 1), sg.SG_FP32)
    gi = sg.Instance(inst)
    log = Trainer(model, gi, TrainConfig(B=4096, steps=400, lr=4e-3, beta=1.0,
                                         optimizer="muon", log_every=100)).run()
    ex = oracle.enumerate_exact(ocfg(m), model.weights().cpu().numpy().astype(np.float64), inst, 1.0)
    spins, logq = model.sample(65536, seed=999)
    out = sg.free_energy(gi.energy(spins), logq, 1.0).cpu().numpy()
    print(f"Muon: F/N exact {ex['F'] / m.N:.6f}  F_IS/N {out[1] / m.N:.6f}  F_q/N {out[0] / m.N:.6f}"
          f"  exact (F_q - F)/N {(ex['Fq'] - ex['F']) / m.N:.2e}")
    assert abs(out[1] - ex["F"]) / m.N <= 1e-3
    assert 0 <= (ex["Fq"] - ex["F"]) / m.N < 2e-3  # the variational gap (KL / beta N)


@pytest.mark.parametrize("shape", [inputs.ModelShape(20, 1, 64, 4), inputs.ModelShape(8, 1, 128, 8),
                                   inputs.ModelShape(12, 1, 96, 6)])
def test_muon_step_tensor_cores_matches_oracle(shape):
    """BF16 models run Muon's Newton-Schulz iteration on tcgen05 (one launch
    for every matrix; the iterate X in BF16, FP32 accumulators).  Three steps
    against the FP64 oracle: the matrices' update within the BF16 bound, the
    momentum and the AdamW parameters as for the FP32 path."""
    import time
    m = shape
    w0 = inputs.make_weights(m, 8)
    model = sg.Model(m, w0, sg.SG_BF16)
    n = model.n_params
    dev = torch.device("cuda")
    mom, am, av = (torch.zeros(n, device=dev) for _ in range(3))
    w, mo, amo, avo = (w0.astype(np.float64).copy(), np.zeros(n), np.zeros(n), np.zeros(n))
    rng = np.random.default_rng(9)
    for step in range(1, 4):
        g = rng.normal(0, 1e-2, n).astype(np.float32)
        model.muon_step(torch.tensor(g, device=dev), mom, am, av, 2e-3, step, mu=0.95,
                        weight_decay=0.1)
        oracle.muon_step(ocfg(m), w, g, mo, amo, avo, 2e-3, 0.95, 0.1, 5, step)
    model.check()
    wg = model.weights().cpu().numpy().astype(np.float64)
    dg, do = wg - w0, w - w0
    mat = np.zeros(n, bool)
    for name, (off, shp) in inputs.offsets(m).items():
        if name.split(".")[-1] in ("Wqkv", "W1", "W2"):
            mat[off:off + int(np.prod(shp))] = True
    rel_mat = np.linalg.norm(dg[mat] - do[mat]) / np.linalg.norm(do[mat])
    rel_rest = np.linalg.norm(dg[~mat] - do[~mat]) / np.linalg.norm(do[~mat])
    # time one step against the FP32 path on the same shape
    m32 = sg.Model(m, w0, sg.SG_FP32)
    gt = torch.tensor(rng.normal(0, 1e-2, n).astype(np.float32), device=dev)
    ts = {}
    for name, mdl in (("bf16 tensor cores", model), ("fp32", m32)):
        mdl.muon_step(gt, mom.clone(), am.clone(), av.clone(), 2e-3, 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            mdl.muon_step(gt, mom.clone(), am.clone(), av.clone(), 2e-3, 4)
        torch.cuda.synchronize()
        ts[name] = (time.perf_counter() - t0) / 5 * 1e3
    print(f"d={m.d}: Muon update rel err matrices {rel_mat:.2e}, other parameters {rel_rest:.2e}; "
          f"step time " + ", ".join(f"{k} {v:.2f} ms" for k, v in ts.items()))
    assert rel_mat < MUON_BF16_TOL
    assert rel_rest < 1e-5
    assert np.allclose(mom.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
