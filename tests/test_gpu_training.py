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
