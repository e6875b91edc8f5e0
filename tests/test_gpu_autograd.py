"""The REINFORCE backward behind torch.autograd (Eq. loss1, Methods "Training
strategy"): loss.backward() through autograd.LogQ and autograd.reinforce_loss
gives the hand-written sg_grad gradient, the FP64 oracle's gradient within the
FP32 bound, and the directional finite difference of the teacher-forced log q."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_22984_gb300 import autograd, inputs, sg

from helpers import ocfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_22984_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


SHAPES = [inputs.ModelShape(20, 2, 32, 4),
          inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7)]


def _case(m, B=64, seed=5):
    w = inputs.make_weights(m, seed)
    s = inputs.random_spins(B, m.N, seed + 1)
    c = (np.random.default_rng(seed).normal(0, 1, B) / B).astype(np.float32)
    return w, s, c


@pytest.mark.parametrize("m", SHAPES)
def test_logq_function_backward_is_sg_grad_and_matches_oracle(m):
    w, s, c = _case(m)
    model = sg.Model(m, w, sg.SG_FP32)
    ts = torch.tensor(s, device="cuda")
    tc = torch.tensor(c, device="cuda")
    wt = model.weights().requires_grad_(True)
    lq = autograd.logq(model, ts, weights=wt)
    assert lq.requires_grad
    (tc * lq).sum().backward()
    g_auto = wt.grad.detach().cpu().numpy()
    g_direct = model.grad(ts, tc).cpu().numpy()
    go, lqo = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    assert np.abs(lq.detach().cpu().numpy() - lqo).max() <= 1e-4 * m.N
    # the same kernels on the same inputs: equal up to FP32 summation order
    assert np.abs(g_auto - g_direct).max() <= 1e-6 * np.abs(g_direct).max()
    rel = np.linalg.norm(g_auto - go) / np.linalg.norm(go)
    assert rel < 1e-4, rel


@pytest.mark.parametrize("precision", [sg.SG_FP32, sg.SG_BF16])
def test_reinforce_loss_backward_fills_weight_grad(precision):
    m = inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7)
    w, s, c = _case(m, B=200, seed=9)
    model = sg.Model(m, w, precision)
    ts = torch.tensor(s, device="cuda")
    tc = torch.tensor(c, device="cuda")
    wt = model.weights().requires_grad_(True)
    loss = autograd.reinforce_loss(model, ts, tc, weights=wt)
    loss.backward()
    g_auto = wt.grad.detach().cpu().numpy()
    go, lqo = oracle.grad(ocfg(m), w, s, c.astype(np.float64))
    tol_lq = 2e-2 if precision == sg.SG_BF16 else 1e-4
    assert abs(loss.item() - float(c.astype(np.float64) @ lqo)) <= tol_lq * m.N * np.abs(c).sum()
    rel = np.linalg.norm(g_auto - go) / np.linalg.norm(go)
    print(f"precision {precision}: reinforce_loss grad rel err {rel:.2e}")
    assert rel < (2e-2 if precision == sg.SG_BF16 else 1e-4)
    # a second backward through a scaled loss scales the gradient (up to the
    # FP32 summation order of the split weight-gradient products, whose
    # partial sums meet in atomics)
    wt.grad = None
    (3.0 * autograd.reinforce_loss(model, ts, tc, weights=wt)).backward()
    g3 = wt.grad.cpu().numpy()
    assert np.abs(g3 - 3.0 * g_auto).max() <= 1e-5 * np.abs(3.0 * g_auto).max()


def test_logq_gradient_matches_finite_differences():
    """Directional derivative of f(w) = sum_b c_b log q_b(w) along random
    directions: central differences of the FP32 teacher-forced log q against
    the autograd gradient (the oracle's FP64 backward is pinned against
    finite differences at 1e-6 on the CPU; here FP32 rounding of f, about
    1e-6 relative, sets the tolerance)."""
    m = inputs.ModelShape(16, 1, 32, 4)
    w, s, c = _case(m, B=128, seed=13)
    c = c * 128  # O(1) coefficients
    model = sg.Model(m, w, sg.SG_FP32)
    ts = torch.tensor(s, device="cuda")
    tc = torch.tensor(c, device="cuda")
    wt = model.weights().requires_grad_(True)
    (tc * autograd.logq(model, ts, weights=wt)).sum().backward()
    g = wt.grad.detach().to(torch.float64)
    w0 = wt.detach().clone()
    rng = np.random.default_rng(3)

    def f(wv):
        model.weights().copy_(wv)
        model.refresh()
        return float((tc.double() * model.logprob(ts).double()).sum())

    for _ in range(4):
        v = torch.tensor(rng.normal(size=w0.numel()), device="cuda")
        v /= v.norm()
        h = 1e-2
        fd = (f((w0.double() + h * v).float()) - f((w0.double() - h * v).float())) / (2 * h)
        an = float(g @ v)
        print(f"directional derivative: autograd {an:.6f}  central difference {fd:.6f}")
        assert abs(fd - an) <= 2e-2 * max(1.0, abs(an))
    model.weights().copy_(w0)
    model.refresh()
