"""Pins of the host-side chain analysis against closed forms."""
import numpy as np

from paper_2606_22984_gb300 import analysis


def ar1(phi, n, chains, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, chains))
    e = rng.standard_normal((n, chains))
    x[0] = e[0] / np.sqrt(1 - phi ** 2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x


def test_tau_of_ar1_matches_closed_form():
    """AR(1) with coefficient phi: tau_int = (1 + phi) / (1 - phi)."""
    for phi in (0.0, 0.5, 0.9):
        x = ar1(phi, 20000, 8, 1)
        tau = analysis.tau_int(x)
        expect = (1 + phi) / (1 - phi)
        assert abs(tau - expect) < 0.1 * expect + 0.05, (phi, tau, expect)


def test_ess_of_independent_samples_is_sample_count():
    x = np.random.default_rng(3).standard_normal((5000, 4))
    e = analysis.ess(x)
    assert 0.8 * 20000 < e < 1.25 * 20000


def test_constant_chain_does_not_divide_by_zero():
    assert analysis.tau_int(np.ones((100, 2))) >= 1e-12
