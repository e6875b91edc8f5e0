"""Host-side analysis of Markov-chain output: integrated autocorrelation time
and effective sample size.  These turn the energy traces that sg_mh_step and
sg_metropolis write on the GPU into the ESS/sec figures; none of the method's
arithmetic is here.

tau_int follows Sokal's automatic windowing: tau(M) = 1 + 2 sum_{k=1..M} rho(k)
with the smallest window M >= c * tau(M) (c = 5), rho averaged over chains.
ESS = (number of samples) / tau.
"""
from __future__ import annotations

import numpy as np


def autocorr(x: np.ndarray, max_lag: int) -> np.ndarray:
    """Normalised autocorrelation rho(0..max_lag) of chains x [n, chains],
    averaged over chains (FFT based)."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n = x.shape[0]
    xc = x - x.mean(axis=0, keepdims=True)
    f = np.fft.rfft(xc, n=2 * n, axis=0)
    acov = np.fft.irfft(f * np.conj(f), axis=0)[: max_lag + 1] / n
    var = acov[0]
    good = var > 0
    if not np.any(good):
        rho = np.zeros(max_lag + 1)
        rho[0] = 1.0
        return rho
    return (acov[:, good] / var[good]).mean(axis=1)


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    """Integrated autocorrelation time with Sokal's window (tau = 1 for
    independent samples)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    rho = autocorr(x, n - 1)
    tau = 1.0
    for M in range(1, n):
        tau = 1.0 + 2.0 * rho[1:M + 1].sum()
        if M >= c * tau:
            return max(tau, 1e-12)
    return max(tau, 1e-12)


def ess(x: np.ndarray, c: float = 5.0) -> float:
    """Effective sample size of chains x [n, chains]: n * chains / tau."""
    x = np.asarray(x, dtype=np.float64)
    chains = 1 if x.ndim == 1 else x.shape[1]
    return x.shape[0] * chains / tau_int(x, c)
