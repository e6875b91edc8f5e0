"""Training loop of the method on the C ABI.  Host orchestration only: every
step of the arithmetic runs in libsg kernels (sampling, local Monte Carlo,
energies, loss weights, the hand-written backward and the optimiser).

One step (Methods "Training strategy", "Variational annealing"; Eq. loss2):
  1. draw B configurations from q (sg_sample);
  2. optionally refine them by a short local Monte Carlo trajectory at the
     current temperature (sg_metropolis) and score the refined
     configurations by the teacher-forced log q (sg_logprob);
  3. energies (sg_energy);
  4. REINFORCE weights of L = E + T ln q (or beta E + ln q at a fixed beta),
     with the likelihood term w of Eq. loss2 (sg_loss_coeff);
  5. gradient through torch.autograd: the surrogate sum_b c_b ln q_b of
     autograd.reinforce_loss, whose forward and backward are one sg_grad
     call, and loss.backward() fills the weight blob's .grad; optimiser step
     on that gradient (sg_adam_step, or sg_muon_step: Muon on the weight
     matrices, AdamW on the rest), weights repacked (sg_model_refresh).
"""
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import torch

from . import autograd, sg


def anneal_temperature(i: int, T0: float, n_warmup: int, n_anneal: int, n_eq: int) -> float:
    """Temperature at training step i of the annealing schedule (Methods
    "Variational annealing"): T0 through the warm-up, then lowered by
    T0 / n_anneal every n_eq steps, reaching 0 after n_warmup + n_eq n_anneal
    steps (and staying there)."""
    if n_anneal < 1 or n_eq < 1:
        raise ValueError("n_anneal and n_eq must be >= 1")
    if i <= n_warmup:
        return float(T0)
    k = (i - n_warmup) // n_eq
    return max(float(T0) - float(T0) / n_anneal * k, 0.0)


@dataclass
class TrainConfig:
    B: int
    steps: int
    lr: float = 1e-3
    beta: Optional[float] = None          # fixed inverse temperature (free-energy form)
    schedule: Optional[Callable[[int], float]] = None  # temperature T(i) (ground-state form)
    lmc_sweeps: int = 0                   # local Monte Carlo sweeps on the samples (0: off)
    w: float = 0.0                        # likelihood (self-distillation) weight of Eq. loss2
    T_floor: float = 1e-3                 # temperature used by the local Monte Carlo at T = 0
    optimizer: str = "adam"               # "adam", or "muon" (Muon + AdamW, sg_muon_step)
    momentum: float = 0.95                # Muon momentum
    weight_decay: float = 0.0             # Muon / AdamW decoupled weight decay
    seed: int = 1
    log_every: int = 50


@dataclass
class TrainLog:
    step: List[int] = field(default_factory=list)
    T: List[float] = field(default_factory=list)
    mean_L: List[float] = field(default_factory=list)
    mean_E: List[float] = field(default_factory=list)
    min_E: List[float] = field(default_factory=list)


class Trainer:
    """REINFORCE training of one model on one instance (Adam or Muon)."""

    def __init__(self, model: "sg.Model", inst: "sg.Instance", cfg: TrainConfig):
        if (cfg.beta is None) == (cfg.schedule is None):
            raise ValueError("give exactly one of beta (fixed) or schedule (temperature)")
        if cfg.optimizer not in ("adam", "muon"):
            raise ValueError("optimizer must be 'adam' or 'muon'")
        self.model, self.inst, self.cfg = model, inst, cfg
        # the master blob as an autograd leaf: backward() writes its .grad
        self.w = model.weights().requires_grad_(True)
        self.m = torch.zeros_like(self.w, requires_grad=False)
        self.v = torch.zeros_like(self.m)
        self.mom = torch.zeros_like(self.m) if cfg.optimizer == "muon" else None
        self.log = TrainLog()

    def temperature(self, i: int) -> float:
        c = self.cfg
        return 1.0 / c.beta if c.schedule is None else float(c.schedule(i))

    def step(self, i: int):
        c, model, inst = self.cfg, self.model, self.inst
        T = self.temperature(i)
        seed = (c.seed << 20) + i
        spins, logq = model.sample(c.B, seed=seed)
        if c.lmc_sweeps > 0:
            inst.metropolis(spins, c.lmc_sweeps, 1.0 / max(T, c.T_floor), seed)
            logq = model.logprob(spins)
        E = inst.energy(spins)
        if c.schedule is None:   # free energy, Eq. loss1: L = beta E + ln q
            a, cc = c.beta, 1.0
        else:                    # ground-state form: L = E + T ln q
            a, cc = 1.0, T
        coeff, mean = sg.loss_coeff(E, logq, a, cc, c.w)
        self.w.grad = None
        autograd.reinforce_loss(model, spins, coeff, weights=self.w).backward()
        grad = self.w.grad
        if self.mom is None:
            sg.adam_step(self.w.detach(), grad, self.m, self.v, c.lr, i + 1)
        else:
            model.muon_step(grad, self.mom, self.m, self.v, c.lr, i + 1, mu=c.momentum,
                            weight_decay=c.weight_decay)
        model.refresh()
        if i % c.log_every == 0 or i == c.steps - 1:
            mv = mean.cpu().numpy()
            self.log.step.append(i)
            self.log.T.append(T)
            self.log.mean_L.append(float(mv[0]))
            self.log.mean_E.append(float(mv[1]))
            self.log.min_E.append(float(E.min().item()))
        return spins, E

    def run(self):
        for i in range(self.cfg.steps):
            self.step(i)
        self.model.check()
        return self.log
