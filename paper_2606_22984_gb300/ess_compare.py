"""Neural independence MH versus single-spin-flip Metropolis: ESS per second.

The transformer (optionally trained first by train.Trainer: variational
annealing from T0 down to the target temperature, local Monte Carlo
refinement of the samples with the self-distillation term of Eq. loss2, Adam
or Muon) proposes whole configurations; sg_mh_step accepts them against the
exact energies, chain by chain.  sg_metropolis runs the classical sweeps on the same instance.  Both
chains' energy traces give tau_int and the ESS (analysis.py); ESS/sec divides by
the GPU time of the calls that produced them (for MH: sampling + energies +
MH; for Metropolis: the sweeps).  Prints one JSON line.

  python -m paper_2606_22984_gb300.ess_compare --workload ea3d10
  python -m paper_2606_22984_gb300.ess_compare --lattice 3 4 --beta 2.0 --d 64 \
      --layers 2 --heads 4 --train-steps 300
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import analysis, build, inputs, sg


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def train(model, inst, a, beta):
    """Variational annealing toward T = 1 / beta (Methods "Variational
    annealing"): T held at T0 for the warm-up, then lowered in n_anneal
    equal decrements every n_eq steps, clamped at 1 / beta; returns the
    trainer's log and the batch free energies of the trained model."""
    from .train import TrainConfig, Trainer, anneal_temperature

    T_target = 1.0 / beta
    T0 = max(a.anneal_T0, T_target)

    def sched(i):
        return max(T_target, anneal_temperature(i, T0, a.anneal_warmup, a.anneal_steps,
                                                 a.anneal_eq))

    cfg = TrainConfig(B=a.train_batch, steps=a.train_steps, lr=a.lr, schedule=sched,
                      lmc_sweeps=a.lmc_sweeps, w=a.w, optimizer=a.optimizer, seed=a.seed,
                      log_every=max(1, a.train_steps // 10))
    log = Trainer(model, inst, cfg).run()
    s, lq = model.sample(a.train_batch, seed=987654)
    out = sg.free_energy(inst.energy(s), lq, beta).cpu().numpy()
    return log, out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="")
    p.add_argument("--lattice", type=int, nargs=2, metavar=("D", "L"), default=None)
    p.add_argument("--beta", type=float, default=None)
    p.add_argument("--d", type=int, default=64)
    p.add_argument("--layers", type=int, default=2)
    p.add_argument("--heads", type=int, default=4)
    p.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    p.add_argument("--train-steps", type=int, default=0)
    p.add_argument("--train-batch", type=int, default=1024)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--optimizer", default="muon", choices=["adam", "muon"])
    p.add_argument("--lmc-sweeps", type=int, default=2, help="local MC sweeps per step (Eq. loss2)")
    p.add_argument("--w", type=float, default=0.05, help="self-distillation weight of Eq. loss2")
    p.add_argument("--anneal-T0", type=float, default=3.0)
    p.add_argument("--anneal-warmup", type=int, default=50)
    p.add_argument("--anneal-steps", type=int, default=20)
    p.add_argument("--anneal-eq", type=int, default=10)
    p.add_argument("--proposals", type=int, default=0, help="proposals per MH step (default: B)")
    p.add_argument("--chains", type=int, default=1024)
    p.add_argument("--mh-steps", type=int, default=4)
    p.add_argument("--replicas", type=int, default=2048)
    p.add_argument("--sweeps", type=int, default=1000)
    p.add_argument("--warmup-sweeps", type=int, default=100)
    p.add_argument("--seed", type=int, default=7)
    a = p.parse_args()
    build.build()
    prec = sg.SG_BF16 if a.precision == "bf16" else sg.SG_FP32
    if a.workload:
        wl = inputs.workloads()[a.workload]
        shape, inst_src, B = wl.model, wl.instance(), wl.B
        beta = a.beta if a.beta is not None else wl.betas[0]
        weights = wl.weights()
        name = wl.name
    else:
        D, L = a.lattice
        W, S = inputs.lattice_mask(D, L)
        N = L ** D
        shape = inputs.ModelShape(N, a.layers, a.d, a.heads, mask_kind=1, W=W, S=S)
        inst_src = inputs.make_ea(D, L, a.seed, pm=True)
        B = a.proposals or 32768
        beta = a.beta if a.beta is not None else 1.0
        weights = inputs.make_weights(shape, a.seed)
        name = f"{D}D EA L={L} +-J periodic, {a.layers}L d{a.d} h{a.heads}, band W={W} S={S}"
    Bp = a.proposals or B
    C = a.chains
    assert Bp % C == 0
    model = sg.Model(shape, weights, prec)
    inst = sg.Instance(inst_src)
    stream = torch.cuda.current_stream()
    log, F_train = train(model, inst, a, beta) if a.train_steps else (None, None)

    # ---- neural MH
    cs, clq = model.sample(C, seed=1)
    cE = inst.energy(cs).double()
    clq = clq.double()
    traces, acc_total, ms_mh = [], 0, 0.0
    for i in range(a.mh_steps):
        e0, e1 = _events()
        e0.record(stream)
        prop, lq = model.sample(Bp, seed=100 + i)
        E = inst.energy(prop)
        acc, tr = sg.mh_step(prop, E, lq, C, beta, 1000 + i, cs, cE, clq, trace=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_mh += e0.elapsed_time(e1)
        traces.append(tr.cpu().numpy())
        acc_total += int(acc.sum().item())
    model.check()
    trace = np.concatenate(traces, axis=0)            # [steps * Bp/C, C]
    burn = trace.shape[0] // 10
    mh_ess = analysis.ess(trace[burn:])
    mh_tau = analysis.tau_int(trace[burn:])
    hist = sg.overlap_hist(cs).cpu().numpy()
    Ns = shape.N
    q = (np.arange(Ns + 1) * 2 - Ns) / Ns
    mh = {"proposals": Bp * a.mh_steps, "chains": C, "acceptance": acc_total / (Bp * a.mh_steps),
          "tau_int_proposals": mh_tau, "ess": mh_ess, "gpu_ms": ms_mh,
          "ess_per_sec": mh_ess / (ms_mh / 1e3), "mean_E_per_spin": float(trace[burn:].mean() / Ns),
          "overlap_mean_abs_q": float((hist * np.abs(q)).sum() / max(1, hist.sum()))}

    # ---- single-spin-flip Metropolis on the same instance
    rs = torch.tensor(inputs.random_spins(a.replicas, Ns, a.seed + 1), device="cuda")
    Em = inst.energy(rs).double()
    inst.metropolis(rs, a.warmup_sweeps, beta, 5, E=Em)
    e0, e1 = _events()
    e0.record(stream)
    Em, trm = inst.metropolis(rs, a.sweeps, beta, 6, E=Em, trace=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_met = e0.elapsed_time(e1)
    trm = trm.cpu().numpy()
    met_ess = analysis.ess(trm)
    met = {"replicas": a.replicas, "sweeps": a.sweeps, "tau_int_sweeps": analysis.tau_int(trm),
           "ess": met_ess, "gpu_ms": ms_met, "ess_per_sec": met_ess / (ms_met / 1e3),
           "mean_E_per_spin": float(trm.mean() / Ns)}
    # an independence chain whose mean energy still differs from the
    # Metropolis chains' has not reached the Boltzmann law: its ESS is not
    # a valid equilibrium figure
    gap = mh["mean_E_per_spin"] - met["mean_E_per_spin"]
    out = {"workload": name, "beta": beta, "precision": a.precision,
           "mean_E_gap_per_spin_mh_minus_metropolis": gap,
           "mh_equilibrated": abs(gap) < 0.01,
           "train_steps": a.train_steps, "train_batch": a.train_batch,
           "training": None if log is None else {
               "optimizer": a.optimizer, "lmc_sweeps": a.lmc_sweeps, "w": a.w,
               "anneal": [a.anneal_T0, a.anneal_warmup, a.anneal_steps, a.anneal_eq],
               "T": log.T, "mean_E_per_spin": [e / Ns for e in log.mean_E]},
           "F_q_per_spin_after_training": None if F_train is None else float(F_train[0] / Ns),
           "F_IS_per_spin_after_training": None if F_train is None else float(F_train[1] / Ns),
           "mh": mh, "metropolis": met,
           "mh_over_metropolis_ess_per_sec": mh["ess_per_sec"] / met["ess_per_sec"]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
