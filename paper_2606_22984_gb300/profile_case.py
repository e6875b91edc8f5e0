"""Run one call of the hot path on a synthetic workload, for profilers (ncu).

  python -m paper_2606_22984_gb300.profile_case --call sample --workload ea2d16 \
      --batch 4096 --precision fp32 --iters 2

Only the named call runs (after its inputs are prepared), so a capture holds
just that call's memory: the model, the inputs and the call's own workspace.
"""
from __future__ import annotations

import argparse

import torch

from . import build, inputs, sg


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--call", default="sample",
                   choices=["sample", "logprob", "grad", "energy", "free_energy", "mh"])
    p.add_argument("--workload", default="ea2d16")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    p.add_argument("--iters", type=int, default=2)
    a = p.parse_args()
    build.build()
    wl = inputs.workloads()[a.workload]
    B = a.batch or wl.B
    prec = sg.SG_BF16 if a.precision == "bf16" else sg.SG_FP32
    model = sg.Model(wl.model, wl.weights(), prec)
    inst = sg.Instance(wl.instance())
    spins, logq = model.sample(B, seed=1)
    E = inst.energy(spins)
    out, coeff = sg.free_energy(E, logq, wl.betas[0], want_coeff=True)
    torch.cuda.synchronize()
    for i in range(a.iters):
        if a.call == "sample":
            model.sample(B, seed=2 + i, spins=spins, logq=logq)
        elif a.call == "logprob":
            model.logprob(spins, logq=logq)
        elif a.call == "grad":
            model.grad(spins, coeff)
        elif a.call == "energy":
            inst.energy(spins, E=E, precision=prec)
        elif a.call == "free_energy":
            sg.free_energy(E, logq, wl.betas[0], out=out, coeff=coeff, want_coeff=True)
        else:
            C = 1024 if B % 1024 == 0 else 1
            cs = spins[:C].clone()
            sg.mh_step(spins, E, logq, C, wl.betas[0], 3 + i, cs, E[:C].double(),
                       logq[:C].double())
    torch.cuda.synchronize()
    print(f"{a.call} x{a.iters} on {wl.name} B={B} {a.precision}: ok")


if __name__ == "__main__":
    main()
