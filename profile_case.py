"""Run one call of the hot path on a synthetic workload, for profilers (ncu).

  python profile_case.py --call sample --workload ea2d16 --batch 4096 \
      --precision fp32 --iters 2

Only the named call runs (after its inputs are prepared), so a capture holds
just that call's memory: the model, the inputs and the call's own workspace.
``--lattice D L`` keeps the workload's model widths but puts it on a D-dim
periodic +-J lattice of side L (band W = L^(D-1), sink W + 1): a smaller case
of the same kernels for captures that replay a launch many times.
``--models n`` samples a group of n models (one launch, B samples in all).
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2606_22984_gb300 import build, inputs, sg  # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--call", default="sample",
                   choices=["sample", "logprob", "grad", "energy", "free_energy", "mh"])
    p.add_argument("--workload", default="ea2d16")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    p.add_argument("--iters", type=int, default=2)
    p.add_argument("--lattice", type=int, nargs=2, metavar=("D", "L"), default=None)
    p.add_argument("--models", type=int, default=1)
    a = p.parse_args()
    build.build()
    wl = inputs.workloads()[a.workload]
    shape, inst_src = wl.model, wl.instance()
    if a.lattice:
        D, L = a.lattice
        W, S = inputs.lattice_mask(D, L)
        shape = inputs.ModelShape(L ** D, shape.n_layers, shape.d, shape.n_heads, d_token=shape.d_token,
                                  d_ff=shape.d_ff, mask_kind=1, W=W, S=S)
        inst_src = inputs.make_ea(D, L, wl.seed, pm=True)
    B = a.batch or wl.B
    prec = sg.SG_BF16 if a.precision == "bf16" else sg.SG_FP32
    weights = (inputs.make_group_weights(shape, wl.seed, a.models) if a.models > 1
               else inputs.make_weights(shape, wl.seed))
    model = sg.Model(shape, weights, prec, n_models=a.models)
    inst = sg.Instance(inst_src)
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
    where = f"{a.lattice[0]}D L={a.lattice[1]} lattice, {wl.name} widths" if a.lattice else wl.name
    print(f"{a.call} x{a.iters} on {where} B={B} {a.precision}: ok")


if __name__ == "__main__":
    main()
