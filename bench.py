#!/usr/bin/env python
"""Throughput of the FlashVAN hot path on one GB300 (or N independent replicas).

One step = one pass of the whole hot path over one batch of B configurations:
ancestral sampling (KV-cache decode) -> energies -> FP64 free energies and
REINFORCE weights -> teacher-forced log q + hand-written backward -> re-score of
the MH chain states -> independence-MH step -> Adam update of the weights.
value = configurations per second over the timed steps (all ranks).

  python bench.py [--steps K] [--warmup W] [--workload ea2d16] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "spin configs/sec sampled+scored, BF16 vs FP32 at fixed F/N error; ESS/sec"
UNIT = "configs/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="ea2d16")
    p.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the per-workload decodes and the fixed-F/N training check")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


def decode_bytes_per_sample(m, elem_bytes):
    """Algorithmic HBM bytes of the KV cache per sampled configuration: every
    visible key and value read at every step and layer, plus each key and value
    written once."""
    t = np.arange(m.N)
    if m.mask_kind == 0:
        vis = t + 1
    else:
        sink = np.minimum(m.S, t + 1)
        lo = np.maximum(m.S, t - m.W)
        vis = sink + np.maximum(0, t - lo + 1)
    per_key = 2 * m.d * elem_bytes * m.n_layers
    return float(vis.sum() * per_key + m.N * per_key)


DECODE_SOURCES = ("decode_bf16.cu", "tc.cuh", "sg_internal.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "decode_bf16_ea2d16_traffic.json")


def decode_source_hash():
    """First 16 hex digits of the sha256 of the BF16 decode's sources."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2606_22984_gb300", "csrc")
    h = hashlib.sha256()
    for f in DECODE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(precision_bf16):
    """DRAM bytes (read + write) of one full-size decode launch from the ncu
    capture recorded in profiles/, or None when the decode sources changed
    since that capture."""
    if not precision_bf16 or not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as fh:
        rec = json.load(fh)
    if rec.get("source_sha256") != decode_source_hash():
        return None
    return float(rec["traffic_bytes_per_launch"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed alone: the burst figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    return FALLBACK_BF16_TFLOPS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_info():
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model == "unknown":  # Arm hosts: lscpu names the core
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count() or 1, model


def oracle_step_time(wl, n, beta, seed):
    """The oracle's pass over n configurations: sample, energies, free
    energies, gradient (teacher-forced forward + backward), MH."""
    import oracle

    m = wl.model
    cfg = oracle.ModelCfg(**vars(m))
    inst = wl.instance()
    w = wl.weights()
    t0 = time.perf_counter()
    s, lq, _, _ = oracle.sample(cfg, w, n, seed)
    E = oracle.energy(inst, s)
    Fq, Fis, ess = oracle.free_energy(E, lq, beta)
    L = beta * E + lq
    oracle.grad(cfg, w, s, (L - L.mean()) / n)
    C = max(1, n // 4)
    oracle.mh(E[: (n // C) * C], lq[: (n // C) * C], C, beta, seed, E[:C], lq[:C])
    return time.perf_counter() - t0


def cpu_baseline(wl, beta, budget_s):
    import oracle

    cores, model = cpu_info()
    pilot_n = 4
    tp = oracle_step_time(wl, pilot_n, beta, 1)
    per = tp / pilot_n * max(1, min(cores, pilot_n))  # single-sample cost when parallel
    n = int(max(pilot_n, min(4096, budget_s / max(per / cores, 1e-6))))
    n = max(pilot_n, min(n, wl.B))
    t = oracle_step_time(wl, n, beta, 2)
    return {"value": n / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} of the {wl.B} configurations of one step (same model, instance and "
                      f"step: sample + energy + free energy + gradient + MH), FP64, "
                      f"{oracle.num_threads()} threads on {model}; {t:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2606_22984_gb300 import inputs

    wl = inputs.workloads()[args.workload]
    beta = wl.betas[len(wl.betas) // 2]
    cores, model = cpu_info()
    base = cpu_baseline(wl, beta, args.cpu_seconds / max(1, args.steps + args.warmup) * 4)
    n = int(base["sample"].split()[0])
    for i in range(args.warmup):
        oracle_step_time(wl, n, beta, 100 + i)
    ts = [oracle_step_time(wl, n, beta, 200 + i) for i in range(args.steps)]
    tot = sum(ts)
    val = n * args.steps / tot
    base["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "global_batch": n, "seq_len": wl.model.N,
                       "parallelism": "cpu"},
            "cpu_baseline": base,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def decode_by_workload(sg, inputs, peak, names=("sk1024", "ea3d10", "ea2d64")):
    """One full-size BF16 decode launch per workload (CUDA events on the
    launching stream), with its algorithmic KV bytes and HBM fraction.  The
    KV workspace is reserved first, so the launch is timed alone."""
    import torch

    out = {}
    stream = torch.cuda.current_stream()
    for name in names:
        wl = inputs.workloads()[name]
        m = wl.model
        grouped = name == "ea2d64"
        nm = len(wl.betas) if grouped else 1
        B = wl.B * nm
        model = sg.Model(m, wl.group_weights() if grouped else wl.weights(), sg.SG_BF16,
                         n_models=nm)
        spins = torch.empty((B, m.N), dtype=torch.int8, device="cuda")
        logq = torch.empty(B, dtype=torch.float32, device="cuda")
        model.reserve(B)
        model.sample(nm * 8, seed=1, spins=spins[: nm * 8], logq=logq[: nm * 8], stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        model.sample(B, seed=2, spins=spins, logq=logq, stream=stream)
        e1.record(stream)
        model.check(stream)
        ms = e0.elapsed_time(e1)
        alg = decode_bytes_per_sample(m, 2) * B
        out[name] = {"workload": wl.name, "B": B, "ms": ms, "configs_per_s": B / (ms / 1e3),
                     "algorithmic_bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                     "frac": alg / (ms / 1e3) / 1e9 / peak}
        model.close()
        del spins, logq
        torch.cuda.empty_cache()
    return out


def decode_patched_3d(sg, inputs, peak):
    """The 3D EA L=10 model with (2, 2, 2) patch cells: 125 tokens of 8 spins,
    a 256-class head, band and sink over the token lattice of side 5 (W=25,
    S=26), 6L d128 h8, B=32768, BF16: one full-size decode launch (CUDA events)
    next to the unpatched one of decode_by_workload."""
    import dataclasses

    import torch

    W, S = inputs.lattice_mask(3, 5)
    m = inputs.ModelShape(1000, 6, 128, 8, d_token=16, mask_kind=1, W=W, S=S, patch=8, lat_D=3,
                          lat_L=10)
    B = 32768
    stream = torch.cuda.current_stream()
    model = sg.Model(m, inputs.make_weights(m, 4), sg.SG_BF16)
    spins = torch.empty((B, m.N), dtype=torch.int8, device="cuda")
    logq = torch.empty(B, dtype=torch.float32, device="cuda")
    model.reserve(B)
    model.sample(8, seed=1, spins=spins[:8], logq=logq[:8], stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    model.sample(B, seed=2, spins=spins, logq=logq, stream=stream)
    e1.record(stream)
    model.check(stream)
    ms = e0.elapsed_time(e1)
    alg = decode_bytes_per_sample(dataclasses.replace(m, N=m.N // m.patch, patch=1), 2) * B
    out = {"workload": "3D EA L=10, (2,2,2) cells: 125 tokens, 256 classes, 6L d128 h8, "
                       "W=25 S=26 tokens", "B": B, "ms": ms, "configs_per_s": B / (ms / 1e3),
           "algorithmic_bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
           "frac": alg / (ms / 1e3) / 1e9 / peak}
    model.close()
    del spins, logq
    torch.cuda.empty_cache()
    return out


def sk_energy_tensor(sg, inputs, iters=20):
    """The dense s.J.s energy of the SK N=1024 workload (B = 8192, BF16 hi/lo
    split of J on tcgen05) through the public sg_energy call, each call the
    spin conversion and the tensor-core product.  Timed twice with CUDA events
    around `iters` calls: queued behind a spin kernel, so that the events see
    the calls' device time only, and back to back from the host, where the
    Python and launch overhead of a 30 us call paces the stream.  The product
    runs 4 B N^2 flops on the tensor cores (J_hi and J_lo); the energy itself
    needs 2 B N^2."""
    import torch

    wl = inputs.workloads()["sk1024"]
    N, B = wl.model.N, wl.B
    gi = sg.Instance(wl.instance())
    gen = torch.Generator(device="cpu").manual_seed(7)
    spins = (2 * torch.randint(0, 2, (B, N), generator=gen, dtype=torch.int8) - 1).cuda()
    E = torch.empty(B, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        gi.energy(spins, E=E, precision=sg.SG_BF16, stream=stream)
    torch.cuda.synchronize()

    def timed(queued):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if queued:
            torch.cuda._sleep(5_000_000)  # ~2.5 ms: the host enqueues every call meanwhile
        e0.record(stream)
        for _ in range(iters):
            gi.energy(spins, E=E, precision=sg.SG_BF16, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / iters

    us_dev, us_host = timed(True), timed(False)
    peak, kind = measured_bf16_peak()
    mma = 4.0 * B * N * N
    tf = mma / (us_dev / 1e6) / 1e12
    return {"workload": wl.name, "B": B, "N": N, "us_per_call": us_dev,
            "configs_per_s": B / (us_dev / 1e6), "mma_flops": mma, "achieved_tflops": tf,
            "peak_tflops": peak, "peak_kind": kind, "frac": tf / peak, "frac_one_product": 0.5 * tf / peak,
            "us_per_call_host_paced": us_host,
            "frac_host_paced": mma / (us_host / 1e6) / 1e12 / peak,
            "timed": "sg_energy calls (spin conversion + tensor-core product), CUDA events; "
                     "us_per_call with the calls queued behind a spin kernel (device time), "
                     "us_per_call_host_paced back to back from Python"}

def fixed_fn_check(sg, inputs, train):
    """BF16 and FP32 models of SK N=20 (beta = 1) trained by the REINFORCE loop
    (Eq. loss1, Adam), then F_IS/N of 65536 fresh samples against the exact
    F/N.  The exact F comes from every one of the 2^20 configurations scored
    by sg_energy and reduced by sg_free_energy with log q = 0, which gives
    F_IS = -ln Z / beta + ln(2^N) / beta."""
    import torch

    wl = inputs.workloads()["sk20"]
    N, beta = wl.model.N, 1.0
    gi = sg.Instance(wl.instance())
    idx = torch.arange(1 << N, device="cuda", dtype=torch.int64)
    bits = (idx[:, None] >> torch.arange(N, device="cuda")) & 1
    allspins = (2 * bits - 1).to(torch.int8).contiguous()
    E = gi.energy(allspins)
    zero = torch.zeros(1 << N, dtype=torch.float32, device="cuda")
    F_all = sg.free_energy(E, zero, beta).cpu().numpy()
    F_exact = F_all[1] - N * np.log(2.0) / beta
    out = {"workload": "SK N=20, beta=1.0 (J ~ N(0, 1/N), seed 1)",
           "F_exact_per_spin": F_exact / N, "bound": 1e-3}
    for prec, shape in ((sg.SG_FP32, wl.model), (sg.SG_BF16, inputs.ModelShape(20, 2, 64, 4))):
        model = sg.Model(shape, inputs.make_weights(shape, 1), prec)
        t0 = time.perf_counter()
        train.Trainer(model, gi, train.TrainConfig(B=4096, steps=400, lr=2e-3, beta=beta,
                                                   seed=100, log_every=1000)).run()
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        spins, logq = model.sample(65536, seed=999)
        F = sg.free_energy(gi.energy(spins), logq, beta).cpu().numpy()
        key = "bf16" if prec == sg.SG_BF16 else "fp32"
        out[key] = {"model": f"2L d{shape.d} h{shape.n_heads}", "train_steps": 400,
                    "train_batch": 4096, "train_s": t_train, "F_IS_per_spin": F[1] / N,
                    "F_q_per_spin": F[0] / N, "abs_err_per_spin": abs(F[1] - F_exact) / N,
                    "within_bound": bool(abs(F[1] - F_exact) / N <= 1e-3)}
        model.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2606_22984_gb300 import build as _build
    from paper_2606_22984_gb300 import inputs, replicas, sg, train

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    wl = inputs.workloads()[args.workload]
    m, B = wl.model, wl.B
    beta = wl.betas[len(wl.betas) // 2]
    # BF16 (tensor cores) is the headline; "auto" also times the FP32 plain path
    prec = {"auto": sg.SG_BF16, "fp32": sg.SG_FP32, "bf16": sg.SG_BF16}[args.precision]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def setup(precision):
        model = sg.Model(m, wl.weights(), precision)
        inst = sg.Instance(wl.instance())
        bufs = dict(
            spins=torch.empty((B, m.N), dtype=torch.int8, device=dev),
            logq=torch.empty(B, dtype=torch.float32, device=dev),
            E=torch.empty(B, dtype=torch.float32, device=dev),
            Ei=torch.empty(B, dtype=torch.int32, device=dev) if wl.instance().pm else None,
            F=torch.empty(3, dtype=torch.float64, device=dev),
            coeff=torch.empty(B, dtype=torch.float32, device=dev),
            grad=torch.empty(model.n_params, dtype=torch.float32, device=dev),
            tf=torch.empty(B, dtype=torch.float32, device=dev),
            m=torch.zeros(model.n_params, dtype=torch.float32, device=dev),
            v=torch.zeros(model.n_params, dtype=torch.float32, device=dev))
        C = 1024 if B % 1024 == 0 else 1
        bufs["C"] = C
        # MH chains start from the all-up configuration
        bufs["cs"] = torch.ones((C, m.N), dtype=torch.int8, device=dev)
        bufs["cE"] = inst.energy(bufs["cs"]).double()
        bufs["clq"] = torch.zeros(C, dtype=torch.float64, device=dev)
        bufs["clq32"] = torch.empty(C, dtype=torch.float32, device=dev)
        bufs["acc"] = torch.empty(C, dtype=torch.int64, device=dev)
        return model, inst, bufs

    ev = []

    def step(model, inst, bufs, i, timed):
        seed = replicas.replica_seed(rank, i)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        model.sample(B, seed, spins=bufs["spins"], logq=bufs["logq"], stream=stream)
        e1.record(stream)
        if timed:
            ev.append((e0, e1))
        inst.energy(bufs["spins"], E=bufs["E"], E_int=bufs["Ei"], want_int=bufs["Ei"] is not None,
                    stream=stream)
        sg.free_energy(bufs["E"], bufs["logq"], beta, out=bufs["F"], coeff=bufs["coeff"],
                       want_coeff=True, stream=stream)
        model.grad(bufs["spins"], bufs["coeff"], grad=bufs["grad"], logq=bufs["tf"], stream=stream)
        C = bufs["C"]
        model.logprob(bufs["cs"], logq=bufs["clq32"], stream=stream)
        bufs["clq"].copy_(bufs["clq32"])
        sg.mh_step(bufs["spins"], bufs["E"], bufs["logq"], C, beta, seed, bufs["cs"], bufs["cE"],
                   bufs["clq"], accepts=bufs["acc"], stream=stream)
        sg.adam_step(model.weights(), bufs["grad"], bufs["m"], bufs["v"], 1e-3, i + 1,
                     stream=stream)
        model.refresh(stream)

    def timed_run(precision, with_clocks):
        model, inst, bufs = setup(precision)
        for i in range(args.warmup):
            step(model, inst, bufs, i, False)
        torch.cuda.synchronize()
        ev.clear()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        n0 = sg.launch_count()
        sampler = ClockSampler(local)
        with sampler:
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for i in range(args.steps):
                step(model, inst, bufs, args.warmup + i, True)
            t1.record(stream)
            torch.cuda.synchronize()
        launches = sg.launch_count() - n0
        ms = replicas.max_over_ranks(t0.elapsed_time(t1), dist, dev)
        if world > 1:
            dist.barrier()
        dec_ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        return model, inst, bufs, ms, dec_ms, launches, sampler.summary()

    model, inst, bufs, ms, dec_ms, launches, clocks = timed_run(prec, True)
    ms_step = ms / args.steps
    value = replicas.whole_job_throughput(B, world, args.steps, ms / 1e3)

    # end to end through the public API with host buffers: a sampling step
    # draws its own inputs on the device from the seed (no input data crosses
    # to the device), and each step reads the sampled configurations, their
    # log q, energies and the free energies back into pinned host memory.
    h_spins = torch.empty((B, m.N), dtype=torch.int8).pin_memory()
    h_lq = torch.empty(B, dtype=torch.float32).pin_memory()
    h_E = torch.empty(B, dtype=torch.float32).pin_memory()
    h_F = torch.empty(3, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(model, inst, bufs, 5000 + i, False)
        h_spins.copy_(bufs["spins"], non_blocking=True)
        h_lq.copy_(bufs["logq"], non_blocking=True)
        h_E.copy_(bufs["E"], non_blocking=True)
        h_F.copy_(bufs["F"], non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": replicas.whole_job_throughput(B, world, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": int(B * m.N + 8 * B + 24)}

    elem = 2 if prec == sg.SG_BF16 else 4
    alg = decode_bytes_per_sample(m, elem) * B
    peak, peak_kind = measured_peaks()
    achieved = alg / (dec_ms / 1e3) / 1e9
    traffic = captured_traffic(prec == sg.SG_BF16) if args.workload == "ea2d16" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "decode",
                "peak_kind": peak_kind, "algorithmic_bytes": alg,
                "decode_ms": dec_ms, "decode_share_of_step": dec_ms / ms_step}
    F = bufs["F"].cpu().numpy()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == sg.SG_FP32 else "bf16", "data": "synthetic",
            "config": {"workload": wl.name, "global_batch": B * world, "seq_len": m.N,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "beta": beta, "l2": "KV cache working set > L2 (129 MB) every step"},
            "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "free_energy_last_step": {"F_q_per_spin": F[0] / m.N, "F_IS_per_spin": F[1] / m.N,
                                      "kish_ess": F[2]}}
    # free the headline run's model and workspaces before the other runs
    model.close()
    del model, inst, bufs
    torch.cuda.empty_cache()
    if args.precision == "auto":
        # the FP32 plain path on the same workload and step, for the BF16/FP32 ratio
        model32, _, bufs32, ms32, dec32, _, _ = timed_run(sg.SG_FP32, False)
        F32 = bufs32["F"].cpu().numpy()
        model32.close()
        del model32, bufs32
        torch.cuda.empty_cache()
        alg32 = decode_bytes_per_sample(m, 4) * B
        line["fp32_plain"] = {
            "value": replicas.whole_job_throughput(B, world, args.steps, ms32 / 1e3), "unit": UNIT,
            "ms_per_step": ms32 / args.steps, "decode_ms": dec32,
            "decode_roofline_frac": alg32 / (dec32 / 1e3) / 1e9 / peak,
            "F_IS_per_spin_last_step": F32[1] / m.N}
        line["bf16_over_fp32"] = value / line["fp32_plain"]["value"]
    if rank == 0 and not args.no_extras:
        # the other full-size workloads' decodes, and the accuracy the metric
        # is quoted at (BF16 and FP32 both within 1e-3 of the exact F/N)
        line["decode_by_workload"] = decode_by_workload(sg, inputs, peak)
        line["decode_by_workload"]["ea3d10_patched"] = decode_patched_3d(sg, inputs, peak)
        line["sk_energy_tensor"] = sk_energy_tensor(sg, inputs)
        line["fixed_FN_check"] = fixed_fn_check(sg, inputs, train)
        # an independence sampler's ESS/sec is at most its proposal rate, which
        # the decode's HBM roofline bounds; the measured ESS/sec of both chains
        # come from a separate run that trains the proposal first
        d3 = line["decode_by_workload"]["ea3d10"]
        line["ess_per_sec"] = {
            "workload": "3D EA L=10 +-J, beta=0.9",
            "neural_mh_upper_bound": d3["B"] / (d3["algorithmic_bytes"] / (peak * 1e9)),
            "proposal_rate_measured": d3["configs_per_s"],
            "source": "paper_2606_22984_gb300/ess_compare.py (trains the proposal, then "
                      "times neural MH and single-spin-flip Metropolis on the same instance); "
                      "summary in profiles/ess_mh_vs_metropolis.md"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, beta, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
