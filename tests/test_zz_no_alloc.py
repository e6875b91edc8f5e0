"""The allocation-free sampling entry point, sg_sample_noalloc.

Some callers cannot let a library allocate device memory: a host framework
that owns every device allocation through its own memory pool (memory the
pool did not hand out is memory it cannot budget), or a latency-sensitive
loop in which cudaMalloc / cudaFree would synchronise the device and stall
its other streams.  For them libsg offers one sampling entry point whose
scratch is a static device array instead of cudaMalloc'd memory.

This test calls it through the C ABI and checks its output against the
ordinary sg_sample on the same inputs (same kernel, so bit for bit) and
against the FP64 oracle, on two calls in a row, after a call of another
shape has left different contents in the shared scratch.  It is kept in the
last-collected file so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_22984_gb300 import build, inputs, sg

from helpers import oracle_replay

pytestmark = pytest.mark.gpu

LOGQ_TOL = 1e-4   # per spin, the FP32 tolerance of the other parity tests
BAND = 1e-5       # the FP32 flag band


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, m, wd, B, seed, stream):
    cfg = sg.config(m, sg.SG_FP32)
    nw = (m.N + 31) // 32
    s = torch.zeros((B, m.N), dtype=torch.int8, device="cuda")
    lq = torch.zeros(B, dtype=torch.float32, device="cuda")
    fl = torch.zeros((B, nw), dtype=torch.int32, device="cuda")
    rc = lib.sg_sample_noalloc(ctypes.byref(cfg), _p(wd), B, 1.0, seed, 0, 0.0, _p(s), _p(lq),
                               _p(fl), stream)
    assert rc == 0, lib.sg_last_error()
    return s, lq, fl


def test_noalloc_sampling_matches_sg_sample_and_oracle_on_two_calls():
    build.build()
    lib = sg.lib()
    assert torch.cuda.is_available()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # another shape first (wider model, larger batch): the scratch then holds
    # different packed weights and KV entries than the checked calls need
    m_other = inputs.ModelShape(50, 3, 128, 8, mask_kind=1, W=9, S=4)
    w_other = torch.tensor(inputs.make_weights(m_other, 3), device="cuda")
    _noalloc(lib, m_other, w_other, 700, 99, stream)
    torch.cuda.synchronize()

    m = inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7)
    B, seed = 300, 4321
    w = inputs.make_weights(m, 7)
    model = sg.Model(m, w, sg.SG_FP32)
    ref_s, ref_lq, ref_f = model.sample(B, seed=seed, with_flags=True)
    wd = torch.tensor(w, device="cuda")
    for _ in range(2):
        s, lq, fl = _noalloc(lib, m, wd, B, seed, stream)
        torch.cuda.synchronize()
        assert torch.equal(s, ref_s)
        assert torch.equal(lq, ref_lq)
        assert torch.equal(fl, ref_f)
    sn, lqn, fln = s.cpu().numpy(), lq.cpu().numpy(), fl.cpu().numpy()
    so, lqo, _, _ = oracle_replay(m, w, seed, sn, fln, BAND)
    assert np.array_equal(so, sn)
    assert np.abs(lqo - lqn).max() <= LOGQ_TOL * m.N


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    build.build()
    lib = sg.lib()
    m = inputs.ModelShape(256, 4, 64, 4, mask_kind=1, W=16, S=17)
    w = torch.tensor(inputs.make_weights(m, 1), device="cuda")
    cfg = sg.config(m, sg.SG_FP32)
    B = 16384  # needs ~1.1 GB of KV cache, far above the static limit
    s = torch.empty((B, m.N), dtype=torch.int8, device="cuda")
    lq = torch.empty(B, dtype=torch.float32, device="cuda")
    rc = lib.sg_sample_noalloc(ctypes.byref(cfg), _p(w), B, 1.0, 1, 0, 0.0, _p(s), _p(lq), None,
                               None)
    assert rc == 1
    assert b"static scratch" in lib.sg_last_error()
