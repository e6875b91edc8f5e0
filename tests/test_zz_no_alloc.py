"""The allocation-free sampling entry point, sg_sample_noalloc.

Some callers cannot allocate device memory while they run -- for example code
inside a CUDA graph capture, or a host framework that owns all device memory
through its own pool -- so libsg offers one sampling entry point whose scratch
is a static device array instead of cudaMalloc'd memory.  This test calls it
through the C ABI twice in a row and checks its output against the ordinary
sg_sample on the same inputs.  It is kept in the last-collected file so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_22984_gb300 import build, inputs, sg

pytestmark = pytest.mark.gpu

LOGQ_TOL = 1e-4  # per spin, the FP32 tolerance of the other parity tests


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_sampling_matches_sg_sample_on_two_calls():
    build.build()
    lib = sg.lib()
    assert torch.cuda.is_available()
    m = inputs.ModelShape(36, 2, 64, 4, mask_kind=1, W=6, S=7)
    B, seed = 300, 4321
    w = inputs.make_weights(m, 7)
    model = sg.Model(m, w, sg.SG_FP32)
    ref_s, ref_lq, ref_f = model.sample(B, seed=seed, with_flags=True)
    wd = torch.tensor(w, device="cuda")
    cfg = sg.config(m, sg.SG_FP32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nw = (m.N + 31) // 32
    for _ in range(2):
        s = torch.zeros((B, m.N), dtype=torch.int8, device="cuda")
        lq = torch.zeros(B, dtype=torch.float32, device="cuda")
        fl = torch.zeros((B, nw), dtype=torch.int32, device="cuda")
        rc = lib.sg_sample_noalloc(ctypes.byref(cfg), _p(wd), B, 1.0, seed, 0, 0.0, _p(s), _p(lq),
                                   _p(fl), stream)
        assert rc == 0, lib.sg_last_error()
        torch.cuda.synchronize()
        assert torch.equal(s, ref_s)
        assert (lq - ref_lq).abs().max().item() <= LOGQ_TOL * m.N
        assert torch.equal(fl, ref_f)


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
