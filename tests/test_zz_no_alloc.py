"""The allocation-free coarse matcher, sv_coarse_match_static.

It exists for callers that cannot allocate device memory when they need a coarse map:
real-time loops that must not wait on the allocator, plugins whose host owns all device
memory.  Its work tables live in a
fixed array inside the library instead of memory a context allocates.

Checked here through the C ABI: two calls in a row (different batches, so the shared
array must be rewritten by the second) give the same disparities as sv_coarse_match and
scores within the coarse tests' 1e-5; oversize calls are refused without launching.
This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2305_11566_gb300 import binding, synth

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5


def _static_call(lib, dps, window, scores=True):
    n = len(dps)
    disp = [torch.full(p.coarse_hw, -1, dtype=torch.int16, device="cuda") for p in dps]
    best = [torch.empty(p.coarse_hw, dtype=torch.float32, device="cuda") for p in dps]
    second = [torch.empty(p.coarse_hw, dtype=torch.float32, device="cuda") for p in dps]
    arr = (binding.SvPair * n)(*[p.sv() for p in dps])
    s = lib.sv_coarse_match_static(arr, n, window, binding._ptrs(disp), binding._ptrs(best), binding._ptrs(second),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s, disp, best, second


@pytest.mark.parametrize("window", [9])
def test_static_matches_context_entry_point_twice(svlib, window):
    ctx = binding.Context(synth.NET_SMALL, window, "fp32")
    try:
        batches = [
            [(synth.make_pair(1242, 375, 190.0, 8100), 48), (synth.make_pair(640, 193, 96.0, 8101), 25)],
            [(synth.make_pair(320, 97, 48.0, 8102), 13), (synth.make_pair(960, 290, 144.0, 8103), 37),
             (synth.make_pair(1242, 375, 190.0, 8104), 48)],
        ]
        for batch in batches:  # two calls in a row on the shared array
            dps = [binding.to_device(p, D) for p, D in batch]
            s, disp, best, second = _static_call(svlib, dps, window)
            assert s == binding.SV_OK
            ref_d, ref_b, ref_s = ctx.coarse_match(dps, scores=True)
            torch.cuda.synchronize()
            for a, b in zip(disp, ref_d):
                assert torch.equal(a, b)
            for a, b in zip(best, ref_b):
                assert (a - b).abs().max().item() <= RHO_TOL
            for a, b in zip(second, ref_s):
                assert (a - b).abs().max().item() <= RHO_TOL
    finally:
        ctx.close()


def test_static_rejects_oversize_calls(svlib):
    p = synth.make_pair(128, 64, 20.0, 8200)
    dp = binding.to_device(p, 8)
    too_many = [dp] * 257
    s, disp, _, _ = _static_call(svlib, too_many, 7)
    assert s == binding.SV_ERR_UNSUPPORTED
    # 16384 x 128 with D = 100: 4 row strips x 43 column groups = 172 jobs per pair
    big = synth.make_pair(16384, 128, 20.0, 8201)
    dpb = binding.to_device(big, 100)
    s, _, _, _ = _static_call(svlib, [dpb], 7)
    assert s == binding.SV_OK
    s, disp, _, _ = _static_call(svlib, [dpb] * 256, 7)  # 256 x 172 jobs > 32768
    assert s == binding.SV_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert bool((disp[0] == -1).all())
    # a side above the library's limit: the same status as sv_coarse_match
    wide = binding.SvPair.from_buffer_copy(dp.sv())
    wide.width = 16400
    wide.pitch = 16400
    arr = (binding.SvPair * 1)(wide)
    assert svlib.sv_coarse_match_static(arr, 1, 7, binding._ptrs([disp[0]]), None, None, None) == \
        binding.SV_ERR_UNSUPPORTED
    assert svlib.sv_coarse_match_static(None, 0, 7, None, None, None, None) == binding.SV_OK
    arr = (binding.SvPair * 1)(dp.sv())
    assert svlib.sv_coarse_match_static(arr, 1, 8, binding._ptrs([disp[0]]), None, None, None) == \
        binding.SV_ERR_INVALID_ARG
