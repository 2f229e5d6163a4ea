"""The no-allocation entry point against the regular one.

obfft_exec_fp64_noalloc serves callers that may not allocate device memory
while they run (cudaMalloc forbidden or too disruptive there, or every byte of
device memory owned by the application's own pool): it keeps its scratch in
device memory reserved when the library loads.  This file is collected last so
that a run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from synth import inputs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2606_23698_gb300 import build as B
    B.build()
    from paper_2606_23698_gb300 import _lib
    return _lib


def _regular(_lib, x, shape, dir):
    plan = _lib.obfft_plan_create(*shape, 1, _lib.OBFFT_MODE_FP64_NATIVE)
    try:
        y = torch.empty_like(x)
        _lib.obfft_exec(plan, x.data_ptr(), y.data_ptr(), dir, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    finally:
        _lib.obfft_destroy(plan)


def _noalloc(_lib, x, y, shape, dir):
    _lib.obfft_exec_fp64_noalloc(x.data_ptr(), y.data_ptr(), *shape, dir,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def test_noalloc_matches_regular_entry_on_two_calls(lib):
    # first call on this device: looks up the reserved arrays (and, with lazy
    # module loading, makes the driver load them); later calls allocate nothing
    warm_in = torch.zeros(8, dtype=torch.complex128, device="cuda")
    warm_out = torch.empty_like(warm_in)
    _noalloc(lib, warm_in, warm_out, (2, 2, 2), -1)
    cases = [((32, 48, 64), -1, S.complex_uniform(11, (32, 48, 64))),
             ((16, 128, 96), +1, S.complex_gaussian(12, (16, 128, 96))),
             # a length-1 first axis: the pass is a device-to-device copy
             ((16, 24, 1), -1, S.complex_uniform(13, (16, 24, 1))),
             ((1, 1, 1), +1, S.complex_uniform(14, (1, 1, 1)))]
    for shape, dir, xh in cases:
        x = xh.to("cuda").contiguous()
        want = _regular(lib, x, shape, dir)
        y = torch.empty_like(x)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        _noalloc(lib, x, y, shape, dir)
        free_after = torch.cuda.mem_get_info()[0]
        got = y.cpu().numpy()
        # same kernels and twiddles as the FP64-native plans: identical bits
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), shape
        assert free_after == free_before, "the no-alloc entry point changed free device memory"


def test_noalloc_rejects_oversize_grid(lib):
    from paper_2606_23698_gb300 import ObfftError
    x = torch.zeros(1, dtype=torch.complex128, device="cuda")
    y = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(ObfftError) as ei:
        lib.obfft_exec_fp64_noalloc(x.data_ptr(), y.data_ptr(), 256, 256, 64, -1, 0)
    assert "exceeds the fixed scratch" in str(ei.value)
