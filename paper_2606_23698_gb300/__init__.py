"""GB300-native Ozaki-Bailey FFT (full-FP64 complex 3-D FFT on FP8/INT8 tensor cores).

The transform runs in libobfft.so (CUDA, sm_103a) behind the C ABI of
include/obfft.h.  This package is its thin Python binding: the same entry
points by name (paper_2606_23698_gb300._lib), a torch-tensor convenience
layer (Plan, fft3), and the autograd Function.  torch only provides device
memory and streams.
"""
from ._lib import (OBFFT_MODE_FP8, OBFFT_MODE_INT8, OBFFT_MODE_FP64_NATIVE, MODES,  # noqa: F401
                   ObfftError, obfft_plan_create, obfft_plan_create_many, obfft_exec,
                   obfft_exec_many, obfft_exec_stage, obfft_destroy, obfft_plan_get_splits,
                   obfft_last_error, obfft_version)
from .api import Plan, PlanMany, fft3, ifft3  # noqa: F401
from .autograd import ObFFT3, fft3_autograd  # noqa: F401
from .slab import SlabPlan, slab_geometry  # noqa: F401
