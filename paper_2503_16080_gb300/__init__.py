"""GB300-native exact modular matrix products for CKKS linear algebra.

Python binding of the C-ABI library ``libmodpp.so`` (declared in
``include/modpp.h``).  Every step of the hot path runs in the library's CUDA
kernels; this package only marshals arguments (device pointers, sizes, the
current CUDA stream) and allocates the caller-side workspace through PyTorch.

The binding is loaded on first use of an API name, so ``synth`` (the seeded
input generators) can be imported on machines without the compiled library.
If the library is missing, every API call raises: there is no fallback.
"""
from __future__ import annotations

_API_NAMES = (
    "modpp_mm", "pc_mm", "pc_mv", "plan_info", "workspace_bytes", "last_status", "Path",
    "ModppError", "lib", "library_path", "profile_enable", "profile_read", "KERNEL_GEMM",
    "KERNEL_SPLIT", "KERNEL_U16", "set_digit_bits", "get_digit_bits", "GroupedPlan",
    "modpp_mm_grouped", "modpp_mm_wide", "set_wide_path", "get_wide_path", "wide_plan_info",
    "selftest_bounded_wait", "set_debug_checks", "get_debug_checks", "modpp_mm_trunc",
    "set_gemm_pair", "get_gemm_pair", "PreparedU",
)
_RING_NAMES = ("Ring",)


def __getattr__(name):
    if name in _API_NAMES:
        from . import api
        return getattr(api, name)
    if name in _RING_NAMES:
        from . import ring
        return getattr(ring, name)
    raise AttributeError(name)
