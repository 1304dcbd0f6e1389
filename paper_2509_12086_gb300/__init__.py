"""GB300-native SAQ encoder (arXiv 2509.12086).

The compute path is the C-ABI library libsaq.so (include/saq.h): CUDA kernels
for sm_103a.  This package is its Python binding; importing it does not load
the library, the first call does (and fails loudly if it is missing).
"""
from ._lib import (Model, SaqError, load, saq_encode, saq_estimate_dist, saq_fit,  # noqa: F401
                   saq_model_create, saq_model_import, saq_plan_search, saq_kernel_launch_count,
                   saq_kernel_timing, saq_kernel_times, saq_quantize_step_ceiling, PRECISIONS,
                   Ingest, saq_set_wait_limit)
