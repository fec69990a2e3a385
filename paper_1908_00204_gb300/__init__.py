"""GB300 (sm_103a) numeric sparse LU refactorization after GLU3.0.

The library itself is C++/CUDA (``csrc/``), exposed through the C ABI of
``include/glu.h``; ``glu`` is its thin Python binding.  Build it in place
with ``paper_1908_00204_gb300.build.build()``.
"""
from . import build  # noqa: F401
from .glu import (GluError, Handle, default_options, glu_analyze, glu_destroy, glu_factor, glu_factor_f32,  # noqa: F401,E501
                  glu_solve_refine, glu_factor_batched, glu_factor_batched_f32, glu_solve_batched,
                  glu_solve_batched_refine, glu_get_factors_batched, glu_get_factors_batched_f32, glu_get_factors_f32,
                  glu_get_deps, glu_get_factors, glu_get_fill, glu_get_levels, glu_get_stats,
                  glu_last_error_info, glu_order_nd, glu_set_stream, glu_solve, glu_solve_noalloc, glu_strerror, glu_sync, load_library,
                  glu_static_pivot, glu_apply_static_pivot, apply_static_pivot)
