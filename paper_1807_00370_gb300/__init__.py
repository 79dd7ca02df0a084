"""GB300-native (sm_103a) cyclic-reduction solver for Hermitian positive
definite block-tridiagonal systems (Neuenhofen, "Review of Cyclic Reduction
for Parallel Solution of Hermitian Positive Definite Block-Tridiagonal
Linear Systems").

The CUDA library libcrsolve.so (C ABI in include/crsolve.h) does all the
work; ``api`` is a thin ctypes binding with the same names.  Importing this
package does not load the library; the first call does, and fails loudly if
it cannot.
"""
from .api import (CRSolveFn, NotPositiveDefinite, Plan, crsolve_backward, crsolve_debug_level_system,
                  crsolve_factor, crsolve_info_get, crsolve_plan_create, crsolve_plan_levels,
                  crsolve_launch_count, crsolve_mixed_precondition, crsolve_mixed_stats, crsolve_peak_probe, crsolve_residual, crsolve_solve, crsolve_solve_host, crsolve_solve_noalloc, crsolve_tile_get, crsolve_tile_get_mixed, crsolve_tile_set, crsolve_tile_set_mixed,
                  crsolve_timing_enable, crsolve_timing_read, solve)
from .batched import (Batch, crsolve_batch_create, crsolve_batch_graph_launch, crsolve_batch_info,
                      crsolve_batch_solve)

__all__ = ["Batch", "crsolve_batch_create", "crsolve_batch_graph_launch", "crsolve_batch_info",
           "crsolve_batch_solve", "CRSolveFn", "NotPositiveDefinite", "Plan", "crsolve_backward", "crsolve_debug_level_system",
           "crsolve_factor", "crsolve_info_get", "crsolve_plan_create", "crsolve_plan_levels",
           "crsolve_launch_count", "crsolve_mixed_precondition", "crsolve_mixed_stats", "crsolve_peak_probe", "crsolve_residual", "crsolve_solve", "crsolve_solve_host", "crsolve_solve_noalloc", "crsolve_tile_get", "crsolve_tile_get_mixed", "crsolve_tile_set", "crsolve_tile_set_mixed",
           "crsolve_timing_enable",
           "crsolve_timing_read", "solve"]
