"""GB300-native interpolation-supplemented lattice Boltzmann solver (ISLBM).

The compute path is the CUDA library libislbm.so (sm_103a); this package is
its Python binding.  See include/islbm.h for the C ABI.
"""
from .islbm import (EXPORTS, KERNEL_VARIANTS, KERNELS, LATTICES, MESH_KINDS, PRECISIONS, STENCILS,
                    Batch, IslbmError, Params, Solver, islbm_autotune, islbm_average_add,
                    islbm_average_get, islbm_average_reset, islbm_create, islbm_debug_bounds, islbm_default_params,
                    islbm_destroy, islbm_get_fields, islbm_get_fields_device,
                    islbm_get_populations, islbm_info, islbm_load, islbm_mass, islbm_mesh_erf,
                    islbm_mesh_tanh, islbm_mesh_uniform, islbm_nusselt, islbm_reduce,
                    islbm_reduce_noalloc, islbm_reynolds, islbm_run_to_steady, islbm_save, islbm_selftest_wait_timeout,
                    islbm_selftest_wait_abort,
                    islbm_set_fields, islbm_set_fields_device, islbm_set_populations,
                    islbm_steady_change, islbm_step, islbm_synchronize, library_path,
                    load_library, islbm_set_row_range, islbm_get_rows, islbm_set_rows,
                    islbm_reduce_sums, islbm_finish_sums, rows_bytes, REDUCTION_SUMS,
                    SUM_MAX_SLOT, islbm_set_allocator, torch_allocator)

__all__ = [n for n in dir() if not n.startswith("_")]
