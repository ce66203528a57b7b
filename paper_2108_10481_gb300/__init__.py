"""GB300 (sm_103a) boundary-element Poisson-Boltzmann solver.

The compute path is libpbbem.so (hand-written CUDA behind the C ABI of
include/pbbem.h); this package only loads it and marshals torch tensors.
"""
from . import spectrum
from .api import (CASES, FORMS, PB_F32, PB_F32_ACCURATE, PB_F64, PB_LAPLACE, PB_MIXED, PB_OP_D, PB_OP_K,
                  PB_OP_M, PB_OP_T, PB_OP_V, PB_YUKAWA, PRECONDS, Params, PBError, pb_energy, pb_init,
                  pb_mesh_load, pb_near_build, pb_op_apply, pb_rhs_charges, pb_solvation_energy, pb_solve, pb_solve_pc, pb_precond_apply, pb_solve_many,
                  pb_system_apply, pb_system_apply_noalloc, pb_version, solve_opts, pb_profile, pb_profile_read, pb_launch_count,
                  PB_KERNEL_PAIR32, PB_KERNEL_PAIR32_ACCURATE, PB_KERNEL_PAIR64, PB_KERNEL_NEAR_ADJ,
                  PB_KERNEL_NEAR_COIN, PB_KERNEL_NEAR_BAND, pb_server_create, pb_submit,
                  pb_server_step, pb_poll, pb_autotune, pb_autotune_plan, pb_selftest_wait, pb_selftest_exp,
                  pb_set_graphs, pb_set_treecode, pb_tree_info, PB_KERNEL_TREE32)
from .api import PB_KERNEL_SPMV, PB_KERNEL_CHEB, PB_KERNEL_KRYLOV, pb_measure_peak
from .api import PB_OK, PB_EINVAL, PB_EMESH, PB_ENOMEM, PB_ENOCONV, PB_ENUMERIC, PB_ECUDA, PB_ETIMEOUT

__all__ = ["CASES", "FORMS", "PRECONDS", "Params", "PBError", "PB_F32", "PB_F32_ACCURATE", "PB_F64",
           "PB_LAPLACE", "PB_MIXED", "PB_OP_D", "PB_OP_K", "PB_OP_M", "PB_OP_T", "PB_OP_V", "PB_YUKAWA",
           "pb_energy", "pb_init", "pb_mesh_load", "pb_near_build", "pb_op_apply", "pb_rhs_charges",
           "pb_solvation_energy", "pb_solve", "pb_solve_pc", "pb_precond_apply", "pb_solve_many", "pb_system_apply", "pb_system_apply_noalloc", "pb_version", "solve_opts", "pb_profile",
           "pb_profile_read", "pb_launch_count", "PB_KERNEL_PAIR32", "PB_KERNEL_PAIR32_ACCURATE", "PB_KERNEL_PAIR64",
           "PB_KERNEL_NEAR_ADJ", "PB_KERNEL_NEAR_COIN", "PB_KERNEL_NEAR_BAND",
           "pb_server_create", "pb_submit", "pb_server_step", "pb_poll", "pb_autotune", "pb_autotune_plan",
           "pb_selftest_wait", "pb_selftest_exp", "pb_set_graphs", "pb_set_treecode", "pb_tree_info", "PB_KERNEL_TREE32",
           "pb_measure_peak", "PB_KERNEL_SPMV", "PB_KERNEL_CHEB", "PB_KERNEL_KRYLOV", "PB_OK", "PB_EINVAL", "PB_EMESH", "PB_ENOMEM", "PB_ENOCONV", "PB_ENUMERIC", "PB_ECUDA", "PB_ETIMEOUT"]
