"""GB300 (sm_103a) implementation of the hybrid-dimensional VAG Darcy solve and
explicit upwind transport (Xing, Masson, Lopez, arXiv 1602.03641).

The compute path is ``libvag.so`` (CUDA, built in-tree by ``build.build()``)
behind the C ABI of ``include/vag.h``; ``vag`` is its ctypes binding.
"""
from .vag import (  # noqa: F401
    Context, System, Server, VagError, assemble_problem, problem_arrays, general_arrays, lib, declared_symbols, launch_count,
    peaceman_wi, is_hex_problem, SHAPE_FACES, VAG_SHAPE_HEX, VAG_SHAPE_TET, VAG_SHAPE_PRISM, VAG_SHAPE_PYRAMID,
    VAG_OK, VAG_EINVAL, VAG_ENOMEM, VAG_EBUDGET, VAG_ENOTCONVERGED, VAG_EBREAKDOWN, VAG_ETIMEOUT,
    VAG_ECUDA, VAG_EMESH, VAG_MEM_HOST, VAG_MEM_DEVICE, VAG_FP64, VAG_MIXED, VAG_MIXED_F16, VAG_FP64_PC32,
    VAG_PC_JACOBI, VAG_PC_CHEBYSHEV, VAG_PC_AMG, VAG_PC_AMG_RS, VAG_KERNEL_SPMV, VAG_KERNEL_SMOOTH, VAG_KERNEL_TRANSPORT_STEP,
    VAG_KERNEL_SPMV32, VAG_KERNEL_CELL_LOCAL, VAG_KRYLOV_CG, VAG_KRYLOV_BICGSTAB, VAG_KRYLOV_GMRES,
)
