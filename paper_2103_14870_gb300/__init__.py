"""GB300-native graph-based FEM fracture (remeshing-free, edge-length hyperelasticity).

The compute path is the CUDA library under ``csrc/`` behind the C ABI in
``include/graphfem.h``; ``graphfem`` is its Python binding.
"""
from .graphfem import (  # noqa: F401
    ASSEMBLY_COLOUR, ASSEMBLY_GATHER, Batch, DRIVER_STRAIN, DRIVER_STRESS, ENERGY_SNH, ENERGY_STVK, FP64, STEP_GRAPH, STEP_STREAM, GNN_FP32_FMA, GNN_PARAM_SHAPES, GNN_PRECOND, GNN_START, GNN_TENSOR_CORES, MASS_CONSISTENT, MASS_LUMPED, QS_SOLVE_FP64, QS_SOLVE_NESTED, MEM_DEVICE, MEM_HOST, MIXED, SOLVE_CG, SOLVE_DISTRIBUTED, SOLVE_KERNELS, SOLVE_NESTED, SOLVE_PERSISTENT, GraphFEMError, Gnn,
    Mesh, load_library,
    bsr_pcg_solve_static, material, mesh_create, mesh_plan,
)
