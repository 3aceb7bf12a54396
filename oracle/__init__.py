"""Plain, slow FP64 CPU oracle for the DG exchange-build hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the C-ABI library and
its Python binding) may import, call or link anything in this package; only
the tests, the smoke check and the CPU-baseline leg of the benchmark use it.

The oracle shares no code with the CUDA path. It restates the discretisation
of Section 5 (auxiliary-grid Poisson problems) and Section 3.4 (SIPDG
Laplacian) of arXiv 2510.21213 directly and solves the resulting discrete
linear systems exactly (dense Cholesky or fast diagonalisation), so that the
multigrid-preconditioned CG of the GPU path can be checked against the exact
solution of the same discrete problem.
"""

from .dg_oracle import (  # noqa: F401
    Mesh,
    gauss_legendre,
    lagrange_eval,
    node_coords,
    quad_weights,
    penalty,
    sipdg_1d,
    assemble_kron,
    assemble_dense,
    boundary_face_nodes,
    boundary_data_direct,
    boundary_data_gausssum,
    gauss_sum_1_over_r,
    rhs,
    solve_dense,
    solve_fdm,
    solve,
    pair_list,
    poisson,
    exchange_build,
    exchange_partial,
    ace_apply,
    jk_apply,
    transfer_matrix,
)
