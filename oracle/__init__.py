"""FP64 CPU oracle for the per-step PISO update (TEST INFRASTRUCTURE ONLY).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA path.
"""
from .piso import (Mesh, Options, Matrix, assemble_C, assemble_P, matvec, matvec_T, grad_p,
                   grad_p_T, divergence, divergence_T, pressure_rhs_vec, correct, outflow_update,
                   piso_step, piso_step_adjoint, mesh_from_case, rollout, rhie_chow_residual,
                   to_sparse)
from . import stats
