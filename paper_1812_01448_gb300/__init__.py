"""Leap-frog Maxwell solver on unstructured triangle meshes, native to GB300 (sm_103a).

The method is the Yee-like scheme of Fadeev's "Numerical simulation of 2D electrodynamic
problems with unstructured triangular meshes": E on edges (eq. 3), B at circumcentres (eq. 4),
plasma current on edges (eqs. 5-6), leap-frog in time (eqs. 14-15), dt from the spectral
radius of M (eq. 20).  The work is done by ``libue.so`` (C ABI in include/ue.h, CUDA kernels in
csrc/); this package is its binding.  Importing it does not load the library; the first call
does, and fails loudly if the library was not built.
"""
from ._native import (UE_DT_GIVEN, UE_DT_LEARNED, UE_DT_POWER, UE_PREC_FP32,  # noqa: F401
                      UE_PREC_FP64, UE_RHO_LEARNED, UE_RHO_POWER, UE_RHO_POWER_FALLBACK,
                      UE_REORDER_GREEDY, UE_REORDER_GREEDY_RINGS, UE_REORDER_KD, UE_REORDER_NONE,
                      UE_REORDER_RCM, UE_VARIANT_BLOCKED,
                      UE_TB_FUSED, UE_TB_SPLIT, UE_VARIANT_PERSISTENT, UE_VARIANT_PLAIN, UEError)
from .api import (Mesh, adam, batch_create, mesh_flip, mesh_relax, mlp_backward, mlp_forward, options,  # noqa: F401
                  power_iteration_static, rho_loss, seg_argmax, triangulate)
