"""phikron: phi_l(-tau*A)v for Kronecker-sum A on one GB300 GPU (arXiv 2211.00696).

The compute path is the CUDA library libphikron.so (include/phikron.h); this package is
its Python binding (``phikron``) and build script (``build``).
"""
from .phikron import (Plan, Batch, Integrator, PhikronError, lib, log_quaderr, quadnodes, setup_quadrature,  # noqa: F401
                      gauss_legendre, clenshaw_curtis, expm_batched, kron_apply_f64,
                      PREC_FP64, PREC_OZAKI_BF16, QUAD_GAUSS, QUAD_CC, QUAD_CC_ADAPTIVE,
                      ERK_EULER, ERK_RK2, ERK_RK3, NONLIN_NONE, NONLIN_ALLEN_CAHN)
