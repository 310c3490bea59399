"""msMINRES-CIQ on one B300: K^{1/2} B and K^{-1/2} B for Gaussian-process
kernel matrices K = K_XX + sigma^2 I (Pleiss et al., NeurIPS 2020).

The compute path is the CUDA library ``libciq.so`` (sources in ``csrc/``,
C ABI in ``include/ciq.h``); this package only marshals arguments to it.
"""
from ._ciq import (CiqError, Kernel, ciq_invsqrt, ciq_invsqrt_batched, ciq_invsqrt_f64,  # noqa: F401
                   ciq_kernel_matrix, ciq_kernel_mvm, ciq_kernel_mvm_f64, ciq_kernel_mvm_noalloc, ciq_lanczos_bounds, ciq_quad_nodes,
                   ciq_sqrt, ciq_sqrt_batched, ciq_sqrt_f64, ciq_stored_mvm, ciq_workspace_bytes, lib, LIB_PATH,
                   ciq_sqrt_dense, ciq_invsqrt_dense, ciq_sqrt_vjp, ciq_invsqrt_vjp,
                   ciq_sqrt_batched_learned, ciq_invsqrt_batched_learned, ciq_mlp_features, ciq_mlp_normaliser,
                   ciq_mlp_init, ciq_mlp_loss_grad, ciq_mlp_train, ciq_mlp_predict, CIQ_MLP_PARAMS,
                   ciq_sqrt_precond, ciq_invsqrt_precond, ciq_pivoted_cholesky, ciq_precond_workspace_bytes,
                   ciq_posterior_sample)
