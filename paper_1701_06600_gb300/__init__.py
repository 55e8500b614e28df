"""GB300 (sm_103a) CPRAND / CPRAND-MIX: randomized CP tensor decomposition (arXiv 1701.06600).

The compute path is libcprand.so (hand-written CUDA kernels behind the C ABI of
include/cprand.h); `binding` marshals torch tensors into it.  Importing this package does not load
the library; the first call does, and fails loudly if the library is not built.
"""
from . import binding  # noqa: F401
from .binding import (cpr_cprand, cpr_cprand_mix, cpr_cprand_batched, cpr_sample_indices,  # noqa: F401
                      cpr_gather_fibers, cpr_sampled_update, cpr_fit_estimate, cpr_mix_tensor,
                      cpr_unmix_factors, cpr_tensor_norm, cpr_default_opts, cpr_sample_size,
                      cpr_status_string, cpr_workspace_size)
