"""GB300 (sm_103a) Chebyshev filter diagonalization: Python binding of libchebfd.so.

The compute path is the C-ABI library built from ``csrc/`` (see
``include/chebfd.h``); this package only marshals arguments.  Importing it
does not load the library; the first call does, and raises if it is missing.
"""
from ._lib import (  # noqa: F401
    C64, C128, R32, R64, ChebFDError, Matrix, chebfd_chebyshev_step, chebfd_convert_block,
    chebfd_filter_block, chebfd_filter_block_df, chebfd_kpm_moments, chebfd_matrix_create_csr,
    chebfd_matrix_create_lattice, chebfd_orthonormalize, chebfd_random_block,
    chebfd_rayleigh_ritz, chebfd_harmonic_ritz, chebfd_residuals, chebfd_scale_bounds,
    chebfd_solve, chebfd_spmv,
    chebfd_window_coeffs, lib, Ensemble, chebfd_ensemble_create, chebfd_ensemble_autotune,
    chebfd_filter_block_noalloc, chebfd_filter_block_host, MLP, chebfd_param_features,
    chebfd_choose_params, pack_params,
    unpack_params, chebfd_solve_batched, chebfd_gram, chebfd_block_update)
