"""Plain FP64 CPU oracle of the ChebFD filter path (Pieper et al., arXiv 1510.04895).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library
``libchebfd.so`` and its Python binding) imports, links or executes this package.
It may be used by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / reference legs of ``bench.py`` - nowhere else.

Every function follows the passage of the paper it cites, in the paper's order
and notation, written for readability rather than speed: numpy / scipy
primitives (a sparse matrix product, a dense Hermitian eigensolver, a DCT, a
sort) serve as single steps, with no blocking, fusion or reordering on top.

Modules
  rng           counter-based SplitMix64 words (published generator)
  lattice       topological-insulator / graphene / diagonal test matrices (CSR)
  sell          SELL-C-sigma storage built from CSR
  coeffs        alpha, beta, window coefficients c_n, kernel factors g_n (Sec. 2.1)
  filter        the filter recurrence of Fig. ChebFD and Chebyshev moments (Sec. 4)
  kpm           stochastic-trace KPM moments, DOS and target count (Sec. 3.1 step 1-2)
  bounds        Lanczos estimate of the spectral interval [a, b] (Sec. 3.1 step 1)
  svqb          rank-revealing SVQB orthonormalisation, plain FP64 Gram (Sec. 3.1 step 6)
  rr            Rayleigh-Ritz pairs and residual norms (Sec. 3.1 step 7)
  solve         the ChebFD outer iteration with ghost rejection (Sec. 3.1 steps 5-8)
  quality       damping factor sigma, quality eta, optimal N_p (Sec. 2.3, 2.4)
  mlp           FP64 reference of the parameter-predicting MLP (no paper counterpart)
"""
