"""chebfd_filter_block_noalloc, the filter for callers that cannot allocate
device memory (its work vectors sit in a fixed array inside the library),
must give the same results as chebfd_filter_block.  Two calls in a row check
that the shared array's leftover contents (and its cleared counters) do not
leak into the next call.  Runs last so that a failure here leaves the rest of
the suite already run."""
import numpy as np
import pytest
import torch

import paper_1510_04895_gb300 as pkg
from oracle import coeffs
from paper_1510_04895_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("single", [False, True])
def test_noalloc_filter_matches_allocating_filter_twice(single):
    H = pkg.chebfd_matrix_create_lattice("topi", 6, 5, 7, t=1.0, m=1.0, W=1.0, seed=3,
                                         also_single=True)
    a, b = -4.8, 4.8
    alpha, beta = coeffs.scaling(a, b)
    gc = pkg.chebfd_window_coeffs(a, b, -0.2, 0.2, 90, "lanczos", 2.0)
    dt = torch.complex64 if single else torch.complex128
    for call, nb in enumerate((64, 80)):        # second call: two panels, other sizes
        X0 = torch.from_numpy(workloads.random_block(10 + call, H.n, nb, True)).to(DEV).to(dt)
        X_ref = X0.clone()
        X_new = X0.clone()
        m_ref = torch.zeros((180, nb), dtype=torch.float64, device=DEV)
        m_new = torch.full((180, nb), 7.0, dtype=torch.float64, device=DEV)
        pkg.chebfd_filter_block(H, alpha, beta, gc, X_ref, moments=m_ref)
        _lib.chebfd_filter_block_noalloc(H, alpha, beta, gc, X_new, moments=m_new)
        torch.cuda.synchronize()
        tol = 1e-11 if not single else 1e-5
        assert _rel(X_new.cpu().numpy(), X_ref.cpu().numpy()) <= tol
        mr = m_ref.cpu().numpy()
        assert np.abs(m_new.cpu().numpy() - mr).max() <= tol * np.abs(mr).max()
        # and without moments
        X_a = X0.clone()
        X_b = X0.clone()
        pkg.chebfd_filter_block(H, alpha, beta, gc, X_a)
        _lib.chebfd_filter_block_noalloc(H, alpha, beta, gc, X_b)
        torch.cuda.synchronize()
        assert _rel(X_b.cpu().numpy(), X_a.cpu().numpy()) <= tol


def test_noalloc_filter_rejects_oversized_requests():
    H = pkg.chebfd_matrix_create_lattice("topi", 64, 64, 8, W=1.0, seed=1, also_single=True)
    gc = pkg.chebfd_window_coeffs(-4.5, 4.5, -0.1, 0.1, 4, "lanczos", 2.0)
    # complex128 panels are 32 columns wide: 2 * N * 32 * 16 B = 128 MiB > 64 MiB
    X = torch.zeros((H.n, 64), dtype=torch.complex128, device=DEV)
    with pytest.raises(pkg.ChebFDError) as e:
        _lib.chebfd_filter_block_noalloc(H, 0.2, 0.0, gc, X)
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_filter_reports_diverging_recurrence_then_recovers():
    """[a, b] = [-1, 1] does not enclose the insulator's spectrum (|E| <= 4):
    T_n(A) grows without bound, the even moments exceed mu_0 and the call
    returns ENUMERIC (the check runs on the device, with a flag in the shared
    array).  A following call with a proper interval succeeds and matches the
    allocating filter: the flag was cleared."""
    H = pkg.chebfd_matrix_create_lattice("topi", 6, 5, 7, t=1.0, m=1.0, W=1.0, seed=3)
    gc = pkg.chebfd_window_coeffs(-1.0, 1.0, -0.2, 0.2, 40, "lanczos", 2.0)
    X = torch.from_numpy(workloads.random_block(21, H.n, 32, True)).to(DEV)
    m = torch.zeros((80, 32), dtype=torch.float64, device=DEV)
    with pytest.raises(pkg.ChebFDError) as e:
        _lib.chebfd_filter_block_noalloc(H, 1.0, 0.0, gc, X, moments=m)
    assert e.value.status == 4
    a, b = -4.8, 4.8
    alpha, beta = coeffs.scaling(a, b)
    gc = pkg.chebfd_window_coeffs(a, b, -0.2, 0.2, 40, "lanczos", 2.0)
    X0 = torch.from_numpy(workloads.random_block(22, H.n, 32, True)).to(DEV)
    X_ref, X_new = X0.clone(), X0.clone()
    m_ref = torch.zeros((80, 32), dtype=torch.float64, device=DEV)
    m_new = torch.zeros((80, 32), dtype=torch.float64, device=DEV)
    pkg.chebfd_filter_block(H, alpha, beta, gc, X_ref, moments=m_ref)
    _lib.chebfd_filter_block_noalloc(H, alpha, beta, gc, X_new, moments=m_new)
    torch.cuda.synchronize()
    assert _rel(X_new.cpu().numpy(), X_ref.cpu().numpy()) <= 1e-11
    mr = m_ref.cpu().numpy()
    assert np.abs(m_new.cpu().numpy() - mr).max() <= 1e-11 * np.abs(mr).max()
