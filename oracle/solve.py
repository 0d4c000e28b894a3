"""The ChebFD iteration, Sec. 3.1 steps 4-8 - oracle side.

Readings of the paper taken here (the paper leaves them open):
* residual threshold: eps is relative, a pair converges when
  ||H v - theta v|| <= eps ||H||, ||H|| = max(|a|, |b|) (Sec. 3.1 step 8);
* ghost Ritz pairs (Sec. 3.1 step 7, 'discard ... if it remains larger than
  sqrt(eps)'): from the second iteration on, an in-window pair is a ghost when
  its residual exceeds sqrt(eps) ||H|| and did not fall by a factor >= 10
  against the residual of the previous iteration's pair nearest in theta;
* convergence (step 8a): at least one accepted in-window pair, and every
  accepted in-window pair below eps ||H||; the window is closed,
  lam_lo <= theta <= lam_hi.  Step 8a holds vacuously for a window without
  eigenvalues; such a window is taken as empty once two successive
  iterations (from the second on) have no in-window Ritz pair that is either
  accepted or still converging, a pair converging when its residual fell to
  at most 0.9 of the previous iteration's nearest pair's.  With a weak
  filter (damping worse than 10x per iteration) the true pairs are
  ghost-flagged but their residuals keep falling, so the iteration goes on
  (or ends unconverged at max_iter); the in-window Ritz values of a window
  without eigenvalues are mixtures of eigenvectors on both sides of it,
  whose residuals stagnate;
* restart (step 8b): the next search block is the full set of Ritz vectors,
  which spans the same space as the orthonormalised filtered block;
* window_inset=f filters with the window W = 1 on [c - (1-f) d, c + (1-f) d]
  inside the target interval [c - d, c + d] (Sec. 2.2 notes that windows with
  W != 1 on part of I_T can converge faster); the window test and the
  convergence test still use the target interval;
* extraction="harmonic" replaces step 7's Ritz pairs by harmonic Ritz pairs
  for the target tau = (lam_lo + lam_hi) / 2 (rr.harmonic_ritz): window
  membership, ghosts and convergence then use their Rayleigh quotients and
  residuals, and the restart block is the set of harmonic vectors;
* search vectors (step 4): SplitMix64 stream 1, column k of n_s, entry 2u-1 at
  word index i*n_s + k (real) or 2(i*n_s + k) + {0, 1} (complex parts);
* locking=True (hard locking of converged pairs, named in Sec. 6): an accepted
  in-window pair whose residual is <= eps ||H|| leaves the search block and
  is kept as found; later filtered blocks are deflated against the locked
  vectors (Y <- Y - L L^H Y, twice) before SVQB, and the search block
  shrinks to n_s minus the locked count.  Pairs are locked four at a time
  (the smallest residuals first; the filter kernels take panel widths in
  multiples of 16 bytes), the rest stay in the block.  Convergence is the
  rule above with the locked pairs counted as accepted and converged;
* adaptive=True (the adaptive choice of N_p that Sec. 6 suggests, with the
  rule of Sec. 2.4): the random start block is a set of n_s stochastic-trace
  probes, so the Chebyshev moments of the first filter (Sec. 4),
  <x_k, T_n(A) x_k> / <x_k, x_k> averaged over the columns, estimate the
  DOS (the KPM of Sec. 3.1 step 1 without extra products).  From them: the
  target count N_T (Eq. DOS:target), the margin delta' at which the count
  of the search interval reaches n_s (Eq. DOS:search), and
  N_p = N_0 S_w / delta' (Sec. 2.4, N_0 of Tab. lanczoskernel at the window
  centre), kept within [N_p / 4, 4 N_p] of the first degree, for every later
  iteration.
"""
import numpy as np

from . import coeffs, filter as filt, kpm, rng, rr, svqb

# N_0 of the Lanczos kernel (mu = 2) at the interval centre c / S_w = 0, 0.1,
# .., 0.9 (Tab. lanczoskernel), linearly interpolated, the last value beyond.
TAB_LANCZOS_N0 = (6.23, 6.20, 6.10, 5.94, 5.71, 5.40, 4.99, 4.46, 3.75, 2.73)


def lanczos_N0(rel_centre):
    x = min(abs(rel_centre), 0.9) * 10.0
    i = min(int(x), 8)
    f = x - i
    return TAB_LANCZOS_N0[i] * (1.0 - f) + TAB_LANCZOS_N0[i + 1] * f


def degree_from_moments(mu, D, a, b, lam_lo, lam_hi, ns, Np0, M_max=1024):
    """(N_T, delta', N_p) from normalised moments mu (Sec. 2.4, Sec. 3.1 steps 2-3):
    the KPM count in the window, the margin where the count of the search
    interval reaches n_s (bisection), N_p = N_0 S_w / delta' within
    [N_p0 / 4, 4 N_p0]."""
    mu = np.asarray(mu[:M_max], dtype=np.float64)
    NT = max(0.0, kpm.count_in_window(mu, D, a, b, lam_lo, lam_hi))
    d_lo, d_hi = 0.0, b - a
    for _ in range(60):
        d = 0.5 * (d_lo + d_hi)
        lo, hi = max(a, lam_lo - d), min(b, lam_hi + d)
        if kpm.count_in_window(mu, D, a, b, lo, hi) < ns:
            d_lo = d
        else:
            d_hi = d
    dprime = max(0.5 * (d_lo + d_hi), 1e-12)
    S_w = 0.5 * (b - a)
    centre = 0.5 * (lam_lo + lam_hi) - 0.5 * (a + b)
    Np = int(round(lanczos_N0(centre / S_w) * S_w / dprime))
    return NT, dprime, int(min(max(Np, max(2, Np0 // 4)), 4 * Np0))


def deflate(Y, L):
    """Y - L (L^H Y): the block with the span of the locked vectors removed
    (hard locking, Sec. 6; L orthonormal)."""
    return Y - L @ (L.conj().T @ Y)


def is_ghost(res, res_prev_nearest, eps, normH):
    """Ghost test of Sec. 3.1 step 7 (reading): an in-window pair whose
    residual stays above sqrt(eps) ||H|| without having fallen tenfold since
    the previous iteration's nearest pair."""
    return res > np.sqrt(eps) * normH and not (res_prev_nearest >= 10.0 * res)


def converging(res, res_prev_nearest):
    """A pair still converging for the empty-window test (reading of Sec. 3.1
    step 8): its residual at most 0.9 of the previous iteration's nearest."""
    return res <= 0.9 * res_prev_nearest


def search_vectors(seed, D, ns, complex_values):
    idx = np.arange(D, dtype=np.uint64)[:, None] * np.uint64(ns) + np.arange(ns, dtype=np.uint64)[None, :]
    if complex_values:
        re = 2 * rng.uniform(seed, rng.STREAM_SEARCH, 2 * idx) - 1
        im = 2 * rng.uniform(seed, rng.STREAM_SEARCH, 2 * idx + np.uint64(1)) - 1
        return re + 1j * im
    return 2 * rng.uniform(seed, rng.STREAM_SEARCH, idx) - 1


def chebfd(H, a, b, lam_lo, lam_hi, ns, Np, eps, kind="lanczos", mu=2.0, seed=0,
           max_iter=40, filter_fn=None, X0=None, complex_values=None, extraction="ritz",
           window_inset=0.0, adaptive=False, locking=False):
    """Run ChebFD; returns a dict with the accepted pairs and the iteration log.

    ``filter_fn(X)``, when given, replaces the recurrence of Fig. ChebFD by
    another evaluation of p[H] X (used for diagonal H, where p[H] X = p(lambda) X)."""
    D = H.shape[0]
    if complex_values is None:
        complex_values = np.iscomplexobj(H.data) if hasattr(H, "data") else False
    alpha, beta = coeffs.scaling(a, b)
    if not 0.0 <= window_inset < 1.0:
        raise ValueError("need 0 <= window_inset < 1")
    c, d = 0.5 * (lam_lo + lam_hi), 0.5 * (lam_hi - lam_lo) * (1.0 - window_inset)
    gc = coeffs.filter_coeffs(a, b, c - d, c + d, Np, kind, mu)
    normH = max(abs(a), abs(b))
    X = search_vectors(seed, D, ns, complex_values) if X0 is None else np.array(X0, copy=True)
    refill = 0
    log = []
    prev = None
    prev_empty = False
    result = None
    n_mvm = 0
    adapted = None
    L = np.zeros((D, 0), dtype=X.dtype)        # locked vectors and their pairs
    lam_L, res_L = np.zeros(0), np.zeros(0)
    for it in range(1, max_iter + 1):
        if adaptive and it == 1:
            m = filt.moments(H, alpha, beta, X, 2 * Np)
            adapted = degree_from_moments(np.mean(m / m[0][None, :], axis=1), D, a, b, lam_lo,
                                          lam_hi, ns, Np)
        Y = filter_fn(X) if filter_fn is not None else filt.filter_block(H, alpha, beta, gc, X)
        n_mvm += X.shape[1] * (len(gc) - 1)
        if adaptive and it == 1:
            gc = coeffs.filter_coeffs(a, b, c - d, c + d, adapted[2], kind, mu)
        for _ in range(2 if L.shape[1] else 0):
            Y = deflate(Y, L)
        Q, rank, refill = svqb.svqb(Y, seed=seed, refill_counter=refill)
        if L.shape[1]:
            # refilled columns are random: deflate once more and re-orthonormalise
            Q = deflate(Q, L)
            Q, _, refill = svqb.svqb(Q, seed=seed, refill_counter=refill)
        if extraction == "harmonic":
            theta, V, res, _ = rr.harmonic_ritz(H, Q, 0.5 * (lam_lo + lam_hi))
        else:
            theta, V, res = rr.rayleigh_ritz(H, Q)
        inwin = (theta >= lam_lo) & (theta <= lam_hi)
        ghost = np.zeros_like(inwin)
        falling = np.zeros_like(inwin)
        if prev is not None:
            pth, pres = prev
            for k in np.nonzero(inwin)[0]:
                j = int(np.argmin(np.abs(pth - theta[k])))
                if is_ghost(res[k], pres[j], eps, normH):
                    ghost[k] = True
                falling[k] = converging(res[k], pres[j])
        acc = inwin & ~ghost
        converged = (bool(acc.any()) or len(lam_L) > 0) and bool(np.all(res[acc] <= eps * normH))
        empty_now = prev is not None and not (acc | (inwin & falling)).any() and not len(lam_L)
        if empty_now and prev_empty:
            converged = True
        prev_empty = empty_now
        log.append(dict(iteration=it, rank=rank, in_window=int(inwin.sum()),
                        ghosts=int(ghost.sum()), accepted=int(acc.sum()),
                        res_min=float(res[acc].min()) if acc.any() else None,
                        res_max=float(res[acc].max()) if acc.any() else None))
        result = dict(theta=np.concatenate([lam_L, theta[acc]]),
                      V=np.concatenate([L, V[:, acc]], axis=1),
                      res=np.concatenate([res_L, res[acc]]), iterations=it,
                      n_mvm=n_mvm, converged=converged, log=log, normH=normH,
                      Np=len(gc) - 1, adapted=adapted, locked=len(lam_L))
        if converged:
            break
        keep = np.ones(len(theta), dtype=bool)
        if locking:
            done = np.nonzero(acc & (res <= eps * normH))[0]
            done = done[np.argsort(res[done], kind="stable")]
            done = np.sort(done[:len(done) // 4 * 4])
            if len(done) and len(theta) - len(done) >= 4:
                L = np.concatenate([L, V[:, done]], axis=1)
                lam_L = np.concatenate([lam_L, theta[done]])
                res_L = np.concatenate([res_L, res[done]])
                keep[done] = False
        prev = (theta[keep], res[keep])
        X = V[:, keep]
    return result
