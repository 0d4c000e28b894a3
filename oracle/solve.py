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
  word index i*n_s + k (real) or 2(i*n_s + k) + {0, 1} (complex parts).
"""
import numpy as np

from . import coeffs, filter as filt, rng, rr, svqb


def search_vectors(seed, D, ns, complex_values):
    idx = np.arange(D, dtype=np.uint64)[:, None] * np.uint64(ns) + np.arange(ns, dtype=np.uint64)[None, :]
    if complex_values:
        re = 2 * rng.uniform(seed, rng.STREAM_SEARCH, 2 * idx) - 1
        im = 2 * rng.uniform(seed, rng.STREAM_SEARCH, 2 * idx + np.uint64(1)) - 1
        return re + 1j * im
    return 2 * rng.uniform(seed, rng.STREAM_SEARCH, idx) - 1


def chebfd(H, a, b, lam_lo, lam_hi, ns, Np, eps, kind="lanczos", mu=2.0, seed=0,
           max_iter=40, filter_fn=None, X0=None, complex_values=None, extraction="ritz",
           window_inset=0.0):
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
    for it in range(1, max_iter + 1):
        Y = filter_fn(X) if filter_fn is not None else filt.filter_block(H, alpha, beta, gc, X)
        Q, rank, refill = svqb.svqb(Y, seed=seed, refill_counter=refill)
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
                if res[k] > np.sqrt(eps) * normH and not (pres[j] >= 10.0 * res[k]):
                    ghost[k] = True
                falling[k] = res[k] <= 0.9 * pres[j]
        acc = inwin & ~ghost
        converged = bool(acc.any()) and bool(np.all(res[acc] <= eps * normH))
        empty_now = prev is not None and not (acc | (inwin & falling)).any()
        if empty_now and prev_empty:
            converged = True
        prev_empty = empty_now
        log.append(dict(iteration=it, rank=rank, in_window=int(inwin.sum()),
                        ghosts=int(ghost.sum()), accepted=int(acc.sum()),
                        res_min=float(res[acc].min()) if acc.any() else None,
                        res_max=float(res[acc].max()) if acc.any() else None))
        result = dict(theta=theta[acc], V=V[:, acc], res=res[acc], iterations=it,
                      n_mvm=it * ns * Np, converged=converged, log=log, normH=normH)
        if converged:
            break
        prev = (theta, res)
        X = V
    return result
