"""Optimisers of Sec. 2.3 over the FP64 oracle (TEST INFRASTRUCTURE).

Levenberg-Marquardt (Sec. 2.3.1).  The paper uses mpfit with a forward-
difference Jacobian of step ~0.1 in every parameter and box constraints; the
details it leaves open are read as follows:
  - step: absolute, per parameter; a forward step that would leave the box is
    taken backwards;
  - damping: solve (J^T J + lambda diag(J^T J)) delta = -J^T r by Cholesky;
    if that fails, lambda *= 10 and retry;
  - trial point clipped to [lo, hi]; accepted when chi2 does not increase
    (lambda /= 10, floor 1e-12), otherwise lambda *= 10;
  - stop when an accepted step lowers chi2 by less than ftol (relative), when
    |delta| <= xtol (|p| + xtol), when lambda > 1e12, or after max_iter
    iterations.
"""
import numpy as np

from . import chi2_batch

FTOL, XTOL, LAMBDA, MAXITER, NONFINITE = 1, 2, 4, 3, 5


def _solve(JTJ, JTr, lam):
    n = JTJ.shape[0]
    for _ in range(12):
        A = JTJ.copy()
        d = np.diag(JTJ).copy()
        d[d <= 0] = 1.0
        A[np.diag_indices(n)] += lam * d
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError:
            lam *= 10.0
            continue
        y = np.linalg.solve(L, -JTr)
        return np.linalg.solve(L.T, y), lam
    return None, lam


def fit_lm(geom, obs, p0, lo, hi, free, fd_step=0.1, max_iter=200, ftol=1e-10, xtol=1e-10, lambda0=1e-3,
           central=False, nthreads=0):
    """Returns (p, chi2, iterations, status)."""
    p = np.array(p0, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    free = list(free)
    steps = np.full(10, float(fd_step)) if np.isscalar(fd_step) else np.asarray(fd_step, dtype=np.float64)
    lam = lambda0
    best = np.nan
    status = 0
    it = 0
    while status == 0:
        batch = [p.copy()]
        hs = []
        for k in free:
            h = steps[k]
            q = p.copy()
            if central:
                q[k] = p[k] + h
                batch.append(q)
                hs.append(2 * h)
            else:
                if p[k] + h > hi[k] and p[k] - h >= lo[k]:
                    h = -h
                q[k] = p[k] + h
                batch.append(q)
                hs.append(h)
        if central:
            for k in free:
                q = p.copy()
                q[k] = p[k] - steps[k]
                batch.append(q)
        c, r = chi2_batch(geom, np.array(batch), obs, want_resid=True, nthreads=nthreads)
        it += 1
        cc = c[0]
        if not np.isfinite(cc):
            status = NONFINITE
            break
        r0 = r[0].ravel()
        nf = len(free)
        if central:
            J = np.stack([(r[1 + j].ravel() - r[1 + nf + j].ravel()) / hs[j] for j in range(nf)], axis=1)
        else:
            J = np.stack([(r[1 + j].ravel() - r0) / hs[j] for j in range(nf)], axis=1)
        d, lam = _solve(J.T @ J, J.T @ r0, lam)
        ct = np.nan
        dn = pn = 0.0
        pt = p.copy()
        if d is not None:
            for j, k in enumerate(free):
                pt[k] = min(max(p[k] + d[j], lo[k]), hi[k])
            dn = float(np.sqrt(np.sum((pt[free] - p[free]) ** 2)))
            pn = float(np.sqrt(np.sum(p[free] ** 2)))
            if dn > 0:
                ct = chi2_batch(geom, pt[None], obs, nthreads=nthreads)[0]
        if np.isfinite(ct) and ct <= cc and dn > 0:
            p = pt
            best = ct
            lam = max(lam * 0.1, 1e-12)
            if (cc - ct) / max(cc, 1e-300) < ftol:
                status = FTOL
            elif dn <= xtol * (pn + xtol):
                status = XTOL
        else:
            best = cc
            lam *= 10.0
            if lam > 1e12:
                status = LAMBDA
        if status == 0 and it >= max_iter:
            status = MAXITER
    return p, best, it, status
