"""Optimisers of Sec. 2.3 over the FP64 oracle (TEST INFRASTRUCTURE).

Levenberg-Marquardt (Sec. 2.3.1).  The paper uses mpfit with a forward-
difference Jacobian of step ~0.1 in every parameter and box constraints; the
details it leaves open are read as follows:
  - step: absolute, per parameter; a forward step that would leave the box is
    taken backwards;
  - damping: solve (J^T J + lambda diag(J^T J)) delta = -J^T r by Cholesky;
    if that fails, lambda *= 10 and retry;
  - trial point clipped to [lo, hi]; accepted when chi2 does not increase;
  - lambda follows the gain ratio rho = (chi2(p) - chi2(p + s)) / (predicted
    decrease of the linearised model, -2 s.J^T r - s.J^T J s) of the clipped
    step s (mpfit steers its step by the same ratio): an accepted step
    multiplies lambda by max(1/10, 1 - (2 rho - 1)^3) (rho = 0 when the
    predicted decrease is not positive; floor 1e-12) and resets nu = 2; a
    rejected one multiplies it by nu and doubles nu (H. B. Nielsen's rule,
    "Damping parameter in Marquardt's method", 1999, with a floor of 1/10
    on the decrease);
  - after a rejected step p is unchanged, so its Jacobian is reused;
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
    """Returns (p, chi2, iterations, status).  An iteration is one damped
    solve and one trial evaluation; the Jacobian is recomputed only after an
    accepted step."""
    p = np.array(p0, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    free = list(free)
    steps = np.full(10, float(fd_step)) if np.isscalar(fd_step) else np.asarray(fd_step, dtype=np.float64)
    lam = lambda0
    nu = 2.0
    best = np.nan
    status = 0
    it = 0
    J = None  # Jacobian at p (None: p moved, recompute)
    while status == 0:
        if J is None:
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
            cc = c[0]
            if not np.isfinite(cc):
                it += 1
                status = NONFINITE
                break
            r0 = r[0].ravel()
            nf = len(free)
            if central:
                J = np.stack([(r[1 + j].ravel() - r[1 + nf + j].ravel()) / hs[j] for j in range(nf)], axis=1)
            else:
                J = np.stack([(r[1 + j].ravel() - r0) / hs[j] for j in range(nf)], axis=1)
            JTJ, JTr = J.T @ J, J.T @ r0
        it += 1
        d, lam = _solve(JTJ, JTr, lam)
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
            s = pt[free] - p[free]
            pred = -(2.0 * (s @ JTr) + s @ JTJ @ s)
            rho = (cc - ct) / pred if pred > 0 else 0.0
            lam = max(lam * max(0.1, 1.0 - (2.0 * rho - 1.0) ** 3), 1e-12)
            nu = 2.0
            p = pt
            best = ct
            J = None
            if (cc - ct) / max(cc, 1e-300) < ftol:
                status = FTOL
            elif dn <= xtol * (pn + xtol):
                status = XTOL
        else:
            best = cc
            lam *= nu
            nu *= 2.0
            if lam > 1e12:
                status = LAMBDA
        if status == 0 and it >= max_iter:
            status = MAXITER
    return p, best, it, status


def grid_search(geom, obs, lo, hi, nodes, fixed, levels, nthreads=0):
    """Nested grids (Sec. 2.3.3) over the oracle: every node's chi2, the best
    node (lowest chi2, ties to the lowest row-major index, NaN worst), then
    a grid of the same size spanning best +- one step, clipped to [lo, hi].
    Returns (best_params, [best index per level], [best chi2 per level],
    [all chi2 per level])."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    fixed = np.asarray(fixed, dtype=np.float64)
    axes = [k for k in range(10) if nodes[k] > 1]
    clo, chi = lo.copy(), hi.copy()
    best_i, best_c, all_c = [], [], []
    bp = fixed.copy()
    for _ in range(levels):
        steps = {k: (chi[k] - clo[k]) / (nodes[k] - 1) for k in axes}
        grids = [clo[k] + np.arange(nodes[k], dtype=np.float64) * steps[k] for k in axes]
        mesh = np.meshgrid(*grids, indexing="ij")  # first axis slowest (row-major)
        N = mesh[0].size
        params = np.tile(fixed, (N, 1))
        for a, k in enumerate(axes):
            params[:, k] = mesh[a].ravel()
        c = chi2_batch(geom, params, obs, nthreads=nthreads)
        key = np.where(np.isnan(c), np.inf, c)
        i = int(np.argmin(key))  # first occurrence = lowest index
        best_i.append(i)
        best_c.append(c[i])
        all_c.append(c)
        bp = params[i].copy()
        for k in axes:
            clo[k] = max(lo[k], bp[k] - steps[k])
            chi[k] = min(hi[k], bp[k] + steps[k])
    return bp, best_i, best_c, all_c


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): uniforms from the top 53 bits,
    normals by Box-Muller (cosine branch)."""
    M = (1 << 64) - 1

    def __init__(self, seed):
        self.s = seed & self.M

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & self.M
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.M
        return z ^ (z >> 31)

    def uniform(self):
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self):
        u1, u2 = self.uniform(), self.uniform()
        u1 = max(u1, 1e-300)
        return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2 * np.pi * u2))


def nested_sample(loglike, lo, hi, n_live, batch, tol=0.5, efr=1.0, seed=1, max_iter=100000, trace=None):
    """Vanilla nested sampling with an ellipsoidal bound (Sec. 2.3.2 reading):
    live points from the uniform prior over [lo, hi]; each iteration draws
    `batch` points uniformly in the live points' bounding ellipsoid (volume
    x 1.1 / efr) that fall inside the box; in draw order each replaces the
    worst live point if its log-likelihood is higher (ln X -= 1/N each);
    stop when ln(Z + Lmax X) - ln Z < tol.  `loglike(params [n][10])`
    returns log L per row.  Returns dict(mean, std, log_z, n_eval, n_iter,
    info) where info is the information H used for the log Z error
    sqrt(H / N).  A dict passed as `trace` receives the trajectory: the
    initial live points and their log L ("live0", "live0_logl"), and per
    iteration the proposals in draw order, their log L and the index of the
    live point each replaced, -1 for none ("props", "logl", "replaced")."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ax = [k for k in range(10) if hi[k] > lo[k]]
    P = len(ax)
    N = n_live
    rng = SplitMix64(seed)
    live = np.tile(lo, (N, 1))
    for i in range(N):
        for k in range(10):
            live[i, k] = lo[k] + (hi[k] - lo[k]) * rng.uniform() if hi[k] > lo[k] else lo[k]
    logl = np.asarray(loglike(live), dtype=np.float64)
    n_eval = N
    if trace is not None:
        trace.update(live0=live.copy(), live0_logl=logl.copy(), props=[], logl=[], replaced=[])
    dead_p, dead_lw, dead_l = [], [], []
    logz, logx = -np.inf, 0.0
    log_shrink = np.log(-np.expm1(-1.0 / N))
    it = 0
    while it < max_iter:
        lmax = logl.max()
        if it > 0 and np.logaddexp(logz, lmax + logx) - logz < tol:
            break
        X = live[:, ax]
        mu = X.mean(axis=0)
        C = (X - mu).T @ (X - mu) / N + np.diag(1e-12 * (hi[ax] - lo[ax]) ** 2)
        Lc = np.linalg.cholesky(C)
        y = np.linalg.solve(Lc, (X - mu).T)
        scale = np.sqrt(np.max(np.sum(y * y, axis=0))) * (1.1 / efr) ** (1.0 / P)
        props = []
        tries = 0
        while len(props) < batch and tries < 1000 * batch:
            tries += 1
            z = np.array([rng.normal() for _ in range(P)])
            rad = rng.uniform() ** (1.0 / P) / np.sqrt(max(float(z @ z), 1e-300))
            v = mu + Lc @ (z * rad * scale)
            if np.all(v >= lo[ax]) and np.all(v <= hi[ax]):
                q = lo.copy()
                q[ax] = v
                props.append(q)
        if not props:
            break
        props = np.array(props)
        lp = np.asarray(loglike(props), dtype=np.float64)
        n_eval += len(props)
        repl = np.full(len(props), -1)
        if trace is not None:
            trace["props"].append(props.copy())
            trace["logl"].append(lp.copy())
            trace["replaced"].append(repl)
        for j in range(len(props)):
            w = int(np.argmin(logl))
            if not lp[j] > logl[w]:
                continue
            repl[j] = w
            lw = logx + log_shrink + logl[w]
            logz = np.logaddexp(logz, lw)
            dead_p.append(live[w].copy())
            dead_lw.append(lw)
            dead_l.append(logl[w])
            logx -= 1.0 / N
            live[w] = props[j]
            logl[w] = lp[j]
        it += 1
    for i in range(N):
        lw = logx - np.log(N) + logl[i]
        logz = np.logaddexp(logz, lw)
        dead_p.append(live[i].copy())
        dead_lw.append(lw)
        dead_l.append(logl[i])
    dead_p = np.array(dead_p)
    wgt = np.exp(np.array(dead_lw) - logz)
    mean = wgt @ dead_p
    std = np.sqrt(wgt @ (dead_p - mean) ** 2)
    info = float(np.sum(wgt * (np.array(dead_l) - logz)))
    return {"mean": mean, "std": std, "log_z": float(logz), "n_eval": n_eval, "n_iter": it, "info": info}


def nested_sample_model(geom, obs, lo, hi, n_live, batch, tol=0.5, efr=1.0, seed=1, nthreads=0, max_iter=100000,
                        trace=None):
    """Nested sampling of the disc model: L = exp(-chi2 / 2) from the oracle;
    outside the parameter domain (chi2 NaN) the likelihood is 0, log L = -inf."""
    def loglike(p):
        c = chi2_batch(geom, p, obs, nthreads=nthreads)
        return np.where(np.isfinite(c), -0.5 * c, -np.inf)
    return nested_sample(loglike, lo, hi, n_live, batch, tol, efr, seed, max_iter=max_iter, trace=trace)
