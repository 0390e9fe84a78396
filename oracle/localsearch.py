"""Local search of Sec. IV.A (TEST INFRASTRUCTURE ONLY): augmented Lagrangian with
BFGS inner minimisation and a strong-Wolfe line search, plus the multistart.

Only tests/ may import this module.  The paper defers the inner algorithms to
Nocedal & Wright, "Numerical Optimization" (2nd ed.); they are written here from
that book: the line search of its Algorithm 3.5 with the zoom of Algorithm 3.6
(cubic interpolation of Eq. 3.59, safeguarded by bisection), BFGS of
Algorithm 6.1 with the inverse-Hessian update of Eq. 6.17 and the initial
scaling of Eq. 6.20.  The outer loop follows the paper's steps 1-5:
lambda_0 = 0, mu_0 > 0; minimise L(lambda_l, mu_l); lambda_{l+1} = lambda_l -
C / mu_l; mu_{l+1} = xi mu_l (0 < xi < 1); warm start; repeat until C = 0 (to a
tolerance).  The objective is given as obj(x) -> (J, grad J, C, grad C) and
the Lagrangian is L = -J - lambda C + C^2 / (2 mu).

Every constant and every decision below is mirrored by the library's native
optimiser, so that both take the same iterates on the same objective.
"""
import math

import numpy as np

C1 = 1e-4          # sufficient decrease
C2 = 0.9           # curvature (strong Wolfe)
LS_MAX = 20        # bracketing iterations
ZOOM_MAX = 30      # zoom iterations
ALPHA_MAX = 1e3    # largest trial step
GROW = 2.0         # step growth while bracketing


def _dot(a, b):
    """Sum of a_i b_i in index order (one rounding per product and per sum)."""
    s = 0.0
    for i in range(len(a)):
        s += float(a[i]) * float(b[i])
    return s


def _matvec(H, v):
    return np.array([_dot(H[i], v) for i in range(H.shape[0])])


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic interpolating (a, fa, ga), (b, fb, gb) (Eq. 3.59),
    or None when it does not exist."""
    if a == b:
        return None
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = gb - ga + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def _zoom_point(lo, flo, glo, hi, fhi, ghi):
    """Cubic step safeguarded to the inner 80% of [lo, hi], else the midpoint."""
    a = _cubic_min(lo, flo, glo, hi, fhi, ghi)
    if a is not None and not math.isfinite(a):
        a = None
    left, right = min(lo, hi), max(lo, hi)
    d = right - left
    if a is None or not (left + 0.1 * d <= a <= right - 0.1 * d):
        a = 0.5 * (lo + hi)
    return a


def line_search(phi, f0, g0, alpha1):
    """Strong-Wolfe step along a descent direction (Algorithms 3.5, 3.6).

    phi(alpha) -> (f, g, payload): the objective, its directional derivative and
    anything the caller wants back for the accepted point; f0, g0 at alpha = 0
    (g0 < 0).  Returns (alpha, f, payload, evaluations, ok).  When no step meets
    both conditions, ok is False and the best point found with sufficient
    decrease is returned (alpha = 0 and payload None if there is none).
    """
    evals = 0
    prev = (0.0, f0, g0, None)
    a = alpha1
    for i in range(LS_MAX):
        f, g, pay = phi(a)
        evals += 1
        cur = (a, f, g, pay)
        # a non-finite value or slope counts as a failed decrease (the step is too long)
        if not (math.isfinite(f) and math.isfinite(g)) or f > f0 + C1 * a * g0 or (i > 0 and f >= prev[1]):
            return _zoom(phi, f0, g0, prev, cur, evals)
        if abs(g) <= -C2 * g0:
            return a, f, pay, evals, True
        if g >= 0.0:
            return _zoom(phi, f0, g0, cur, prev, evals)
        prev = cur
        a = min(GROW * a, ALPHA_MAX)
    return prev[0], prev[1], prev[3], evals, False


def _zoom(phi, f0, g0, lo, hi, evals):
    """lo, hi = (alpha, f, g, payload); lo has sufficient decrease and the lower f."""
    for _ in range(ZOOM_MAX):
        a = _zoom_point(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
        f, g, pay = phi(a)
        evals += 1
        cur = (a, f, g, pay)
        if not (math.isfinite(f) and math.isfinite(g)) or f > f0 + C1 * a * g0 or f >= lo[1]:
            hi = cur
        else:
            if abs(g) <= -C2 * g0:
                return a, f, pay, evals, True
            if g * (hi[0] - lo[0]) >= 0.0:
                hi = lo
            lo = cur
    return lo[0], lo[1], lo[3], evals, False


def bfgs(fg, x0, gtol=1e-6, max_iter=200):
    """Minimise fg(x) -> (f, grad, aux) from x0 (Algorithm 6.1).  Returns dict(x, f, g,
    aux, iters, evals, status); status "converged" (max |g| <= gtol), "max_iter" or
    "line_search" (no step meeting the strong Wolfe conditions; the best point with
    sufficient decrease, if any, is taken first)."""
    x = np.array(x0, dtype=np.float64)
    n = x.size
    f, g, aux = fg(x)
    evals = 1
    if not (math.isfinite(f) and all(math.isfinite(v) for v in g)):
        return dict(x=x, f=f, g=g, aux=aux, iters=0, evals=evals, status="invalid")
    H = np.eye(n)
    first = True
    for k in range(max_iter):
        if np.max(np.abs(g)) <= gtol:
            return dict(x=x, f=f, g=g, aux=aux, iters=k, evals=evals, status="converged")
        p = -_matvec(H, g)
        gp = _dot(p, g)
        if not gp < 0.0:  # not a descent direction: restart from the gradient
            H = np.eye(n)
            p = -g
            gp = _dot(p, g)
        alpha1 = min(1.0, 1.0 / math.sqrt(_dot(g, g))) if first else 1.0

        def phi(a, x=x, p=p):
            xa = x + a * p
            fa, ga, auxa = fg(xa)
            return fa, _dot(ga, p), (xa, ga, auxa)
        a, fa, pay, ne, ok = line_search(phi, f, gp, alpha1)
        evals += ne
        if pay is None:
            return dict(x=x, f=f, g=g, aux=aux, iters=k, evals=evals, status="line_search")
        xn, gn, auxn = pay
        s = xn - x
        y = gn - g
        ys = _dot(y, s)
        if ys > 0.0:
            if first:
                H = (ys / _dot(y, y)) * np.eye(n)  # Eq. 6.20
            rho = 1.0 / ys
            Hy = _matvec(H, y)
            H = (H - rho * (np.outer(s, Hy) + np.outer(Hy, s))
                 + (rho * rho * _dot(y, Hy) + rho) * np.outer(s, s))  # Eq. 6.17
        first = False
        x, f, g, aux = xn, fa, gn, auxn
        if not ok:
            return dict(x=x, f=f, g=g, aux=aux, iters=k + 1, evals=evals, status="line_search")
    status = "converged" if np.max(np.abs(g)) <= gtol else "max_iter"
    return dict(x=x, f=f, g=g, aux=aux, iters=max_iter, evals=evals, status=status)


def augmented_lagrangian(obj, x0, mu0=1.0, xi=0.5, outer=10, gtol=1e-6, ctol=1e-8, max_iter=200):
    """Steps 1-4 of Sec. IV.A from x0.  obj(x) -> (J, gJ, C, gC).  Returns dict(x, J, C,
    lam, mu, outer, evals, history, status): status 0 = |C| <= ctol reached, 1 = `outer`
    inner minimisations run, 2 = the objective is not finite where an inner
    minimisation starts."""
    lam, mu = 0.0, mu0
    x = np.array(x0, dtype=np.float64)
    evals = 0
    history = []
    J = C = None
    for l in range(outer):
        def fg(z, lam=lam, mu=mu):
            Jz, gJ, Cz, gC = obj(z)
            L = -Jz - lam * Cz + Cz * Cz / (2.0 * mu)
            return L, -np.asarray(gJ) - (lam - Cz / mu) * np.asarray(gC), (Jz, Cz)
        r = bfgs(fg, x, gtol=gtol, max_iter=max_iter)
        evals += r["evals"]
        x = r["x"]
        J, C = r["aux"]
        history.append(dict(J=J, C=C, lam=lam, mu=mu, iters=r["iters"], status=r["status"]))
        if r["status"] == "invalid":
            return dict(x=x, J=J, C=C, lam=lam, mu=mu, outer=l + 1, evals=evals, history=history,
                        status=2)
        if abs(C) <= ctol:
            return dict(x=x, J=J, C=C, lam=lam, mu=mu, outer=l + 1, evals=evals, history=history,
                        status=0)
        lam = lam - C / mu
        mu = xi * mu
    return dict(x=x, J=J, C=C, lam=lam, mu=mu, outer=outer, evals=evals, history=history, status=1)


def multistart(obj, starts, **kw):
    """Step 5: the local search from every start; returns the runs and the index of the
    best feasible one (largest J among |C| <= ctol, else largest J)."""
    runs = [augmented_lagrangian(obj, x0, **kw) for x0 in starts]
    ctol = kw.get("ctol", 1e-8)
    feas = [i for i, r in enumerate(runs) if abs(r["C"]) <= ctol] or list(range(len(runs)))
    best = max(feas, key=lambda i: runs[i]["J"])
    return runs, best
