"""Oracle: minimax tau and omega grids (Sec. 2: the non-uniform tau_j, omega_k grids the paper
takes from GreenX).

Test infrastructure only (see the package docstring).  Slow: mpmath at 50 digits.

The paper does not print the grids; GreenX's tables are not available here (and none is written
from memory).  What the grids are is fixed by their defining property, restated here in scaled
units x = D / dmin on [1, R], R = dmax / dmin (transition energies D in [dmin, dmax]):

* time grid (tau_j, a_j), j = 1..n: the n-term exponential sum closest to 1/x in the maximum
  norm, min max_x |1/x - sum_j a_j exp(-tau_j x)|  (1/x = int_0^inf exp(-x tau) d tau, the
  Laplace form of an energy denominator, discretised);
* frequency grid (omega_k, W_k): the n-term sum closest to 1/x in the maximum norm among
  (1/pi) sum_k W_k 4x^2 / (x^2 + omega_k^2)^2  (pi/x = int_0^inf (2x/(x^2 + w^2))^2 dw: the
  squared Lorentzian of a transition, the frequency integral of the leading term of the RPA
  integrand, so W_k are weights of int_0^inf d omega).

Both are nonlinear Chebyshev problems; their solutions are characterised by equioscillation:
the error takes its maximum modulus, with alternating signs, at (at least) 2n + 1 points of
[1, R].  The solver here is the Remez exchange for that characterisation: solve the 2n + 1
equations r(x_i) = (-1)^i E for the 2n parameters and E (Newton, mpmath), move the x_i to the
extrema of the new error curve, repeat until the extrema are level.  Terms are added one at a
time from n = 1 on a range R_g >= R wide enough that n terms stay above ~1e-6, each new term
starting from a least-squares fit (numpy, only a starting point); the solution is then carried
from R_g down to R by continuation, each step starting from the previous range's solution and
its extrema mapped onto the new range.  The result is fixed by the equioscillation conditions,
which the tests check on a dense sample independently of this solver.

Range: ranges so narrow that n terms would fit below ~1e-9 are degenerate (the parameters are
then fixed only by rounding), so R_eff = max(R, R_floor(n)), R_floor(n) = exp(n pi^2 / ln 1e9)
/ 8 (the asymptotic error exp(-n pi^2 / ln(8R)) of exponential sums of 1/x), rounded up to
1/8 octave: R_b = 2^{ceil(8 log2 R_eff) / 8}.  The grid covers [1, R_b], hence [1, R].
Physical units: tau_j = tau_j^ / dmin, omega_k = dmin omega_k^, W_k = dmin W_k^; Gamma is the
least-squares fit of grid.fit_gamma on [dmin, R_b dmin].
"""
from __future__ import annotations

import math

import mpmath as mp
import numpy as np

DPS = 50
FLOOR_ERR = 1e-9


def r_floor(n):
    """Smallest range ratio the n-point grids are built for (module docstring)."""
    return math.exp(n * math.pi ** 2 / math.log(1.0 / FLOOR_ERR)) / 8.0


def range_ratio(n, dmin, dmax):
    """R_b: the range ratio an n-point grid for transitions in [dmin, dmax] is built for."""
    r = max(dmax / dmin, r_floor(n), 1.0)
    return 2.0 ** (math.ceil(8.0 * math.log2(r)) / 8.0)


def _sample(R, m):
    """x = R^{u^2}, u uniform on [0, 1] (the error lobes are narrowest near x = 1)."""
    return [R ** (u * u) for u in np.linspace(0.0, 1.0, m)]


# ---------------------------------------------------------------------------------------------
# the two families, parameters p = (log a_1..n, log t_1..n); value and gradient at x (mpmath)

def _tau_val(p, x):
    n = len(p) // 2
    return mp.fsum(mp.exp(p[j]) * mp.exp(-mp.exp(p[n + j]) * x) for j in range(n))


def _tau_grad(p, x):
    n = len(p) // 2
    g = []
    for j in range(n):
        a, t = mp.exp(p[j]), mp.exp(p[n + j])
        g.append(a * mp.exp(-t * x))
    for j in range(n):
        a, t = mp.exp(p[j]), mp.exp(p[n + j])
        g.append(-a * t * x * mp.exp(-t * x))
    return g


def _om_val(p, x):
    n = len(p) // 2
    return mp.fsum(mp.exp(p[k]) * 4 * x ** 2 / (x ** 2 + mp.exp(2 * p[n + k])) ** 2 for k in range(n)) / mp.pi


def _om_grad(p, x):
    n = len(p) // 2
    g = [mp.exp(p[k]) * 4 * x ** 2 / (x ** 2 + mp.exp(2 * p[n + k])) ** 2 / mp.pi for k in range(n)]
    for k in range(n):
        w, o2 = mp.exp(p[k]), mp.exp(2 * p[n + k])
        g.append(-w * 16 * x ** 2 * o2 / (x ** 2 + o2) ** 3 / mp.pi)
    return g


FAMILIES = {"tau": (_tau_val, _tau_grad), "omega": (_om_val, _om_grad)}


def error_curve(kind, p, x):
    """r(x) = 1/x - phi(x; p) in scaled units (mpmath number)."""
    return 1 / mp.mpf(x) - FAMILIES[kind][0](p, mp.mpf(x))


# ---------------------------------------------------------------------------------------------
# numpy least squares (starting points only)

def _np_family(kind, p, x):
    n = len(p) // 2
    a, t = np.exp(p[:n]), np.exp(p[n:])
    if kind == "tau":
        E = np.exp(-np.outer(x, t))
        f = E @ a
        J = np.hstack([E * a, -(E * a) * (x[:, None] * t)])
    else:
        D = x[:, None] ** 2 + t[None] ** 2
        L = 4 * x[:, None] ** 2 / D ** 2 / math.pi
        f = L @ a
        J = np.hstack([L * a, -a * 16 * x[:, None] ** 2 * t ** 2 / D ** 3 / math.pi])
    return f, J


def _least_squares(kind, p, R, weights=None, m=1500, iters=300):
    """Levenberg-Marquardt fit of 1/x on m log-spaced points of [1, R] (weighted)."""
    xs = np.array(_sample(R, m))
    w = np.ones(m) if weights is None else weights
    p = p.copy()
    lam = 1e-3
    f, J = _np_family(kind, p, xs)
    r = (1 / xs - f) * w
    cost = r @ r
    for _ in range(iters):
        Jw = J * w[:, None]
        A, g = Jw.T @ Jw, Jw.T @ r
        dA = np.diag(A) + 1e-12 * np.diag(A).max()
        improved = False
        while lam < 1e14:
            try:
                d = np.linalg.solve(A + lam * np.diag(dA), g)
            except np.linalg.LinAlgError:
                lam *= 10
                continue
            mx = np.abs(d).max()
            if mx > 0.5:
                d *= 0.5 / mx
            fn, Jn = _np_family(kind, p + d, xs)
            rn = (1 / xs - fn) * w
            cn = rn @ rn
            if np.isfinite(cn) and cn < cost:
                done = cost - cn < 1e-13 * cost
                p, f, J, r, cost = p + d, fn, Jn, rn, cn
                lam = max(lam / 3, 1e-12)
                improved = True
                break
            lam *= 4
        if not improved or done:
            break
    return p


def _start(kind, p_prev, R, variant=0):
    """Starting point for n + 1 terms from the n-term solution (None: one term).  variant 0 puts
    the new term beyond the largest parameter, 1 below the smallest, v >= 2 in the middle of the
    (v - 1)-th widest gap; None when that variant does not exist."""
    if p_prev is None:
        if variant:
            return None
        p = np.array([0.0, 0.0]) if kind == "tau" else np.array([math.log(math.pi), math.log(math.sqrt(R))])
    else:
        n = len(p_prev) // 2
        o = np.argsort(p_prev[n:])
        la, lt = list(p_prev[:n][o]), list(p_prev[n:][o])
        if n == 1:
            if variant > 1:
                return None
            d = 1.0 if variant == 0 else -1.0
            lt, la = [lt[0] - 1.5 * d, lt[0] + d], [la[0] - 1.0, la[0]]
        elif variant <= 1:
            if variant == 0:
                lt.append(2 * lt[-1] - lt[-2])
                la.append(2 * la[-1] - la[-2])
            else:
                lt.insert(0, 2 * lt[0] - lt[1])
                la.insert(0, 2 * la[0] - la[1])
            c = sum(lt) / len(lt)
            lt = [c + (v - c) * math.sqrt(n / (n + 1.0)) for v in lt]
        else:
            gaps = sorted(((lt[j + 1] - lt[j], j) for j in range(n - 1)), reverse=True)
            if variant - 2 >= len(gaps):
                return None
            j = gaps[variant - 2][1]
            lt.insert(j + 1, 0.5 * (lt[j] + lt[j + 1]))
            la.insert(j + 1, 0.5 * (la[j] + la[j + 1]) - math.log(2.0))
        p = np.array(la + lt)
    xs = np.array(_sample(R, 1500))
    w = np.ones(len(xs))
    for _ in range(6):   # least squares, reweighted towards the largest errors (Lawson-like)
        p = _least_squares(kind, p, R, w)
        f, _ = _np_family(kind, p, xs)
        e = np.abs(1 / xs - f)
        w = w * np.sqrt(e / e.max()) + 1e-3
        w /= w.max()
    return p


# ---------------------------------------------------------------------------------------------
# Remez exchange (mpmath)

def _extrema(kind, p, R, m):
    """Alternating extrema of r on [1, R]: endpoints and the interior maxima of |r| (golden search)."""
    xs = [mp.mpf(x) for x in _sample(R, m)]
    xs[-1] = mp.mpf(R)
    e = [error_curve(kind, p, x) for x in xs]
    idx = [0] + [i for i in range(1, m - 1) if (abs(e[i]) >= abs(e[i - 1]) and abs(e[i]) >= abs(e[i + 1])
                                                  and mp.sign(e[i - 1]) == mp.sign(e[i]) == mp.sign(e[i + 1]))] + [m - 1]
    pts = []
    for i in idx:
        if i in (0, m - 1):
            x = xs[i]
        else:   # maximise |r| on [x_{i-1}, x_{i+1}] in log x
            lo, hi = mp.log(xs[i - 1]), mp.log(xs[i + 1])
            g = (mp.sqrt(5) - 1) / 2
            c, d = hi - g * (hi - lo), lo + g * (hi - lo)
            fc, fd = abs(error_curve(kind, p, mp.exp(c))), abs(error_curve(kind, p, mp.exp(d)))
            for _ in range(45):
                if fc > fd:
                    hi, d, fd = d, c, fc
                    c = hi - g * (hi - lo)
                    fc = abs(error_curve(kind, p, mp.exp(c)))
                else:
                    lo, c, fc = c, d, fd
                    d = lo + g * (hi - lo)
                    fd = abs(error_curve(kind, p, mp.exp(d)))
            x = mp.exp((lo + hi) / 2)
        pts.append((x, error_curve(kind, p, x)))
    # one point per run of equal sign: the largest |r|
    alt = []
    for x, v in pts:
        if alt and mp.sign(v) == mp.sign(alt[-1][1]):
            if abs(v) > abs(alt[-1][1]):
                alt[-1] = (x, v)
        else:
            alt.append((x, v))
    return alt


def _level(kind, p, xs, E):
    """Newton on r(x_i; p) - (-1)^i E = 0, i = 0..2n (2n + 1 unknowns: p and E)."""
    val, grad = FAMILIES[kind]
    n2 = len(p)
    p = [mp.mpf(v) for v in p]
    for _ in range(60):
        F = mp.matrix(n2 + 1, 1)
        J = mp.matrix(n2 + 1, n2 + 1)
        for i, x in enumerate(xs):
            s = 1 if i % 2 == 0 else -1
            F[i] = 1 / x - val(p, x) - s * E
            g = grad(p, x)
            for j in range(n2):
                J[i, j] = -g[j]
            J[i, n2] = -s
        d = mp.lu_solve(J, -F)
        step = mp.mpf(1)
        mx = max(abs(d[j]) for j in range(n2))
        if mx > mp.mpf("0.5"):
            step = mp.mpf("0.5") / mx
        p = [p[j] + step * d[j] for j in range(n2)]
        E = E + step * d[n2]
        if step == 1 and mx < mp.mpf(10) ** (-(DPS - 10)):
            break
    return p, E


def remez(kind, p0, R, tol=1e-13, iters=40, ref=None):
    """Levels the error curve of the family from p0 on [1, R]; returns (p, max |r|, extrema) or
    None.  ref: 2n + 1 points to level on first (a previous range's extrema mapped onto [1, R])."""
    n2 = len(p0)
    p = [mp.mpf(v) for v in p0]
    m = max(400, 60 * n2)
    if ref is not None and len(ref) == n2 + 1:
        E0 = mp.fsum((1 if i % 2 == 0 else -1) * error_curve(kind, p, x) for i, x in enumerate(ref)) / (n2 + 1)
        p, _ = _level(kind, p, ref, E0)
    for _ in range(iters):
        alt = _extrema(kind, p, R, m)
        if len(alt) < n2 + 1:
            return None
        # n2 + 1 consecutive alternating extrema holding the largest of them
        big = max(range(len(alt)), key=lambda i: abs(alt[i][1]))
        s0 = min(max(0, big - n2 // 2), len(alt) - n2 - 1)
        seg = alt[s0:s0 + n2 + 1]
        emax = max(abs(v) for _, v in alt)
        emin = min(abs(v) for _, v in seg)
        xs = [x for x, _ in seg]
        if (emax - emin) / emax < tol:   # level, and no other extremum above the level
            return p, emax, xs
        E0 = mp.sign(seg[0][1]) * mp.fsum(abs(v) for _, v in seg) / len(seg)
        p, _ = _level(kind, p, xs, E0)
    return None


def minimax_scaled(kind, n, R):
    """Scaled minimax parameters on [1, R]: returns (a[n], t[n]) ascending in t and max |r|."""
    mp.mp.dps = DPS
    Rg = max(R, math.exp(n * math.pi ** 2 / math.log(1e6)) / 8.0)
    p_prev, res = None, None
    for k in range(1, n + 1):
        for variant in range(8):
            start = _start(kind, p_prev, Rg, variant)
            if start is None:
                break
            res = remez(kind, start, Rg)
            if res is not None:
                break
        if res is None:
            raise RuntimeError("minimax %s grid: no level error curve at %d terms, R = %g" % (kind, k, Rg))
        p_prev = np.array([float(v) for v in res[0]])
    p, emax, ref = res
    Rc, f = Rg, 1.25
    while Rc > R:   # continuation to R: extrema mapped by log x -> log x log Rn / log Rc
        Rn = max(R, Rc / f)
        sc = mp.log(Rn) / mp.log(Rc)
        rq = [mp.mpf(1)] + [mp.exp(mp.log(x) * sc) for x in ref[1:-1]] + [mp.mpf(Rn)]
        step = remez(kind, p, Rn, ref=rq)
        if step is None:
            f = math.sqrt(f)
            if f < 1.01:
                raise RuntimeError("minimax %s grid: continuation stalled at R = %g" % (kind, Rc))
            continue
        p, emax, ref = step
        Rc, f = Rn, min(2.0, f * 1.5)
    n_ = len(p) // 2
    a = [mp.exp(v) for v in p[:n_]]
    t = [mp.exp(v) for v in p[n_:]]
    order = sorted(range(n_), key=lambda j: t[j])
    return [a[j] for j in order], [t[j] for j in order], emax


def make_minimax_grid(n, dmin, dmax):
    """tau[n], omega[n], w_omega[n] and gamma[n][n] in Ha units, the time grid's weights a_tau[n]
    (1/D ~ sum_j a_tau_j exp(-D tau_j)), R_b and the largest errors of the two fits (scaled units)."""
    from . import grid as ogrid
    R = range_ratio(n, dmin, dmax)
    a, t, et = minimax_scaled("tau", n, R)
    w, o, eo = minimax_scaled("omega", n, R)
    tau = np.array([float(v) for v in t]) / dmin
    omega = np.array([float(v) for v in o]) * dmin
    w_omega = np.array([float(v) for v in w]) * dmin
    gamma = ogrid.fit_gamma(tau, omega, dmin, R * dmin)
    a_tau = np.array([float(v) for v in a]) / dmin   # 1/D ~ sum_j a_tau_j exp(-D tau_j)
    return dict(tau=tau, omega=omega, w_omega=w_omega, gamma=gamma, a_tau=a_tau, r_eff=R, err_tau=float(et),
                err_omega=float(eo))
