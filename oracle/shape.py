"""FP64 solver of the axisymmetric equilibrium droplet shape (App. B).

TEST INFRASTRUCTURE ONLY: the yardstick for the simulated equilibria (through
eq. L2-error_equilibrium), imported by tests/.  Plain numpy/scipy; no code
shared with the CUDA library.

The surface is r = R0 g(u), u = cos(phi) in [-1, 1], phi the polar angle
from +z about an origin midway between the top and the bottom of the drop
(eq. bc: g(1) = g(-1)).  The normal force balance, eq. YL,

    k = [u g g' - g^2 - (1 - u^2) g g''] / [(1 - u^2) g'^2 + g^2]^(3/2)
        + (u g' + 3 g) / (g [(1 - u^2) g'^2 + g^2]^(1/2))
        + (m-1)(n-1)/((n-m) eps) (1 + cos theta_eq) [(eps/h)^n - (eps/h)^m],

with eps = xi / R0, k = dp R0 / sigma and the height above the substrate
h = u g(u) + g(-1) + delta, holds at every grid point together with eq. bc
and the volume constraint eq. volconstr (integral of g^3 du = 2); the
unknowns are g at the grid points, delta and k.  Second-order finite
differences on a grid uniform in u (at u = +-1 the terms with 1 - u^2
vanish and one-sided first derivatives are used); the volume integral by the
trapezoidal rule; Newton's method with the Jacobian from central
differences, continued from the sphere down to the wanted angle.
"""
from __future__ import annotations

import numpy as np


_COEF = {}


def _coefficients(u):
    """Weights of the three-point second-order formulas on the grid u
    (uniform or not); one-sided for g' at the ends."""
    key = (u.size, float(u[0]), float(u[1]), float(u[-2]), float(u.sum()))
    if key not in _COEF:
        h1, h2 = u[1:-1] - u[:-2], u[2:] - u[1:-1]
        du = (u[-1] - u[0]) / (u.size - 1)
        if np.max(np.abs(np.diff(u) - du)) < 1e-12 * abs(du):
            h1 = h2 = np.full(u.size - 2, du)   # a uniform grid: the symmetric formulas exactly
        d1 = (-h2 / (h1 * (h1 + h2)), (h2 - h1) / (h1 * h2), h1 / (h2 * (h1 + h2)))
        d2 = (2.0 / (h1 * (h1 + h2)), -2.0 / (h1 * h2), 2.0 / (h2 * (h1 + h2)))
        a, b = u[1] - u[0], u[2] - u[1]
        e0 = (-(2 * a + b) / (a * (a + b)), (a + b) / (a * b), -a / (b * (a + b)))
        a, b = u[-1] - u[-2], u[-2] - u[-3]
        e1 = ((2 * a + b) / (a * (a + b)), -(a + b) / (a * b), a / (b * (a + b)))
        if len(_COEF) > 64:
            _COEF.clear()
        _COEF[key] = (d1, d2, e0, e1)
    return _COEF[key]


def _derivs(g, u):
    """First and second derivatives of g(u) on the grid u (the terms with
    1 - u^2 vanish at the ends, where only g' is needed)."""
    d1, d2, e0, e1 = _coefficients(u)
    gd = np.empty_like(g)
    gdd = np.zeros_like(g)
    gd[1:-1] = d1[0] * g[:-2] + d1[1] * g[1:-1] + d1[2] * g[2:]
    gdd[1:-1] = d2[0] * g[:-2] + d2[1] * g[1:-1] + d2[2] * g[2:]
    gd[0] = e0[0] * g[0] + e0[1] * g[1] + e0[2] * g[2]
    gd[-1] = e1[0] * g[-1] + e1[1] * g[-2] + e1[2] * g[-3]
    return gd, gdd


def curvature(g, u):
    """div(n) R0 of the surface r = R0 g(u) (the first two terms of eq. YL)."""
    gd, gdd = _derivs(g, u)
    s = 1.0 - u * u
    Q = np.sqrt(s * gd * gd + g * g)
    return (u * g * gd - g * g - s * g * gdd) / Q ** 3 + (u * gd + 3 * g) / (g * Q)


def wall_term(g, u, delta, eps, theta, n=6, m=3):
    h = u * g + g[0] + delta
    A = (m - 1) * (n - 1) / ((n - m) * eps) * (1.0 + np.cos(theta))
    return A * ((eps / h) ** n - (eps / h) ** m)


def residual(x, u, eps, theta, n=6, m=3, wall=True):
    g, delta, k = x[:-2], x[-2], x[-1]
    r = curvature(g, u) - k
    if wall:
        r = r + wall_term(g, u, delta, eps, theta, n, m)
    vol = np.trapezoid(g ** 3, u) - 2.0
    return np.concatenate([r, [g[-1] - g[0], vol]])


def _jacobian(x, u, eps, theta, n, m):
    """Sparse central-difference Jacobian.  Row i of the grid equations
    depends on g[i-1 .. i+1] (g[0 .. 2] and g[-3 ..] at the ends), on g[0]
    through h, on delta and on k; so the columns of g[1 .. -2] are perturbed
    three at a time (every third one), the volume row is differentiated
    exactly, and the remaining columns one by one."""
    from scipy import sparse
    N = x.size - 2
    rows, cols, vals = [], [], []
    hstep = lambda v: 1e-7 * max(1.0, abs(v))

    def diff(idx):
        xp, xm = x.copy(), x.copy()
        hs = np.array([hstep(x[j]) for j in idx])
        xp[idx] += hs
        xm[idx] -= hs
        return residual(xp, u, eps, theta, n, m) - residual(xm, u, eps, theta, n, m), hs

    for j in (0, N - 1, N, N + 1):            # g(-1), g(1), delta, k: full columns
        d, hs = diff(np.array([j]))
        nz = np.flatnonzero(d[:N])
        rows += list(nz)
        cols += [j] * nz.size
        vals += list(d[nz] / (2 * hs[0]))
    for c in range(3):
        idx = np.arange(1 + c, N - 1, 3)
        d, hs = diff(idx)
        for j, hj in zip(idx, hs):
            rr = {r for r in (j - 1, j, j + 1) if 0 <= r < N}
            if j <= 2:
                rr.add(0)
            if j >= N - 3:
                rr.add(N - 1)
            for r in rr:
                rows.append(r)
                cols.append(j)
                vals.append(d[r] / (2 * hj))
    w = np.empty(N)                             # trapezoid weights on the grid
    w[1:-1] = 0.5 * (u[2:] - u[:-2])
    w[0], w[-1] = 0.5 * (u[1] - u[0]), 0.5 * (u[-1] - u[-2])
    rows += [N + 1] * N                         # volume row: d/dg of trapezoid(g^3)
    cols += list(range(N))
    vals += list(3.0 * x[:N] ** 2 * w)
    rows += [N, N]                              # g(1) - g(-1)
    cols += [0, N - 1]
    vals += [-1.0, 1.0]
    return sparse.csc_matrix((vals, (rows, cols)), shape=(x.size, x.size))


def _newton(x, u, eps, theta, n, m, tol=1e-10, max_iter=60):
    # the residual cannot be evaluated more accurately than rounding over the
    # finest spacing squared (second differences): accept down to that floor
    floor = 100.0 * np.finfo(float).eps / np.min(np.diff(u)) ** 2
    tol = max(tol, floor)
    for _ in range(max_iter):
        F = residual(x, u, eps, theta, n, m)
        if np.max(np.abs(F)) < tol:
            return x, True
        from scipy.sparse.linalg import spsolve
        J = _jacobian(x, u, eps, theta, n, m)
        dx = spsolve(J, -F)
        if np.max(np.abs(dx)) < 1e-13:     # at the round-off floor of the residual
            return x + dx, np.max(np.abs(F)) < max(1e-8, floor)
        # backtracking: heights above the substrate stay positive and the
        # residual norm decreases (Armijo)
        f0 = np.linalg.norm(F)
        lam = 1.0
        while lam > 1e-6:
            xn = x + lam * dx
            if (np.all(u * xn[:-2] + xn[0] + xn[-2] > 0) and np.all(xn[:-2] > 0)
                    and np.linalg.norm(residual(xn, u, eps, theta, n, m)) < (1.0 - 1e-4 * lam) * f0):
                break
            lam *= 0.5
        x = x + lam * dx
    return x, np.max(np.abs(residual(x, u, eps, theta, n, m))) < max(1e-8, floor)


def cap_g(u, theta):
    """Eq. gcap with c from the volume constraint: the spherical cap of angle
    theta, origin at its mid-height (the solution without the wall term)."""
    c2 = np.cos(theta / 2) ** 2
    base = -c2 * u + np.sqrt(1.0 - c2 * c2 * (1.0 - u * u))
    c = (2.0 / np.trapezoid(base ** 3, u)) ** (1.0 / 3.0)
    return c * base, c


def solve(theta, eps, n_grid=401, n=6, m=3, steps=None):
    """Equilibrium profile for contact angle theta (radians) and eps = xi/R0.
    Continuation: from a nearly non-wetting sphere down to theta at
    eps0 = max(eps, 0.1), then down to eps.  Returns (u, g, delta, k)."""
    u = np.linspace(-1.0, 1.0, n_grid)
    eps0 = max(eps, 0.1)
    if steps is None:
        steps = max(4, int(np.ceil((np.pi - theta) / 0.1)))
    x = None
    for th in np.linspace(np.pi - 0.15, theta, steps):
        if x is None:
            g0, c = cap_g(u, th)
            x = np.concatenate([g0, [eps0, 2.0 / c]])
        x, ok = _newton(x, u, eps0, th, n, m)
        if not ok:
            raise RuntimeError(f"no convergence at theta = {th:.4f}")
    e_prev = eps0
    for e in np.geomspace(eps0, eps, max(1, int(np.ceil(20 * np.log10(eps0 / eps)))) + 1)[1:]:
        x = x.copy()
        x[-2] *= e / e_prev                    # the film thickness follows eps
        x, ok = _newton(x, u, e, theta, n, m)
        if not ok:
            raise RuntimeError(f"no convergence at eps = {e:.4g}")
        e_prev = e
    return u, x[:-2], x[-2], x[-1]


def graded_grid(n, uc, beta):
    """n points on [-1, 1] clustered about uc: u = uc + sinh(x) / beta with x
    uniform (spacing about 1 / beta times finer at uc than far from it)."""
    a, b = np.arcsinh((-1.0 - uc) * beta), np.arcsinh((1.0 - uc) * beta)
    u = uc + np.sinh(np.linspace(a, b, n)) / beta
    u[0], u[-1] = -1.0, 1.0
    return u


def _sharpest(u, g):
    _, gdd = _derivs(g, u)
    return u[np.argmax(np.abs(gdd[2:-2])) + 2]


def solve_graded(theta, eps, n_grid=1601, beta=30.0, eps_start=0.05):
    """Like solve, for small eps: solve at eps_start on a uniform grid, then
    continue in eps on a grid graded about the sharpest turn of the profile
    (the contact-line region, whose width shrinks with eps), moving the grid
    with it.  Returns (u, g, delta, k)."""
    u, g, d, k = solve(theta, eps_start, n_grid=min(n_grid, 1601))
    uc = _sharpest(u, g)
    uu = graded_grid(n_grid, uc, beta)
    x = np.concatenate([np.interp(uu, u, g), [d, k]])
    x, ok = _newton(x, uu, eps_start, theta, 6, 3)       # settle on the graded grid first
    if not ok:
        raise RuntimeError(f"no convergence on the graded grid at eps = {eps_start:.4g}")
    e_prev = eps_start
    for e in np.geomspace(eps_start, eps, max(2, int(np.ceil(40 * np.log10(eps_start / eps)))) + 1)[1:]:
        x = x.copy()
        x[-2] *= e / e_prev
        x, ok = _newton(x, uu, e, theta, 6, 3)
        if not ok:
            raise RuntimeError(f"no convergence at eps = {e:.4g}")
        e_prev = e
        uc2 = _sharpest(uu, x[:-2])
        if abs(uc2 - uc) > 0.02:              # the turn moved: regrid about it
            uc, un = uc2, graded_grid(n_grid, uc2, beta)
            x = np.concatenate([np.interp(un, uu, x[:-2]), x[-2:]])
            uu = un
            x, ok = _newton(x, uu, e, theta, 6, 3)
            if not ok:
                raise RuntimeError(f"no convergence after regridding at eps = {e:.4g}")
    return uu, x[:-2], x[-2], x[-1]


def angle_from_height(g):
    """Eq. angleh with the half-height l = (g(1) + g(-1)) / 2 (R0 = 1)."""
    ell = 0.5 * (g[-1] + g[0])
    if ell ** 3 >= 1.0:
        return np.pi
    return 2.0 * np.arctan(np.sqrt(3.0 * ell ** 3 / (1.0 - ell ** 3)))


def profile_phi(u, g, phi):
    """g at polar angles phi (linear in u)."""
    return np.interp(np.cos(phi), u, g)


def centroid_height(u, g):
    """Height of the volume centroid above the origin of r = g(u) (R0 = 1):
    the z-moment of the body, 2 pi int g^4 u du / 4, over its volume,
    2 pi int g^3 du / 3 (trapezoidal in u)."""
    return 0.75 * np.trapezoid(g ** 4 * u, u) / np.trapezoid(g ** 3, u)


def profile_about_centroid(u, g, phi):
    """The surface r = g(u) re-expressed as the distance G(phi) from the
    body's volume centroid at polar angle phi about that point (the form in
    which a simulated profile is measured: node distances from the
    droplet's centroid)."""
    zc = centroid_height(u, g)
    x = g * np.sqrt(np.clip(1.0 - u * u, 0.0, None))
    z = g * u - zc
    r = np.hypot(x, z)
    ph = np.arctan2(x, z)                      # 0 at the top, pi at the bottom
    order = np.argsort(ph)
    return np.interp(phi, ph[order], r[order])


def e_l2(phi, g_sim, g_theo):
    """Eq. L2-error_equilibrium on samples phi (trapezoidal in phi)."""
    return np.sqrt(np.trapezoid((g_sim - g_theo) ** 2, phi) / np.trapezoid(g_theo ** 2, phi))


def film_thickness(eps, k, theta, n=6, m=3):
    """Planar-film gap of App. C for (n, m) = (6, 3): delta =
    eps (2 / (1 + sqrt(1 + 4 beta)))^(1/3), beta = (n-m) eps k /
    ((m-1)(n-1)(1 + cos theta))."""
    assert (n, m) == (6, 3)
    beta = (n - m) * eps * k / ((m - 1) * (n - 1) * (1.0 + np.cos(theta)))
    return eps * (2.0 / (1.0 + np.sqrt(1.0 + 4.0 * beta))) ** (1.0 / 3.0)
