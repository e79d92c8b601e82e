"""Independent reference mathematics for the tests (mpmath / long double).

Closed-form two-body propagation through orbital elements (Kepler's equation
in its elliptic and hyperbolic forms) and a long-double classical RK4. None of
this is taken from the oracle or the CUDA library.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

mp.mp.dps = 40


def _vec(a):
    return [mp.mpf(float(t)) for t in a]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _norm(a):
    return mp.sqrt(_dot(a, a))


def propagate_two_body(mu, x0, v0, t):
    """State after time t on the conic through (x0, v0) about mass parameter mu.

    Elliptic (E - e sin E = M) or hyperbolic (e sinh H - H = M) Kepler
    equation solved in 40-digit arithmetic. Returns float64 arrays.
    """
    mu = mp.mpf(float(mu))
    t = mp.mpf(float(t))
    x = _vec(x0)
    v = _vec(v0)
    r = _norm(x)
    v2 = _dot(v, v)
    hvec = _cross(x, v)
    hn = _norm(hvec)
    eps = v2 / 2 - mu / r
    vxh = _cross(v, hvec)
    evec = [vxh[k] / mu - x[k] / r for k in range(3)]
    e = _norm(evec)
    rv = _dot(x, v)
    Pq = [evec[k] / e for k in range(3)]
    hh = [hvec[k] / hn for k in range(3)]
    Qq = _cross(hh, Pq)
    if eps < 0:
        a = -mu / (2 * eps)
        n = mp.sqrt(mu / a ** 3)
        cE = (1 - r / a) / e
        sE = rv / (e * mp.sqrt(mu * a))
        E0 = mp.atan2(sE, cE)
        M = E0 - e * mp.sin(E0) + n * t
        E = mp.findroot(lambda E_: E_ - e * mp.sin(E_) - M, M)
        b = mp.sqrt(1 - e * e)
        xp = a * (mp.cos(E) - e)
        yp = a * b * mp.sin(E)
        rr = a * (1 - e * mp.cos(E))
        vxp = -mp.sqrt(mu * a) / rr * mp.sin(E)
        vyp = mp.sqrt(mu * a) / rr * b * mp.cos(E)
    else:
        A = mu / (2 * eps)
        n = mp.sqrt(mu / A ** 3)
        chH = (1 + r / A) / e
        shH = rv / (e * mp.sqrt(mu * A))
        H0 = mp.asinh(shH)
        M = e * mp.sinh(H0) - H0 + n * t
        H = mp.findroot(lambda H_: e * mp.sinh(H_) - H_ - M, mp.asinh(M / e))
        b = mp.sqrt(e * e - 1)
        xp = A * (e - mp.cosh(H))
        yp = A * b * mp.sinh(H)
        rr = A * (e * mp.cosh(H) - 1)
        vxp = -mp.sqrt(mu * A) / rr * mp.sinh(H)
        vyp = mp.sqrt(mu * A) / rr * b * mp.cosh(H)
    xo = np.array([float(xp * Pq[k] + yp * Qq[k]) for k in range(3)])
    vo = np.array([float(vxp * Pq[k] + vyp * Qq[k]) for k in range(3)])
    return xo, vo


def stumpff_mp(z, k):
    """c_k(z) in closed form at 40 digits."""
    z = mp.mpf(float(z))
    if z == 0:
        return 1.0 / float(mp.factorial(k))
    if z > 0:
        u = mp.sqrt(z)
        c = [mp.cos(u), mp.sin(u) / u, (1 - mp.cos(u)) / z, (u - mp.sin(u)) / (u * z)][k]
    else:
        u = mp.sqrt(-z)
        c = [mp.cosh(u), mp.sinh(u) / u, (mp.cosh(u) - 1) / (-z), (mp.sinh(u) - u) / (u * (-z))][k]
    return float(c)


def rk4_longdouble(deriv, y0, T, nsteps):
    """Classical fourth-order Runge-Kutta in numpy long double."""
    y = np.array(y0, dtype=np.longdouble)
    h = np.longdouble(T) / nsteps
    half = np.longdouble(0.5)
    six = np.longdouble(6)
    for _ in range(nsteps):
        k1 = deriv(y)
        k2 = deriv(y + half * h * k1)
        k3 = deriv(y + half * h * k2)
        k4 = deriv(y + h * k3)
        y = y + h / six * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def newton_barycentric_deriv(G, masses):
    """Right-hand side of the full Newtonian (N+1)-body problem in an inertial
    frame; state [x (n,3), v (n,3)] flattened, long double."""
    ms = np.asarray(masses, dtype=np.longdouble)
    n = ms.shape[0]
    Gl = np.longdouble(G)

    def f(y):
        x = y[: 3 * n].reshape(n, 3)
        v = y[3 * n:].reshape(n, 3)
        d = x[None, :, :] - x[:, None, :]          # d[i, j] = x_j - x_i
        r2 = (d * d).sum(-1)
        np.fill_diagonal(r2, 1)
        inv3 = 1 / (r2 * np.sqrt(r2))
        np.fill_diagonal(inv3, 0)
        a = Gl * (ms[None, :, None] * d * inv3[:, :, None]).sum(1)
        return np.concatenate([v.reshape(-1), a.reshape(-1)])

    return f
