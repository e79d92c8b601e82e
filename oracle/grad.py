"""Differentiable CPU reference of the integrator step (test infrastructure only).

Only the tests may import this module; the product path never does. It
restates, in plain PyTorch float64 on the CPU, the step of the hybrid
symplectic method for a system with no close encounters, so that
``torch.autograd`` gives the exact derivative of the discrete map and serves
as the reference for the library's adjoint kernels.

The step is B(h/2) C(h/2) A(h) C(h/2) B(h/2) (Eq. H with the splitting of
Eqs. Ha, Hb, Hc):

* B, the interaction kick of Eq. Hb: v_i += (h/2) G sum_j m_j w(r_ij) (x_j - x_i) / r_ij^3
  with w = K - r dK/dr, K the changeover function (1 beyond rc);
* C, the drift of Eq. Hc: x_i += (h/2) P / m0 with P = sum_j m_j v_j;
* A, the Kepler part of Eq. Ha: each body moves on its two-body orbit about
  mu = G m0 (Gauss f and g functions of the universal anomaly s).

The method only sends bodies to the direct solver when a pair comes within
its critical radius; ``step`` refuses such a state (RuntimeError), so the map
it differentiates is the whole step. Not pinned by itself: the tests pin it
against central finite differences of the C oracle's forward and against the
symplectic structure of the step's Jacobian.
"""
from __future__ import annotations

import torch

G_GAUSS = 2.959122082855911e-4


def changeover(r, rc):
    """K(r) of the changeover (the paragraph after Eq. Hc) in the infinitely
    smooth reading: y = (r - 0.1 rc) / (0.9 rc), K = f(y) / (f(y) + f(1 - y)),
    f(y) = exp(-1/y) for y > 0 and 0 otherwise."""
    y = (r - 0.1 * rc) / (0.9 * rc)
    yc = y.clamp(1e-300, 1.0 - 1e-16)
    f = torch.where(y > 0, torch.exp(-1.0 / yc), torch.zeros_like(y))
    g = torch.where(y < 1, torch.exp(-1.0 / (1.0 - yc)), torch.zeros_like(y))
    return f / (f + g)


def kick_accel(x, m, rc, G=G_GAUSS):
    """Acceleration of Eq. Hb: a_i = G sum_{j != i} m_j w_ij (x_j - x_i) / r_ij^3,
    w = K - r dK/dr with rc_ij = max(rc_i, rc_j). Also returns the smallest
    r_ij^2 / rc_ij^2 (below 1: a close encounter)."""
    n = x.shape[0]
    d = x.unsqueeze(0) - x.unsqueeze(1)  # d[i, j] = x_j - x_i
    r2 = (d * d).sum(-1)
    eye = torch.eye(n, dtype=torch.bool)
    r2s = torch.where(eye, torch.ones_like(r2), r2)
    r = torch.sqrt(r2s)
    rcij = torch.maximum(rc.unsqueeze(0), rc.unsqueeze(1))
    inside = r < rcij
    # w = K - r dK/dr; dK/dr by autograd of K along r only where it matters
    if bool(inside.any()):
        rr = r.detach().requires_grad_(True)
        K = changeover(rr, rcij)
        (dK,) = torch.autograd.grad(K.sum(), rr, create_graph=True)
        w_in = changeover(r, rcij) - r * dK
        w = torch.where(inside, w_in, torch.ones_like(r))
    else:
        w = torch.ones_like(r)
    coef = G * m.unsqueeze(0) * w / (r2s * r)
    coef = torch.where(eye, torch.zeros_like(coef), coef)
    a = (coef.unsqueeze(-1) * d).sum(1)
    ratio = torch.where(eye, torch.full_like(r2, float("inf")), r2 / (rcij * rcij))
    return a, float(ratio.detach().min())


def energy(x, v, m, m0=1.0, G=G_GAUSS):
    """Total energy E = H_A + H_B + H_C of Eqs. Ha-Hc: the changeover K
    cancels between the close part of H_A and H_B, so
    E = sum m v^2 / 2 - sum G m0 m / |x| - sum_{i<j} G m_i m_j / r_ij
        + |sum m v|^2 / (2 m0).
    x, v (n, 3) heliocentric positions and barycentric velocities, m (n,)
    (absorbed bodies are left out by the caller). Differentiable by autograd."""
    n = x.shape[0]
    kin = 0.5 * (m * (v * v).sum(1)).sum()
    star = -(G * m0 * m / torch.sqrt((x * x).sum(1))).sum()
    d = x.unsqueeze(0) - x.unsqueeze(1)
    iu = torch.triu_indices(n, n, 1)
    r = torch.sqrt((d[iu[0], iu[1]] ** 2).sum(-1))
    pair = -(G * m[iu[0]] * m[iu[1]] / r).sum()
    P = (m.unsqueeze(1) * v).sum(0)
    return kin + star + pair + (P * P).sum() / (2.0 * m0)


def stumpff(z):
    """Stumpff functions c0..c3 of z (elementwise): the power series of c2 and
    c3 at |z| / 4^q <= 0.1, c0 = 1 - z c2, c1 = 1 - z c3 there, and q
    applications of the argument-quadrupling identities."""
    q = torch.zeros_like(z, dtype=torch.long)
    za = z.detach().abs()
    while bool((za / 4.0 ** q > 0.1).any()):
        q = q + (za / 4.0 ** q > 0.1).long()
    zs = z / (4.0 ** q).to(z.dtype)
    c2 = torch.zeros_like(zs)
    c3 = torch.zeros_like(zs)
    term2, term3 = torch.ones_like(zs) / 2.0, torch.ones_like(zs) / 6.0
    for k in range(12):
        c2 = c2 + term2
        c3 = c3 + term3
        term2 = term2 * (-zs) / ((2 * k + 3) * (2 * k + 4))
        term3 = term3 * (-zs) / ((2 * k + 4) * (2 * k + 5))
    c0 = 1.0 - zs * c2
    c1 = 1.0 - zs * c3
    for level in range(int(q.max()) if q.numel() else 0):
        act = q > level
        n0 = 2.0 * c0 * c0 - 1.0
        n1 = c0 * c1
        n2 = 0.5 * c1 * c1
        n3 = 0.25 * (c2 + c0 * c3)
        c0 = torch.where(act, n0, c0)
        c1 = torch.where(act, n1, c1)
        c2 = torch.where(act, n2, c2)
        c3 = torch.where(act, n3, c3)
    return c0, c1, c2, c3


def kepler(x, v, h, mu):
    """Two-body drift of Eq. Ha's first sum by h for every body: universal
    Kepler equation r0 G1 + eta G2 + mu G3 = h in s (G_k = s^k c_k(beta s^2),
    beta = 2 mu / r0 - v^2, eta = x . v), solved by Newton's method on
    detached values; one Newton update on the attached graph then carries the
    implicit derivative ds = -F_p / F_s. Gauss f, g, fdot, gdot give x', v'."""
    r0 = torch.sqrt((x * x).sum(-1))
    eta = (x * v).sum(-1)
    beta = 2.0 * mu / r0 - (v * v).sum(-1)

    def F(s, r0, eta, beta):
        c0, c1, c2, c3 = stumpff(beta * s * s)
        G1, G2, G3 = s * c1, s * s * c2, s * s * s * c3
        return r0 * G1 + eta * G2 + mu * G3 - h, r0 * c0 + eta * G1 + mu * G2

    with torch.no_grad():
        s = torch.full_like(r0, h) / r0
        for _ in range(40):
            f, fp = F(s, r0, eta, beta)
            ds = f / fp
            s = s - ds
        if not bool((ds.abs() <= 1e-13 * s.abs()).all()):
            raise RuntimeError("Kepler solve did not converge")
    s = s.detach()
    f, fp = F(s, r0, eta, beta)
    s = s - f / fp.detach() + (f / fp.detach()).detach()  # value s, derivative -F_p / F_s
    c0, c1, c2, c3 = stumpff(beta * s * s)
    G1, G2 = s * c1, s * s * c2
    r = r0 * c0 + eta * G1 + mu * G2
    fm = 1.0 - mu * G2 / r0
    gg = r0 * G1 + eta * G2
    fd = -mu * G1 / (r * r0)
    gd = 1.0 - mu * G2 / r
    xn = fm.unsqueeze(-1) * x + gg.unsqueeze(-1) * v
    vn = fd.unsqueeze(-1) * x + gd.unsqueeze(-1) * v
    return xn, vn


def step(x, v, m, rc, h, m0=1.0, G=G_GAUSS):
    """One step B(h/2) C(h/2) A(h) C(h/2) B(h/2) with the kick of Eq. Hb
    evaluated at the step's start and end positions. Raises RuntimeError if
    any pair is inside its critical radius at the trial (post-drift) or start
    positions, i.e. if the method would use its direct solver."""
    mu = G * m0
    a, q0 = kick_accel(x, m, rc, G)
    v = v + 0.5 * h * a
    x = x + 0.5 * h * (m.unsqueeze(-1) * v).sum(0) / m0
    x, v = kepler(x, v, h, mu)
    a, q1 = kick_accel(x, m, rc, G)
    if min(q0, q1) < 1.0:
        raise RuntimeError("close encounter: the reference covers encounter-free steps only")
    x = x + 0.5 * h * (m.unsqueeze(-1) * v).sum(0) / m0
    v = v + 0.5 * h * a
    return x, v


def integrate(x, v, m, rc, h, nsteps, m0=1.0, G=G_GAUSS):
    for _ in range(nsteps):
        x, v = step(x, v, m, rc, h, m0, G)
    return x, v


def gradient(x0, v0, m0_bodies, rc, h, nsteps, gx, gv, gm, m0=1.0, G=G_GAUSS):
    """Gradient of L = <gx, x_T> + <gv, v_T> + <gm, m_T> with respect to
    (x_0, v_0, m_0) by reverse-mode automatic differentiation of ``integrate``.
    Masses are constant without mergers, so m_T = m_0."""
    x = torch.tensor(x0, dtype=torch.float64, requires_grad=True)
    v = torch.tensor(v0, dtype=torch.float64, requires_grad=True)
    m = torch.tensor(m0_bodies, dtype=torch.float64, requires_grad=True)
    rct = torch.tensor(rc, dtype=torch.float64)
    xT, vT = integrate(x, v, m, rct, h, nsteps, m0, G)
    L = (xT * torch.as_tensor(gx)).sum() + (vT * torch.as_tensor(gv)).sum() + (
        m * torch.as_tensor(gm)).sum()
    L.backward()
    return x.grad.numpy(), v.grad.numpy(), m.grad.numpy()
