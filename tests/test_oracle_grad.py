"""Pins of the differentiable CPU reference (oracle/grad.py).

It is held to things other than itself: the C oracle's forward (values), the
C oracle's forward again through central finite differences (derivatives),
and the symplectic structure of the step (Mercury-type splittings of Eqs.
Ha-Hc are compositions of Hamiltonian flows, so the Jacobian M of one step in
the canonical pair (x, p = m v) satisfies M^T Omega M = Omega).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad as og  # noqa: E402
from oracle import nbref  # noqa: E402
from paper_2604_09184_b300 import ics  # noqa: E402

G = ics.G_GAUSS


def small_disk(n, seed):
    d = ics.make_disk(n, 2.0, 0.8, 2.5, 0.02, 0.01, 8.0, seed=seed)
    p = nbref.params(dt_rcrit=d.dt)
    rc = np.array([nbref.rcrit(p, d.x[i], d.v[i], d.m[i]) for i in range(n)])
    return d, p, rc


def oracle_final(p, x, v, m, R, rc, steps, dt):
    s = nbref.RefSystem(p, x, v, m, R, rc=rc)
    assert s.step(steps, dt) == 0
    st = s.state()
    assert s.stats()["groups"] == 0
    return st["x"], st["v"]


def test_forward_matches_c_oracle():
    d, p, rc = small_disk(8, 4101)
    steps = 30
    xr, vr = oracle_final(p, d.x, d.v, d.m, d.R, rc, steps, d.dt)
    with torch.no_grad():
        xt, vt = og.integrate(torch.tensor(d.x), torch.tensor(d.v), torch.tensor(d.m),
                              torch.tensor(rc), d.dt, steps)
    ex = np.linalg.norm(xt.numpy() - xr, axis=1) / np.linalg.norm(xr, axis=1)
    ev = np.linalg.norm(vt.numpy() - vr, axis=1) / np.linalg.norm(vr, axis=1)
    assert ex.max() < 1e-13 and ev.max() < 1e-13, (ex.max(), ev.max())


def test_kick_inside_rc_matches_c_oracle():
    """The changeover branch (w = K - r dK/dr < 1) of the reference kick against
    the C oracle's force on a configuration with pairs inside rc."""
    rng = np.random.default_rng(7)
    n = 10
    x = np.column_stack([1.0 + 0.002 * rng.standard_normal(n), 0.002 * rng.standard_normal(n),
                         0.0005 * rng.standard_normal(n)])
    m = 1e-7 * (1 + rng.random(n))
    rc = 0.0015 * (1 + rng.random(n))
    a_ref, pairs = nbref.forces(x, m, rc, G)
    assert len(pairs) > 0
    a, qmin = og.kick_accel(torch.tensor(x), torch.tensor(m), torch.tensor(rc), G)
    assert qmin < 1.0
    err = np.abs(a.detach().numpy() - a_ref).max() / np.abs(a_ref).max()
    assert err < 1e-13, err


def test_gradient_matches_finite_differences_of_c_oracle():
    d, p, rc = small_disk(5, 4102)
    steps = 8
    rng = np.random.default_rng(11)
    gx, gv = rng.standard_normal((5, 3)), rng.standard_normal((5, 3)) * 50.0
    gm = np.zeros(5)
    dx, dv, dm = og.gradient(d.x, d.v, d.m, rc, d.dt, steps, gx, gv, gm)

    def loss(x, v, m):
        xr, vr = oracle_final(p, x, v, m, d.R, rc, steps, d.dt)
        return float((gx * xr).sum() + (gv * vr).sum())

    # masses: a larger relative step keeps the loss change far above its rounding
    for arr, grad, rel in ((d.x, dx, 1e-6), (d.v, dv, 1e-6), (d.m, dm, 1e-3)):
        for idx in np.ndindex(arr.shape):
            h = rel * max(abs(arr[idx]), 1e-3 if arr is not d.m else 1e-12)
            xp = [d.x.copy(), d.v.copy(), d.m.copy()]
            xm = [d.x.copy(), d.v.copy(), d.m.copy()]
            k = 0 if arr is d.x else (1 if arr is d.v else 2)
            xp[k][idx] += h
            xm[k][idx] -= h
            fd = (loss(*xp) - loss(*xm)) / (2 * h)
            scale = np.abs(grad).max()
            assert abs(fd - grad[idx]) <= 2e-6 * scale, (k, idx, fd, grad[idx])


@pytest.mark.parametrize("steps", [1, 4])
def test_step_jacobian_is_symplectic(steps):
    d, p, rc = small_disk(3, 4103)
    m = torch.tensor(d.m)
    rct = torch.tensor(rc)

    def flow(z):
        x = z[:9].reshape(3, 3)
        v = (z[9:].reshape(3, 3)) / m.unsqueeze(-1)
        xT, vT = og.integrate(x, v, m, rct, d.dt, steps)
        return torch.cat([xT.reshape(-1), (m.unsqueeze(-1) * vT).reshape(-1)])

    z0 = torch.cat([torch.tensor(d.x).reshape(-1), (m.unsqueeze(-1) *
                                                     torch.tensor(d.v)).reshape(-1)])
    M = torch.autograd.functional.jacobian(flow, z0).numpy()
    Om = np.zeros((18, 18))
    Om[:9, 9:] = np.eye(9)
    Om[9:, :9] = -np.eye(9)
    # every entry of M^T Omega M - Omega against the size of the terms that
    # cancel in it (|M|^T |Omega| |M|): rounding leaves ~1e-16 of that scale
    resid = M.T @ Om @ M - Om
    scale = np.abs(M).T @ np.abs(Om) @ np.abs(M)
    assert np.max(np.abs(resid) / scale) <= 1e-12
    # the check is not vacuous: M is far from the identity (x depends on p / m)
    assert np.abs(M - np.eye(18)).max() > 1e3


def _energy_system(seed, n=6):
    """Bodies with a sizeable net momentum (so the Eq. Hc term matters)."""
    rng = np.random.default_rng(seed)
    m = np.array([1e-3, 3e-4, 5e-5, 2e-6, 7e-7, 4e-8, 1e-9, 2e-9][:n])
    r = rng.uniform(0.7, 6.0, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    x = np.stack([r * np.cos(ph), r * np.sin(ph), rng.normal(0, 0.05, n)], 1)
    vk = np.sqrt(G / r)
    v = np.stack([-vk * np.sin(ph), vk * np.cos(ph), np.zeros(n)], 1) + rng.normal(0, 2e-3, (n, 3))
    return x, v, m


def _c_energy(x, v, m):
    s = nbref.RefSystem(nbref.params(merge=0), x, v, m, np.full(len(m), 1e-6))
    return s.energy_momentum()["E"]


@pytest.mark.parametrize("seed", [11, 12])
def test_energy_matches_c_oracle_and_its_gradient_central_differences(seed):
    """og.energy equals the C oracle's E (pinned to the inertial-frame
    Newtonian energy) and its autograd gradient equals central differences of
    the C oracle's E in every coordinate, velocity and mass."""
    x, v, m = _energy_system(seed)
    xt, vt, mt = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in (x, v, m))
    E = og.energy(xt, vt, mt)
    Ec = _c_energy(x, v, m)
    assert abs(E.item() - Ec) <= 1e-14 * abs(Ec)
    gx, gv, gm = torch.autograd.grad(E, (xt, vt, mt))
    for arr, g, rel in ((x, gx, 1e-6), (v, gv, 1e-6), (m, gm, 1e-6)):
        flat = arr.reshape(-1)
        for k in range(flat.size):
            h = rel * max(abs(flat[k]), 1e-3 if arr is not m else 1e-12)
            up = [a.copy() for a in (x, v, m)]
            dn = [a.copy() for a in (x, v, m)]
            which = 0 if arr is x else (1 if arr is v else 2)
            up[which].reshape(-1)[k] += h
            dn[which].reshape(-1)[k] -= h
            fd = (_c_energy(*up) - _c_energy(*dn)) / (2 * h)
            ad = g.reshape(-1)[k].item()
            # truncation O(h^2) plus the rounding noise of E itself over 2h
            noise = 64 * np.spacing(abs(Ec)) / (2 * h)
            assert abs(fd - ad) <= 2e-6 * abs(ad) + noise, (which, k, fd, ad, noise)
