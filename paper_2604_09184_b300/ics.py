"""Seeded synthetic planetesimal disks (the inputs of every test and benchmark).

This module only draws initial conditions; it holds none of the integrator's
arithmetic, so both the CUDA library and the CPU oracle can be fed from it.

The workloads follow the paper's disks (section "The GENGA code" and the
three studies of section "New results from GPU N-body simulations"):
equal-mass planetesimals around a solar-mass star, a minimum-mass-solar-nebula
surface density Sigma ~ a^-1.5 (so dN/da ~ a^-0.5), nearly circular and
coplanar orbits, optionally Jupiter and Saturn analogues.

Units: AU, day, solar mass. Positions are heliocentric, velocities
barycentric (democratic heliocentric coordinates).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G_GAUSS = 2.959122082855911e-4          # k^2, k = 0.01720209895 (AU^3 Msun^-1 day^-2)
M_EARTH = 1.0 / 332946.0487             # Msun
M_JUPITER = 1.0 / 1047.3486
M_SATURN = 1.0 / 3497.898
MSUN_G = 1.98847e33                     # g
AU_CM = 1.495978707e13                  # cm
R_JUPITER = 7.1492e9 / AU_CM            # AU
R_SATURN = 6.0268e9 / AU_CM             # AU
SEED_BASE = 2604_09184


@dataclasses.dataclass
class Disk:
    x: np.ndarray      # (n, 3) heliocentric positions, AU
    v: np.ndarray      # (n, 3) barycentric velocities, AU/day
    m: np.ndarray      # (n,) masses, Msun
    R: np.ndarray      # (n,) physical radii, AU
    dt: float          # nominal time step, day
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def _radius(m, rho=2.0, f=1.0):
    """Radius of a sphere of mass m (Msun) and bulk density rho (g/cm^3), times f."""
    return f * np.cbrt(3.0 * m * MSUN_G / (4.0 * math.pi * rho)) / AU_CM


def _kepler_E(M, e):
    """Eccentric anomaly from mean anomaly (elliptic), vectorised Newton."""
    E = M + e * np.sin(M)
    for _ in range(50):
        d = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - d
        if np.all(np.abs(d) < 1e-15):
            break
    return E


def elements_to_state(mu, a, e, inc, Om, om, M):
    """Heliocentric position and velocity of elliptic orbits."""
    E = _kepler_E(M, e)
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = a * b * sE
    n = np.sqrt(mu / a ** 3)
    rr = a * (1.0 - e * cE)
    vxp = -a * n * sE / (rr / a)
    vyp = a * n * b * cE / (rr / a)
    cO, sO, co, so, ci, si = np.cos(Om), np.sin(Om), np.cos(om), np.sin(om), np.cos(inc), np.sin(inc)
    P = np.stack([cO * co - sO * so * ci, sO * co + cO * so * ci, so * si], axis=-1)
    Q = np.stack([-cO * so - sO * co * ci, -sO * so + cO * co * ci, co * si], axis=-1)
    x = xp[:, None] * P + yp[:, None] * Q
    v = vxp[:, None] * P + vyp[:, None] * Q
    return x, v


def _to_barycentric(vhel, m, m0):
    return vhel - (m[:, None] * vhel).sum(0) / (m0 + m.sum())


def planetesimal_disk(rng, n, m_total, a_min, a_max, sig_e, sig_i, m0=1.0, rho=2.0,
                      f_radius=1.0):
    """Elements of n equal-mass planetesimals with dN/da ~ a^-0.5 on [a_min, a_max]."""
    u = rng.random(n)
    a = (math.sqrt(a_min) + u * (math.sqrt(a_max) - math.sqrt(a_min))) ** 2
    e = np.minimum(rng.rayleigh(sig_e, n), 0.9)
    inc = rng.rayleigh(sig_i, n)
    Om = rng.random(n) * 2 * math.pi
    om = rng.random(n) * 2 * math.pi
    M = rng.random(n) * 2 * math.pi
    m = np.full(n, m_total / n)
    return dict(a=a, e=e, inc=inc, Om=Om, om=om, M=M, m=m, R=_radius(m, rho, f_radius))


def make_disk(n, m_total_earth, a_min, a_max, sig_e, sig_i, dt, seed, giants=(),
              m0=1.0, f_radius=1.0, name="") -> Disk:
    """A planetesimal disk plus optional giant planets ('J', 'S'), giants first."""
    rng = np.random.Generator(np.random.PCG64(seed))
    els = []
    for g in giants:
        a, e, mg, Rg = {"J": (5.2, 0.048, M_JUPITER, R_JUPITER),
                        "S": (9.58, 0.056, M_SATURN, R_SATURN)}[g]
        ang = rng.random(3) * 2 * math.pi
        els.append(dict(a=np.array([a]), e=np.array([e]), inc=np.array([0.0]),
                        Om=ang[:1], om=ang[1:2], M=ang[2:], m=np.array([mg]),
                        R=np.array([Rg])))
    if n > 0:
        els.append(planetesimal_disk(rng, n, m_total_earth * M_EARTH, a_min, a_max, sig_e,
                                     sig_i, m0=m0, f_radius=f_radius))
    cat = {k: np.concatenate([d[k] for d in els]) for k in els[0]}
    mu = G_GAUSS * (m0 + cat["m"])
    x, vh = elements_to_state(mu, cat["a"], cat["e"], cat["inc"], cat["Om"], cat["om"], cat["M"])
    v = _to_barycentric(vh, cat["m"], m0)
    return Disk(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v),
                m=np.ascontiguousarray(cat["m"]), R=np.ascontiguousarray(cat["R"]), dt=dt,
                name=name)


# ---------------------------------------------------------------------------
# The five workloads (sizes, time steps and step counts).
# ---------------------------------------------------------------------------
TOY_DISK = dict(n=256, m_total_earth=2.0, a_min=0.7, a_max=1.3, sig_e=0.01, sig_i=0.005,
                dt=6.0, steps=1000)
MMSN_16K = dict(n=16384, m_total_earth=5.0, a_min=0.5, a_max=4.0, sig_e=0.01, sig_i=0.005,
                dt=6.0, steps=10_000, giants=("J", "S"))
MMSN_64K = dict(n=65536, m_total_earth=5.0, a_min=0.5, a_max=4.0, sig_e=0.01, sig_i=0.005,
                dt=6.0, steps=1000, giants=("J", "S"))
ADJOINT_2K = dict(n=2048, m_total_earth=1.0, a_min=0.7, a_max=1.3, sig_e=0.01, sig_i=0.005,
                  dt=6.0, steps=2000, giants=("J",))
WORKLOADS = {"toy_disk_256": (0, TOY_DISK), "mmsn_16k_js": (1, MMSN_16K),
             "mmsn_64k_js": (2, MMSN_64K), "adjoint_2k_j": (4, ADJOINT_2K)}


def workload(name: str, n: int | None = None, f_radius: float = 1.0, seed_offset: int = 0) -> Disk:
    """One of the named workloads; n overrides the planetesimal count (small cases)."""
    idx, cfg = WORKLOADS[name]
    cfg = dict(cfg)
    cfg.pop("steps")
    if n is not None:
        cfg["n"] = n
    return make_disk(seed=SEED_BASE + idx + seed_offset, f_radius=f_radius, name=name, **cfg)


def ensemble(n_systems=4096, n_lo=16, n_hi=512, seed=SEED_BASE + 3, m0=1.0):
    """Independent systems for the batched mode: N log-uniform in [n_lo, n_hi],
    total mass uniform in [0.5, 5] Earth masses, a on [0.5, 2] AU,
    e and i Rayleigh(0.02, 0.01), dt = 3 days."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi + 1), n_systems))).astype(int)
    ns = np.clip(ns, n_lo, n_hi)
    mt = rng.uniform(0.5, 5.0, n_systems)
    disks = []
    for k in range(n_systems):
        sub = int(rng.integers(0, 2**62))
        disks.append(make_disk(int(ns[k]), float(mt[k]), 0.5, 2.0, 0.02, 0.01, 3.0, seed=sub,
                               m0=m0, name="ensemble"))
    return disks
