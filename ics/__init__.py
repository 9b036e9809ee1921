"""Seeded synthetic particle sets for the tree-method workloads.

This module only draws inputs: it holds none of the tree method's arithmetic,
and both the oracle tests and the CUDA path take their particles from it.
Random numbers come from numpy's counter-based Philox generator keyed by the
seed, so a (model, N, seed) triple always gives the same particles.

Models (G = 1 throughout, equal particle masses m = M/N):

* ``plummer``   Plummer (1911) sphere, total mass 1, scale radius 1. Radii by
                inverting M(<r) = r^3 / (1 + r^2)^(3/2) at a uniform mass
                fraction X in [0, 0.999) (the 0.1% outermost mass is dropped,
                as in Aarseth, Henon & Wielen 1974); speeds by von Neumann
                rejection from g(q) = q^2 (1 - q^2)^(7/2), q = v / v_esc;
                isotropic directions. Virial ratio 0.5; ``virial`` rescales
                velocities to Q = K/|W| using the analytic W = -3 pi / 32.
* ``uniform_sphere``  cold uniform sphere of radius 1 (the workload the paper
                measures on, Section 6.1).
* ``galaxy``    Hernquist (1990) halo (mass fraction 0.8, scale 1, truncated at
                r = 100) plus an exponential disk (mass fraction 0.2, scale
                length 0.1, sech^2 scale height 0.01), equal particle masses.
                Halo velocities are isotropic Gaussian with sigma = v_c / sqrt(3);
                disk particles move on circular orbits from the enclosed mass
                plus a 10% isotropic dispersion (velocities are only used to
                drift particles; one force evaluation does not depend on them).
* ``batch``     several independent Plummer spheres with N log-uniform in
                [2^lo, 2^hi] and virial ratio uniform in [q_lo, q_hi],
                seeds base+k.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Particles:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def pos(self):
        return self.x, self.y, self.z

    def vel(self):
        return self.vx, self.vy, self.vz


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _isotropic(g: np.random.Generator, n: int):
    cos_t = g.uniform(-1.0, 1.0, n)
    phi = g.uniform(0.0, 2.0 * np.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t


def plummer(n: int, seed: int, virial: float | None = None, x_max: float = 0.999) -> Particles:
    g = rng(seed)
    X = g.uniform(0.0, x_max, n)
    X = np.maximum(X, 1e-300)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    ux, uy, uz = _isotropic(g, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = g.uniform(0.0, 1.0, todo.size)
        yy = g.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    v = q * np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    wx, wy, wz = _isotropic(g, n)
    if virial is not None:
        v = v * np.sqrt(virial / 0.5)
    m = np.full(n, 1.0 / n)
    return Particles(r * ux, r * uy, r * uz, v * wx, v * wy, v * wz, m)


def uniform_sphere(n: int, seed: int) -> Particles:
    g = rng(seed)
    r = g.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    ux, uy, uz = _isotropic(g, n)
    z0 = np.zeros(n)
    return Particles(r * ux, r * uy, r * uz, z0, z0.copy(), z0.copy(), np.full(n, 1.0 / n))


def _exp_disk_radius(u: np.ndarray, rd: float) -> np.ndarray:
    """Invert M(<R)/M = 1 - (1 + R/rd) exp(-R/rd) by bisection."""
    lo = np.zeros_like(u)
    hi = np.full_like(u, 60.0)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        f = 1.0 - (1.0 + mid) * np.exp(-mid)
        lo = np.where(f < u, mid, lo)
        hi = np.where(f < u, hi, mid)
    return 0.5 * (lo + hi) * rd


def galaxy(n: int, seed: int, halo_frac: float = 0.8, a: float = 1.0, r_trunc: float = 100.0,
           rd: float = 0.1, zd: float = 0.01) -> Particles:
    g = rng(seed)
    nh = int(round(n * halo_frac))
    nd = n - nh
    m_part = 1.0 / n
    mh_tot = nh * m_part
    md_tot = nd * m_part
    # Hernquist halo: M(<r)/M = (r / (r + a))^2, truncated at r_trunc.
    xmax = (r_trunc / (r_trunc + a)) ** 2
    X = g.uniform(0.0, xmax, nh)
    sx = np.sqrt(X)
    rh = a * sx / (1.0 - sx)
    ux, uy, uz = _isotropic(g, nh)
    # Disk: exponential in R, sech^2 in z.
    Rd = _exp_disk_radius(g.uniform(0.0, 0.999, nd), rd)
    ph = g.uniform(0.0, 2.0 * np.pi, nd)
    zz = zd * np.arctanh(np.clip(2.0 * g.uniform(0.0, 1.0, nd) - 1.0, -0.999999, 0.999999))

    def m_enc(r):
        mh = mh_tot * np.minimum((r / (r + a)) ** 2 / xmax, 1.0)
        x = r / rd
        md = md_tot * np.minimum((1.0 - (1.0 + x) * np.exp(-x)) / 0.999, 1.0)
        return mh + md

    vch = np.sqrt(m_enc(rh) / np.maximum(rh, 1e-6))
    sig = vch / np.sqrt(3.0)
    vhx, vhy, vhz = (g.normal(0.0, 1.0, nh) * sig for _ in range(3))
    vcd = np.sqrt(m_enc(Rd) / np.maximum(Rd, 1e-6))
    vdx = -vcd * np.sin(ph) + 0.1 * vcd * g.normal(0.0, 1.0, nd)
    vdy = vcd * np.cos(ph) + 0.1 * vcd * g.normal(0.0, 1.0, nd)
    vdz = 0.1 * vcd * g.normal(0.0, 1.0, nd)
    x = np.concatenate([rh * ux, Rd * np.cos(ph)])
    y = np.concatenate([rh * uy, Rd * np.sin(ph)])
    z = np.concatenate([rh * uz, zz])
    vx = np.concatenate([vhx, vdx])
    vy = np.concatenate([vhy, vdy])
    vz = np.concatenate([vhz, vdz])
    return Particles(x, y, z, vx, vy, vz, np.full(n, m_part))


def batch(n_systems: int = 32, seed_base: int = 100, log2_lo: float = 12.0,
          log2_hi: float = 20.0, q_lo: float = 0.3, q_hi: float = 0.7):
    """Independent Plummer spheres of uneven size. Returns a list of
    (Particles, virial ratio) and the per-system sizes."""
    g = rng(seed_base)
    sizes = np.rint(2.0 ** g.uniform(log2_lo, log2_hi, n_systems)).astype(np.int64)
    qs = g.uniform(q_lo, q_hi, n_systems)
    systems = [plummer(int(sizes[k]), seed_base + k, virial=float(qs[k])) for k in range(n_systems)]
    return systems, sizes, qs


# Named workloads: the sizes and parameters the tree method is run on.
WORKLOADS = {
    "plummer_16k": dict(model="plummer", n=16384, seed=1, eps=1.0 / 256, theta=0.5, n_grp=64,
                        quad=False),
    "plummer_1m": dict(model="plummer", n=1 << 20, seed=2, eps=1.0 / 1024, theta=0.5, n_grp=256,
                       quad=False, n_reuse=4, dt=1.0 / 256),
    "galaxy_8m": dict(model="galaxy", n=1 << 23, seed=3, eps=1.0 / 2048, theta=0.4, n_grp=512,
                      quad=True),
    "plummer_4m_mixed": dict(model="plummer", n=1 << 22, seed=4, eps=1.0 / 1024, theta=0.6,
                             n_grp=256, quad=True),
    "uniform_4m": dict(model="uniform_sphere", n=1 << 22, seed=5, eps=1.0 / 1024, theta=0.5,
                       n_grp=256, quad=False),
    # 32 Plummer systems, N log-uniform in [2^12, 2^20], virial ratio in [0.3, 0.7]
    "batch32": dict(model="batch", n=None, seed=100, eps=1.0 / 512, theta=0.5, n_grp=64,
                    quad=False, n_systems=32),
}


def make_batch(n_systems: int = 32, seed_base: int = 100):
    """Concatenated particles of ``batch`` and the system offsets."""
    systems, sizes, qs = batch(n_systems, seed_base)
    cat = Particles(*(np.concatenate([getattr(p, a) for p in systems])
                      for a in ("x", "y", "z", "vx", "vy", "vz", "m")))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return cat, off, qs


def plummer_search_radii(p: Particles, n_nb: float) -> np.ndarray:
    """Search radii for a Plummer sphere of scale radius 1: h_i such that a
    sphere of radius h_i around particle i holds n_nb particles on average
    under the analytic number density N (3 / 4 pi) (1 + r^2)^(-5/2), i.e.
    h_i = (n_nb / N)^(1/3) (1 + r_i^2)^(5/6). Input generation only."""
    r2 = p.x * p.x + p.y * p.y + p.z * p.z
    return (n_nb / p.n) ** (1.0 / 3.0) * (1.0 + r2) ** (5.0 / 6.0)


def make(model: str, n: int, seed: int) -> Particles:
    if model == "plummer":
        return plummer(n, seed)
    if model == "uniform_sphere":
        return uniform_sphere(n, seed)
    if model == "galaxy":
        return galaxy(n, seed)
    raise KeyError(model)
