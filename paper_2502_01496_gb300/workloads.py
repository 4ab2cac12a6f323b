"""Seeded synthetic particle sets for the force evaluation.

This module only draws inputs: positions, masses, smoothing lengths and the
per-system parameters of a batch.  It holds none of the method's arithmetic and
is shared by the tests, the benchmark and the smoke check; the oracle receives
plain arrays and never imports it.

Recipes (units G = 1, Sec. 2 Eq. 1):
  * ``plummer``   -- Plummer sphere, scale radius b, total mass M, equal masses;
                     r = b / sqrt(X^(-2/3) - 1), X ~ U(0, 0.999), isotropic.
  * ``polytrope_binary`` -- two n = 1 polytropes (the paper's neutron-star model,
                     Sec. 6), each built from a jittered cubic lattice cut to a
                     ball and stretch-mapped radially so that the enclosed mass
                     fraction (sin xi - xi cos xi)/pi, xi = pi r / R, matches the
                     lattice point's rank along the mass coordinate; smoothing
                     lengths h = h_fact (m / rho)^(1/3) (Eq. 39) from the analytic
                     density rho_c sin(xi)/xi, floored at 0.01 rho_c.
  * ``uniform_clumps`` -- half uniform in the unit cube, half in 64 Gaussian
                     clumps (sigma 0.01), masses log-uniform over one decade.
  * ``plummer_batch`` -- many Plummer systems with log-uniform sizes and
                     uniform theta.
Seeds: ``seed = 20250203 + 1000 * config_index + system_index`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 20250203


def seed_for(config_index: int, system_index: int = 0) -> int:
    return BASE_SEED + 1000 * int(config_index) + int(system_index)


@dataclass
class ParticleSet:
    x: np.ndarray                 # (n, 3) float64, caller order
    m: np.ndarray                 # (n,) float64
    h: np.ndarray | None          # (n,) float64 smoothing lengths, or None (Plummer softening)
    soft_kind: int                # 0 Plummer softening, 1 M4 kernel softening
    eps: float                    # Plummer softening length
    name: str

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    sz = np.sqrt(1.0 - cz * cz)
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def plummer(n: int, seed: int, *, M: float = 1.0, b: float = 1.0, eps: float = 0.01,
            xmax: float = 0.999) -> ParticleSet:
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, xmax, n)
    r = b / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    m = np.full(n, M / n)
    return ParticleSet(x=x, m=m, h=None, soft_kind=0, eps=eps, name=f"plummer{n}")


def plummer_velocities(x: np.ndarray, seed: int, *, M: float = 1.0, b: float = 1.0) -> np.ndarray:
    """Equilibrium velocities of a Plummer sphere by rejection sampling of
    q = v / v_esc with density q^2 (1 - q^2)^(7/2) (Aarseth, Henon & Wielen 1974)."""
    rng = np.random.default_rng(seed + 7)
    n = x.shape[0]
    r = np.linalg.norm(x, axis=1)
    vesc = np.sqrt(2.0 * M) * (r * r + b * b) ** -0.25
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qa = rng.uniform(0.0, 1.0, todo.size)
        ya = rng.uniform(0.0, 0.1, todo.size)
        ok = ya < qa * qa * (1.0 - qa * qa) ** 3.5
        q[todo[ok]] = qa[ok]
        todo = todo[~ok]
    return (q * vesc)[:, None] * _isotropic(rng, n)


def _mass_fraction_n1(xi: np.ndarray) -> np.ndarray:
    return (np.sin(xi) - xi * np.cos(xi)) / np.pi


def _invert_mass_fraction_n1(f: np.ndarray) -> np.ndarray:
    lo = np.zeros_like(f)
    hi = np.full_like(f, np.pi)
    for _ in range(60):                       # bisection: the fraction is monotone in xi
        mid = 0.5 * (lo + hi)
        below = _mass_fraction_n1(mid) < f
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def polytrope_ball(n: int, rng: np.random.Generator, *, R: float = 1.0, M: float = 1.0,
                   h_fact: float = 1.2, rho_floor: float = 0.01):
    a = (4.0 * np.pi / (3.0 * n)) ** (1.0 / 3.0) * R
    k = int(np.ceil(R / a)) + 2
    g = np.arange(-k, k + 1, dtype=np.float64) * a
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    rad = np.linalg.norm(lat, axis=1)
    keep = np.lexsort((np.arange(rad.size), rad))[:n]
    p = lat[keep] + rng.uniform(-0.1 * a, 0.1 * a, (n, 3))
    ru = np.linalg.norm(p, axis=1)
    rank = np.empty(n)
    rank[np.lexsort((np.arange(n), ru))] = np.arange(n)
    xi = _invert_mass_fraction_n1((rank + 0.5) / n)
    r = xi * R / np.pi
    x = p * (r / np.where(ru > 0, ru, 1.0))[:, None]
    m = np.full(n, M / n)
    rho_c = np.pi * M / (4.0 * R ** 3)
    rho = np.maximum(rho_c * np.sinc(xi / np.pi), rho_floor * rho_c)
    h = h_fact * (m / rho) ** (1.0 / 3.0)
    return x, m, h


def polytrope_binary(n_per_star: int, seed: int, *, R: float = 1.0, sep: float = 4.0,
                     M: float = 1.0) -> ParticleSet:
    rng = np.random.default_rng(seed)
    xs, ms, hs = [], [], []
    for sgn in (-1.0, 1.0):
        x, m, h = polytrope_ball(n_per_star, rng, R=R, M=M)
        x[:, 0] += sgn * 0.5 * sep
        xs.append(x), ms.append(m), hs.append(h)
    return ParticleSet(x=np.concatenate(xs), m=np.concatenate(ms), h=np.concatenate(hs),
                       soft_kind=1, eps=0.0, name=f"binary_polytrope_2x{n_per_star}")


def binary_velocities(ps: ParticleSet, *, sep: float = 4.0) -> np.ndarray:
    """Circular orbit of the two stars about their common centre of mass."""
    n = ps.n // 2
    mtot = ps.m.sum()
    v = 0.5 * np.sqrt(mtot / sep)
    out = np.zeros_like(ps.x)
    out[:n, 1] = -v
    out[n:, 1] = v
    return out


def uniform_clumps(n: int, seed: int, *, n_clumps: int = 64, sigma: float = 0.01,
                   eps: float = 1e-3) -> ParticleSet:
    rng = np.random.default_rng(seed)
    nu = n // 2
    nc = n - nu
    xu = rng.uniform(0.0, 1.0, (nu, 3))
    centres = rng.uniform(0.0, 1.0, (n_clumps, 3))
    which = np.arange(nc) % n_clumps
    xc = centres[which] + rng.normal(0.0, sigma, (nc, 3))
    x = np.concatenate([xu, xc])
    m = np.exp(rng.uniform(0.0, np.log(10.0), n))
    m /= m.sum()
    return ParticleSet(x=x, m=m, h=None, soft_kind=0, eps=eps, name=f"uniform_clumps{n}")


@dataclass
class Batch:
    systems: list
    theta: np.ndarray
    eps: np.ndarray


def plummer_batch(n_sys: int, config_index: int = 3, *, nmin: int = 2048, nmax: int = 262144,
                  theta_lo: float = 0.3, theta_hi: float = 1.0, eps: float = 0.01) -> Batch:
    rng = np.random.default_rng(seed_for(config_index))
    sizes = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), n_sys))).astype(np.int64)
    thetas = rng.uniform(theta_lo, theta_hi, n_sys)
    systems = [plummer(int(sizes[k]), seed_for(config_index, k), eps=eps) for k in range(n_sys)]
    return Batch(systems=systems, theta=thetas, eps=np.full(n_sys, eps))
