"""Closed-curve samplers for the Nystrom discretisation (Sec. 3.1).

A curve is sampled at N equispaced parameters theta_j = 2*pi*j/N, j = 0..N-1.
For a counter-clockwise parametrisation gamma(theta) the sampler returns

* x_j, y_j           the node gamma(theta_j)
* nx_j, ny_j         the unit normal (gamma_2', -gamma_1')/|gamma'|, which points
                     out of the bounded region Omega_1 (into Omega_0, Sec. 2)
* w_j                the trapezoidal weight |gamma'(theta_j)| * 2*pi/N (Sec. 3.1)
* kappa_j            the signed curvature, positive on a convex curve

Every curve here is a "Fourier star" r(theta) = 1 + sum_m a_m cos(m*theta + phi_m)
in polar form; the unit disk is the case with no modes.  The samples are
computed in float64 from the closed-form derivatives of r(theta).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Curve:
    """Sampled closed curve (structure of arrays, float64, length N)."""

    x: np.ndarray
    y: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    w: np.ndarray
    kappa: np.ndarray
    name: str = "curve"

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self) -> Tuple[np.ndarray, ...]:
        return (self.x, self.y, self.nx, self.ny, self.w, self.kappa)


def fourier_star_at(theta, modes: Sequence[Tuple[int, float, float]] = ()) -> Dict[str, np.ndarray]:
    """Closed-form geometry of r(theta) = 1 + sum a*cos(m*theta + phi) at arbitrary parameters.

    Returns the point (x, y), the outward unit normal (nx, ny), the parametrisation speed
    v = |gamma'|, its first two derivatives dv, ddv with respect to theta, and the signed
    curvature kappa, all as float64 arrays shaped like ``theta``.
    """
    theta = np.asarray(theta, dtype=np.float64)
    r = np.ones_like(theta)
    d1 = np.zeros_like(theta)
    d2 = np.zeros_like(theta)
    d3 = np.zeros_like(theta)
    for m, a, phi in modes:
        arg = m * theta + phi
        r = r + a * np.cos(arg)
        d1 = d1 - a * m * np.sin(arg)
        d2 = d2 - a * m * m * np.cos(arg)
        d3 = d3 + a * m * m * m * np.sin(arg)
    c, s = np.cos(theta), np.sin(theta)
    # derivatives of gamma = r (cos, sin) up to third order
    x, y = r * c, r * s
    dx, dy = d1 * c - r * s, d1 * s + r * c
    ddx = d2 * c - 2.0 * d1 * s - r * c
    ddy = d2 * s + 2.0 * d1 * c - r * s
    dddx = d3 * c - 3.0 * d2 * s - 3.0 * d1 * c + r * s
    dddy = d3 * s + 3.0 * d2 * c - 3.0 * d1 * s - r * c
    v = np.sqrt(dx * dx + dy * dy)
    g12 = dx * ddx + dy * ddy
    dv = g12 / v
    ddv = (ddx * ddx + ddy * ddy + dx * dddx + dy * dddy) / v - g12 * g12 / v**3
    return {"x": x, "y": y, "nx": dy / v, "ny": -dx / v, "v": v, "dv": dv, "ddv": ddv,
            "kappa": (dx * ddy - dy * ddx) / v**3}


def fourier_star(n: int, modes: Sequence[Tuple[int, float, float]] = (), name: str = "star") -> Curve:
    """Sample r(theta) = 1 + sum a*cos(m*theta + phi) over (m, a, phi) in ``modes``."""
    if n <= 0:
        raise ValueError("n must be positive")
    theta = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n
    g = fourier_star_at(theta, modes)
    w = g["v"] * (2.0 * np.pi / n)
    return Curve(g["x"], g["y"], g["nx"], g["ny"], w, g["kappa"], name)


def disk(n: int) -> Curve:
    """Unit circle: nodes (cos, sin), normals equal to the nodes, w = 2*pi/N, kappa = 1."""
    return fourier_star(n, (), name="disk")


def star(n: int, amp: float = 0.3, m: int = 5) -> Curve:
    """Star r(theta) = 1 + amp*cos(m*theta)."""
    return fourier_star(n, ((m, amp, 0.0),), name=f"star{m}")


def random_star_batch(count: int, seed: int, n_min: int = 2048, n_max: int = 32768,
                      k_range: Tuple[float, float] = (5.0, 40.0),
                      ratio_range: Tuple[float, float] = (1.2, 2.0)) -> List[Dict]:
    """Random scatterers r = 1 + sum_{m=2..8} a_m cos(m*theta + phi_m), a_m ~ U(0, 0.05).

    Node counts are drawn log-uniformly in [n_min, n_max] (any integer, so leaf
    boxes come out uneven); k_ext ~ U(k_range), k_int = k_ext * U(ratio_range),
    eps0 = 1, eps1 = (k_int / k_ext)^2.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        a = rng.uniform(0.0, 0.05, size=7)
        phi = rng.uniform(0.0, 2.0 * np.pi, size=7)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        n = min(max(n, n_min), n_max)
        k0 = float(rng.uniform(*k_range))
        k1 = k0 * float(rng.uniform(*ratio_range))
        modes = tuple((m, float(a[m - 2]), float(phi[m - 2])) for m in range(2, 9))
        out.append({"curve": fourier_star(n, modes, name=f"rstar{i}"), "k0": k0, "k1": k1,
                    "eps0": 1.0, "eps1": (k1 / k0) ** 2})
    return out


# Named workloads.  eps0 = 1 and eps1 = (k1/k0)^2 follow k_i = omega*sqrt(eps_i) (Sec. 2)
# with eps0 = 1 as in Sec. 6.
WORKLOADS: Dict[str, Dict] = {
    "disk512": dict(curve=("disk", 512), k0=5.0, k1=8.0, leaf=64, nproxy=32, tol=1e-10),
    "star16k": dict(curve=("star", 16384), k0=20.0, k1=30.0, leaf=128, nproxy=64, tol=1e-10),
    "star64k": dict(curve=("star", 65536), k0=40.0, k1=60.0, leaf=128, nproxy=64, tol=1e-10),
    "star262k": dict(curve=("star", 262144), k0=100.0, k1=150.0, leaf=128, nproxy=64, tol=1e-8),
}

# Batch of independent random scatterers (random_star_batch), solved in one handle.
BATCH_WORKLOADS: Dict[str, Dict] = {
    "batch64": dict(count=64, seed=2024, n_min=2048, n_max=32768, leaf=128, nproxy=64, tol=1e-10),
}


def batch_workload(name: str, count: int | None = None, n_max: int | None = None) -> Dict:
    """The named batch workload with its sampled scatterers; ``count`` / ``n_max`` shrink it."""
    spec = dict(BATCH_WORKLOADS[name])
    cnt = spec.pop("count") if count is None else count
    spec.pop("count", None)
    seed = spec.pop("seed")
    lo, hi = spec.pop("n_min"), spec.pop("n_max")
    if n_max is not None:
        hi = n_max
        lo = min(lo, hi)
    spec["problems"] = random_star_batch(cnt, seed, lo, hi)
    spec["name"] = name
    return spec


def workload(name: str, n: int | None = None) -> Dict:
    """Return the named workload with its sampled curve; ``n`` overrides the node count."""
    spec = dict(WORKLOADS[name])
    kind, n0 = spec.pop("curve")
    n = n0 if n is None else n
    spec["curve"] = disk(n) if kind == "disk" else star(n)
    spec["eps0"] = 1.0
    spec["eps1"] = (spec["k1"] / spec["k0"]) ** 2
    spec["name"] = name
    return spec
