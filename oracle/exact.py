"""Closed-form solution of the transmission problem (Sec. 2) on the unit disk.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Separation of variables, independent of any boundary integral formulation.
With the incident plane wave u_in = exp(i k0 x1) = sum_n i^n J_n(k0 r) e^{i n theta}:
    exterior  u_0 = u_in + sum_n a_n H_n(k0 r) e^{i n theta}
    interior  u_1 = sum_n b_n J_n(k1 r) e^{i n theta}
The interface conditions of Sec. 2 at r = 1 (nu = radial direction, into Omega_0):
    i^n J_n(k0) + a_n H_n(k0)                   = b_n J_n(k1)               (continuity of u)
    (k0/eps0) [i^n J_n'(k0) + a_n H_n'(k0)]     = (k1/eps1) b_n J_n'(k1)    (continuity of q)
The boundary unknowns are u(theta) = sum_n b_n J_n(k1) e^{i n theta} and
q(theta) = (k1/eps1) sum_n b_n J_n'(k1) e^{i n theta}.
"""

from __future__ import annotations

import numpy as np
from scipy import special as _sp


def disk_coefficients(k0: float, k1: float, eps0: float, eps1: float, nmax: int):
    """(n, a_n, b_n) for |n| <= nmax."""
    n = np.arange(-nmax, nmax + 1)
    jk0, jk1 = _sp.jv(n, k0), _sp.jv(n, k1)
    djk0, djk1 = _sp.jvp(n, k0), _sp.jvp(n, k1)
    hk0, dhk0 = _sp.hankel1(n, k0), _sp.h1vp(n, k0)
    inc = (1j) ** (n % 4)
    # [ -H_n(k0)            J_n(k1)          ] [a]   [ i^n J_n(k0)          ]
    # [ -(k0/e0) H_n'(k0)   (k1/e1) J_n'(k1) ] [b] = [ (k0/e0) i^n J_n'(k0) ]
    m11, m12 = -hk0, jk1
    m21, m22 = -(k0 / eps0) * dhk0, (k1 / eps1) * djk1
    r1, r2 = inc * jk0, (k0 / eps0) * inc * djk0
    det = m11 * m22 - m12 * m21
    a = (r1 * m22 - m12 * r2) / det
    b = (m11 * r2 - r1 * m21) / det
    return n, a, b


def disk_solution(theta: np.ndarray, k0: float, k1: float, eps0: float, eps1: float,
                  extra_terms: int = 40):
    """(q, u) on the unit circle at parameters ``theta``; series truncated at |n| <= k1 + extra."""
    nmax = int(np.ceil(max(k0, k1))) + extra_terms
    n, a, b = disk_coefficients(k0, k1, eps0, eps1, nmax)
    ph = np.exp(1j * np.outer(theta, n))
    u = ph @ (b * _sp.jv(n, k1))
    q = ph @ ((k1 / eps1) * b * _sp.jvp(n, k1))
    return q, u
