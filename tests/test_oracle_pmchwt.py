"""Pins of the PMCHWT comparator oracle (oracle/pmchwt.py), against the disk's Bessel-series
solution and the Muller-like system, not against itself:

* first-order convergence to the exact disk solution (the O(h) rate of Sec. 6) for eps0 = 1
  and eps0 = 2 (the latter pins the 1/eps0 of the flux right-hand side);
* planted mistakes stop the convergence: a doubled 1/tau^2 correction, the right-hand side
  without 1/eps0, the free terms of the Muller-like system added;
* the row-scaled matrix is complex symmetric off the diagonal (and on it: PMCHWT has no
  free terms), bit for bit;
* on a star its solution approaches the O(h^3) Muller-like solution at first order.
"""

import math

import numpy as np
import pytest

from oracle import kernels as OK
from oracle import pmchwt as PM
from oracle.exact import disk_solution
from synth import disk, star


def _disk_errors(prm, solve, ns=(128, 256, 512)):
    errs = []
    for n in ns:
        th = 2 * np.pi * np.arange(n) / n
        q, u = disk_solution(th, prm.k0, prm.k1, prm.eps0, prm.eps1)
        ex = np.concatenate([q, u])
        x = solve(disk(n), prm)
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    return errs


@pytest.mark.parametrize("eps0", [1.0, 2.0])
def test_pmchwt_first_order_on_disk(eps0):
    prm = OK.Params.from_wavenumbers(5.0, 8.0, eps0=eps0)
    e = _disk_errors(prm, PM.pmchwt_solve)
    orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert all(0.9 <= o <= 1.2 for o in orders), orders
    assert e[-1] < 0.012


def _with_diag_scale(scale):
    orig = PM.diag_N

    def dn(k, w, kappa):
        return orig(k, w, kappa) + (scale - 1.0) * (-math.pi / (6.0 * w * w))
    return dn


@pytest.mark.parametrize("mistake", ["double_tau2", "rhs_eps", "free_terms"])
def test_planted_mistakes_stop_convergence(mistake, monkeypatch):
    prm = OK.Params.from_wavenumbers(5.0, 8.0, eps0=2.0)
    if mistake == "double_tau2":
        monkeypatch.setattr(PM, "diag_N", _with_diag_scale(2.0))
        solve = PM.pmchwt_solve
    elif mistake == "rhs_eps":
        def solve(c, p):
            uin, dudn = OK.incident_plane_wave(c, p.k0)
            f = np.concatenate([-uin, dudn]) * np.concatenate([c.w, c.w])
            return np.linalg.solve(PM.pmchwt_matrix(c, p), f)
    else:
        def solve(c, p):
            A = PM.pmchwt_matrix(c, p)
            n = c.n
            half = 0.5 * (p.eps0 + p.eps1) * c.w
            A[np.arange(n), n + np.arange(n)] -= half
            A[n + np.arange(n), np.arange(n)] += half
            return np.linalg.solve(A, PM.pmchwt_rhs(c, p))
    e = _disk_errors(prm, solve)
    assert e[-1] > 0.05 or math.log2(e[-2] / e[-1]) < 0.5, e


def test_pmchwt_matrix_symmetric_bitwise():
    prm = OK.Params.from_wavenumbers(3.0, 6.0)
    A = PM.pmchwt_matrix(star(300), prm)
    assert np.array_equal(A, A.T)


def test_pmchwt_approaches_muller_solution_first_order():
    prm = OK.Params.from_wavenumbers(5.0, 8.0)
    ref = OK.dense_solve(star(1024), prm)
    d = []
    for n in (128, 256, 512):
        s = 1024 // n
        r = np.concatenate([ref[:1024][::s], ref[1024:][::s]])
        d.append(np.linalg.norm(PM.pmchwt_solve(star(n), prm) - r) / np.linalg.norm(r))
    assert 0.8 <= math.log2(d[0] / d[1]) <= 1.3 and 0.8 <= math.log2(d[1] / d[2]) <= 1.3, d
