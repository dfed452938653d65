"""Pins of the PMCHWT comparator oracle (oracle/pmchwt.py), against the disk's Bessel-series
solution and the Muller-like system, not against itself:

* first-order convergence to the exact disk solution (the O(h) rate of Sec. 6) for eps0 = 1
  and eps0 = 2 (the latter pins the 1/eps0 of the flux right-hand side);
* planted mistakes stop the convergence: a doubled 1/tau^2 correction, the right-hand side
  without 1/eps0, the free terms of the Muller-like system added;
* the row-scaled matrix is complex symmetric off the diagonal (and on it: PMCHWT has no
  free terms), bit for bit;
* on a star its solution approaches the O(h^3) Muller-like solution at first order;
* the corrected hypersingular diagonal equals the constant term of the off-diagonal kernel's
  expansion about the node, on circles of several radii (the kappa^2 / 24 pi term) and on
  stars, whose non-uniform parametrisation speed adds the speed term; planted mistakes
  (speed term dropped, kappa for kappa^2, kappa^2 / 8 pi) fail that limit.
"""

import math

import numpy as np
import pytest

from oracle import kernels as OK
from oracle import pmchwt as PM
from oracle.exact import disk_solution
from synth import disk, fourier_star_at, star


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

    def dn(k, w, kappa, hs=0.0):
        return orig(k, w, kappa, hs) + (scale - 1.0) * (-math.pi / (6.0 * w * w))
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


# ---- the hypersingular diagonal constant, pinned by the kernel's own expansion ----
#
# In the parameter tau of the equispaced rule, f(tau) = N_k(gamma(t), gamma(t + tau)) v(t + tau)
# = A / tau^2 + L log|tau| + C + O(tau) with A = 1 / (2 pi v), L = -(k^2 / 4 pi) v.  The
# zeta-corrected rule's node value is [C + L log(h / 2 pi)] / v - pi / (6 w^2), so
#     diag_N(k, w, kappa, hs) + pi / (6 w^2) + (k^2 / 4 pi) log(h / 2 pi) = C / v
# must hold for every h.  C is measured from the off-diagonal kernel (pinned by finite
# differences of G) at closed-form curve points, from the symmetric mean of f(+tau), f(-tau).

def _geometry(kind, th):
    if kind.startswith("circle"):
        rad = float(kind[len("circle"):])
        one = np.ones_like(th)
        return {"x": rad * np.cos(th), "y": rad * np.sin(th), "nx": np.cos(th), "ny": np.sin(th),
                "v": rad * one, "dv": 0 * one, "ddv": 0 * one, "kappa": one / rad}
    modes = {"star3": ((3, 0.2, 0.0),), "star5": ((5, 0.3, 0.0),),
             "fourier": ((2, 0.1, 0.3), (7, 0.04, 1.1))}[kind]
    return fourier_star_at(th, modes)


def _hyp_constant(kind, tau, k, th):
    p = _geometry(kind, th)
    f = []
    for s in (1, -1):
        q = _geometry(kind, th + s * tau)
        dx, dy = p["x"] - q["x"], p["y"] - q["y"]
        r = np.hypot(dx, dy)
        a = dx * p["nx"] + dy * p["ny"]
        b = dx * q["nx"] + dy * q["ny"]
        nn = p["nx"] * q["nx"] + p["ny"] * q["ny"]
        _, _, _, nk = OK._layer_kernels(k, r, a, b, nn)
        f.append(nk * q["v"])
    v = p["v"]
    return (0.5 * (f[0] + f[1]) - 1.0 / (2 * np.pi * v * tau**2) + (k * k / (4 * np.pi)) * v * math.log(tau)) / v


def _hyp_constant_error(kind, tau, k=2.0, n=1024):
    """max over nodes of |C / v (from the kernel, Richardson-extrapolated from tau and tau/2)
    - the rule's constant| on n nodes of the curve."""
    th = 2 * np.pi * np.arange(n) / n
    h = 2 * np.pi / n
    c_num = (4 * _hyp_constant(kind, tau / 2, k, th) - _hyp_constant(kind, tau, k, th)) / 3
    p = _geometry(kind, th)
    w = p["v"] * h
    # the speed term from the sampled weights (what the discretisation sees)
    hs = OK.hypersingular_speed_term(w) if not kind.startswith("circle") else np.zeros(n)
    c_rule = PM.diag_N(k, w, p["kappa"], hs) + np.pi / (6 * w * w) + (k * k / (4 * np.pi)) * math.log(h / (2 * np.pi))
    return np.max(np.abs(c_num - c_rule))


@pytest.mark.parametrize("kind", ["circle0.5", "circle3", "star3", "star5", "fourier"])
def test_hypersingular_diagonal_is_the_kernel_constant(kind):
    # extrapolated truncation error O(tau^4 log tau) until rounding in the 1/tau^2
    # subtraction takes over near tau = 1e-3
    e_coarse, e_fine = _hyp_constant_error(kind, 8e-3), _hyp_constant_error(kind, 2e-3)
    assert e_fine < 2e-5 and (e_fine < 5e-6 or e_coarse / e_fine > 16), (e_coarse, e_fine)


def test_speed_term_matches_closed_form_derivatives():
    """The central differences of the sampled weights give v'/v and v''/v of the curve."""
    for modes in (((3, 0.2, 0.0),), ((5, 0.3, 0.0),), ((2, 0.1, 0.3), (7, 0.04, 1.1))):
        for n in (1024, 4096):
            th = 2 * np.pi * np.arange(n) / n
            g = fourier_star_at(th, modes)
            h = 2 * np.pi / n
            exact = (g["ddv"] / (6 * g["v"]) - g["dv"] ** 2 / (4 * g["v"] ** 2)) * h * h / (2 * np.pi)
            got = OK.hypersingular_speed_term(g["v"] * h)
            scale = np.max(np.abs(exact))
            # order-16 differences: truncation negligible here; rounding grows like n^2
            assert np.max(np.abs(got - exact)) <= 1e-9 * scale, (modes, n)
    assert np.max(np.abs(OK.hypersingular_speed_term(np.full(50, 0.3)))) < 1e-16  # a circle
    from fractions import Fraction as F
    assert OK.central_weights(2, 1) == [F(1, 12), F(-2, 3), 0, F(2, 3), F(-1, 12)]
    assert OK.central_weights(2, 2) == [F(-1, 12), F(4, 3), F(-5, 2), F(4, 3), F(-1, 12)]


_PLANTED_N = {
    "no_speed_term": lambda orig: (lambda k, w, kappa, hs=0.0: orig(k, w, kappa, 0.0 * hs)),
    "kappa_not_squared": lambda orig: (lambda k, w, kappa, hs=0.0: orig(k, w, kappa, hs)
                                       + (kappa - kappa * kappa) / (24 * math.pi)),
    "kappa2_over_8pi": lambda orig: (lambda k, w, kappa, hs=0.0: orig(k, w, kappa, hs)
                                     + kappa * kappa * (1 / (8 * math.pi) - 1 / (24 * math.pi))),
}


@pytest.mark.parametrize("mistake,kind", [("no_speed_term", "star3"), ("no_speed_term", "star5"),
                                          ("kappa_not_squared", "circle0.5"),
                                          ("kappa_not_squared", "circle3"),
                                          ("kappa2_over_8pi", "circle3")])
def test_planted_hypersingular_mistakes_fail_the_limit(mistake, kind, monkeypatch):
    monkeypatch.setattr(PM, "diag_N", _PLANTED_N[mistake](PM.diag_N))
    assert _hyp_constant_error(kind, 2e-3) > 1e-3
