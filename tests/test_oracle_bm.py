"""Pins of the Burton-Miller comparator oracle (oracle/bm.py) against the disk's Bessel-series
solution: first-order convergence for eps0 = 1 and 2; the sign printed in the paper for the
alpha eps0 (D* + I/2) term, a dropped alpha N term and a dropped free term do not converge."""

import math

import numpy as np
import pytest

from oracle import bm as BM
from oracle import kernels as OK
from oracle.exact import disk_solution
from synth import disk


def _errors(prm, solve, ns=(128, 256, 512)):
    out = []
    for n in ns:
        th = 2 * np.pi * np.arange(n) / n
        q, u = disk_solution(th, prm.k0, prm.k1, prm.eps0, prm.eps1)
        ex = np.concatenate([q, u])
        x = solve(disk(n), prm)
        out.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    return out


@pytest.mark.parametrize("eps0", [1.0, 2.0])
def test_bm_first_order_on_disk(eps0):
    prm = OK.Params.from_wavenumbers(5.0, 8.0, eps0=eps0)
    e = _errors(prm, BM.bm_solve)
    orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert all(0.9 <= o <= 1.2 for o in orders), orders
    assert e[-1] < 0.01


def _variant(kind):
    def solve(c, p):
        A = BM.bm_matrix(c, p)
        n = c.n
        pts = OK.Points.from_curve(c)
        alpha = 1j / p.k0
        if kind == "printed_sign":
            # +alpha eps0 (D*0 + I/2): flip the sign of that term of the (1, q) block
            _, _, ds0, _ = OK._layer_kernels(p.k0, *_geom(pts))
            i = np.arange(n)
            ds0[i, i] = OK.diag_D(c.kappa)
            corr = 2 * alpha * p.eps0 * (ds0 * c.w[None, :])
            corr[i, i] += 2 * alpha * p.eps0 * 0.5
            A[:n, :n] += corr
        elif kind == "no_alphaN":
            _, _, _, n0 = OK._layer_kernels(p.k0, *_geom(pts))
            i = np.arange(n)
            from oracle.pmchwt import diag_N
            n0[i, i] = diag_N(p.k0, c.w, c.kappa, pts.hs)
            A[:n, n:] -= alpha * n0 * c.w[None, :]
        else:  # no free term in the interior trace row
            i = np.arange(n)
            A[n + i, n + i] -= 0.5
        return np.linalg.solve(A, BM.bm_rhs(c, p))
    return solve


def _geom(pts):
    dx = pts.x[:, None] - pts.x[None, :]
    dy = pts.y[:, None] - pts.y[None, :]
    r = np.sqrt(dx * dx + dy * dy)
    np.fill_diagonal(r, 1.0)
    a = dx * pts.nx[:, None] + dy * pts.ny[:, None]
    b = dx * pts.nx[None, :] + dy * pts.ny[None, :]
    nn = pts.nx[:, None] * pts.nx[None, :] + pts.ny[:, None] * pts.ny[None, :]
    return r, a, b, nn


@pytest.mark.parametrize("kind", ["printed_sign", "no_alphaN", "no_free_term"])
def test_planted_bm_mistakes_do_not_converge(kind):
    prm = OK.Params.from_wavenumbers(5.0, 8.0, eps0=2.0)
    e = _errors(prm, _variant(kind))
    assert e[-1] > 0.05 or math.log2(e[-2] / e[-1]) < 0.5, e
