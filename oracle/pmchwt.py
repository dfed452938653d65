"""Symmetric PMCHWT comparator (Sec. 3.2, Eq. symmetric_pmchwt), oracle in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Same unknowns as the Muller-like system (q = (1/eps) du/dnu, u), same row scaling by W:
    A11 = -(eps0 S_k0 + eps1 S_k1)          A12 = D_k0 + D_k1
    A21 = D*_k0 + D*_k1                     A22 = -(N_k0 / eps0 + N_k1 / eps1)
    rhs = [-W u_in ; (1/eps0) W du_in/dnu]
(the sum of the exterior and interior representation formulas and of their normal
derivatives: the free terms cancel, and the hypersingular parts of N_k0, N_k1 add).

One-point corrected diagonal of the hypersingular kernel (the paper does not print it;
reading): near the diagonal the Laplace part of N_k is 1/(2 pi sigma^2) + kappa^2/(24 pi)
+ O(sigma^2) in arclength sigma (exact constant on a circle).  In the parameter tau of the
equispaced rule, the kernel times the source's speed v = |gamma'| is A/tau^2 + C + O(tau)
with A = 1/(2 pi v) and C/v = kappa^2/(24 pi) + (v''/6 - v'^2/(4v))/(2 pi v^3) (the odd
1/tau term vanishes).  The zeta-corrected trapezoidal rule for FP int f(tau) dtau adds
-2 zeta(2) A / h = -pi^2 A / (3h) at the node plus the constant C, so the diagonal entry
(per weight w_i = v_i h) is -pi / (6 w_i^2) + kappa^2/(24 pi) + s_i / w_i^2, where s_i is
the speed term of kernels.hypersingular_speed_term (zero on a circle), plus the
log-singular and constant terms of N_k - N_0 (those of the Muller-like N difference for
one wavenumber):
    N~_k(i,i) = (s_i - pi/6) / w_i^2 + kappa_i^2/(24 pi) + (i/8) k^2
                - k^2 (log(k/2) + gamma_E)/(4 pi) + k^2/(8 pi) - (k^2/(4 pi)) log(w_i / 2 pi).
The rule is first order (the error of the corrected 1/tau^2 rule is O(h)), which is the
O(h) convergence the paper reports for PMCHWT.  S~, D~, D*~ as in kernels.py.
"""

from __future__ import annotations

import math

import numpy as np

from .kernels import EULER_GAMMA, Params, Points, _layer_kernels, diag_D, diag_S, incident_plane_wave


def diag_N(k: float, w, kappa, hs=0.0):
    """One-point corrected N~_k(i,i) (reading in the module docstring); hs is the node's
    speed term (kernels.hypersingular_speed_term)."""
    c = (0.125j * k * k - (k * k / (4.0 * math.pi)) * (math.log(k / 2.0) + EULER_GAMMA) + k * k / (8.0 * math.pi))
    return ((hs - math.pi / 6.0) / (w * w) + kappa * kappa / (24.0 * math.pi) + c
            - (k * k / (4.0 * math.pi)) * np.log(w / (2.0 * math.pi)))


def pmchwt_blocks(obs: Points, src: Points, prm: Params, scaled: bool = True):
    """(A11, A12, A21, A22) of the (row-scaled, or unscaled with scaled=False) PMCHWT system."""
    e0, e1 = prm.eps0, prm.eps1
    dx = obs.x[:, None] - src.x[None, :]
    dy = obs.y[:, None] - src.y[None, :]
    same = (obs.gid[:, None] == src.gid[None, :]) & (obs.gid[:, None] >= 0)
    r = np.sqrt(dx * dx + dy * dy)
    r = np.where(same, 1.0, r)
    a = dx * obs.nx[:, None] + dy * obs.ny[:, None]
    b = dx * src.nx[None, :] + dy * src.ny[None, :]
    nn = obs.nx[:, None] * src.nx[None, :] + obs.ny[:, None] * src.ny[None, :]
    g0, d0, ds0, n0 = _layer_kernels(prm.k0, r, a, b, nn)
    g1, d1, ds1, n1 = _layer_kernels(prm.k1, r, a, b, nn)
    ks = e0 * g0 + e1 * g1
    kd = d0 + d1
    kds = ds0 + ds1
    kn = n0 / e0 + n1 / e1
    if same.any():
        oi, si = np.nonzero(same)
        wi, ki, hi = obs.w[oi], obs.kappa[oi], obs.hs[oi]
        ks[oi, si] = e0 * diag_S(prm.k0, wi) + e1 * diag_S(prm.k1, wi)
        dd = diag_D(ki)
        kd[oi, si] = 2.0 * dd
        kds[oi, si] = 2.0 * dd
        kn[oi, si] = diag_N(prm.k0, wi, ki, hi) / e0 + diag_N(prm.k1, wi, ki, hi) / e1
    if scaled:
        wgt = obs.w[:, None] * src.w[None, :]
    else:
        wgt = np.broadcast_to(src.w[None, :], dx.shape)
    return -(wgt * ks), wgt * kd, wgt * kds, -(wgt * kn)


def pmchwt_matrix(curve, prm: Params, scaled: bool = True) -> np.ndarray:
    """The 2N x 2N PMCHWT matrix, unknowns [q; u], equations [sum of traces; sum of fluxes]."""
    pts = Points.from_curve(curve)
    blk = pmchwt_blocks(pts, pts, prm, scaled)
    return np.block([[blk[0], blk[1]], [blk[2], blk[3]]])


def pmchwt_rhs(curve, prm: Params, angle: float = 0.0, scaled: bool = True) -> np.ndarray:
    """[-W u_in ; (1/eps0) W du_in/dnu] (without W for scaled=False)."""
    uin, dudn = incident_plane_wave(curve, prm.k0, angle)
    f = np.concatenate([-uin, dudn / prm.eps0])
    if scaled:
        f = f * np.concatenate([curve.w, curve.w])
    return f


def pmchwt_solve(curve, prm: Params, angle: float = 0.0, scaled: bool = True) -> np.ndarray:
    """Dense LU solution [q; u] of the PMCHWT system."""
    return np.linalg.solve(pmchwt_matrix(curve, prm, scaled), pmchwt_rhs(curve, prm, angle, scaled))


def pmchwt_entries(obs: Points, obs_eq, src: Points, src_comp, prm: Params, scaled: bool = True) -> np.ndarray:
    """Dense block A[(p, e), (q, c)] of the PMCHWT system for (point, equation) rows and
    (point, unknown) columns (e, c in {0, 1} as in kernels.entries)."""
    obs_eq = np.asarray(obs_eq, dtype=np.int64)
    src_comp = np.asarray(src_comp, dtype=np.int64)
    blk = pmchwt_blocks(obs, src, prm, scaled)
    e = obs_eq[:, None]
    c = src_comp[None, :]
    return np.where(e == 0, np.where(c == 0, blk[0], blk[1]), np.where(c == 0, blk[2], blk[3]))
