"""Burton-Miller comparator (Sec. 6, Eq. bm), oracle in FP64 (non-symmetric; unscaled).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Unknowns ordered [q; u] as in the Muller-like system (q = (1/eps) du/dnu).  From the
exterior representation formula (trace: (D0 - I/2) u - eps0 S0 q = -u_in; normal
derivative: -N0 u + eps0 (D*0 + I/2) q = q_in) and the interior trace equation
((D1 + I/2) u - eps1 S1 q = 0):
    row 1 = trace - alpha * normal derivative (exterior), alpha = i / k0:
        [-eps0 S0 - alpha eps0 (D*0 + I/2),  D0 - I/2 + alpha N0]   rhs  -u_in - alpha du_in/dnu
    row 2 = interior trace:
        [-eps1 S1,                           D1 + I/2]               rhs  0
Reading: the paper prints +alpha eps0 (D*0 + I/2) in row 1 together with the same u
column and right-hand side; with the sign conventions of the Muller-like system (pinned
by its third-order disk convergence) only the form above is consistent, and the printed
sign does not converge (tests/test_oracle_bm.py).  Every kernel entry is Z~(x_i, y_j) w_j
(unscaled); the diagonal is one-point corrected as in kernels.py and pmchwt.py, so the
hypersingular N0 makes the rule first order.
"""

from __future__ import annotations

import numpy as np

from .kernels import Params, Points, _layer_kernels, diag_D, diag_S, incident_plane_wave
from .pmchwt import diag_N


def bm_blocks(obs: Points, src: Points, prm: Params, scaled: bool = False):
    """(A11, A12, A21, A22) of the Burton-Miller system ([q; u] columns)."""
    e0, e1 = prm.eps0, prm.eps1
    alpha = 1j / prm.k0
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
    if same.any():
        oi, si = np.nonzero(same)
        wi, ki, hi = obs.w[oi], obs.kappa[oi], obs.hs[oi]
        g0[oi, si] = diag_S(prm.k0, wi)
        g1[oi, si] = diag_S(prm.k1, wi)
        dd = diag_D(ki)
        d0[oi, si] = dd
        ds0[oi, si] = dd
        d1[oi, si] = dd
        n0[oi, si] = diag_N(prm.k0, wi, ki, hi)
    wgt = obs.w[:, None] * src.w[None, :] if scaled else np.broadcast_to(src.w[None, :], dx.shape)
    a11 = wgt * (-e0 * g0 - alpha * e0 * ds0)
    a12 = wgt * (d0 + alpha * n0)
    a21 = wgt * (-e1 * g1)
    a22 = wgt * d1
    if same.any():
        ftw = obs.w[oi] if scaled else np.ones(len(oi))
        a11[oi, si] += -alpha * e0 * 0.5 * ftw
        a12[oi, si] += -0.5 * ftw
        a22[oi, si] += 0.5 * ftw
    return a11, a12, a21, a22


def bm_matrix(curve, prm: Params, scaled: bool = False) -> np.ndarray:
    pts = Points.from_curve(curve)
    blk = bm_blocks(pts, pts, prm, scaled)
    return np.block([[blk[0], blk[1]], [blk[2], blk[3]]])


def bm_rhs(curve, prm: Params, angle: float = 0.0, scaled: bool = False) -> np.ndarray:
    """[-u_in - alpha du_in/dnu ; 0] (times W for scaled=True)."""
    uin, dudn = incident_plane_wave(curve, prm.k0, angle)
    f = np.concatenate([-uin - (1j / prm.k0) * dudn, np.zeros_like(uin)])
    if scaled:
        f = f * np.concatenate([curve.w, curve.w])
    return f


def bm_solve(curve, prm: Params, angle: float = 0.0, scaled: bool = False) -> np.ndarray:
    return np.linalg.solve(bm_matrix(curve, prm, scaled), bm_rhs(curve, prm, angle, scaled))


def bm_entries(obs: Points, obs_eq, src: Points, src_comp, prm: Params, scaled: bool = False) -> np.ndarray:
    obs_eq = np.asarray(obs_eq, dtype=np.int64)
    src_comp = np.asarray(src_comp, dtype=np.int64)
    blk = bm_blocks(obs, src, prm, scaled)
    e = obs_eq[:, None]
    c = src_comp[None, :]
    return np.where(e == 0, np.where(c == 0, blk[0], blk[1]), np.where(c == 0, blk[2], blk[3]))
