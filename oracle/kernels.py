"""Matrix entries of the symmetric Muller-like Nystrom system (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (Sec. 3.1, Sec. 3.2):
    G_k(x, y)       = (i/4) H_0^(1)(k r),  r = |x - y|                       (2-D fundamental solution)
    dG/dnu(y)       = (i k/4) H_1(k r) (d . nu_y) / r,  d = x - y              (kernel of D_k)
    dG/dnu(x)       = -(i k/4) H_1(k r) (d . nu_x) / r                         (kernel of D_k^*)
    d2G/dnu(x)dnu(y)= (i k/4) [ H_1(kr)/r nu_x.nu_y
                              + (d.nu_x)(d.nu_y)/r (k H_0(kr)/r - 2 H_1(kr)/r^2) ]  (kernel of N_k)
These follow from differentiating G_k with H_0' = -H_1 and H_1'(z) = H_0(z) - H_1(z)/z.

Row-scaled blocks (Eq. 15, block form in Sec. 4.1), W = diag(w):
    A11 = -(eps0^2 S_k0 - eps1^2 S_k1)
    A12 = eps0 (D_k0 - W/2) - eps1 (D_k1 + W/2)
    A21 = eps0 (D*_k0 + W/2) - eps1 (D*_k1 - W/2)
    A22 = -(N_k0 - N_k1)
with [Z]_ij = w_i Z~(x_i, y_j) w_j for every layer operator Z (Sec. 3.1).

The baseline ("Base") matrix is the unscaled system of Sec. 6 (naive Muller-like),
i.e. the same blocks with every row divided by w_i: [Z']_ij = Z~(x_i, y_j) w_j and
free terms -/+ (eps0 + eps1)/2 I.

One-point corrected diagonal (Sec. 3.1).  The paper uses the lowest-order zeta
correction but does not print the terms.  Reading used here: for a kernel
A log|x - y| + B + o(1) on the curve, the punctured trapezoidal rule plus the
diagonal value A log(w_i / 2 pi) + B integrates to O(h^3) (the zeta-function
constant 2 zeta'(0) = -log 2 pi gives the h log(h / 2 pi) weight; log|gamma'| comes
from the smooth ratio |gamma(t) - gamma(s)| / |t - s|).  This gives
    S~_k(i,i)        = i/4 - (1/2 pi) (gamma_E + log(k w_i / 4 pi))
    D~(i,i) = D*~(i,i) = -kappa_i / (4 pi)       (the continuous limit of the kernel)
    (N_k0 - N_k1)~(i,i) = (i/8)(k0^2 - k1^2)
                        - (1/4 pi)[k0^2 (log(k0/2) + gamma_E) - k1^2 (log(k1/2) + gamma_E)]
                        + (k0^2 - k1^2)/(8 pi) - ((k0^2 - k1^2)/(4 pi)) log(w_i / 2 pi)
The hypersingular parts of N_k0 and N_k1 are identical and cancel, so only the
difference is ever corrected.

Right-hand side (Eq. 15): [-eps0 W u_in ; W d(u_in)/dnu].  The paper prints
(1/eps0) W q_in for the second row; deriving the system from Green's
representation (Sec. 2, with nu pointing into Omega_0) gives W d(u_in)/dnu.
The two agree for eps0 = 1, which holds in every workload; the
transparent-obstacle test pins the derived form for eps0 != 1.

Symmetry (Eq. syms): every off-diagonal pair is evaluated by one expression
whose inputs change only by exact negations under the swap (p, q) -> (q, p),
so A_pq = A_qp^T holds bit for bit away from the diagonal.
"""

from __future__ import annotations

import dataclasses
import math
from fractions import Fraction
from typing import Optional, Sequence, Tuple

import numpy as np
from scipy import special as _sp

EULER_GAMMA = 0.57721566490153286060651209008240243


@dataclasses.dataclass
class Params:
    """Material and wave parameters (Sec. 2): k_i = omega sqrt(eps_i)."""

    k0: float
    k1: float
    eps0: float = 1.0
    eps1: float = 1.0

    @staticmethod
    def from_wavenumbers(k0: float, k1: float, eps0: float = 1.0) -> "Params":
        """eps1 = eps0 (k1/k0)^2, the relation k_i = omega sqrt(eps_i) of Sec. 2."""
        return Params(k0, k1, eps0, eps0 * (k1 / k0) ** 2)


def central_weights(m: int, order: int):
    """Weights c_{-m..m} of the central difference of the given derivative order with
    2m + 1 equispaced points (unit spacing), as exact rationals: the unique weights that
    reproduce every polynomial of degree <= 2m, i.e. sum_j c_j j^p = order! [p = order]
    for p = 0..2m (solved by Gaussian elimination over the rationals)."""
    js = list(range(-m, m + 1))
    size = 2 * m + 1
    rows = [[Fraction(j) ** p for j in js] + [Fraction(math.factorial(order) if p == order else 0)]
            for p in range(size)]
    for c in range(size):
        piv = next(r for r in range(c, size) if rows[r][c] != 0)
        rows[c], rows[piv] = rows[piv], rows[c]
        for r in range(size):
            if r != c and rows[r][c] != 0:
                f = rows[r][c] / rows[c][c]
                rows[r] = [a - f * b for a, b in zip(rows[r], rows[c])]
    return [rows[i][size] / rows[i][i] for i in range(size)]


def hypersingular_speed_term(w, m: int = 8) -> np.ndarray:
    """Speed-dependent part of the constant term of the hypersingular diagonal, per node.

    With the parametrisation speed v = |gamma'| sampled as the trapezoidal weights
    w_j = v(theta_j) h, the Laplace hypersingular kernel times the source's weight has the
    expansion A / tau^2 + C + O(tau) in the parameter offset tau, with A = 1 / (2 pi v) and
    C / v = kappa^2 / (24 pi) + (v''/6 - v'^2 / (4 v)) / (2 pi v^3) (a change of variables
    from arclength, where the constant is kappa^2 / (24 pi)).  In index units (derivatives
    with respect to j, so h drops out) the second part is s_j / w_j^2 with
        s_j = (l2_j / 6 - l1_j^2 / 4) / (2 pi),   l1 = (dw/dj) / w,   l2 = (d^2 w/dj^2) / w,
    and this function returns s (dimensionless; zero on a circle).  The derivatives of the
    periodic sequence w are central differences of order 2m (m = 8, fewer on very short
    curves), which are exact to rounding for the smooth curves used here.
    """
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[0]
    m = max(0, min(m, (n - 1) // 2))
    if m == 0:
        return np.zeros(n)
    c1 = [float(c) for c in central_weights(m, 1)]
    c2 = [float(c) for c in central_weights(m, 2)]
    d1 = np.zeros(n)
    d2 = np.zeros(n)
    for k, j in enumerate(range(-m, m + 1)):
        sh = np.roll(w, -j)  # sh[i] = w[i + j] (periodic)
        d1 += c1[k] * sh
        d2 += c2[k] * sh
    l1, l2 = d1 / w, d2 / w
    return (l2 / 6.0 - l1 * l1 / 4.0) / (2.0 * math.pi)


@dataclasses.dataclass
class Points:
    """A set of points: curve nodes (gid >= 0 is the node index) or proxy points (gid = -1).

    hs is the per-node speed term of the hypersingular diagonal (hypersingular_speed_term);
    zero for proxy points and where not given.
    """

    x: np.ndarray
    y: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    w: np.ndarray
    kappa: np.ndarray
    gid: np.ndarray
    hs: Optional[np.ndarray] = None

    def __post_init__(self):
        if self.hs is None:
            self.hs = np.zeros(self.x.shape[0])

    @staticmethod
    def from_curve(curve) -> "Points":
        n = curve.x.shape[0]
        return Points(curve.x, curve.y, curve.nx, curve.ny, curve.w, curve.kappa,
                      np.arange(n, dtype=np.int64), hypersingular_speed_term(curve.w))

    def fields(self):
        return (self.x, self.y, self.nx, self.ny, self.w, self.kappa, self.gid, self.hs)

    def take(self, idx) -> "Points":
        idx = np.asarray(idx, dtype=np.int64)
        return Points(*(v[idx] for v in self.fields()))

    @staticmethod
    def circle(cx: float, cy: float, radius: float, count: int) -> "Points":
        """Proxy ring (Sec. 4.1): equispaced points, outward radial normal, weight 2 pi R / P."""
        phi = 2.0 * np.pi * np.arange(count, dtype=np.float64) / count
        c, s = np.cos(phi), np.sin(phi)
        return Points(cx + radius * c, cy + radius * s, c, s,
                      np.full(count, 2.0 * np.pi * radius / count), np.zeros(count),
                      np.full(count, -1, dtype=np.int64))

    def __len__(self) -> int:
        return int(self.x.shape[0])


def hankel01(z: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """H_0^(1)(z), H_1^(1)(z) = J_n(z) + i Y_n(z) for real z > 0 (library Bessel functions)."""
    return _sp.j0(z) + 1j * _sp.y0(z), _sp.j1(z) + 1j * _sp.y1(z)


def _layer_kernels(k: float, r, a, b, nn):
    """Kernels of S_k, D_k, D*_k, N_k at separation r (c-A1 forms above).

    a = d.nu_obs, b = d.nu_src, nn = nu_obs.nu_src, d = x_obs - x_src.
    """
    h0, h1 = hankel01(k * r)
    g = 0.25j * h0
    c1 = (0.25j * k) * h1
    d = c1 * (b / r)
    ds = -(c1 * (a / r))
    n = c1 * (nn / r) + (0.25j * k) * ((a * b) / r) * (k * h0 / r - 2.0 * h1 / (r * r))
    return g, d, ds, n


def diag_S(k: float, w):
    """One-point corrected S~_k(i,i) (reading derived in the module docstring)."""
    return 0.25j - (1.0 / (2.0 * math.pi)) * (EULER_GAMMA + np.log(k * w / (4.0 * math.pi)))


def diag_D(kappa):
    """D~(i,i) = D*~(i,i) = -kappa_i / (4 pi): the continuous diagonal limit of the D kernel."""
    return -kappa / (4.0 * math.pi)


def diag_Ndiff(k0: float, k1: float, w):
    """One-point corrected (N_k0 - N_k1)~(i,i) (reading derived in the module docstring)."""
    dk2 = k0 * k0 - k1 * k1
    c = (0.125j * dk2
         - (1.0 / (4.0 * math.pi)) * (k0 * k0 * (math.log(k0 / 2.0) + EULER_GAMMA)
                                      - k1 * k1 * (math.log(k1 / 2.0) + EULER_GAMMA))
         + dk2 / (8.0 * math.pi))
    return c - (dk2 / (4.0 * math.pi)) * np.log(w / (2.0 * math.pi))


def kernel_blocks(obs: Points, src: Points, prm: Params, scaled: bool = True):
    """The four blocks (A11, A12, A21, A22) between every obs point and every src point.

    ``scaled`` selects the row-scaled symmetric system (Eq. 15); otherwise the
    unscaled baseline system of Sec. 6.  Pairs with the same node (gid equal and
    >= 0) receive the corrected diagonal and the free terms.
    """
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
    ks = e0 * e0 * g0 - e1 * e1 * g1
    kd = e0 * d0 - e1 * d1
    kds = e0 * ds0 - e1 * ds1
    kn = n0 - n1
    if same.any():
        oi, si = np.nonzero(same)
        wi = obs.w[oi]
        ks[oi, si] = e0 * e0 * diag_S(prm.k0, wi) - e1 * e1 * diag_S(prm.k1, wi)
        dd = diag_D(obs.kappa[oi])
        kd[oi, si] = e0 * dd - e1 * dd
        kds[oi, si] = e0 * dd - e1 * dd
        kn[oi, si] = diag_Ndiff(prm.k0, prm.k1, wi)
    if scaled:
        wgt = obs.w[:, None] * src.w[None, :]
        ftw = obs.w
    else:
        wgt = np.broadcast_to(src.w[None, :], dx.shape)
        ftw = np.ones_like(obs.w)
    a11 = -(wgt * ks)
    a12 = wgt * kd
    a21 = wgt * kds
    a22 = -(wgt * kn)
    if same.any():
        half = 0.5 * (e0 + e1) * ftw[oi]
        a12[oi, si] -= half
        a21[oi, si] += half
    return a11, a12, a21, a22


def entries(obs: Points, obs_eq, src: Points, src_comp, prm: Params, scaled: bool = True,
            chunk: int = 1 << 22) -> np.ndarray:
    """Dense block A[(p, e), (q, c)] for obs list (point p, equation e) x src list (point q, unknown c).

    e = 0 is the first equation row of Eq. 15 and e = 1 the second; c = 0 is the
    flux unknown q and c = 1 the trace unknown u.  ``obs``/``src`` give one point
    per row/column (repeats allowed).
    """
    obs_eq = np.asarray(obs_eq, dtype=np.int64)
    src_comp = np.asarray(src_comp, dtype=np.int64)
    m, n = len(obs), len(src)
    out = np.empty((m, n), dtype=np.complex128)
    if m == 0 or n == 0:
        return out
    step = max(1, chunk // max(n, 1))
    for i0 in range(0, m, step):
        i1 = min(m, i0 + step)
        blk = kernel_blocks(obs.take(np.arange(i0, i1)), src, prm, scaled)
        e = obs_eq[i0:i1, None]
        c = src_comp[None, :]
        out[i0:i1] = np.where(e == 0, np.where(c == 0, blk[0], blk[1]),
                              np.where(c == 0, blk[2], blk[3]))
    return out


def dense_matrix(curve, prm: Params, scaled: bool = True) -> np.ndarray:
    """The full 2N x 2N matrix with unknowns ordered [q_1..q_N, u_1..u_N] (Eq. 15 / Sec. 6)."""
    pts = Points.from_curve(curve)
    n = len(pts)
    both = Points(*(np.concatenate([v, v]) for v in pts.fields()))
    lab = np.concatenate([np.zeros(n, np.int64), np.ones(n, np.int64)])
    return entries(both, lab, both, lab, prm, scaled)


def incident_plane_wave(curve, k0: float, angle: float = 0.0):
    """u_in = exp(i k0 (x cos a + y sin a)) and its normal derivative at the nodes (Sec. 6)."""
    ca, sa = math.cos(angle), math.sin(angle)
    uin = np.exp(1j * k0 * (curve.x * ca + curve.y * sa))
    dudn = 1j * k0 * (curve.nx * ca + curve.ny * sa) * uin
    return uin, dudn


def rhs(curve, prm: Params, angle: float = 0.0, scaled: bool = True) -> np.ndarray:
    """Right-hand side [-eps0 W u_in ; W du_in/dnu] (row-scaled) or without W (baseline)."""
    uin, dudn = incident_plane_wave(curve, prm.k0, angle)
    f = np.concatenate([-prm.eps0 * uin, dudn])
    if scaled:
        f = f * np.concatenate([curve.w, curve.w])
    return f


def dense_solve(curve, prm: Params, angle: float = 0.0, scaled: bool = True) -> np.ndarray:
    """Reference solution [q; u] by dense LU with partial pivoting (LAPACK getrf/getrs)."""
    return np.linalg.solve(dense_matrix(curve, prm, scaled), rhs(curve, prm, angle, scaled))


def matvec_rows(curve, prm: Params, x: np.ndarray, rows: Optional[Sequence[int]] = None,
                scaled: bool = True) -> np.ndarray:
    """(A x)[rows] evaluated on the fly, rows indexing the 2N equations (no matrix stored)."""
    pts = Points.from_curve(curve)
    n = len(pts)
    rows = np.arange(2 * n) if rows is None else np.asarray(rows, dtype=np.int64)
    both = Points(*(np.concatenate([v, v]) for v in pts.fields()))
    lab = np.concatenate([np.zeros(n, np.int64), np.ones(n, np.int64)])
    out = np.empty(rows.shape[0], dtype=np.complex128)
    step = max(1, (1 << 21) // (2 * n))
    for i0 in range(0, rows.shape[0], step):
        rr = rows[i0:i0 + step]
        out[i0:i0 + step] = entries(both.take(rr), lab[rr], both, lab, prm, scaled) @ x
    return out
