"""Proxy-method HSS compression, factorisation and solve (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 4 step by step:

* Tree (Sec. 4.1, Theorem 1 setting): a binary tree over the node index order.
  A box [b, e) splits into [b, b + (e-b)//2) and the rest; all leaves sit at
  depth L = ceil(log2(N / leaf)).  Box centre = mean of the box's nodes, radius
  rho = largest node distance from the centre (readings: the paper only asks
  for a virtual boundary enclosing Gamma_i).
* Proxy method (Sec. 4.1, Table 2): the proxy ring has P points on the circle of
  radius proxy_factor * rho; the near set is every active point of another box
  of the same level strictly inside that circle (reading of "a neighborhood of
  Gamma_i").  M_R has rows = near (point, equation) pairs that are active in the
  compressed system, then the P proxy points for equation 1 and for equation 2;
  its columns are the box's active unknowns, flux part then trace part.
* Column ID (Sec. 4.1): Householder QR with column pivoting on each half of M_R;
  the pivot is the largest remaining column 2-norm (recomputed every step, ties
  to the lowest column index); stop at the first |R_kk| <= tol |R_00| (or at the
  fixed rank k_l = ceil(a^(L-l) k_L), Sec. 4.3).  T = R11^{-1} R12 and
  R^h = [I T] Pi^T.
* Symmetric mode: L_i = R_i^T (Eq. low-rank_R), plain transpose.
* Non-symmetric baseline: M_L (rows = the box's active equations, columns = near
  active unknowns then proxy sources) gets a row ID of each half; per half the
  row and column ranks are raised to their maximum so that R_i A_ii^{-1} L_i is
  square (reading: the paper's fixed-rank runs have equal ranks by construction).
* Factorisation (Sec. 4.2): Atilde_i = (R_i D_i^{-1} L_i)^{-1}; a parent's diagonal
  block is [[Atilde_c1, A(I_c1, J_c2)], [A(I_c2, J_c1), Atilde_c2]] with the
  children's skeleton rows I and columns J; the root block is LU-factorised.
* Solve (Sec. 4.2): up pass g = D^{-1} f, f~ = Atilde R g; root solve; down pass
  x = g - X (f~ - Atilde y) with X = D^{-1} L.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np
import scipy.linalg as sla

from .kernels import Params, Points, entries, rhs


# ----------------------------------------------------------------------------- ID


def cpqr_id(m: np.ndarray, tol: float, rank: Optional[int] = None):
    """Column interpolative decomposition M[:, perm] ~= M[:, perm[:r]] [I T].

    Householder QR with column pivoting; the remaining column norms are
    recomputed at every step.  With ``rank`` given the factorisation runs for
    exactly min(rank, m, n) steps, else it stops at the first step k whose
    pivot norm |R_kk| is <= tol * |R_00|.
    Returns (r, perm, T) with T of shape (r, n - r).
    """
    a = np.array(m, dtype=np.complex128, copy=True)
    rows, cols = a.shape
    perm = np.arange(cols)
    kmax = min(rows, cols) if rank is None else min(rows, cols, rank)
    ref = None
    k = 0
    while k < kmax:
        norms = np.sqrt(np.sum(np.abs(a[k:, k:]) ** 2, axis=0))
        j = k + int(np.argmax(norms))
        piv = norms[j - k]
        if ref is None:
            ref = piv
        if rank is None and (piv <= tol * ref or piv == 0.0):
            break
        if j != k:
            a[:, [k, j]] = a[:, [j, k]]
            perm[[k, j]] = perm[[j, k]]
        x = a[k:, k].copy()
        nx = np.linalg.norm(x)
        if nx == 0.0:
            break
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * nx
        v = x
        v[0] -= alpha
        v /= np.linalg.norm(v)
        a[k:, k:] -= 2.0 * np.outer(v, v.conj() @ a[k:, k:])
        k += 1
    r = k
    if r == 0:
        return 0, perm, np.zeros((0, cols), dtype=np.complex128)
    r11 = np.triu(a[:r, :r])
    t = sla.solve_triangular(r11, a[:r, r:], lower=False)
    return r, perm, t


def interp_matrix(r: int, perm: np.ndarray, t: np.ndarray) -> np.ndarray:
    """R = [I T] Pi^T as a dense r x n matrix (column perm[c] of R is column c of [I T])."""
    n = perm.shape[0]
    out = np.zeros((r, n), dtype=np.complex128)
    out[:, perm[:r]] = np.eye(r)
    out[:, perm[r:]] = t
    return out


# ----------------------------------------------------------------------------- tree


@dataclasses.dataclass
class Box:
    level: int
    index: int
    begin: int
    end: int
    cx: float = 0.0
    cy: float = 0.0
    rho: float = 0.0
    children: Tuple[int, ...] = ()
    # active sets per half h (0: flux columns / eq-1 rows, 1: trace columns / eq-2 rows)
    act: List[np.ndarray] = dataclasses.field(default_factory=list)
    actrow: List[np.ndarray] = dataclasses.field(default_factory=list)
    # column ID (from M_R) and row ID (from M_L; equal to the column ID when symmetric)
    rank: List[int] = dataclasses.field(default_factory=list)
    perm: List[np.ndarray] = dataclasses.field(default_factory=list)
    T: List[np.ndarray] = dataclasses.field(default_factory=list)
    rrank: List[int] = dataclasses.field(default_factory=list)
    rperm: List[np.ndarray] = dataclasses.field(default_factory=list)
    rT: List[np.ndarray] = dataclasses.field(default_factory=list)
    nproxy: int = 0
    # factorisation
    lu: object = None
    X: Optional[np.ndarray] = None
    At: Optional[np.ndarray] = None

    @property
    def skel(self):
        return [self.act[h][self.perm[h][: self.rank[h]]] for h in (0, 1)]

    @property
    def skelrow(self):
        return [self.actrow[h][self.rperm[h][: self.rrank[h]]] for h in (0, 1)]


def tree_depth(n: int, leaf: int) -> int:
    return 0 if n <= leaf else int(math.ceil(math.log2(n / leaf)))


def build_tree(curve, leaf: int) -> List[List[Box]]:
    """levels[l] lists the boxes of level l (root = level 0)."""
    n = curve.x.shape[0]
    depth = tree_depth(n, leaf)
    levels: List[List[Box]] = [[Box(0, 0, 0, n)]]
    for l in range(1, depth + 1):
        cur: List[Box] = []
        for parent in levels[l - 1]:
            mid = parent.begin + (parent.end - parent.begin) // 2
            i0 = len(cur)
            cur.append(Box(l, i0, parent.begin, mid))
            cur.append(Box(l, i0 + 1, mid, parent.end))
            parent.children = (i0, i0 + 1)
        levels.append(cur)
    for lev in levels:
        for b in lev:
            xs, ys = curve.x[b.begin:b.end], curve.y[b.begin:b.end]
            b.cx, b.cy = float(np.mean(xs)), float(np.mean(ys))
            b.rho = float(np.max(np.hypot(xs - b.cx, ys - b.cy))) if b.end > b.begin else 0.0
    return levels


# ----------------------------------------------------------------------------- solver


@dataclasses.dataclass
class Options:
    leaf: int = 64
    nproxy: int = 32
    proxy_factor: float = 1.5
    tol: float = 1e-10
    symmetric: bool = True
    fixed_rank_kL: int = 0        # > 0 selects the fixed-rank schedule of Sec. 4.3
    rank_scale_a: float = 1.15


def proxy_count(opts: Options, prm: Params, radius: float) -> int:
    """Proxy points on a ring of the given radius: at least ``nproxy``, and enough to
    resolve the fields of the larger wavenumber on that ring (2 k R + 32, rounded up
    to a multiple of 8).  Reading: the paper fixes no count."""
    kmax = max(prm.k0, prm.k1)
    need = int(math.ceil((2.0 * kmax * radius + 32.0) / 8.0)) * 8
    return max(opts.nproxy, need)


def _rows_points(pts: Points, ids_by_eq) -> Tuple[Points, np.ndarray]:
    ids = np.concatenate([np.asarray(i, dtype=np.int64) for i in ids_by_eq])
    lab = np.concatenate([np.full(len(i), e, dtype=np.int64) for e, i in enumerate(ids_by_eq)])
    return pts.take(ids), lab


def _stack(a: Points, b: Points) -> Points:
    return Points(*(np.concatenate([u, v]) for u, v in zip(a.fields(), b.fields())))


class HSS:
    """Oracle HSS solver: ``compress()``, ``factor()``, ``solve(f)``."""

    def __init__(self, curve, prm: Params, opts: Options):
        self.curve, self.prm, self.opts = curve, prm, opts
        self.pts = Points.from_curve(curve)
        self.n = curve.x.shape[0]
        self.levels = build_tree(curve, opts.leaf)
        self.depth = len(self.levels) - 1
        self.scaled = opts.symmetric

    # -- helpers
    def _fixed_rank(self, level: int) -> Optional[int]:
        if self.opts.fixed_rank_kL <= 0:
            return None
        return int(math.ceil(self.opts.rank_scale_a ** (self.depth - level) * self.opts.fixed_rank_kL))

    def near(self, box: Box, level: List[Box], which: str):
        """Per half h, the active points of other boxes of this level inside the proxy circle."""
        radius = self.opts.proxy_factor * box.rho
        out = []
        for h in (0, 1):
            sel = []
            for other in level:
                if other is box:
                    continue
                ids = other.actrow[h] if which == "row" else other.act[h]
                if len(ids) == 0:
                    continue
                d = np.hypot(self.curve.x[ids] - box.cx, self.curve.y[ids] - box.cy)
                sel.append(ids[d < radius])
            out.append(np.concatenate(sel) if sel else np.zeros(0, dtype=np.int64))
        return out

    def proxy_points(self, box: Box) -> Points:
        radius = self.opts.proxy_factor * box.rho
        box.nproxy = proxy_count(self.opts, self.prm, radius)
        return Points.circle(box.cx, box.cy, radius, box.nproxy)

    def m_r(self, box: Box, level: List[Box]) -> np.ndarray:
        """Proxy interaction matrix M_R: observations on Gamma_i', sources on Gamma_i (Table 2)."""
        nr = self.near(box, level, "row")
        prx = self.proxy_points(box)
        obs, lab = _rows_points(self.pts, nr)
        pl = np.concatenate([np.zeros(len(prx), np.int64), np.ones(len(prx), np.int64)])
        obs = _stack(obs, _stack(prx, prx))
        lab = np.concatenate([lab, pl])
        src, comp = _rows_points(self.pts, box.act)
        return entries(obs, lab, src, comp, self.prm, self.scaled)

    def m_l(self, box: Box, level: List[Box]) -> np.ndarray:
        """Proxy interaction matrix M_L: observations on Gamma_i, sources on Gamma_i' (Table 2)."""
        nc = self.near(box, level, "col")
        prx = self.proxy_points(box)
        src, comp = _rows_points(self.pts, nc)
        pl = np.concatenate([np.zeros(len(prx), np.int64), np.ones(len(prx), np.int64)])
        src = _stack(src, _stack(prx, prx))
        comp = np.concatenate([comp, pl])
        obs, lab = _rows_points(self.pts, box.actrow)
        return entries(obs, lab, src, comp, self.prm, self.scaled)

    # -- compression (Sec. 4.1)
    def compress(self):
        opts = self.opts
        for l in range(self.depth, 0, -1):
            level = self.levels[l]
            for box in level:
                if l == self.depth:
                    ids = np.arange(box.begin, box.end, dtype=np.int64)
                    box.act = [ids, ids]
                    box.actrow = [ids, ids]
                else:
                    c1, c2 = (self.levels[l + 1][c] for c in box.children)
                    box.act = [np.concatenate([c1.skel[h], c2.skel[h]]) for h in (0, 1)]
                    box.actrow = [np.concatenate([c1.skelrow[h], c2.skelrow[h]]) for h in (0, 1)]
            fixed = self._fixed_rank(l)
            for box in level:
                mr = self.m_r(box, level)
                n0 = len(box.act[0])
                halves = [mr[:, :n0], mr[:, n0:]]
                box.rank, box.perm, box.T = [], [], []
                for h in (0, 1):
                    r, p, t = cpqr_id(halves[h], opts.tol, fixed)
                    box.rank.append(r)
                    box.perm.append(p)
                    box.T.append(t)
                if opts.symmetric:
                    box.rrank, box.rperm, box.rT = box.rank, box.perm, box.T
                    continue
                ml = self.m_l(box, level)
                m0 = len(box.actrow[0])
                rhalves = [ml[:m0, :].T, ml[m0:, :].T]
                box.rrank, box.rperm, box.rT = [], [], []
                for h in (0, 1):
                    r, p, t = cpqr_id(rhalves[h], opts.tol, fixed)
                    k = max(r, box.rank[h])
                    if r < k:
                        r, p, t = cpqr_id(rhalves[h], opts.tol, k)
                    if box.rank[h] < k:
                        box.rank[h], box.perm[h], box.T[h] = cpqr_id(halves[h], opts.tol, k)
                    box.rrank.append(r)
                    box.rperm.append(p)
                    box.rT.append(t)
        return self

    # -- factorisation (Sec. 4.2)
    def _positions(self, box: Box, level: int):
        """Position of each active unknown (per half, in active-set order) in the box's
        diagonal-block ordering: leaf [flux; trace], parent [child1 (flux; trace); child2 (...)]."""
        if level == self.depth:
            n = box.end - box.begin
            return [np.arange(n), n + np.arange(n)]
        c1, c2 = (self.levels[level + 1][c] for c in box.children)
        a1 = c1.rank[0] + c1.rank[1]
        pos = []
        for h in (0, 1):
            o1 = 0 if h == 0 else c1.rank[0]
            o2 = a1 + (0 if h == 0 else c2.rank[0])
            pos.append(np.concatenate([o1 + np.arange(c1.rank[h]), o2 + np.arange(c2.rank[h])]))
        return pos

    def _diag_block(self, box: Box, level: int) -> np.ndarray:
        if level == self.depth:
            ids = np.arange(box.begin, box.end, dtype=np.int64)
            obs, lab = _rows_points(self.pts, [ids, ids])
            return entries(obs, lab, obs, lab, self.prm, self.scaled)
        c1, c2 = (self.levels[level + 1][c] for c in box.children)
        r1, l1 = _rows_points(self.pts, c1.skelrow)
        r2, l2 = _rows_points(self.pts, c2.skelrow)
        s1, k1 = _rows_points(self.pts, c1.skel)
        s2, k2 = _rows_points(self.pts, c2.skel)
        top = np.hstack([c1.At, entries(r1, l1, s2, k2, self.prm, self.scaled)])
        bot = np.hstack([entries(r2, l2, s1, k1, self.prm, self.scaled), c2.At])
        return np.vstack([top, bot])

    def _basis(self, box: Box, level: int, row: bool) -> np.ndarray:
        """Dense R^T (row=False) or L (row=True) in the box's diagonal-block ordering."""
        pos = self._positions(box, level)
        rank = box.rrank if row else box.rank
        perm = box.rperm if row else box.perm
        tt = box.rT if row else box.T
        size = sum(len(p) for p in pos)
        out = np.zeros((size, rank[0] + rank[1]), dtype=np.complex128)
        for h in (0, 1):
            c0 = 0 if h == 0 else rank[0]
            rmat = interp_matrix(rank[h], perm[h], tt[h])  # rank x n_h
            out[pos[h], c0:c0 + rank[h]] = rmat.T
        return out

    def factor(self):
        if self.depth == 0:
            root = self.levels[0][0]
            root.lu = sla.lu_factor(self._diag_block_leafroot())
            return self
        for l in range(self.depth, 0, -1):
            for box in self.levels[l]:
                d = self._diag_block(box, l)
                box.lu = sla.lu_factor(d)
                lmat = self._basis(box, l, row=True)
                box.X = sla.lu_solve(box.lu, lmat)
                rt = self._basis(box, l, row=False)
                box.At = np.linalg.inv(rt.T @ box.X)
        root = self.levels[0][0]
        root.lu = sla.lu_factor(self._diag_block(root, 0))
        return self

    def _diag_block_leafroot(self):
        ids = np.arange(self.n, dtype=np.int64)
        obs, lab = _rows_points(self.pts, [ids, ids])
        return entries(obs, lab, obs, lab, self.prm, self.scaled)

    # -- solve (Sec. 4.2)
    def solve(self, f: np.ndarray) -> np.ndarray:
        """Solve with the system's own right-hand side f ([eq1 rows; eq2 rows], 2N)."""
        n = self.n
        if self.depth == 0:
            return sla.lu_solve(self.levels[0][0].lu, f)
        g, ft = {}, {}
        for l in range(self.depth, 0, -1):
            for box in self.levels[l]:
                if l == self.depth:
                    fb = np.concatenate([f[box.begin:box.end], f[n + box.begin:n + box.end]])
                else:
                    c1, c2 = (self.levels[l + 1][c] for c in box.children)
                    fb = np.concatenate([ft[(l + 1, c1.index)], ft[(l + 1, c2.index)]])
                gb = sla.lu_solve(box.lu, fb)
                rt = self._basis(box, l, row=False)
                g[(l, box.index)] = gb
                ft[(l, box.index)] = box.At @ (rt.T @ gb)
        root = self.levels[0][0]
        c1, c2 = (self.levels[1][c] for c in root.children)
        y = {0: sla.lu_solve(root.lu, np.concatenate([ft[(1, c1.index)], ft[(1, c2.index)]]))}
        x = np.empty(2 * n, dtype=np.complex128)
        ys = {(0, 0): y[0]}
        for l in range(1, self.depth + 1):
            for parent in self.levels[l - 1]:
                yp = ys[(l - 1, parent.index)]
                c1, c2 = (self.levels[l][c] for c in parent.children)
                a1 = c1.rank[0] + c1.rank[1]
                for c, yc in ((c1, yp[:a1]), (c2, yp[a1:])):
                    xb = g[(l, c.index)] - c.X @ (ft[(l, c.index)] - c.At @ yc)
                    if l == self.depth:
                        m = c.end - c.begin
                        x[c.begin:c.end] = xb[:m]
                        x[n + c.begin:n + c.end] = xb[m:]
                    else:
                        ys[(l, c.index)] = xb
        return x

    # -- reporting
    def ranks(self):
        """Per level (leaf first): list of (rank_flux, rank_trace) per box."""
        return [[tuple(b.rank) for b in self.levels[l]] for l in range(self.depth, 0, -1)]


def hss_solve(curve, prm: Params, opts: Options, angle: float = 0.0):
    """Compress, factor and solve; returns (x, solver).  x = [q; u]."""
    s = HSS(curve, prm, opts).compress().factor()
    return s.solve(rhs(curve, prm, angle, opts.symmetric)), s
