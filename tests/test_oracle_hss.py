"""Pins of the oracle's ID and HSS solver.

* the column ID recovers the exact rank of a rank-k product and reproduces it to
  rounding; its pivot order equals LAPACK's pivoted QR when the column norms are
  well separated; fixed-rank mode stops at the requested rank;
* with every ID kept at full rank the multilevel elimination of Sec. 4.2 is exact, so
  it equals dense LU to rounding (pins the block algebra and orderings);
* at tol 1e-10 the symmetric single-ID solver and the two-ID baseline agree with
  dense LU (Example 2: the symmetric formulation does not degrade accuracy);
* the proxy-method basis reproduces the whole far block row of a leaf box;
* the fixed-rank schedule follows k_l = ceil(a^(L-l) k_L) (Sec. 4.3).
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hss as H
from oracle import kernels as K
from synth import disk, star, workload


def _rng():
    return np.random.default_rng(7)


def test_id_recovers_exact_rank():
    rng = _rng()
    for m, n, k in ((60, 40, 9), (200, 90, 31), (30, 50, 30)):
        a = (rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))) @ \
            (rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n)))
        r, perm, t = H.cpqr_id(a, 1e-12)
        assert r == k
        rec = a[:, perm[:r]] @ H.interp_matrix(r, perm, t)
        assert np.linalg.norm(rec - a) <= 1e-12 * np.linalg.norm(a)


def test_id_pivots_match_lapack_pivoted_qr():
    rng = _rng()
    m, n = 80, 40
    a = (rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))) * (0.5 ** np.arange(n))[rng.permutation(n)]
    r, perm, _ = H.cpqr_id(a, 0.0, rank=12)
    _, _, p = sla.qr(a, pivoting=True, mode="economic")
    assert list(perm[:12]) == list(p[:12])


def test_id_fixed_rank_and_tolerance_stop():
    rng = _rng()
    a = rng.normal(size=(50, 30)) * (10.0 ** -np.arange(30))
    r, _, t = H.cpqr_id(a, 0.0, rank=7)
    assert r == 7 and t.shape == (7, 23)
    r, perm, t = H.cpqr_id(a, 1e-6)
    # the stop is the first pivot norm <= tol * first pivot norm
    q, rr, p = sla.qr(a, pivoting=True)
    d = np.abs(np.diag(rr))
    assert r == int(np.argmax(d <= 1e-6 * d[0]))


def test_full_rank_hss_equals_dense_lu():
    c = star(256)
    prm = K.Params.from_wavenumbers(6.0, 9.0)
    for sym in (True, False):
        x, s = H.hss_solve(c, prm, H.Options(leaf=32, nproxy=32, tol=1e-300, symmetric=sym))
        xd = K.dense_solve(c, prm, scaled=sym)
        assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


@pytest.mark.parametrize("sym", [True, False], ids=["sym", "base"])
def test_disk512_hss_matches_dense(sym):
    w = workload("disk512")
    prm = K.Params(w["k0"], w["k1"], w["eps0"], w["eps1"])
    x, s = H.hss_solve(w["curve"], prm, H.Options(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"],
                                                  symmetric=sym))
    xd = K.dense_solve(w["curve"], prm)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert all(0 < r < 64 for lev in s.ranks()[:1] for box in lev for r in box)


@pytest.mark.slow
def test_star_sym_and_base_agree_with_dense():
    c = star(1024)
    prm = K.Params.from_wavenumbers(20.0, 30.0)
    xd = K.dense_solve(c, prm)
    for sym in (True, False):
        x, _ = H.hss_solve(c, prm, H.Options(leaf=128, nproxy=64, tol=1e-10, symmetric=sym))
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_proxy_basis_reproduces_far_block_row():
    c = star(1024)
    prm = K.Params.from_wavenumbers(20.0, 30.0)
    s = H.HSS(c, prm, H.Options(leaf=128, nproxy=64, tol=1e-10))
    s.compress()
    leaf = s.levels[-1][3]
    ids = np.arange(leaf.begin, leaf.end)
    other = np.setdiff1d(np.arange(c.n), ids)
    pts = K.Points.from_curve(c)
    obs, lab = H._rows_points(pts, [other, other])
    src, comp = H._rows_points(pts, [ids, ids])
    blk = K.entries(obs, lab, src, comp, prm)
    n = len(ids)
    for h in (0, 1):
        half = blk[:, h * n:(h + 1) * n]
        r, perm, t = leaf.rank[h], leaf.perm[h], leaf.T[h]
        rec = half[:, perm[:r]] @ H.interp_matrix(r, perm, t)
        assert np.linalg.norm(rec - half) <= 1e-8 * np.linalg.norm(half)


def test_fixed_rank_schedule():
    c = disk(512)
    prm = K.Params.from_wavenumbers(5.0, 8.0)
    s = H.HSS(c, prm, H.Options(leaf=64, nproxy=32, fixed_rank_kL=20, rank_scale_a=1.15)).compress()
    depth = s.depth
    for i, lev in enumerate(s.ranks()):
        level = depth - i
        want = math.ceil(1.15 ** (depth - level) * 20)
        for box in lev:
            for r in box:
                assert r == want
