"""Batched solve of many independent scatterers in one handle, through the C ABI.

* a batch of random star scatterers of uneven size and different wavenumbers
  (the random_star_batch family: r = 1 + sum_m a_m cos(m theta + phi_m)): every
  problem's block of the batch solution within 1e-8 of the oracle's dense LU of
  that problem alone, in both modes;
* a batch mixing a problem whose tree is a single leaf (its root at height 0) with
  deeper trees, and problems given in any order;
* the batch and single-problem handles give the same solution per problem;
* the batch's kernel launches follow the tallest tree and largest blocks, not the number
  of problems.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import kernels as OK  # noqa: E402
from synth import random_star_batch, star  # noqa: E402


@pytest.fixture(scope="module")
def solver_mod():
    from paper_2609_33216_b300 import solver
    assert torch.cuda.is_available()
    return solver


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _batch(solver_mod, probs, mode="sym", **kw):
    b = solver_mod.BatchSolver([p["curve"] for p in probs], [p["k0"] for p in probs], [p["k1"] for p in probs],
                               [p["eps0"] for p in probs], [p["eps1"] for p in probs], mode=mode, **kw)
    b.compress()
    b.factor()
    x = b.solve(b.rhs(0.0))
    torch.cuda.synchronize()
    return x.cpu().numpy(), b


@pytest.fixture(scope="module")
def small_batch():
    probs = random_star_batch(5, seed=11, n_min=300, n_max=1800, k_range=(5.0, 25.0))
    dense = [OK.dense_solve(p["curve"], OK.Params(p["k0"], p["k1"], p["eps0"], p["eps1"])) for p in probs]
    return probs, dense


@pytest.mark.parametrize("mode", ["sym", "base"])
def test_batch_matches_dense_per_problem(solver_mod, small_batch, mode):
    probs, dense = small_batch
    x, b = _batch(solver_mod, probs, mode, leaf=64, nproxy=32, tol=1e-10)
    assert b.rows == 2 * sum(p["curve"].n for p in probs)
    assert len(set(b.depths)) > 1  # uneven trees
    for c, xd in enumerate(dense):
        xc = x[b.row0[c]:b.row0[c] + 2 * b.ns[c]]
        assert _rel(xc, xd) <= 1e-8, (c, _rel(xc, xd))
    b.close()


def test_batch_with_single_leaf_problem(solver_mod, small_batch):
    probs, dense = small_batch
    tiny = random_star_batch(1, seed=5, n_min=40, n_max=60, k_range=(3.0, 6.0))[0]
    dt = OK.dense_solve(tiny["curve"], OK.Params(tiny["k0"], tiny["k1"], tiny["eps0"], tiny["eps1"]))
    order = [2, 0, 4]
    mixed = [probs[order[0]], tiny, probs[order[1]], probs[order[2]]]
    ref = [dense[order[0]], dt, dense[order[1]], dense[order[2]]]
    x, b = _batch(solver_mod, mixed, "sym", leaf=64, nproxy=32, tol=1e-10)
    assert b.depths[1] == 0
    for c, xd in enumerate(ref):
        xc = x[b.row0[c]:b.row0[c] + 2 * b.ns[c]]
        assert _rel(xc, xd) <= 1e-8, (c, _rel(xc, xd))
    b.close()


def test_batch_agrees_with_single_handles(solver_mod):
    probs = random_star_batch(3, seed=3, n_min=2048, n_max=6000, k_range=(10.0, 30.0))
    x, b = _batch(solver_mod, probs, "sym", leaf=128, nproxy=64, tol=1e-10)
    for c, p in enumerate(probs):
        s = solver_mod.Solver(p["curve"], p["k0"], p["k1"], p["eps0"], p["eps1"], leaf=128, nproxy=64, tol=1e-10)
        s.compress()
        s.factor()
        xs = s.solve(s.rhs(0.0)).cpu().numpy()
        xc = x[b.row0[c]:b.row0[c] + 2 * b.ns[c]]
        # different sketch draws per handle: agreement at the ID tolerance, not bitwise
        assert _rel(xc, xs) <= 1e-8, (c, _rel(xc, xs))
        # per-problem ranks are those of a handle holding that problem alone, within a few
        lv = b.depths[c]
        rb = np.array(b.ranks(c, lv))
        rs = np.array(s.ranks(lv))
        assert np.abs(rb - rs).max() <= 2
        s.close()
    b.close()


def test_batch_launches_do_not_grow_with_problem_count(solver_mod):
    from paper_2609_33216_b300 import symhss as S
    probs = random_star_batch(6, seed=8, n_min=1000, n_max=4000, k_range=(5.0, 20.0))
    n0 = S.lib.symhss_launch_count()
    x, b = _batch(solver_mod, probs, "sym", leaf=128, nproxy=64, tol=1e-10)
    batch_launches = S.lib.symhss_launch_count() - n0
    b.close()
    singles = []
    for p in probs:
        n0 = S.lib.symhss_launch_count()
        x, b = _batch(solver_mod, [p], "sym", leaf=128, nproxy=64, tol=1e-10)
        singles.append(S.lib.symhss_launch_count() - n0)
        b.close()
    # one launch per kernel and height: the blocked LU adds panel launches for the largest
    # block of a height, and a batched height of >= 32 blocks takes the tensor-core path (64-column
    # blocks, two launches per product) that a single problem's few blocks do not, so the batch
    # may exceed its largest single problem by a bounded factor; it stays far below their sum
    assert batch_launches <= 1.5 * max(singles), (batch_launches, singles)
    assert batch_launches <= 0.4 * sum(singles), (batch_launches, singles)


def test_batch_set_curves_and_multiple_rhs(solver_mod):
    probs = random_star_batch(3, seed=21, n_min=500, n_max=1500, k_range=(5.0, 15.0))
    b = solver_mod.BatchSolver([p["curve"] for p in probs], [p["k0"] for p in probs], [p["k1"] for p in probs],
                               leaf=64, nproxy=32, tol=1e-10)
    moved = []
    for p in probs:  # same node counts, shifted curves
        c = p["curve"]
        moved.append(type(c)(c.x + 0.25, c.y - 0.5, c.nx, c.ny, c.w, c.kappa, c.name))
    b.set_curves(moved)
    b.compress()
    b.factor()
    f = torch.stack([b.rhs(0.0), b.rhs(0.7)])
    x = b.solve(f).cpu().numpy()
    for c, p in enumerate(probs):
        prm = OK.Params(p["k0"], p["k1"], p["eps0"], p["eps1"])
        for j, ang in enumerate([0.0, 0.7]):
            xd = OK.dense_solve(moved[c], prm, angle=ang)
            xc = x[j, b.row0[c]:b.row0[c] + 2 * b.ns[c]]
            assert _rel(xc, xd) <= 1e-8
    b.close()
