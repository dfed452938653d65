"""End-to-end GPU solver parity against the FP64 oracle, through the C ABI.

* unit disk, 512 nodes (k0 = 5, k1 = 8, leaf 64, 32-point rings, tol 1e-10): symmetric and
  baseline solutions within 1e-8 of the oracle's dense LU, and within the discretisation
  error of the Bessel-series solution (Example 2);
* a star with 2048 nodes at k0 = 20, k1 = 30 (leaf 128): both modes within 1e-8 of dense LU;
  GPU leaf ranks within one of the oracle's;
* the transparent obstacle (k1 = k0, eps1 = eps0 = 2.5) returns u = u_in, q = du_in/dnu / eps0;
* several right-hand sides at once, host-buffer solve, curve replacement and uneven trees;
* the 16384-node star at k0 = 20, k1 = 30 (the benchmark workload): sampled rows of the
  residual, evaluated by the oracle one row at a time, and agreement of both modes;
* error paths: calls out of order are refused without touching the device.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import hss as OH  # noqa: E402
from oracle import kernels as OK  # noqa: E402
from oracle.exact import disk_solution  # noqa: E402
from synth import disk, fourier_star, star, workload  # noqa: E402


@pytest.fixture(scope="module")
def solver_mod():
    from paper_2609_33216_b300 import solver
    assert torch.cuda.is_available()
    return solver


def _run(solver_mod, curve, prm: OK.Params, mode="sym", angle=0.0, **kw):
    s = solver_mod.Solver(curve, prm.k0, prm.k1, prm.eps0, prm.eps1, mode=mode, **kw)
    s.compress()
    s.factor()
    x = s.solve(s.rhs(angle))
    torch.cuda.synchronize()
    return x.cpu().numpy(), s


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mode", ["sym", "base"])
def test_disk512_matches_dense_and_bessel(solver_mod, mode):
    w = workload("disk512")
    prm = OK.Params(w["k0"], w["k1"], w["eps0"], w["eps1"])
    x, s = _run(solver_mod, w["curve"], prm, mode, leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    xd = OK.dense_solve(w["curve"], prm)
    assert _rel(x, xd) <= 1e-8
    th = 2 * np.pi * np.arange(512) / 512
    q, u = disk_solution(th, prm.k0, prm.k1, prm.eps0, prm.eps1)
    assert _rel(x, np.concatenate([q, u])) <= 1.2e-5
    s.close()


@pytest.mark.parametrize("mode", ["sym", "base"])
def test_star2048_matches_dense(solver_mod, mode):
    c = star(2048)
    prm = OK.Params.from_wavenumbers(20.0, 30.0)
    xd = OK.dense_solve(c, prm)
    x, s = _run(solver_mod, c, prm, mode, leaf=128, nproxy=64, tol=1e-10)
    assert _rel(x, xd) <= 1e-8
    s.close()
    # the plain ID (no sketch) reproduces the oracle's ranks
    x, s = _run(solver_mod, c, prm, mode, leaf=128, nproxy=64, tol=1e-10, oversample=0)
    assert _rel(x, xd) <= 1e-8
    oracle = OH.HSS(c, prm, OH.Options(leaf=128, nproxy=64, tol=1e-10, symmetric=(mode == "sym"))).compress()
    depth = oracle.depth
    gpu_leaf = s.ranks(depth)
    ora_leaf = oracle.ranks()[0]
    for g, o in zip(gpu_leaf, ora_leaf):
        assert abs(g[0] - o[0]) <= 1 and abs(g[1] - o[1]) <= 1
    s.close()


def test_transparent_obstacle_exact(solver_mod):
    c = star(1024)
    prm = OK.Params(4.0, 4.0, 2.5, 2.5)
    x, s = _run(solver_mod, c, prm, "sym", leaf=64, nproxy=32, tol=1e-12)
    uin, dudn = OK.incident_plane_wave(c, prm.k0)
    np.testing.assert_allclose(x[1024:], uin, atol=1e-11)
    np.testing.assert_allclose(x[:1024], dudn / prm.eps0, atol=1e-10)
    s.close()


def test_multiple_rhs_host_solve_and_set_curve(solver_mod):
    c = fourier_star(1500, ((2, 0.1, 0.3), (7, 0.03, 1.0)))  # uneven tree: 16 leaves of 93 or 94 nodes
    prm = OK.Params.from_wavenumbers(12.0, 18.0)
    s = solver_mod.Solver(c, prm.k0, prm.k1, prm.eps0, prm.eps1, leaf=128, nproxy=64, tol=1e-10)
    s.compress()
    s.factor()
    f = torch.stack([s.rhs(0.0), s.rhs(1.1)])
    x = s.solve(f).cpu().numpy()
    for i, ang in enumerate((0.0, 1.1)):
        xd = OK.dense_solve(c, prm, angle=ang)
        assert _rel(x[i], xd) <= 1e-8
    xh = s.solve_host(f.cpu().numpy())
    np.testing.assert_allclose(xh, x, rtol=0, atol=1e-14 * np.abs(x).max())
    c2 = fourier_star(1500, ((3, 0.12, 0.0),))
    s.set_curve(c2)
    s.compress()
    s.factor()
    x2 = s.solve(s.rhs(0.0)).cpu().numpy()
    assert _rel(x2, OK.dense_solve(c2, prm)) <= 1e-8
    s.close()


def test_small_problem_without_tree(solver_mod):
    c = disk(100)
    prm = OK.Params.from_wavenumbers(3.0, 5.0)
    x, s = _run(solver_mod, c, prm, "sym", leaf=128)
    assert _rel(x, OK.dense_solve(c, prm)) <= 1e-12
    s.close()


def test_calls_out_of_order_are_refused(solver_mod):
    from paper_2609_33216_b300 import symhss as S
    s = solver_mod.Solver(disk(256), 5.0, 8.0, leaf=64)
    with pytest.raises(S.SymhssError) as e:
        s.factor()
    assert e.value.code == S.SYMHSS_ERR_STATE
    with pytest.raises(S.SymhssError) as e:
        s.solve(torch.zeros(512, dtype=torch.complex128, device="cuda"))
    assert e.value.code == S.SYMHSS_ERR_STATE
    s.close()


def test_benchmark_workload_residual_and_modes(solver_mod):
    w = workload("star16k")
    prm = OK.Params(w["k0"], w["k1"], w["eps0"], w["eps1"])
    c = w["curve"]
    kw = dict(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    xs, s = _run(solver_mod, c, prm, "sym", **kw)
    xb, b = _run(solver_mod, c, prm, "base", **kw)
    assert _rel(xs, xb) <= 1e-8
    rng = np.random.default_rng(5)
    rows = rng.choice(2 * c.n, 48, replace=False)
    f = OK.rhs(c, prm)
    res = OK.matvec_rows(c, prm, xs, rows) - f[rows]
    assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(f[rows])
    st = s.stats()
    assert st.depth == 7 and st.nboxes_leaf == 128
    s.close()
    b.close()


@pytest.mark.slow
def test_benchmark_workload_matches_oracle_hss(solver_mod):
    """GPU symmetric solver vs the oracle's symmetric HSS on the 16384-node star."""
    w = workload("star16k")
    prm = OK.Params(w["k0"], w["k1"], w["eps0"], w["eps1"])
    c = w["curve"]
    x, s = _run(solver_mod, c, prm, "sym", leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"])
    s.close()
    xo, _ = OH.hss_solve(c, prm, OH.Options(leaf=w["leaf"], nproxy=w["nproxy"], tol=w["tol"]))
    assert _rel(x, xo) <= 1e-8


def test_sketched_and_plain_ids_agree(solver_mod):
    """The randomized-sketch ID (default) and the ID of the full proxy matrices (oversample 0)
    give the same solution to the solver tolerance, in both modes."""
    c = star(2048)
    prm = OK.Params.from_wavenumbers(20.0, 30.0)
    xd = OK.dense_solve(c, prm)
    for mode in ("sym", "base"):
        xs, s1 = _run(solver_mod, c, prm, mode, leaf=128, nproxy=64, tol=1e-10)
        xp, s2 = _run(solver_mod, c, prm, mode, leaf=128, nproxy=64, tol=1e-10, oversample=0)
        assert _rel(xs, xd) <= 1e-8 and _rel(xp, xd) <= 1e-8
        assert s1.stats().kernel_launches[5] > 0 and s2.stats().kernel_launches[5] == 0
        s1.close()
        s2.close()
