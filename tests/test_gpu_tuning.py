"""Launch tuning and the autotuner (symhss_set_tuning / symhss_autotune): every tunable only
changes launch shapes, so every setting gives the same solution (bit for bit: the same
arithmetic runs in other blocks or streams), and the autotuner returns a valid setting with
the handle left factorised."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from synth import star  # noqa: E402


@pytest.fixture(scope="module")
def mods():
    from paper_2609_33216_b300 import solver as SV
    from paper_2609_33216_b300 import symhss as S
    assert torch.cuda.is_available()
    return SV, S


def test_every_tuning_gives_the_same_solution(mods):
    SV, S = mods
    s = SV.Solver(star(6000), 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10)
    ref = None
    for la, pt, ch, cm, pc in [(0, 1024, 0, 16, 1), (1, 1024, 0, 16, 8), (0, 256, 8, 1, 16), (1, 512, 32, 4, 2),
                               (0, 512, 16, 8, 4)]:
        S.symhss_set_tuning(s.h, lu_lookahead=la, lu_panel_threads=pt, tile_loop_chunk=ch, id_cluster_max=cm,
                            lu_panel_cluster=pc)
        s.compress()
        s.factor()
        x = s.solve(s.rhs(0.0)).cpu().numpy()
        if ref is None:
            ref = x
        else:
            assert np.array_equal(x, ref), (la, pt, ch, cm, pc, np.abs(x - ref).max())
    with pytest.raises(S.SymhssError):
        S.symhss_set_tuning(s.h, lu_panel_threads=300)
    s.close()


def test_autotune_returns_valid_setting_and_leaves_handle_factored(mods):
    SV, S = mods
    s = SV.Solver(star(4096), 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10)
    t = S.symhss_autotune(s.h, reps=1)
    assert t.lu_lookahead in (0, 1) and t.lu_panel_threads in (256, 512, 1024)
    assert t.tile_loop_chunk in (0, 8, 16, 32) and t.id_cluster_max in (1, 2, 4, 8, 16)
    assert t.lu_panel_cluster in (1, 2, 4, 8, 16) and t.lu_tc in (0, 1, 2) and t.lu_outer in (16, 32, 64)
    assert S.symhss_get_tuning(s.h).as_dict() == t.as_dict()
    x = s.solve(s.rhs(0.0))  # factorised by the autotuner
    assert torch.isfinite(torch.view_as_real(x)).all()
    s.close()


def test_tensor_core_and_fp64_factorisations_agree(mods):
    """lu_tc = 1 (blocked LU and solves with tensor-core updates, column blocks of lu_outer = 64, 32
    or 16), lu_tc = 0 (16-column LU and unblocked solves on the FP64 pipe) and lu_tc = 2 (the first
    at levels of >= 32 blocks) factorise the same compressed system: the solutions agree to FP64
    rounding amplified by the blocks' conditioning (<= 1e-11 relative)."""
    SV, S = mods
    s = SV.Solver(star(6000), 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10)
    xs = []
    for tc, outer in ((1, 64), (0, 64), (2, 64), (1, 16), (1, 32), (2, 16)):
        S.symhss_set_tuning(s.h, lu_tc=tc, lu_outer=outer)
        s.compress()
        s.factor()
        xs.append(s.solve(s.rhs(0.0)).cpu().numpy())
    for i in (0, 2, 3, 4, 5):
        assert np.linalg.norm(xs[i] - xs[1]) / np.linalg.norm(xs[1]) <= 1e-11, i
    s.close()


@pytest.mark.parametrize("mode,precision", [("sym", "fp64"), ("base", "fp64"), ("sym", "mixed")])
def test_pipelined_build_matches_compress_then_factor(mods, mode, precision):
    """symhss_build runs the compression of height t + 1 on a second stream while height t is
    factorised: the same kernels on the same data, so the solution is bit for bit that of
    symhss_compress followed by symhss_factor, with the same launch count and ranks."""
    SV, S = mods
    s = SV.Solver(star(6000), 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10, mode=mode, precision=precision)
    s.compress()
    s.factor()
    ref = s.solve(s.rhs(0.0)).cpu().numpy()
    st0 = s.stats()
    r0 = [list(s.ranks(lev)) for lev in range(1, st0.depth + 1)]
    for _ in range(2):
        s.build()
        x = s.solve(s.rhs(0.0)).cpu().numpy()
        assert np.array_equal(x, ref), np.abs(x - ref).max()
    st1 = s.stats()
    assert st1.ms_build > 0
    assert list(st1.kernel_launches) == list(st0.kernel_launches)
    assert [list(s.ranks(lev)) for lev in range(1, st1.depth + 1)] == r0
    s.close()


def test_pipelined_build_batch_and_single_leaf(mods):
    SV, S = mods
    from synth import random_star_batch
    probs = random_star_batch(4, seed=17, n_min=40, n_max=5000, k_range=(5.0, 25.0))
    args = ([p["curve"] for p in probs], [p["k0"] for p in probs], [p["k1"] for p in probs],
            [p["eps0"] for p in probs], [p["eps1"] for p in probs])
    b = SV.BatchSolver(*args, leaf=64, nproxy=32, tol=1e-10)
    b.compress()
    b.factor()
    ref = b.solve(b.rhs(0.0)).cpu().numpy()
    b.build()
    x = b.solve(b.rhs(0.0)).cpu().numpy()
    assert np.array_equal(x, ref)
    b.close()
    # a handle whose tree is a single leaf: nothing to compress, the build only factorises
    t = SV.Solver(star(100), 5.0, 8.0, leaf=128, nproxy=32, tol=1e-10)
    t.compress()
    t.factor()
    r1 = t.solve(t.rhs(0.0)).cpu().numpy()
    t.build()
    assert np.array_equal(t.solve(t.rhs(0.0)).cpu().numpy(), r1)
    t.close()
