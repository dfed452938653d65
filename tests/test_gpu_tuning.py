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
    assert t.lu_panel_cluster in (1, 2, 4, 8, 16)
    assert S.symhss_get_tuning(s.h).as_dict() == t.as_dict()
    x = s.solve(s.rhs(0.0))  # factorised by the autotuner
    assert torch.isfinite(torch.view_as_real(x)).all()
    s.close()
