"""Fixed-rank compression (Sec. 4.3, Theorem `order`: k_l = ceil(a^(L - l) k_L), with the paper's
k_L = 30 and a = 1.15) end to end on the GPU, against the oracle's fixed-rank HSS.

With the sketch off (oversample = 0) the GPU takes the same plain pivoted-QR IDs of the proxy
matrices as the oracle, so both build the same fixed-rank approximation: every level's ranks
follow the schedule exactly, and the two solutions agree to 1e-8 relative although the
approximation itself differs from the dense solution (the paper's ranks are smaller than this
problem's tolerance-chosen ones).
"""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import kernels as OK  # noqa: E402
from oracle.hss import HSS, Options  # noqa: E402
from synth import star  # noqa: E402


@pytest.mark.parametrize("mode", ["sym", "base"])
def test_fixed_rank_solver_matches_oracle_fixed_rank_hss(mode):
    from paper_2609_33216_b300.solver import Solver
    assert torch.cuda.is_available()
    c = star(2048)
    prm = OK.Params.from_wavenumbers(5.0, 8.0)
    kl, a = 30, 1.15
    s = Solver(c, prm.k0, prm.k1, prm.eps0, prm.eps1, mode=mode, leaf=128, nproxy=64, tol=1e-10,
               fixed_rank_kL=kl, rank_scale_a=a, oversample=0)
    s.compress()
    s.factor()
    x = s.solve(s.rhs(0.0)).cpu().numpy()
    depth = s.stats().depth
    for lvl in range(1, depth + 1):
        want = math.ceil(a ** (depth - lvl) * kl)
        got = np.asarray(s.ranks(lvl))
        # every box has more columns and rows than the schedule's rank here
        assert np.all(got == want), (lvl, got, want)
    s.close()
    h = HSS(c, prm, Options(leaf=128, nproxy=64, tol=1e-10, symmetric=(mode == "sym"), fixed_rank_kL=kl,
                            rank_scale_a=a))
    h.compress()
    h.factor()
    xo = h.solve(OK.rhs(c, prm, scaled=(mode == "sym")))
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
