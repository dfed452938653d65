"""Failure paths of the solver handle, driven from the host without faulting the GPU:

* a rank limit below the ranks the tolerance needs stops the compression with
  SYMHSS_ERR_RANK_OVERFLOW; with the limit lifted the same handle compresses, factorises and
  solves, bit for bit like a fresh handle;
* a device-memory budget below the compression's needs makes its allocations fail as on a full
  device (SYMHSS_ERR_NOMEM); with the budget lifted the same handle recovers, and a budget that
  holds the whole factorisation changes nothing;
* calls out of order return SYMHSS_ERR_STATE.
(The bounded waits of the tensor-core kernels are driven to their limits in test_gpu_kernels.py.)
"""

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


def _solver(SV):
    return SV.Solver(star(2048), 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10)


def _run(s):
    s.compress()
    s.factor()
    return s.solve(s.rhs(0.0)).cpu().numpy()


def test_rank_limit_overflow_and_recovery(mods):
    SV, S = mods
    ref = _solver(SV)
    x_ref = _run(ref)
    ref.close()
    s = _solver(SV)
    S.symhss_set_rank_limit(s.h, 5)
    with pytest.raises(S.SymhssError) as exc:
        s.compress()
    assert exc.value.code == S.SYMHSS_ERR_RANK_OVERFLOW
    with pytest.raises(S.SymhssError) as exc:
        s.factor()  # nothing compressed
    assert exc.value.code == S.SYMHSS_ERR_STATE
    S.symhss_set_rank_limit(s.h, 0)
    assert np.array_equal(_run(s), x_ref)
    S.symhss_set_rank_limit(s.h, 1000)  # above every rank: no effect
    assert np.array_equal(_run(s), x_ref)
    s.close()


def test_memory_budget_failure_and_recovery(mods):
    SV, S = mods
    ref = _solver(SV)
    x_ref = _run(ref)
    ref.close()
    s = _solver(SV)
    S.symhss_set_memory_limit(s.h, 1 << 20)  # 1 MiB: far below what the compression needs
    with pytest.raises(S.SymhssError) as exc:
        s.compress()
    assert exc.value.code == S.SYMHSS_ERR_NOMEM
    S.symhss_set_memory_limit(s.h, 0)
    assert np.array_equal(_run(s), x_ref)
    used = S.symhss_stats(s.h).device_bytes
    S.symhss_set_memory_limit(s.h, 4 * used + (64 << 20))
    assert np.array_equal(_run(s), x_ref)
    s.close()
