"""The column-ID entry point that allocates no device memory (for callers under a fixed
device-memory budget, inside an allocator they do not own, or on paths that cannot take
cudaMalloc's device-wide synchronisation) returns what symhss_column_id returns.

Two calls in a row (different batch sizes, so the shared scratch array is reused) are each
compared with the allocating entry point on copies of the same input; a batch above the
scratch capacity is refused on the host.  This file is collected last on purpose.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _batch(seed, batch, m, n, k):
    rng = np.random.default_rng(seed)
    a = (rng.normal(size=(batch, m, k)) + 1j * rng.normal(size=(batch, m, k))) @ \
        (rng.normal(size=(batch, k, n)) + 1j * rng.normal(size=(batch, k, n)))
    a += 1e-9 * (rng.normal(size=a.shape) + 1j * rng.normal(size=a.shape))
    return np.ascontiguousarray(np.transpose(a, (0, 2, 1)))  # column-major per matrix


def _run(fn, cm, m, n, tol):
    batch = cm.shape[0]
    a = torch.as_tensor(cm).to("cuda")
    rank = torch.zeros(batch, dtype=torch.int32, device="cuda")
    perm = torch.zeros((batch, n), dtype=torch.int32, device="cuda")
    st = (n // 2) * ((n + 1) // 2)
    t = torch.zeros((batch, st), dtype=torch.complex128, device="cuda")
    fn(a.data_ptr(), m, n, m, m * n, batch, tol, -1, rank.data_ptr(), perm.data_ptr(), t.data_ptr(), st,
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rank.cpu().numpy(), perm.cpu().numpy(), t.cpu().numpy()


def test_noalloc_column_id_matches_allocating_entry_point():
    from paper_2609_33216_b300 import symhss as S
    for seed, batch, m, n, k in ((1, 7, 96, 64, 21), (2, 19, 150, 90, 37)):
        cm = _batch(seed, batch, m, n, k)
        r0, p0, t0 = _run(S.symhss_column_id, cm.copy(), m, n, 1e-7)
        r1, p1, t1 = _run(S.symhss_column_id_noalloc, cm.copy(), m, n, 1e-7)
        np.testing.assert_array_equal(r1, r0)
        np.testing.assert_array_equal(p1, p0)
        assert np.all(r1 == k)
        for b in range(batch):
            used = r0[b] * (n - r0[b])
            np.testing.assert_allclose(t1[b, :used], t0[b, :used], rtol=1e-12, atol=0)


def test_noalloc_rejects_batch_above_capacity():
    from paper_2609_33216_b300 import symhss as S
    import ctypes as C
    rc = S.lib.symhss_column_id_noalloc(C.c_void_p(16), 4, 4, 4, 16, 4097, 1e-8, -1, C.c_void_p(16),
                                        C.c_void_p(16), C.c_void_p(16), 4, None)
    assert rc == S.SYMHSS_ERR_INVALID
