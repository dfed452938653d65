"""GPU parity of the building blocks against the oracle, through the C ABI.

* tile generator (kernel-entry evaluation of Eq. 15 / Sec. 6 baseline) vs the oracle's
  entries, on curve nodes (with the corrected diagonal) and proxy points;
* bit-exact transpose symmetry of the GPU's own row-scaled matrix (Eq. syms);
* batched column ID vs the oracle's pivoted-QR ID (ranks, interpolation residual);
* batched LU / solve vs a dense solve.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import hss as OH  # noqa: E402
from oracle import kernels as OK  # noqa: E402
from synth import disk, fourier_star, star  # noqa: E402


@pytest.fixture(scope="module")
def S():
    from paper_2609_33216_b300 import symhss
    assert torch.cuda.is_available()
    return symhss


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _points(S, pts: OK.Points):
    # the Muller-like entries do not use the hypersingular speed term: none is passed
    arrs = [_dev(v) for v in (pts.x, pts.y, pts.nx, pts.ny, pts.w, pts.kappa)]
    ids = _dev(pts.gid.astype(np.int32), torch.int32)
    st = S.points_struct(len(pts), [a.data_ptr() for a in arrs], ids.data_ptr())
    return st, arrs + [ids]


def gpu_block(S, prm: OK.Params, obs: OK.Points, obs_eq, src: OK.Points, src_comp, scaled=True):
    ost, keep1 = _points(S, obs)
    sst, keep2 = _points(S, src)
    eq = _dev(np.asarray(obs_eq, np.int32), torch.int32)
    comp = _dev(np.asarray(src_comp, np.int32), torch.int32)
    m, n = len(obs), len(src)
    out = torch.zeros((n, m), dtype=torch.complex128, device="cuda")  # column-major m x n
    p = S.params(prm.k0, prm.k1, prm.eps0, prm.eps1)
    S.symhss_kernel_block(p, ost, eq.data_ptr(), sst, comp.data_ptr(), scaled, out.data_ptr(), m,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


def _assert_entries_close(got, ref):
    """Both sides evaluate each entry in FP64 from Hankel values accurate to ~1e-15; the
    N-kernel difference of far pairs cancels terms up to ~100x the result, so entries agree
    to ~1e-13 relative, plus an absolute floor of 1e-14 of the block's largest entry."""
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    assert np.all(err <= 2e-13 * np.abs(ref) + 1e-14 * scale), (err.max(), scale)


def test_hankel_matches_mpmath(S):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    x = np.concatenate([np.geomspace(1e-5, 500.0, 1500), np.linspace(3.9, 4.1, 41), np.linspace(19.9, 20.1, 41)])
    dx = _dev(x)
    out = torch.zeros(2 * len(x), dtype=torch.complex128, device="cuda")
    S.symhss_hankel01(dx.data_ptr(), len(x), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for n in (0, 1):
        ref = np.array([complex(mp.hankel1(n, float(v))) for v in x])
        rel = np.abs(got[n * len(x):(n + 1) * len(x)] - ref) / np.abs(ref)
        assert rel.max() <= 5e-15, (n, rel.max(), x[np.argmax(rel)])


def test_pivot_reciprocal_within_ulps_of_exact(S):
    """The LU panels' pivot reciprocal (conj(a) / |a|^2, 1 / |a|^2 by two Newton steps from the
    hardware's approximate reciprocal; Smith's division outside [2^-996, 2^997)) against the
    exact 1 / a in rational arithmetic: each component within 4 units of 2^-53 |1 / a| (the
    rounding of |a|^2, of the reciprocal and of the final products), and zero gives no finite
    value."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    mag = 10.0 ** rng.uniform(-290, 290, 3000)
    ph = rng.uniform(0, 2 * np.pi, 3000)
    a = mag * np.exp(1j * ph)
    edge = np.array([1.0, -1.0, 1j, -1j, 2.0 ** -500 + 0j, 2.0 ** 498, 3.0 - 4.0j, 1e-160 + 1e-161j,
                     1e155 - 1e154j, 2.0 ** -510 * (1 + 1j), 2.0 ** 511 * (1 - 1j)])
    a = np.concatenate([a, edge])
    dev = torch.as_tensor(a).to("cuda")
    out = torch.empty_like(dev)
    S.symhss_pivot_reciprocal(dev.data_ptr(), len(a), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for v, g in zip(a, got):
        x, y = Fraction(float(v.real)), Fraction(float(v.imag))
        s2 = x * x + y * y
        ex, ey = x / s2, -y / s2
        scale = abs(complex(float(ex), float(ey)))
        tol = 4 * 2.0 ** -53 * scale
        assert abs(float(Fraction(float(g.real)) - ex)) <= tol and abs(float(Fraction(float(g.imag)) - ey)) <= tol, (v, g)
    z = torch.zeros(1, dtype=torch.complex128, device="cuda")
    S.symhss_pivot_reciprocal(z.data_ptr(), 1, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert not np.isfinite(out[:1].cpu().numpy()).all()


@pytest.mark.parametrize("scaled", [True, False], ids=["scaled", "unscaled"])
def test_tiles_match_oracle_on_nodes_and_proxies(S, scaled):
    c = fourier_star(300, ((3, 0.2, 0.1), (5, 0.05, 0.7)))
    prm = OK.Params(9.0, 17.0, 1.3, 3.1)
    pts = OK.Points.from_curve(c)
    rng = np.random.default_rng(3)
    rows = rng.choice(300, 200, replace=False)
    cols = rng.choice(300, 170, replace=False)
    cols[:40] = rows[:40]  # coincident nodes: corrected diagonal and free terms
    ring = OK.Points.circle(0.2, -0.1, 0.7, 64)
    obs = OH._stack(pts.take(rows), ring)
    eq = np.concatenate([rng.integers(0, 2, 200), np.repeat([0, 1], 32)])
    src = pts.take(cols)
    comp = rng.integers(0, 2, 170)
    ref = OK.entries(obs, eq, src, comp, prm, scaled)
    got = gpu_block(S, prm, obs, eq, src, comp, scaled)
    _assert_entries_close(got, ref)


def test_gpu_matrix_symmetric_bit_exact(S):
    c = star(333)
    prm = OK.Params(6.0, 11.0, 1.3, 3.4)
    pts = OK.Points.from_curve(c)
    both = OH._stack(pts, pts)
    lab = np.concatenate([np.zeros(333, int), np.ones(333, int)])
    a = gpu_block(S, prm, both, lab, both, lab, True)
    n = 333
    i = np.arange(n)
    skew = a - a.T
    ft = skew[i, n + i].copy()
    skew[i, n + i] = 0
    skew[n + i, i] = 0
    assert np.count_nonzero(skew) == 0
    np.testing.assert_allclose(ft, -(prm.eps0 + prm.eps1) * c.w, rtol=1e-14)
    ref = OK.dense_matrix(c, prm)
    _assert_entries_close(a, ref)


def _id_gpu(S, mats, tol, fixed=-1):
    b, m, n = mats.shape
    a = torch.as_tensor(np.ascontiguousarray(np.transpose(mats, (0, 2, 1)))).to("cuda")  # column-major
    rank = torch.zeros(b, dtype=torch.int32, device="cuda")
    perm = torch.zeros((b, n), dtype=torch.int32, device="cuda")
    st = max(1, (n // 2) * ((n + 1) // 2))
    t = torch.zeros((b, st), dtype=torch.complex128, device="cuda")
    S.symhss_column_id(a.data_ptr(), m, n, m, m * n, b, tol, fixed, rank.data_ptr(), perm.data_ptr(),
                       t.data_ptr(), st, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = []
    for i in range(b):
        r = int(rank[i])
        tt = t[i, : r * (n - r)].cpu().numpy().reshape(n - r, r).T if r else np.zeros((0, n))
        out.append((r, perm[i].cpu().numpy().astype(np.int64), tt))
    return out


def test_column_id_matches_oracle_on_proxy_blocks(S):
    c = star(1024)
    prm = OK.Params.from_wavenumbers(20.0, 30.0)
    solver = OH.HSS(c, prm, OH.Options(leaf=128, nproxy=64, tol=1e-10))
    lev = solver.levels[-1]
    for b in lev:
        ids = np.arange(b.begin, b.end)
        b.act = [ids, ids]
        b.actrow = [ids, ids]
    mats = []
    for b in lev[:4]:
        mr = solver.m_r(b, lev)
        mats += [mr[:, :128], mr[:, 128:]]
    got = [_id_gpu(S, m[None], 1e-10)[0] for m in mats]
    for mtx, (r, perm, t) in zip(mats, got):
        r0, p0, t0 = OH.cpqr_id(mtx, 1e-10)
        assert abs(r - r0) <= 1
        assert sorted(perm.tolist()) == list(range(mtx.shape[1]))
        # T = R11^{-1} R12 with |R_rr| ~ tol |R_00| is ill-conditioned by design: compare the
        # interpolation residual (what the ID guarantees), not T entry by entry
        rec = mtx[:, perm[:r]] @ OH.interp_matrix(r, perm, t)
        assert np.linalg.norm(rec - mtx) <= 1e-9 * np.linalg.norm(mtx)
        rec0 = mtx[:, p0[:r0]] @ OH.interp_matrix(r0, p0, t0)
        assert np.linalg.norm(rec - mtx) <= 10 * max(np.linalg.norm(rec0 - mtx), 1e-12 * np.linalg.norm(mtx))


def test_column_id_exact_rank_and_fixed_rank(S):
    rng = np.random.default_rng(11)
    mats = []
    for k in (3, 17, 40):
        a = (rng.normal(size=(90, k)) + 1j * rng.normal(size=(90, k))) @ \
            (rng.normal(size=(k, 60)) + 1j * rng.normal(size=(k, 60)))
        mats.append(a)
    got = _id_gpu(S, np.stack(mats), 1e-12)
    for a, (r, perm, t), k in zip(mats, got, (3, 17, 40)):
        assert r == k
        rec = a[:, perm[:r]] @ OH.interp_matrix(r, perm, t)
        assert np.linalg.norm(rec - a) <= 1e-11 * np.linalg.norm(a)
    got = _id_gpu(S, np.stack(mats), 0.0, fixed=9)
    assert all(r == 9 for r, _, _ in got)


@pytest.mark.parametrize("n", [1, 7, 64, 257])
def test_lu_batched_solves(S, n):
    for nrhs, batch in ((3, 5), (37, 5), (80, 60)):  # per-block CTA path, blocked 8- and 16-column paths
        _lu_solve_case(S, n, nrhs, batch)


def _lu_solve_case(S, n, nrhs, batch):
    rng = np.random.default_rng(n + nrhs)
    a = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n)) + 3 * np.eye(n)
    b = rng.normal(size=(batch, n, nrhs)) + 1j * rng.normal(size=(batch, n, nrhs))
    da = torch.as_tensor(np.ascontiguousarray(np.transpose(a, (0, 2, 1)))).to("cuda")
    db = torch.as_tensor(np.ascontiguousarray(np.transpose(b, (0, 2, 1)))).to("cuda")
    piv = torch.zeros((batch, n), dtype=torch.int32, device="cuda")
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    S.symhss_lu_batched(da.data_ptr(), n, n, n * n, batch, piv.data_ptr(), info.data_ptr(), s)
    S.symhss_lu_solve_batched(da.data_ptr(), n, n, n * n, piv.data_ptr(), db.data_ptr(), nrhs, n, nrhs * n, batch, s)
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0
    x = np.transpose(db.cpu().numpy(), (0, 2, 1))
    for i in range(batch):
        ref = np.linalg.solve(a[i], b[i])
        assert np.linalg.norm(x[i] - ref) <= 1e-12 * np.linalg.cond(a[i]) * np.linalg.norm(ref), (n, nrhs)


@pytest.mark.parametrize("n,nrhs,batch", [(500, 280, 2), (257, 130, 4), (130, 600, 1), (64 * 5, 17, 31)])
def test_lu_inverse_blocked_solves(S, n, nrhs, batch):
    """Many right-hand sides on few blocks (< 32): the blocked solve forms the inverses of its
    64-row diagonal blocks (unit-lower and upper) and applies them as tensor-core products, the
    off-diagonal blocks as before; ragged last block, one and several matrices."""
    _lu_solve_case(S, n, nrhs, batch)


@pytest.mark.parametrize("n,nrhs,batch", [(600, 1, 1), (1000, 2, 3), (130, 1, 9), (2048, 1, 1), (300, 4, 20)])
def test_lu_cluster_solves(S, n, nrhs, batch):
    """Few right-hand sides on few large blocks: the solve runs on a thread-block cluster per
    (block, right-hand side), 32-row blocks owned in turn, ragged last block."""
    _lu_solve_case(S, n, nrhs, batch)


def test_lu_reports_singular_block(S):
    n = 6
    a = np.eye(n, dtype=np.complex128)
    a[3, 3] = 0.0
    da = torch.as_tensor(np.ascontiguousarray(a.T)).to("cuda")
    piv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.symhss_lu_batched(da.data_ptr(), n, n, n * n, 1, piv.data_ptr(), info.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert int(info[0]) == 4


def _splitmix(x):
    x = x + np.uint64(0x9E3779B97F4A7C15)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def _omega(seed, b, s, m):
    """Rademacher matrix of the sketch from its published counter-based definition (splitmix64)."""
    i = np.arange(s, dtype=np.uint64)[:, None]
    k = np.arange(m, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        h = _splitmix(np.uint64(seed) ^ (np.uint64(b) * np.uint64(0xD1B54A32D192ED03)) ^
                      (i * np.uint64(0x8CB92BA72F3D8DD7)) ^ k)
    return np.where((h >> np.uint64(63)) != 0, -1.0, 1.0)


@pytest.mark.parametrize("m,n,s,batch", [(64, 16, 8, 1), (384, 128, 64, 3), (830, 265, 170, 2), (1000, 3, 40, 1)])
def test_tensor_core_sketch_matches_fp64_product(S, m, n, s, batch):
    """Y = Omega M on the tensor cores (exact 8-bit slices, FP32 accumulation) equals the FP64 product
    to rounding: column-relative error <= 4e-15 (seven FP64 additions of exact slice products)."""
    rng = np.random.default_rng(m + n)
    mats = (rng.normal(size=(batch, m, n)) + 1j * rng.normal(size=(batch, m, n))) * \
        np.exp(3 * rng.normal(size=(batch, 1, n)))
    mats[:, :, 0] *= 1e-30
    da = torch.as_tensor(np.ascontiguousarray(np.transpose(mats, (0, 2, 1)))).to("cuda")
    y = torch.zeros((batch, n, s), dtype=torch.complex128, device="cuda")
    seed = 987654321
    S.symhss_sketch(da.data_ptr(), m, n, m, m * n, batch, s, seed, y.data_ptr(), s, s * n,
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    yg = np.transpose(y.cpu().numpy(), (0, 2, 1))
    for b in range(batch):
        ref = _omega(seed, b, s, m) @ mats[b]
        err = np.abs(yg[b] - ref).max(axis=0) / np.abs(ref).max(axis=0)
        assert err.max() <= 4e-15, (b, err.max())


def test_sketch_wait_timeout_returns_status_and_device_stays_usable(S):
    """Every wait of the sketch kernel is bounded in time.  With a 1 ns limit the waits for the
    bulk copies and MMAs expire: the kernel drains what it has in flight, frees its tensor
    memory and reports SYMHSS_ERR_TIMEOUT.  With the default limit restored, the same call on
    the same (still usable) device gives the FP64 product again."""
    m, n, s, batch = 300, 70, 48, 3
    rng = np.random.default_rng(42)
    mats = rng.normal(size=(batch, m, n)) + 1j * rng.normal(size=(batch, m, n))
    da = torch.as_tensor(np.ascontiguousarray(np.transpose(mats, (0, 2, 1)))).to("cuda")
    y = torch.zeros((batch, n, s), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    seed = 5
    try:
        S.symhss_set_wait_limit_ns(1)
        with pytest.raises(S.SymhssError) as exc:
            S.symhss_sketch(da.data_ptr(), m, n, m, m * n, batch, s, seed, y.data_ptr(), s, s * n, stream)
        assert exc.value.code == S.SYMHSS_ERR_TIMEOUT
    finally:
        S.symhss_set_wait_limit_ns(0)
    torch.cuda.synchronize()
    S.symhss_sketch(da.data_ptr(), m, n, m, m * n, batch, s, seed, y.data_ptr(), s, s * n, stream)
    torch.cuda.synchronize()
    yg = np.transpose(y.cpu().numpy(), (0, 2, 1))
    for b in range(batch):
        ref = _omega(seed, b, s, m) @ mats[b]
        err = np.abs(yg[b] - ref).max(axis=0) / np.abs(ref).max(axis=0)
        assert err.max() <= 4e-15, (b, err.max())


def _zgemm_case(rng, m, n, k, batch, spread):
    a = (rng.normal(size=(batch, m, k)) + 1j * rng.normal(size=(batch, m, k)))
    b = (rng.normal(size=(batch, k, n)) + 1j * rng.normal(size=(batch, k, n)))
    a *= np.exp(spread * rng.normal(size=(batch, m, 1)))  # rows and columns of very different scale
    b *= np.exp(spread * rng.normal(size=(batch, 1, n)))
    if m > 3 and k > 2:
        a[:, 1, :] = 0.0  # an all-zero row
        a[:, 2, 1] *= 1e-40  # an entry far below its row's maximum
    c = rng.normal(size=(batch, m, n)) + 1j * rng.normal(size=(batch, m, n))
    return a, b, c


def _colmajor(x):
    """(batch, rows, cols) -> device tensor laid out column-major per matrix."""
    return torch.as_tensor(np.ascontiguousarray(np.transpose(x, (0, 2, 1)))).to("cuda")


@pytest.mark.parametrize("m,n,k,batch", [(1, 1, 1, 1), (37, 5, 3, 2), (128, 32, 64, 1), (300, 70, 64, 3),
                                         (192, 192, 64, 2), (257, 33, 100, 2), (64, 61, 17, 4)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tensor_core_zgemm_matches_fp64_product(S, m, n, k, batch, mode):
    """C = A B, C -= A B, C += A B on the tensor cores (exact 7-bit slices, FP32 accumulation of
    integers below 2^24, int64 recombination) against numpy's FP64 product: every entry within
    8 k 2^-52 max_l|A(i,l)| max_l|B(l,j)| (the FP64 bound with row and column maxima)."""
    rng = np.random.default_rng(1000 * m + 10 * n + k + mode)
    a, b, c = _zgemm_case(rng, m, n, k, batch, spread=3.0)
    da, db, dc = _colmajor(a), _colmajor(b), _colmajor(c)
    S.symhss_zgemm(da.data_ptr(), m, m * k, db.data_ptr(), k, k * n, dc.data_ptr(), m, m * n, m, n, k, batch, mode,
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = np.transpose(dc.cpu().numpy(), (0, 2, 1))
    prod = a @ b
    ref = {0: prod, 1: c - prod, 2: c + prod}[mode]
    amax = np.maximum(np.abs(a.real), np.abs(a.imag)).max(axis=2)   # (batch, m)
    bmax = np.maximum(np.abs(b.real), np.abs(b.imag)).max(axis=1)   # (batch, n)
    bound = 8 * k * 2.0 ** -52 * amax[:, :, None] * bmax[:, None, :] + 4 * 2.0 ** -52 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_tensor_core_zgemm_timeout_and_recovery(S):
    """With the timeout probe on, the product's last MMA wait targets a phase that nothing
    completes and expires after the 1 ms limit: SYMHSS_ERR_TIMEOUT after the kernel drained its
    MMAs; with the probe off and the default limit the same call then gives the product."""
    rng = np.random.default_rng(9)
    m, n, k, batch = 200, 40, 64, 2
    a, b, c = _zgemm_case(rng, m, n, k, batch, spread=1.0)
    da, db = _colmajor(a), _colmajor(b)
    dc = torch.zeros((batch, n, m), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    try:
        S.symhss_set_wait_limit_ns(1_000_000)
        S.symhss_set_timeout_probe(True)
        with pytest.raises(S.SymhssError) as exc:
            S.symhss_zgemm(da.data_ptr(), m, m * k, db.data_ptr(), k, k * n, dc.data_ptr(), m, m * n, m, n, k,
                           batch, 0, stream)
        assert exc.value.code == S.SYMHSS_ERR_TIMEOUT
    finally:
        S.symhss_set_timeout_probe(False)
        S.symhss_set_wait_limit_ns(0)
    S.symhss_zgemm(da.data_ptr(), m, m * k, db.data_ptr(), k, k * n, dc.data_ptr(), m, m * n, m, n, k, batch, 0,
                   stream)
    torch.cuda.synchronize()
    got = np.transpose(dc.cpu().numpy(), (0, 2, 1))
    assert np.abs(got - a @ b).max() <= 1e-12 * np.abs(a @ b).max()
