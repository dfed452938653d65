"""Accuracy of the matrix entries at the node spacing of the large workloads.

Off the diagonal, the second-row/second-column block needs N_k0 - N_k1, a difference of two
hypersingular kernels whose 1/r^2 parts cancel; at the spacing of the 65536- and 262144-node
stars (h ~ 1e-4 and 2.4e-5) the difference is evaluated in FP64 as the difference of the two
kernels, as Sec. 3.1 writes the operators.  These tests measure what that costs: every entry
block of nearest-neighbour pairs (index offsets 1, 2, 3, 7, 40) is compared with the kernel
formulas evaluated by mpmath at 30 digits from the same FP64 inputs.  Measured (oracle, worst of
30 pairs): S blocks 5e-16 relative; D and D* blocks 3e-12 at offset 1, because d . nu ~ kappa r^2 / 2
cancels in the geometry (a loss of about 1 / (kappa r) digits' worth); the N difference 8e-12,
because its 1/r^2 parts cancel (a ratio of about 1 / (k^2 r^2 |log r|)).  All are four or more
orders below the ID tolerances of those workloads (1e-10, 1e-8), so the plain FP64 difference is
kept and the small-r series of the difference is not needed; the residuals those workloads show
are set by the compression, not by the entries.
"""

import math

import numpy as np
import pytest

from oracle import kernels as OK
from synth import star

mp = pytest.importorskip("mpmath")

CASES = [(65536, 40.0, 60.0), (262144, 100.0, 150.0)]
OFFSETS = (1, 2, 3, 7, 40)


def _mp_blocks(xo, yo, nxo, nyo, wo, xs, ys, nxs, nys, ws, k0, k1, e0, e1):
    """[A11 A12; A21 A22] of the row-scaled system (Eq. 15) for one off-diagonal pair, in mpmath."""
    mp.mp.dps = 30
    X = [mp.mpf(v) for v in (xo, yo, nxo, nyo, wo, xs, ys, nxs, nys, ws)]
    xo, yo, nxo, nyo, wo, xs, ys, nxs, nys, ws = X
    dx, dy = xo - xs, yo - ys
    r = mp.sqrt(dx * dx + dy * dy)
    a = dx * nxo + dy * nyo
    b = dx * nxs + dy * nys
    nn = nxo * nxs + nyo * nys

    def layer(k):
        k = mp.mpf(k)
        h0, h1 = mp.hankel1(0, k * r), mp.hankel1(1, k * r)
        g = mp.mpc(0, 0.25) * h0
        c1 = mp.mpc(0, 0.25) * k * h1
        d = c1 * b / r
        ds = -c1 * a / r
        nk = c1 * nn / r + mp.mpc(0, 0.25) * k * (a * b / r) * (k * h0 / r - 2 * h1 / (r * r))
        return g, d, ds, nk

    g0, d0, ds0, n0 = layer(k0)
    g1, d1, ds1, n1 = layer(k1)
    w = wo * ws
    e0, e1 = mp.mpf(e0), mp.mpf(e1)
    return [-w * (e0 * e0 * g0 - e1 * e1 * g1), w * (e0 * d0 - e1 * d1),
            w * (e0 * ds0 - e1 * ds1), -w * (n0 - n1)]


def _pairs(n):
    rng = np.random.default_rng(n)
    base = rng.choice(n, 6, replace=False)
    return [(int(i), int((i + o) % n)) for i in base for o in OFFSETS]


def _reference(c, prm, pairs):
    ref = np.empty((len(pairs), 4), dtype=np.complex128)
    for p, (i, j) in enumerate(pairs):
        blk = _mp_blocks(c.x[i], c.y[i], c.nx[i], c.ny[i], c.w[i], c.x[j], c.y[j], c.nx[j], c.ny[j], c.w[j],
                         prm.k0, prm.k1, prm.eps0, prm.eps1)
        ref[p] = [complex(v) for v in blk]
    return ref


def _rel_errors(got, ref):
    return np.abs(got - ref) / np.abs(ref)


@pytest.mark.parametrize("n,k0,k1", CASES)
def test_oracle_entries_at_fine_spacing(n, k0, k1):
    c = star(n)
    prm = OK.Params.from_wavenumbers(k0, k1)
    pairs = _pairs(n)
    ref = _reference(c, prm, pairs)
    pts = OK.Points.from_curve(c)
    got = np.empty_like(ref)
    for p, (i, j) in enumerate(pairs):
        blk = OK.kernel_blocks(pts.take([i]), pts.take([j]), prm)
        got[p] = [blk[q][0, 0] for q in range(4)]
    err = _rel_errors(got, ref)
    # S block: FP64 rounding of the Hankel values; D, D*: the geometric cancellation; N: the
    # cancellation of the two hypersingular parts
    assert err[:, 0].max() <= 1e-14, err[:, 0].max()
    assert err[:, 1:3].max() <= 2e-11, err[:, 1:3].max()
    assert err[:, 3].max() <= 1e-10, err[:, 3].max()


@pytest.mark.gpu
@pytest.mark.parametrize("n,k0,k1", CASES)
def test_gpu_tile_entries_at_fine_spacing(n, k0, k1):
    torch = pytest.importorskip("torch")
    from paper_2609_33216_b300 import symhss as S
    assert torch.cuda.is_available()
    c = star(n)
    prm = OK.Params.from_wavenumbers(k0, k1)
    pairs = _pairs(n)
    ref = _reference(c, prm, pairs)
    obs = np.array([i for i, _ in pairs])
    src = np.array([j for _, j in pairs])

    def dev(a, dt=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)

    def pts(idx):
        arrs = [dev(v[idx]) for v in (c.x, c.y, c.nx, c.ny, c.w, c.kappa)]
        ids = dev(idx.astype(np.int32), torch.int32)
        return S.points_struct(len(idx), [a.data_ptr() for a in arrs], ids.data_ptr()), arrs + [ids]

    m = len(pairs)
    # rows: each observation point twice (eq 0, eq 1); columns: each source twice (comp 0, 1)
    o2 = np.repeat(obs, 2)
    s2 = np.repeat(src, 2)
    ost, k1_ = pts(o2)
    sst, k2_ = pts(s2)
    eq = dev(np.tile([0, 1], m).astype(np.int32), torch.int32)
    comp = dev(np.tile([0, 1], m).astype(np.int32), torch.int32)
    out = torch.zeros((2 * m, 2 * m), dtype=torch.complex128, device="cuda")
    p = S.params(prm.k0, prm.k1, prm.eps0, prm.eps1)
    S.symhss_kernel_block(p, ost, eq.data_ptr(), sst, comp.data_ptr(), True, out.data_ptr(), 2 * m,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    blk = out.cpu().numpy().T  # row-major (2m x 2m)
    got = np.empty_like(ref)
    for q in range(m):
        got[q] = [blk[2 * q, 2 * q], blk[2 * q, 2 * q + 1], blk[2 * q + 1, 2 * q], blk[2 * q + 1, 2 * q + 1]]
    err = _rel_errors(got, ref)
    assert err[:, 0].max() <= 1e-14, err[:, 0].max()
    assert err[:, 1:3].max() <= 2e-11, err[:, 1:3].max()
    assert err[:, 3].max() <= 1e-10, err[:, 3].max()
