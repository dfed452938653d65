"""The learned rank / skeleton proposer on the GPU, against its FP64 oracle (oracle/mlp.py):

* box features of a compressed handle equal the oracle's feature definition evaluated on the
  same curve and boxes; rank targets equal the handle's ID ranks;
* the network's forward pass, loss and gradient (FP16 weights, FP32 accumulation) match the
  oracle's FP64 evaluation of the same FP16 weights; one Adam step matches the oracle's;
* training on plain-ID data of generated scatterers lowers the loss, and the trained network
  proposes ranks of held-out boxes closely;
* attached to a solver it sizes the sketches from its proposals: every sketched ID passes the
  residual check (or is redone as a plain ID), the solution is unchanged to 1e-8, and the
  ID-side kernel time (sketch, ID, residual check, features and network) with and without the
  network is measured and printed (the gain the network brings on this GPU).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402
from synth import random_star_batch, star  # noqa: E402


@pytest.fixture(scope="module")
def mods():
    from paper_2609_33216_b300 import proposer as P
    from paper_2609_33216_b300 import solver as SV
    from paper_2609_33216_b300 import symhss as S
    assert torch.cuda.is_available()
    return P, SV, S


def _rand_batch(seed, B):
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(B, 128)) * 0.5).astype(np.float32)
    yr = rng.uniform(0.2, 0.8, size=(B, 2)).astype(np.float32)
    ys = rng.uniform(0, 1, size=(B, 64)).astype(np.float32)
    mk = (rng.uniform(size=(B, 64)) < 0.7).astype(np.float32)
    return x, yr, ys, mk


def test_features_and_targets_match_oracle(mods):
    P, SV, S = mods
    c = star(4096)
    s = SV.Solver(c, 20.0, 30.0, leaf=128, nproxy=64, tol=1e-10, oversample=0)
    s.compress()
    x, yr, ys, mk, meta, geo = S.symhss_training_data(s.h)
    assert x.shape[0] == sum(2 ** l for l in range(1, s.stats().depth + 1))
    for i in range(x.shape[0]):
        pr, lev, hgt, b, L, n0, n1, mn, npx, _ = meta[i]
        f = M.box_features(c.x, c.y, c.kappa, b, b + L, geo[i, 0], geo[i, 1], geo[i, 2], 20.0, 30.0, 1e-10, hgt,
                           n0, n1, mn, npx)
        assert np.abs(x[i] - f).max() <= 1e-6 * max(1.0, np.abs(f).max())
    for lev in range(1, s.stats().depth + 1):
        ranks = np.array(s.ranks(lev))
        rows = np.where(meta[:, 1] == lev)[0]
        assert np.allclose(yr[rows], np.log2(1 + ranks) / 8, atol=1e-7)
        # skeleton fractions: per half, the counted skeleton nodes add up to the rank
        assert np.all(mk[rows].sum(1) > 0)
    s.close()


def test_forward_loss_grad_and_adam_match_oracle(mods):
    P, SV, S = mods
    net = P.Proposer(seed=3, max_batch=256)
    rng = np.random.default_rng(4)
    p = net.params().astype(np.float64)
    p[-128:] = rng.normal(size=128) * 0.1  # non-zero last bias
    net.set_params(p.astype(np.float32))
    x, yr, ys, mk = _rand_batch(5, 200)
    dev = [torch.from_numpy(a).cuda() for a in (x, yr, ys, mk)]
    p16 = net.params_fp16().astype(np.float64)
    assert np.array_equal(p16, M.fp16(net.params()))
    out = net.forward(dev[0]).cpu().numpy()
    o_ref, _ = M.forward(p16, x.astype(np.float64))
    assert np.abs(out - o_ref).max() <= 1e-5 * np.abs(o_ref).max()
    loss, g = net.loss_grad(*dev)
    l_ref, g_ref = M.loss_and_grad(p16, x.astype(np.float64), yr, ys, mk)
    assert abs(loss - l_ref) <= 1e-5 * abs(l_ref)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    # one Adam step (first step: -lr * g / (|g| + eps)) from the same state
    master = net.params().astype(np.float64)
    net.step(*dev, lr=1e-3)
    w1 = net.params().astype(np.float64)
    w_ref, _, _ = M.adam_step(master, np.zeros_like(master), np.zeros_like(master), g_ref, step=1, lr=1e-3)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    assert np.abs(w1 - w_ref)[big].max() <= 1e-6
    net.close()


@pytest.fixture(scope="module")
def trained(mods):
    P, SV, S = mods
    probs = [dict(curve=star(8192), k0=20.0, k1=30.0)]
    probs += random_star_batch(5, seed=31, n_min=2048, n_max=16384, k_range=(5.0, 40.0))
    for p in probs:
        p.setdefault("eps1", (p["k1"] / p["k0"]) ** 2)
    data = P.collect(probs, leaf=128, nproxy=64, tol=1e-10)
    net = P.Proposer(seed=0, max_batch=4096)
    losses = net.train(data, steps=1500, batch=256, lr=2e-3, seed=1)
    return net, data, losses


def test_training_lowers_loss_and_predicts_held_out_ranks(mods, trained):
    P, SV, S = mods
    net, data, losses = trained
    assert losses[-1] < 0.2 * losses[0]
    held = random_star_batch(1, seed=404, n_min=8000, n_max=9000, k_range=(15.0, 30.0))[0]
    x, yr, *_ = P.collect([held], leaf=128, nproxy=64, tol=1e-10)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    r_hat = P.predicted_ranks(out)
    r = np.exp2(8.0 * yr.astype(np.float64)) - 1.0
    rel = np.abs(r_hat - r) / np.maximum(r, 1.0)
    assert np.median(rel) <= 0.12, np.median(rel)


def test_attached_proposer_keeps_solution_and_reports_id_time(mods, trained):
    P, SV, S = mods
    net, _, _ = trained
    held = random_star_batch(1, seed=405, n_min=15000, n_max=16000, k_range=(20.0, 30.0))[0]

    def run(with_net):
        s = SV.Solver(held["curve"], held["k0"], held["k1"], held["eps0"], held["eps1"], leaf=128, nproxy=64,
                      tol=1e-10)
        if with_net:
            net.attach(s, margin=1.3)
        for _ in range(3):  # warm-up, then the timed repetition is the last one
            s.compress()
            s.factor()
            x = s.solve(s.rhs(0.0))
        torch.cuda.synchronize()
        st = s.stats()
        side = sum(st.kernel_ms[k] for k in (S.K_ID, S.K_SKETCH, S.K_CHECK, S.K_MLP))
        out = (x.cpu().numpy(), side, st.proposals, st.sketch_redo, st.check_failed, st.check_max_ratio,
               st.proposal_rank_err)
        s.close()
        return out

    x0, side0, n0, redo0, fail0, ratio0, _ = run(False)
    x1, side1, n1, redo1, fail1, ratio1, err1 = run(True)
    assert n0 == 0 and n1 > 0
    assert err1 < 0.25
    assert ratio0 <= 1e-10 and ratio1 <= 1e-10
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) <= 1e-8
    print(f"\nID-side ms without / with the proposer: {side0:.2f} / {side1:.2f} "
          f"(redone IDs {redo0} / {redo1}, failed checks {fail0} / {fail1}, rank error {err1:.3f})")
    # no gain is asserted: the pivoted QR's cost on this GPU is set by the number of pivot
    # steps (the rank), not by the sketch height the network shrinks; a proposal far below
    # the rank makes a thin sketch whose ID is redone on the full matrix (each redone ID is a
    # full pivoted QR of a proxy matrix, about 2 ms each at this size, while the default path's
    # leaf sketches are sized from the analytic rank estimate and need no redo).  The bound
    # only guards against a pathological slowdown: 2 ms per redone ID on top of twice the
    # default path.
    assert side1 <= 2.0 * side0 + 2.0 * max(redo1, 1) + 2.0


def test_proposer_gain_on_high_frequency_star(mods):
    """The high-frequency star workload (262144 nodes, k 100 / 150, tol 1e-8): the default rank estimate
    (1.7x the rank one level down) is too thin where ranks grow faster, so IDs are continued
    or redone; the trained network sizes the sketches and the ID-side time drops."""
    P, SV, S = mods
    from synth import workload
    net = P.train_default(seed=0, steps=3000)
    w = workload("star262k")

    def run(with_net):
        s = SV.Solver(w["curve"], w["k0"], w["k1"], w["eps0"], w["eps1"], leaf=w["leaf"], nproxy=w["nproxy"],
                      tol=w["tol"])
        if with_net:
            net.attach(s, margin=1.3)
        for _ in range(2):
            s.compress()
            s.factor()
            x = s.solve(s.rhs(0.0))
        torch.cuda.synchronize()
        st = s.stats()
        side = sum(st.kernel_ms[k] for k in (S.K_ID, S.K_SKETCH, S.K_CHECK, S.K_MLP))
        out = x.cpu().numpy(), side, st.sketch_redo, st.check_failed, st.check_max_ratio
        s.close()
        torch.cuda.empty_cache()
        return out

    x0, side0, redo0, fail0, r0 = run(False)
    x1, side1, redo1, fail1, r1 = run(True)
    print(f"\nstar262k ID-side ms without / with the proposer: {side0:.1f} / {side1:.1f} "
          f"(redone {redo0} / {redo1}, failed checks {fail0} / {fail1})")
    assert r0 <= w["tol"] and r1 <= w["tol"]
    # both solutions equally good: sampled rows of the residual, evaluated by the oracle
    from oracle import kernels as OK
    prm = OK.Params(w["k0"], w["k1"], w["eps0"], w["eps1"])
    n = w["curve"].n
    rows = np.random.default_rng(12).choice(2 * n, size=16, replace=False)
    f = OK.rhs(w["curve"], prm)[rows]
    res = [np.linalg.norm(OK.matvec_rows(w["curve"], prm, x, rows=rows) - f) / np.linalg.norm(f) for x in (x0, x1)]
    diff = np.linalg.norm(x1 - x0) / np.linalg.norm(x0)
    print(f"sampled residual without / with: {res[0]:.2e} / {res[1]:.2e}; solution difference {diff:.2e}")
    assert res[1] <= max(2.0 * res[0], 1e-6)
    assert diff <= 1e-4
    assert side1 < side0
    net.close()
