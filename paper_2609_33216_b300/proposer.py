"""Learned rank / skeleton proposer: training data, GPU training and attachment to a solver.

Argument marshalling around the C ABI (``symhss_mlp_*``, ``symhss_training_data``,
``symhss_set_proposer``): the features, the network's forward and backward passes and the
Adam updates all run in the library's kernels; this module shuffles samples on the host,
copies them to the device and loops over minibatches.

Training data are the plain column IDs (no sketch) of generated scatterers: every
compressed box contributes its features, its two ranks and where its skeleton lies.
"""

from __future__ import annotations

import ctypes as C
import math
from typing import Iterable, List, Optional

import numpy as np
import torch

from . import symhss as S


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (the last layer scaled by 1/4, unused outputs zero), zero biases."""
    rng = np.random.default_rng(seed)
    w = S.MLP_WIDTH
    parts = []
    for li in range(3):
        bound = math.sqrt(6.0 / w) * (0.25 if li == 2 else 1.0)
        W = rng.uniform(-bound, bound, size=(w, w))
        if li == 2:
            W[66:, :] = 0.0
        parts += [W.ravel(), np.zeros(w)]
    return np.concatenate(parts).astype(np.float32)


class Proposer:
    """A proposer network on cuda:0 (FP32 master weights, FP16 evaluation copy)."""

    def __init__(self, params: Optional[np.ndarray] = None, max_batch: int = 4096, seed: int = 0):
        p = init_params(seed) if params is None else np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (S.MLP_PARAMS,):
            raise ValueError("params must have SYMHSS_MLP_PARAMS entries")
        self.max_batch = max_batch
        h = C.c_void_p()
        S.check(S.lib.symhss_mlp_create(p.ctypes.data, max_batch, C.byref(h)), "symhss_mlp_create")
        self.h = h

    def params(self) -> np.ndarray:
        out = np.empty(S.MLP_PARAMS, np.float32)
        S.check(S.lib.symhss_mlp_get_params(self.h, out.ctypes.data, None), "symhss_mlp_get_params")
        return out

    def params_fp16(self) -> np.ndarray:
        out = np.empty(S.MLP_PARAMS, np.float16)
        S.check(S.lib.symhss_mlp_get_params(self.h, None, out.ctypes.data), "symhss_mlp_get_params")
        return out

    def set_params(self, p: np.ndarray) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        S.check(S.lib.symhss_mlp_set_params(self.h, p.ctypes.data), "symhss_mlp_set_params")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        out = torch.empty((x.shape[0], S.MLP_WIDTH), dtype=torch.float32, device=x.device)
        S.check(S.lib.symhss_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(out.data_ptr()),
                                         C.c_void_p(_stream())), "symhss_mlp_forward")
        return out

    def loss_grad(self, x, yr, ys, mask):
        """Loss (float) and gradient (numpy float32) on one device batch."""
        loss = C.c_double()
        g = np.empty(S.MLP_PARAMS, np.float32)
        S.check(S.lib.symhss_mlp_loss_grad(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(yr.data_ptr()),
                                           C.c_void_p(ys.data_ptr()), C.c_void_p(mask.data_ptr()), x.shape[0],
                                           C.byref(loss), g.ctypes.data, C.c_void_p(_stream())),
                "symhss_mlp_loss_grad")
        return loss.value, g

    def step(self, x, yr, ys, mask, lr: float, want_loss: bool = False):
        loss = C.c_double()
        S.check(S.lib.symhss_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(yr.data_ptr()),
                                            C.c_void_p(ys.data_ptr()), C.c_void_p(mask.data_ptr()), x.shape[0],
                                            float(lr), C.byref(loss) if want_loss else None,
                                            C.c_void_p(_stream())), "symhss_mlp_train_step")
        return loss.value if want_loss else None

    def train(self, data, steps: int = 2000, batch: int = 512, lr: float = 2e-3, seed: int = 0,
              lr_final: float = 2e-4) -> List[float]:
        """Adam on shuffled minibatches of (x, y_rank, y_skel, mask) host arrays; returns the
        loss of the first batch of every epoch."""
        x, yr, ys, mk = (np.ascontiguousarray(a, dtype=np.float32) for a in data[:4])
        n = x.shape[0]
        batch = min(batch, n, self.max_batch)
        rng = np.random.default_rng(seed)
        losses = []
        done = 0
        while done < steps:
            order = rng.permutation(n)
            dev = [torch.from_numpy(np.ascontiguousarray(a[order])).cuda() for a in (x, yr, ys, mk)]
            for b0 in range(0, n - batch + 1, batch):
                if done >= steps:
                    break
                frac = done / max(1, steps - 1)
                rate = lr * (lr_final / lr) ** frac  # geometric decay
                sl = [d[b0:b0 + batch] for d in dev]
                loss = self.step(*sl, lr=rate, want_loss=(b0 == 0))
                if loss is not None:
                    losses.append(loss)
                done += 1
        torch.cuda.synchronize()
        return losses

    def attach(self, solver, margin: float = 1.3) -> None:
        """Let `solver` (Solver or BatchSolver) size its sketches from this network's ranks."""
        S.check(S.lib.symhss_set_proposer(solver.h, self.h, margin), "symhss_set_proposer")
        solver._proposer = self

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            S.lib.symhss_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def detach(solver) -> None:
    S.check(S.lib.symhss_set_proposer(solver.h, None, 1.0), "symhss_set_proposer")
    solver._proposer = None


def predicted_ranks(out: np.ndarray) -> np.ndarray:
    """Rank proposals (flux, trace) from network outputs: 2^(8 o) - 1."""
    return np.exp2(8.0 * np.asarray(out, dtype=np.float64)[:, :2]) - 1.0


def collect(problems: Iterable[dict], leaf: int, nproxy: int, tol: float, mode: str = "sym"):
    """Training samples from plain IDs (no sketch) of each problem {curve, k0, k1, eps0, eps1}."""
    from .solver import Solver
    xs, yrs, yss, mks, metas = [], [], [], [], []
    for p in problems:
        s = Solver(p["curve"], p["k0"], p["k1"], p.get("eps0", 1.0), p.get("eps1"), mode=mode, leaf=leaf,
                   nproxy=nproxy, tol=tol, oversample=0)
        s.compress()
        x, yr, ys, mk, meta, _ = S.symhss_training_data(s.h, _stream())
        xs.append(x)
        yrs.append(yr)
        yss.append(ys)
        mks.append(mk)
        metas.append(meta)
        s.close()
    return (np.concatenate(xs), np.concatenate(yrs), np.concatenate(yss), np.concatenate(mks),
            np.concatenate(metas))


def training_problems(scale: int = 1) -> List[dict]:
    """Generated scatterers of the disk / star families at the benchmark wavenumber ranges
    (unit disk 512 nodes at k 5/8; r = 1 + 0.3 cos 5 theta at 16384 nodes, k 20/30, and
    65536 / scale nodes at k 40/60 and 80/120; random stars r = 1 + sum a_m cos(m theta + phi_m)
    at k 5..60), each at ID tolerances 1e-10 and 1e-8 through `collect`."""
    from synth import disk, random_star_batch, star
    probs = [dict(curve=disk(512), k0=5.0, k1=8.0),
             dict(curve=star(16384 // scale), k0=20.0, k1=30.0),
             dict(curve=star(65536 // scale), k0=40.0, k1=60.0),
             dict(curve=star(65536 // scale), k0=80.0, k1=120.0)]
    probs += random_star_batch(6, seed=77, n_min=4096 // scale, n_max=32768 // scale, k_range=(5.0, 60.0))
    for p in probs:
        p.setdefault("eps0", 1.0)
        p.setdefault("eps1", (p["k1"] / p["k0"]) ** 2)
    return probs


def train_default(seed: int = 0, steps: int = 3000, scale: int = 1, tols=(1e-10, 1e-8)) -> "Proposer":
    """Collect plain-ID data of `training_problems` at each tolerance and train a network."""
    probs = training_problems(scale)
    parts = [collect(probs, leaf=128, nproxy=64, tol=t) for t in tols]
    data = tuple(np.concatenate([p[k] for p in parts]) for k in range(5))
    net = Proposer(seed=seed, max_batch=4096)
    net.train(data, steps=steps, batch=512, seed=seed)
    net.data_size = data[0].shape[0]
    return net
