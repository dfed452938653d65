"""Torch-facing wrapper of the C ABI: device buffers and streams come from torch.

Every method forwards to one C entry point; no arithmetic of the solver happens here.
"""

from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import symhss as S


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One scatterer: ``compress()``, ``factor()``, ``solve(rhs)`` on cuda:0."""

    def __init__(self, curve, k0: float, k1: float, eps0: float = 1.0, eps1: Optional[float] = None,
                 mode: str = "sym", curve_on_device: bool = False, formulation: str = "muller",
                 precision: str = "fp64", **params):
        if eps1 is None:
            eps1 = eps0 * (k1 / k0) ** 2
        self.n = int(curve.n)
        self.mode = S.SYMHSS_SYM if mode == "sym" else S.SYMHSS_NONSYM
        form = {"muller": S.SYMHSS_MULLER, "pmchwt": S.SYMHSS_PMCHWT, "bm": S.SYMHSS_BM}[formulation]
        prec = S.SYMHSS_MIXED if precision == "mixed" else S.SYMHSS_FP64
        self.prm = S.params(k0, k1, eps0, eps1, mode=self.mode, formulation=form, precision=prec, **params)
        self._keep = []
        cs = self._curve_struct(curve, curve_on_device)
        self.h = S.symhss_create(cs, self.prm, _stream())

    def _curve_struct(self, curve, on_device: bool) -> S.symhss_curve:
        arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in curve.arrays()]
        if on_device:
            tens = [torch.from_numpy(a).to("cuda") for a in arrays]
            self._keep = tens
            return S.curve_struct(self.n, [t.data_ptr() for t in tens], S.SYMHSS_DEVICE)
        self._keep = arrays
        return S.curve_struct(self.n, [a.ctypes.data for a in arrays], S.SYMHSS_HOST)

    def set_curve(self, curve, on_device: bool = False) -> None:
        S.symhss_set_curve(self.h, self._curve_struct(curve, on_device), _stream())

    def compress(self) -> None:
        S.symhss_compress(self.h, _stream())

    def factor(self) -> None:
        S.symhss_factor(self.h, _stream())

    def build(self) -> None:
        """compress() and factor(), pipelined over tree heights on two streams."""
        S.symhss_build(self.h, _stream())

    def rhs(self, angle: float = 0.0) -> torch.Tensor:
        f = torch.empty(2 * self.n, dtype=torch.complex128, device="cuda")
        S.symhss_rhs_plane_wave(self.h, angle, f.data_ptr(), _stream())
        return f

    def solve(self, rhs: torch.Tensor) -> torch.Tensor:
        """rhs: complex128 on cuda, shape (2n,) or (nrhs, 2n) (each row one right-hand side)."""
        rhs = rhs.contiguous()
        nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
        x = torch.empty_like(rhs)
        S.symhss_solve(self.h, rhs.data_ptr(), x.data_ptr(), nrhs, _stream())
        return x

    def matvec(self, x: torch.Tensor) -> torch.Tensor:
        """y = A_hss x (FP64 compressed operator); x like solve's right-hand side."""
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x)
        S.check(S.lib.symhss_matvec(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs,
                                    C.c_void_p(_stream())), "symhss_matvec")
        return y

    def set_refinement(self, steps: int) -> None:
        S.check(S.lib.symhss_set_refinement(self.h, steps), "symhss_set_refinement")

    def solve_host(self, rhs: np.ndarray) -> np.ndarray:
        rhs = np.ascontiguousarray(rhs, dtype=np.complex128)
        nrhs = 1 if rhs.ndim == 1 else rhs.shape[0]
        x = np.empty_like(rhs)
        S.symhss_solve_host(self.h, rhs.ctypes.data, x.ctypes.data, nrhs, _stream())
        return x

    def stats(self) -> S.symhss_stats_t:
        return S.symhss_stats(self.h)

    def ranks(self, level: int):
        return S.symhss_level_ranks(self.h, level)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            S.symhss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent scatterers in one handle: every tree height of every problem
    runs in one launch per kernel.  Vectors stack the problems' [eq1; eq2] blocks."""

    def __init__(self, curves, k0s, k1s, eps0s=None, eps1s=None, mode: str = "sym", **params):
        cnt = len(curves)
        if eps0s is None:
            eps0s = [1.0] * cnt
        if eps1s is None:
            eps1s = [e0 * (k1 / k0) ** 2 for e0, k0, k1 in zip(eps0s, k0s, k1s)]
        self.mode = S.SYMHSS_SYM if mode == "sym" else S.SYMHSS_NONSYM
        self.prms = [S.params(k0, k1, e0, e1, mode=self.mode, **params)
                     for k0, k1, e0, e1 in zip(k0s, k1s, eps0s, eps1s)]
        self._keep = []
        self.h = S.symhss_create_batch(self._curve_structs(curves), self.prms, _stream())
        self.ns, self.depths, self.row0 = S.symhss_batch_info(self.h)
        self.rows = 2 * sum(self.ns)

    def _curve_structs(self, curves):
        keep, out = [], []
        for c in curves:
            arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in c.arrays()]
            keep.append(arrays)
            out.append(S.curve_struct(int(c.n), [a.ctypes.data for a in arrays], S.SYMHSS_HOST))
        self._keep = keep
        return out

    def set_curves(self, curves) -> None:
        S.symhss_set_curves(self.h, self._curve_structs(curves), _stream())

    def compress(self) -> None:
        S.symhss_compress(self.h, _stream())

    def factor(self) -> None:
        S.symhss_factor(self.h, _stream())

    def build(self) -> None:
        """compress() and factor(), pipelined over tree heights on two streams."""
        S.symhss_build(self.h, _stream())

    def rhs(self, angle: float = 0.0) -> torch.Tensor:
        f = torch.empty(self.rows, dtype=torch.complex128, device="cuda")
        S.symhss_rhs_plane_wave(self.h, angle, f.data_ptr(), _stream())
        return f

    def solve(self, rhs: torch.Tensor) -> torch.Tensor:
        rhs = rhs.contiguous()
        nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
        x = torch.empty_like(rhs)
        S.symhss_solve(self.h, rhs.data_ptr(), x.data_ptr(), nrhs, _stream())
        return x

    def matvec(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x)
        S.check(S.lib.symhss_matvec(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs,
                                    C.c_void_p(_stream())), "symhss_matvec")
        return y

    def set_refinement(self, steps: int) -> None:
        S.check(S.lib.symhss_set_refinement(self.h, steps), "symhss_set_refinement")

    def block(self, v: torch.Tensor, c: int) -> torch.Tensor:
        """Problem c's [eq1; eq2] block of a batch vector."""
        return v[..., self.row0[c]:self.row0[c] + 2 * self.ns[c]]

    def stats(self) -> S.symhss_stats_t:
        return S.symhss_stats(self.h)

    def ranks(self, problem: int, level: int):
        return S.symhss_problem_ranks(self.h, problem, level)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            S.symhss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
