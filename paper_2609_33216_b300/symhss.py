"""ctypes binding of libsymhss.so (C ABI in include/symhss.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  Device buffers are passed as raw pointers (e.g. ``tensor.data_ptr()``
of a torch tensor on ``cuda:0``), streams as ``torch.cuda.current_stream().cuda_stream``.
There is no fallback: if the library is missing, importing this module raises.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsymhss.so")

SYMHSS_OK = 0
SYMHSS_ERR_INVALID = -1
SYMHSS_ERR_NOMEM = -2
SYMHSS_ERR_CUDA = -3
SYMHSS_ERR_RANK_OVERFLOW = -4
SYMHSS_ERR_SINGULAR = -5
SYMHSS_ERR_TIMEOUT = -6
SYMHSS_ERR_STATE = -7
SYMHSS_ERR_DEVICE = -8

SYMHSS_SYM = 0
SYMHSS_NONSYM = 1
SYMHSS_FP64 = 0
SYMHSS_MIXED = 1
SYMHSS_MULLER = 0
SYMHSS_PMCHWT = 1
SYMHSS_BM = 2
SYMHSS_HOST = 0
SYMHSS_DEVICE = 1
SYMHSS_MAX_LEVELS = 32
K_TILES, K_ID, K_GETRF, K_GETRS, K_OTHER, K_SKETCH, K_CHECK, K_MLP = 0, 1, 2, 3, 4, 5, 6, 7
K_NAMES = ["tiles", "id", "getrf", "getrs", "other", "sketch", "check", "mlp"]
MLP_PARAMS = 49536
MLP_WIDTH = 128

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class symhss_curve(C.Structure):
    _fields_ = [("n", C.c_int), ("x", C.c_void_p), ("y", C.c_void_p), ("nx", C.c_void_p),
                ("ny", C.c_void_p), ("w", C.c_void_p), ("kappa", C.c_void_p), ("location", C.c_int)]


class symhss_params(C.Structure):
    _fields_ = [("k0", C.c_double), ("k1", C.c_double), ("eps0", C.c_double), ("eps1", C.c_double),
                ("tol", C.c_double), ("leaf", C.c_int), ("nproxy", C.c_int), ("proxy_factor", C.c_double),
                ("mode", C.c_int), ("precision", C.c_int), ("fixed_rank_kL", C.c_int),
                ("rank_scale_a", C.c_double), ("oversample", C.c_int), ("formulation", C.c_int),
                ("seed", C.c_uint64)]


class symhss_stats_t(C.Structure):
    _fields_ = [("n", C.c_int), ("depth", C.c_int), ("nboxes_leaf", C.c_int), ("root_size", C.c_int),
                ("max_rank", C.c_int * 2), ("level_max_rank", (C.c_int * 2) * SYMHSS_MAX_LEVELS),
                ("level_mean_rank", (C.c_double * 2) * SYMHSS_MAX_LEVELS),
                ("level_nproxy", C.c_int * SYMHSS_MAX_LEVELS),
                ("ms_compress", C.c_double), ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("ms_tiles", C.c_double), ("ms_id", C.c_double), ("ms_lu", C.c_double),
                ("ms_basis", C.c_double), ("pairs_evaluated", C.c_longlong), ("id_count", C.c_longlong),
                ("flops_lu", C.c_double), ("flops_id", C.c_double), ("device_bytes", C.c_longlong),
                ("kernel_ms", C.c_double * 8), ("kernel_launches", C.c_longlong * 8),
                ("kernel_work", C.c_double * 8), ("sketch_redo", C.c_longlong),
                ("check_failed", C.c_longlong), ("check_max_ratio", C.c_double), ("proposals", C.c_longlong),
                ("proposal_rank_err", C.c_double), ("proposal_under", C.c_longlong), ("ms_build", C.c_double)]


class symhss_tuning(C.Structure):
    _fields_ = [("lu_lookahead", C.c_int), ("lu_panel_threads", C.c_int), ("tile_loop_chunk", C.c_int),
                ("id_cluster_max", C.c_int), ("lu_panel_cluster", C.c_int), ("lu_tc", C.c_int),
                ("lu_outer", C.c_int), ("reserved", C.c_int * 1)]

    def as_dict(self):
        return {k: getattr(self, k) for k in ("lu_lookahead", "lu_panel_threads", "tile_loop_chunk", "id_cluster_max",
                                              "lu_panel_cluster", "lu_tc", "lu_outer")}


class symhss_points(C.Structure):
    _fields_ = [("n", C.c_int), ("x", C.c_void_p), ("y", C.c_void_p), ("nx", C.c_void_p),
                ("ny", C.c_void_p), ("w", C.c_void_p), ("kappa", C.c_void_p), ("id", C.c_void_p),
                ("hs", C.c_void_p)]


# (name, restype, argtypes) of every exported symbol
_SIGNATURES = [
    ("symhss_strerror", C.c_char_p, [C.c_int]),
    ("symhss_params_default", C.c_int, [C.POINTER(symhss_params)]),
    ("symhss_create", C.c_int, [C.POINTER(symhss_curve), C.POINTER(symhss_params), C.c_void_p,
                                C.POINTER(C.c_void_p)]),
    ("symhss_set_curve", C.c_int, [C.c_void_p, C.POINTER(symhss_curve), C.c_void_p]),
    ("symhss_create_batch", C.c_int, [C.POINTER(symhss_curve), C.POINTER(symhss_params), C.c_int, C.c_void_p,
                                      C.POINTER(C.c_void_p)]),
    ("symhss_set_curves", C.c_int, [C.c_void_p, C.POINTER(symhss_curve), C.c_int, C.c_void_p]),
    ("symhss_batch_info", C.c_int, [C.c_void_p, _ip, _ip, _ip, C.POINTER(C.c_longlong)]),
    ("symhss_compress", C.c_int, [C.c_void_p, C.c_void_p]),
    ("symhss_factor", C.c_int, [C.c_void_p, C.c_void_p]),
    ("symhss_build", C.c_int, [C.c_void_p, C.c_void_p]),
    ("symhss_rhs_plane_wave", C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    ("symhss_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("symhss_solve_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("symhss_matvec", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("symhss_set_refinement", C.c_int, [C.c_void_p, C.c_int]),
    ("symhss_stats", C.c_int, [C.c_void_p, C.POINTER(symhss_stats_t)]),
    ("symhss_level_ranks", C.c_int, [C.c_void_p, C.c_int, _ip]),
    ("symhss_problem_ranks", C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip]),
    ("symhss_destroy", C.c_int, [C.c_void_p]),
    ("symhss_mlp_create", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    ("symhss_mlp_set_params", C.c_int, [C.c_void_p, C.c_void_p]),
    ("symhss_mlp_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("symhss_mlp_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("symhss_mlp_loss_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    ("symhss_mlp_train_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                        C.c_float, C.POINTER(C.c_double), C.c_void_p]),
    ("symhss_mlp_destroy", C.c_int, [C.c_void_p]),
    ("symhss_set_proposer", C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    ("symhss_get_tuning", C.c_int, [C.c_void_p, C.POINTER(symhss_tuning)]),
    ("symhss_set_tuning", C.c_int, [C.c_void_p, C.POINTER(symhss_tuning)]),
    ("symhss_autotune", C.c_int, [C.c_void_p, C.c_int, C.POINTER(symhss_tuning), C.c_void_p]),
    ("symhss_training_data", C.c_int, [C.c_void_p, _ip, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    ("symhss_launch_count", C.c_longlong, []),
    ("symhss_hankel01", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("symhss_pivot_reciprocal", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("symhss_speed_terms", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("symhss_set_wait_limit_ns", C.c_int, [C.c_longlong]),
    ("symhss_set_timeout_probe", C.c_int, [C.c_int]),
    ("symhss_set_rank_limit", C.c_int, [C.c_void_p, C.c_int]),
    ("symhss_set_memory_limit", C.c_int, [C.c_void_p, C.c_longlong]),
    ("symhss_zgemm", C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_void_p, C.c_int, C.c_longlong, C.c_void_p,
                               C.c_int, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    ("symhss_kernel_block", C.c_int, [C.POINTER(symhss_params), C.POINTER(symhss_points), C.c_void_p,
                                      C.POINTER(symhss_points), C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                      C.c_void_p]),
    ("symhss_column_id", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_double,
                                   C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    ("symhss_column_id_noalloc", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_int,
                                           C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong,
                                           C.c_void_p]),
    ("symhss_sketch", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_int,
                                C.c_ulonglong, C.c_void_p, C.c_int, C.c_longlong, C.c_void_p]),
    ("symhss_lu_batched", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    ("symhss_lu_solve_batched", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_longlong, C.c_void_p, C.c_void_p,
                                          C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_void_p]),
]

SYMBOLS = [s[0] for s in _SIGNATURES]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2609_33216_b300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class SymhssError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib.symhss_strerror(code).decode()} ({code})")


def check(code: int, what: str = "symhss") -> None:
    if code != SYMHSS_OK:
        raise SymhssError(code, what)


def params(k0: float, k1: float, eps0: float = 1.0, eps1: float = 1.0, **kw) -> symhss_params:
    """Default parameters with the given wavenumbers / materials and field overrides."""
    p = symhss_params()
    check(lib.symhss_params_default(C.byref(p)), "symhss_params_default")
    p.k0, p.k1, p.eps0, p.eps1 = k0, k1, eps0, eps1
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def curve_struct(n: int, ptrs, location: int) -> symhss_curve:
    """ptrs: six pointers (x, y, nx, ny, w, kappa) as ints."""
    return symhss_curve(n, *[C.c_void_p(int(p)) for p in ptrs], location)


def symhss_create(curve: symhss_curve, prm: symhss_params, stream: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    check(lib.symhss_create(C.byref(curve), C.byref(prm), C.c_void_p(stream), C.byref(h)), "symhss_create")
    return h


def symhss_create_batch(curves, prms, stream: int = 0) -> C.c_void_p:
    """curves: list of symhss_curve, prms: list of symhss_params (same length)."""
    cnt = len(curves)
    ca = (symhss_curve * cnt)(*curves)
    pa = (symhss_params * cnt)(*prms)
    h = C.c_void_p()
    check(lib.symhss_create_batch(ca, pa, cnt, C.c_void_p(stream), C.byref(h)), "symhss_create_batch")
    return h


def symhss_set_curves(h, curves, stream: int = 0) -> None:
    cnt = len(curves)
    ca = (symhss_curve * cnt)(*curves)
    check(lib.symhss_set_curves(h, ca, cnt, C.c_void_p(stream)), "symhss_set_curves")


def symhss_batch_info(h):
    """(n, depth, row0) lists, one entry per problem."""
    cnt = C.c_int()
    check(lib.symhss_batch_info(h, C.byref(cnt), None, None, None), "symhss_batch_info")
    n = (C.c_int * cnt.value)()
    d = (C.c_int * cnt.value)()
    r = (C.c_longlong * cnt.value)()
    check(lib.symhss_batch_info(h, None, n, d, r), "symhss_batch_info")
    return list(n), list(d), list(r)


def symhss_problem_ranks(h, problem: int, level: int):
    out = (C.c_int * (2 * (1 << level)))()
    check(lib.symhss_problem_ranks(h, problem, level, out), "symhss_problem_ranks")
    return [(out[2 * b], out[2 * b + 1]) for b in range(1 << level)]


def symhss_set_curve(h, curve: symhss_curve, stream: int = 0) -> None:
    check(lib.symhss_set_curve(h, C.byref(curve), C.c_void_p(stream)), "symhss_set_curve")


def symhss_compress(h, stream: int = 0) -> None:
    check(lib.symhss_compress(h, C.c_void_p(stream)), "symhss_compress")


def symhss_factor(h, stream: int = 0) -> None:
    check(lib.symhss_factor(h, C.c_void_p(stream)), "symhss_factor")


def symhss_build(h, stream: int = 0) -> None:
    check(lib.symhss_build(h, C.c_void_p(stream)), "symhss_build")


def symhss_rhs_plane_wave(h, angle: float, rhs_ptr: int, stream: int = 0) -> None:
    check(lib.symhss_rhs_plane_wave(h, angle, C.c_void_p(rhs_ptr), C.c_void_p(stream)), "symhss_rhs_plane_wave")


def symhss_solve(h, rhs_ptr: int, x_ptr: int, nrhs: int = 1, stream: int = 0) -> None:
    check(lib.symhss_solve(h, C.c_void_p(rhs_ptr), C.c_void_p(x_ptr), nrhs, C.c_void_p(stream)), "symhss_solve")


def symhss_solve_host(h, rhs_ptr: int, x_ptr: int, nrhs: int = 1, stream: int = 0) -> None:
    check(lib.symhss_solve_host(h, C.c_void_p(rhs_ptr), C.c_void_p(x_ptr), nrhs, C.c_void_p(stream)),
          "symhss_solve_host")


def symhss_stats(h) -> symhss_stats_t:
    st = symhss_stats_t()
    check(lib.symhss_stats(h, C.byref(st)), "symhss_stats")
    return st


def symhss_level_ranks(h, level: int):
    out = (C.c_int * (2 * (1 << level)))()
    check(lib.symhss_level_ranks(h, level, out), "symhss_level_ranks")
    return [(out[2 * b], out[2 * b + 1]) for b in range(1 << level)]


def symhss_destroy(h) -> None:
    check(lib.symhss_destroy(h), "symhss_destroy")


def symhss_pivot_reciprocal(a_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    check(lib.symhss_pivot_reciprocal(C.c_void_p(a_ptr), n, C.c_void_p(out_ptr), C.c_void_p(stream)),
          "symhss_pivot_reciprocal")


def symhss_hankel01(x_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    check(lib.symhss_hankel01(C.c_void_p(x_ptr), n, C.c_void_p(out_ptr), C.c_void_p(stream)), "symhss_hankel01")


def points_struct(n: int, ptrs, id_ptr: int, hs_ptr: int = 0) -> symhss_points:
    """ptrs: six device pointers (x, y, nx, ny, w, kappa); hs_ptr: speed terms or 0 (none)."""
    return symhss_points(n, *[C.c_void_p(int(p)) for p in ptrs], C.c_void_p(int(id_ptr)),
                         C.c_void_p(int(hs_ptr)) if hs_ptr else None)


def symhss_speed_terms(w) -> "np.ndarray":
    """Speed terms of the hypersingular diagonal for one curve's weights (host arrays)."""
    import numpy as np
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty_like(w)
    check(lib.symhss_speed_terms(w.ctypes.data_as(C.c_void_p), int(w.shape[0]), out.ctypes.data_as(C.c_void_p)),
          "symhss_speed_terms")
    return out


def symhss_kernel_block(prm: symhss_params, obs: symhss_points, obs_eq: int, src: symhss_points, src_comp: int,
                        scaled: bool, out: int, ld: int, stream: int = 0) -> None:
    check(lib.symhss_kernel_block(C.byref(prm), C.byref(obs), C.c_void_p(obs_eq), C.byref(src),
                                  C.c_void_p(src_comp), int(bool(scaled)), C.c_void_p(out), ld,
                                  C.c_void_p(stream)), "symhss_kernel_block")


def symhss_column_id(a: int, m: int, n: int, lda: int, stride_a: int, batch: int, tol: float, fixed_rank: int,
                     rank: int, perm: int, t: int, stride_t: int, stream: int = 0) -> None:
    check(lib.symhss_column_id(C.c_void_p(a), m, n, lda, stride_a, batch, tol, fixed_rank, C.c_void_p(rank),
                               C.c_void_p(perm), C.c_void_p(t), stride_t, C.c_void_p(stream)), "symhss_column_id")


def symhss_column_id_noalloc(a: int, m: int, n: int, lda: int, stride_a: int, batch: int, tol: float,
                             fixed_rank: int, rank: int, perm: int, t: int, stride_t: int, stream: int = 0) -> None:
    check(lib.symhss_column_id_noalloc(C.c_void_p(a), m, n, lda, stride_a, batch, tol, fixed_rank, C.c_void_p(rank),
                                       C.c_void_p(perm), C.c_void_p(t), stride_t, C.c_void_p(stream)),
          "symhss_column_id_noalloc")


def symhss_sketch(a: int, m: int, n: int, lda: int, stride_a: int, batch: int, s: int, seed: int, y: int, ldy: int,
                  stride_y: int, stream: int = 0) -> None:
    check(lib.symhss_sketch(C.c_void_p(a), m, n, lda, stride_a, batch, s, seed, C.c_void_p(y), ldy, stride_y,
                            C.c_void_p(stream)), "symhss_sketch")


def symhss_zgemm(a: int, lda: int, stride_a: int, b: int, ldb: int, stride_b: int, c: int, ldc: int, stride_c: int,
                 m: int, n: int, k: int, batch: int, mode: int, stream: int = 0) -> None:
    """mode 0: C = A B, 1: C -= A B, 2: C += A B (batched, column-major complex128, device pointers)."""
    check(lib.symhss_zgemm(C.c_void_p(a), lda, stride_a, C.c_void_p(b), ldb, stride_b, C.c_void_p(c), ldc, stride_c,
                           m, n, k, batch, mode, C.c_void_p(stream)), "symhss_zgemm")


def symhss_set_rank_limit(h, max_rank: int) -> None:
    check(lib.symhss_set_rank_limit(h, int(max_rank)), "symhss_set_rank_limit")


def symhss_set_memory_limit(h, nbytes: int) -> None:
    check(lib.symhss_set_memory_limit(h, int(nbytes)), "symhss_set_memory_limit")


def symhss_set_timeout_probe(on: bool) -> None:
    check(lib.symhss_set_timeout_probe(int(bool(on))), "symhss_set_timeout_probe")


def symhss_set_wait_limit_ns(ns: int) -> None:
    check(lib.symhss_set_wait_limit_ns(int(ns)), "symhss_set_wait_limit_ns")


def symhss_lu_batched(a: int, n: int, lda: int, stride_a: int, batch: int, ipiv: int, info: int,
                      stream: int = 0) -> None:
    check(lib.symhss_lu_batched(C.c_void_p(a), n, lda, stride_a, batch, C.c_void_p(ipiv), C.c_void_p(info),
                                C.c_void_p(stream)), "symhss_lu_batched")


def symhss_lu_solve_batched(lu: int, n: int, lda: int, stride_a: int, ipiv: int, b: int, nrhs: int, ldb: int,
                            stride_b: int, batch: int, stream: int = 0) -> None:
    check(lib.symhss_lu_solve_batched(C.c_void_p(lu), n, lda, stride_a, C.c_void_p(ipiv), C.c_void_p(b), nrhs,
                                      ldb, stride_b, batch, C.c_void_p(stream)), "symhss_lu_solve_batched")


def symhss_training_data(h, stream: int = 0):
    """(x, y_rank, y_skel, mask, meta, geo) numpy arrays of the handle's last compression."""
    import numpy as np
    cnt = C.c_int(0)
    check(lib.symhss_training_data(h, C.byref(cnt), None, None, None, None, None, None, C.c_void_p(stream)),
          "symhss_training_data")
    n = cnt.value
    x = np.zeros((n, MLP_WIDTH), np.float32)
    yr = np.zeros((n, 2), np.float32)
    ys = np.zeros((n, 64), np.float32)
    mk = np.zeros((n, 64), np.float32)
    meta = np.zeros((n, 10), np.int32)
    geo = np.zeros((n, 3), np.float64)
    if n:
        check(lib.symhss_training_data(h, C.byref(cnt), x.ctypes.data, yr.ctypes.data, ys.ctypes.data, mk.ctypes.data,
                                       meta.ctypes.data, geo.ctypes.data, C.c_void_p(stream)), "symhss_training_data")
    return x, yr, ys, mk, meta, geo


def symhss_get_tuning(h) -> symhss_tuning:
    t = symhss_tuning()
    check(lib.symhss_get_tuning(h, C.byref(t)), "symhss_get_tuning")
    return t


def symhss_set_tuning(h, **kw) -> None:
    t = symhss_get_tuning(h)
    for k, v in kw.items():
        setattr(t, k, v)
    check(lib.symhss_set_tuning(h, C.byref(t)), "symhss_set_tuning")


def symhss_autotune(h, reps: int = 2, stream: int = 0) -> symhss_tuning:
    t = symhss_tuning()
    check(lib.symhss_autotune(h, reps, C.byref(t), C.c_void_p(stream)), "symhss_autotune")
    return t
