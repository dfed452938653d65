"""The C-ABI library loads without a GPU and exports every symbol include/symhss.h declares;
host-side argument validation rejects bad input before touching the device."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "symhss.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(symhss_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2609_33216_b300 import symhss as S
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(S.lib, name), name
    assert set(names) <= set(S.SYMBOLS)


def test_struct_sizes_match_header_layout():
    from paper_2609_33216_b300 import symhss as S
    # params: 5 doubles, 2 ints, 1 double, 3 ints (+pad), 1 double, 2 ints, uint64
    assert C.sizeof(S.symhss_params) == 96
    assert C.sizeof(S.symhss_curve) == 4 + 4 + 6 * 8 + 8


def test_invalid_arguments_rejected_on_host():
    from paper_2609_33216_b300 import symhss as S
    import numpy as np
    n = 64
    arrs = [np.ones(n) for _ in range(6)]
    cs = S.curve_struct(n, [a.ctypes.data for a in arrs], S.SYMHSS_HOST)
    h = C.c_void_p()
    for bad in (dict(k0=-1.0), dict(tol=-1.0), dict(leaf=0), dict(nproxy=4), dict(proxy_factor=1.0),
                dict(mode=7), dict(precision=3), dict(fixed_rank_kL=-2), dict(eps1=float("nan"))):
        kw = dict(k0=1.0, k1=2.0)
        kw.update(bad)
        p = S.params(kw.pop("k0"), kw.pop("k1"), **kw)
        assert S.lib.symhss_create(C.byref(cs), C.byref(p), None, C.byref(h)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_create(None, None, None, C.byref(h)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_compress(None, None) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_destroy(None) == S.SYMHSS_OK
    assert S.lib.symhss_strerror(S.SYMHSS_ERR_SINGULAR) == b"singular diagonal block"
    assert S.lib.symhss_column_id(None, 4, 4, 2, 16, 1, 1e-3, -1, None, None, None, 4, None) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_lu_batched(None, 4, 2, 16, 1, None, None, None) == S.SYMHSS_ERR_INVALID


def test_batch_create_rejects_mismatched_shared_fields_on_host():
    from paper_2609_33216_b300 import symhss as S
    import numpy as np
    n = 64
    arrs = [np.ones(n) for _ in range(6)]
    cs = S.curve_struct(n, [a.ctypes.data for a in arrs], S.SYMHSS_HOST)
    curves = (S.symhss_curve * 2)(cs, cs)
    h = C.c_void_p()
    for field, value in (("tol", 1e-6), ("leaf", 32), ("nproxy", 48), ("mode", S.SYMHSS_NONSYM),
                         ("oversample", 0), ("seed", 7), ("proxy_factor", 2.0)):
        p0 = S.params(1.0, 2.0)
        p1 = S.params(3.0, 4.0, 1.0, 2.0)  # wavenumbers and materials may differ
        setattr(p1, field, value)
        prms = (S.symhss_params * 2)(p0, p1)
        assert S.lib.symhss_create_batch(curves, prms, 2, None, C.byref(h)) == S.SYMHSS_ERR_INVALID, field
    prms = (S.symhss_params * 2)(S.params(1.0, 2.0), S.params(1.0, -2.0))
    assert S.lib.symhss_create_batch(curves, prms, 2, None, C.byref(h)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_create_batch(curves, prms, 0, None, C.byref(h)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_create_batch(None, prms, 2, None, C.byref(h)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_set_curves(None, curves, 2, None) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_batch_info(None, None, None, None, None) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_problem_ranks(None, 0, 1, None) == S.SYMHSS_ERR_INVALID


def test_tuning_calls_validate_on_host():
    from paper_2609_33216_b300 import symhss as S
    t = S.symhss_tuning()
    assert S.lib.symhss_get_tuning(None, C.byref(t)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_set_tuning(None, C.byref(t)) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_autotune(None, 1, None, None) == S.SYMHSS_ERR_INVALID


def test_speed_terms_match_oracle_on_host():
    """symhss_speed_terms (host code: closed-form difference weights) against the oracle's
    speed term (difference weights solved over the rationals) on sampled curves."""
    from paper_2609_33216_b300 import symhss as S
    import numpy as np
    from oracle import kernels as OK
    from synth import fourier_star, random_star_batch, star
    curves = [star(300), star(16384), fourier_star(97, ((3, 0.2, 0.0),)), fourier_star(5, ((2, 0.1, 0.0),))]
    curves += [p["curve"] for p in random_star_batch(2, 11, 2048, 4096)]
    for c in curves:
        got = S.symhss_speed_terms(c.w)
        ref = OK.hypersingular_speed_term(c.w)
        # s enters the diagonal as (s - pi/6) / w^2: summation-order rounding of ~1e-16
        assert np.max(np.abs(got - ref)) <= 1e-15, c.name
    with pytest.raises(RuntimeError):
        S.symhss_speed_terms(np.array([1.0, -1.0, 1.0]))


def test_limits_reject_null_handles():
    from paper_2609_33216_b300 import symhss as S
    assert S.lib.symhss_set_rank_limit(None, 10) == S.SYMHSS_ERR_INVALID
    assert S.lib.symhss_set_memory_limit(None, 1 << 20) == S.SYMHSS_ERR_INVALID
