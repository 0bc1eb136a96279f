"""The C-ABI library loads, exports every entry point include/exp.h declares, and
validates its arguments on the host (no GPU needed for these paths)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_03682_gb300 import build, expgb
    build.build()
    return expgb.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(exp_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"exp_create", "exp_init_integrals", "exp_ccsd_iterate", "exp_energy"} <= names
    for n in names:
        assert hasattr(lib, n), n


def _cfg(expgb, **over):
    io = np.array(over.pop("irrep_occ", [2, 2]), np.int32)
    iv = np.array(over.pop("irrep_virt", [3, 3]), np.int32)
    eo = np.linspace(-2, -1, int(io.sum()))
    ev = np.linspace(1, 2, int(iv.sum()))
    keep = [io, iv, eo, ev]
    d = dict(n_inst=1, n_occ=int(io.sum()), n_virt=int(iv.sum()), n_irrep=len(io), precision=0,
             n_slices=5, diis_dim=6, conv_tol=1e-9, max_iter=10, guess=0)
    d.update(over)
    cfg = expgb.Config(d["n_inst"], d["n_occ"], d["n_virt"], d["n_irrep"],
                       io.ctypes.data_as(C.POINTER(C.c_int32)), iv.ctypes.data_as(C.POINTER(C.c_int32)),
                       eo.ctypes.data_as(C.POINTER(C.c_double)), ev.ctypes.data_as(C.POINTER(C.c_double)),
                       d["precision"], d["n_slices"], d["diis_dim"], d["conv_tol"], d["max_iter"], d["guess"], 0.0,
                       d.get("n_active", 0), None, d.get("level_shift", 0.0), d.get("packed", 1),
                       d.get("n_slices_major", 0), d.get("denom_shift", 0.0), d.get("denom_shift_n", 1),
                       d.get("real_arith", 0))
    return cfg, keep


@pytest.mark.parametrize("bad", [dict(n_occ=5), dict(n_irrep=17), dict(diis_dim=9), dict(conv_tol=0.0),
                                 dict(max_iter=0), dict(precision=7), dict(precision=1, n_slices=2),
                                 dict(n_inst=0), dict(n_active=2), dict(level_shift=-1.0),
                                 dict(precision=1, n_slices=5, n_slices_major=2),
                                 dict(precision=1, n_slices=5, n_slices_major=7),
                                 dict(denom_shift=-0.1), dict(denom_shift=0.2, denom_shift_n=0),
                                 dict(real_arith=2)])
def test_create_rejects_bad_config_on_host(lib, bad):
    from paper_2004_03682_gb300 import expgb
    cfg, keep = _cfg(expgb, **bad)
    a = expgb.Allocator(expgb.ALLOC_FN(lambda n, u: None), expgb.FREE_FN(lambda p, u: None), None)
    h = C.c_void_p()
    st = lib.exp_create(C.byref(cfg), C.byref(a), None, C.byref(h))
    assert st == 1, (st, lib.exp_last_error(None))
    assert not h.value
    assert len(lib.exp_last_error(None)) > 0


def test_null_arguments_rejected(lib):
    assert lib.exp_create(None, None, None, None) == 1
    assert lib.exp_init_integrals(None, None, None, None) == 1
    assert lib.exp_ccsd_iterate(None, 1, None, None) == 1
    assert lib.exp_energy(None, 0, None, None) == 1
    lib.exp_destroy(None)


def test_zgemm_rejects_bad_arguments_on_host(lib):
    """exp_zgemm validates shape, precision, slice count and the double-single K limit
    before any device work (the operand pointers are never touched here)."""
    from paper_2004_03682_gb300 import expgb
    a = expgb.Allocator(expgb.ALLOC_FN(lambda n, u: None), expgb.FREE_FN(lambda p, u: None), None)
    fake = C.c_void_p(256)

    def call(prec, slices, M, N, K):
        return lib.exp_zgemm(C.byref(a), None, prec, slices, M, N, K, fake, fake, fake, 1.0, 0.0, 0)

    assert call(expgb.EXP_EMU_DS, 5, 4, 4, 17) == 1
    assert b"16" in lib.exp_last_error(None)
    assert call(7, 5, 4, 4, 4) == 1
    assert call(expgb.EXP_EMU_BF16, 2, 4, 4, 4) == 1
    assert call(expgb.EXP_FP64, 5, 0, 4, 4) == 1
    assert lib.exp_zgemm(None, None, expgb.EXP_FP64, 5, 4, 4, 4, fake, fake, fake, 1.0, 0.0, 0) == 1


def test_profile_top_rejects_null_context(lib):
    ms, macs = C.c_double(), C.c_double()
    assert lib.exp_profile_top(None, 1, None, 0, C.byref(ms), C.byref(macs)) == 1


@pytest.mark.parametrize("L,M,m", [(1, 1, 3), (2, 1, 4), (1, 1, 6), (3, 0, 5)])
def test_pade_zero_matches_oracle_on_the_host(lib, L, M, m):
    """exp_pade_zero (host code of the library, no GPU) against the oracle's fit."""
    from oracle import intruder
    from paper_2004_03682_gb300 import expgb
    rng = np.random.default_rng(m + 7 * L)
    x = np.sort(rng.uniform(0.001, 0.1, m))
    vals = (-1.33 + 0.002j) + (0.5 + 0.1j) * x / (1 + 2.0 * x) + 1e-7 * rng.standard_normal(m)
    got = expgb.pade_zero(x, vals, L, M)
    ref = intruder.pade_zero(x, vals, L, M)
    assert abs(got - ref) < 1e-9 * abs(ref)


def test_pade_zero_rejects_too_few_points(lib):
    from paper_2004_03682_gb300 import expgb
    with pytest.raises(expgb.ExpError) as e:
        expgb.pade_zero([0.1, 0.2], [1.0, 2.0], 1, 1)
    assert e.value.status == 1
