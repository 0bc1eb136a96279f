"""Pins for the two T1 / F_mi terms the GPU path forms from intermediates of the same
iteration instead of as products of their own (exact identities; the oracle keeps
the textbook terms of Eq. (amplitudes)):

  -1/2 sum_mef <ma||ef> t_im^ef = 1/2 sum_m X_am,im - sum_e Y_ae t_i^e,
      X_amij = sum_ef <am||ef> tau_ij^ef,  Y_ae = sum_mf t_m^f <ma||fe>;
  1/2 sum_nef <mn||ef> taut_in^ef = sum_n X2_mn,in - 1/2 sum_e t_i^e F_me,
      X2_mnij = 1/2 sum_ef <mn||ef> tau_ij^ef,  F_me = sum_nf t_n^f <mn||ef>.

Both rest on tau - t2 = 2 (taut - t2) = t_i^e t_j^f - t_i^f t_j^e and on the
antisymmetry of the integrals in e, f, which the recipe builds in exactly; checked
here on the recipe's integrals with t1 != 0, and shown to fail when that antisymmetry
is broken (so the check has teeth)."""
import numpy as np
import pytest

from oracle import ccsd, integrals
from paper_2004_03682_gb300 import synthetic as syn


def _case(no, nv, G, seed):
    prob = syn.make_problem(seed, no, nv, G)
    b = ccsd.Blocks(integrals.integrals(prob), integrals.fock(prob), no)
    t1, t2 = syn.trial_amplitudes(prob, seed + 1, t1_max=0.2, t2_max=0.2)
    return b, t1, t2


def _r1_term(Vovvv, Vvovv, t1, t2):
    es = ccsd.es
    direct = -0.5 * es("imef,maef->ia", t2, Vovvv)
    X = es("amef,ijef->amij", Vvovv, ccsd.tau(t1, t2))
    Y = es("mf,mafe->ae", t1, Vovvv)
    return direct, 0.5 * es("amim->ia", X) - es("ae,ie->ia", Y, t1)


def _fmi_term(Voovv, t1, t2):
    es = ccsd.es
    direct = 0.5 * es("inef,mnef->mi", ccsd.tau_tilde(t1, t2), Voovv)
    X2 = 0.5 * es("ijef,mnef->mnij", ccsd.tau(t1, t2), Voovv)
    Fme = es("nf,mnef->me", t1, Voovv)
    return direct, es("mnin->mi", X2) - 0.5 * es("me,ie->mi", Fme, t1)


@pytest.mark.parametrize("no,nv,G", [(3, 7, 1), (4, 10, 2), (6, 14, 4)])
def test_r1_term_from_x_and_y(no, nv, G):
    b, t1, t2 = _case(no, nv, G, 700 + no + nv + G)
    direct, rewritten = _r1_term(b.v("ovvv"), b.v("vovv"), t1, t2)
    assert np.max(np.abs(direct)) > 0
    np.testing.assert_allclose(rewritten, direct, atol=1e-13 * np.max(np.abs(direct)), rtol=0)


@pytest.mark.parametrize("no,nv,G", [(3, 7, 1), (4, 10, 2), (6, 14, 4)])
def test_fmi_term_from_w_mnij_and_f_me(no, nv, G):
    b, t1, t2 = _case(no, nv, G, 750 + no + nv + G)
    direct, rewritten = _fmi_term(b.v("oovv"), t1, t2)
    assert np.max(np.abs(direct)) > 0
    np.testing.assert_allclose(rewritten, direct, atol=1e-13 * np.max(np.abs(direct)), rtol=0)


def test_rewrites_need_the_antisymmetry():
    """With the e, f antisymmetry of the integrals broken, both identities fail."""
    b, t1, t2 = _case(4, 10, 1, 799)
    rng = np.random.default_rng(0)
    noise = lambda a: a + 0.1 * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape))
    Vovvv = noise(b.v("ovvv"))
    d, r = _r1_term(Vovvv, -Vovvv.transpose(1, 0, 2, 3), t1, t2)
    assert np.max(np.abs(r - d)) > 1e-6 * np.max(np.abs(d))
    d, r = _fmi_term(noise(b.v("oovv")), t1, t2)
    assert np.max(np.abs(r - d)) > 1e-6 * np.max(np.abs(d))
