"""GPU parity of the CC2 method (method = CC2) against the CPU oracle's residual_cc2.

The GPU evaluates the CC2 doubles from the T1-dressed DF factors; the oracle follows
the appendix's W intermediates. Both are the same integral of exp(-T1) H exp(T1), so
they agree to rounding: FP64 residuals within 1e-12 of max(1, max|S|) element-wise,
energies after fixed iterations within 1e-11 Eh (split precision: 1e-9).
"""
import numpy as np
import pytest

from oracle import ccsd_ref as R
from paper_2103_08473_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccsd():
    from paper_2103_08473_gb300 import build, ccsd as mod
    mod.load(build.build())
    return mod


def _sys(o, v, naux, seed, scale, fock_scale):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    fock = None
    if fock_scale:
        fock = f + inputs.random_hermitian(o + v, seed + 500, scale=fock_scale)
        f = fock
    return s, f, fock


def _maxrel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("o,v,naux,seed,scale,fs", [
    (3, 5, 7, 401, 0.3, 0.1),
    (5, 13, 20, 402, 0.2, 0.05),
    (7, 37, 50, 403, 0.1, 0.02),
    (1, 4, 6, 404, 0.3, 0.0),       # one occupied spinor
])
def test_cc2_residual_matches_oracle(ccsd, o, v, naux, seed, scale, fs):
    s, f, fock = _sys(o, v, naux, seed, scale, fs)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    S1, S2 = R.residual_cc2(f, V, t1, t2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, method=ccsd.METHOD_CC2) as cc:
        r1, r2 = cc.residual(t1, t2)
        hvv = cc.get_tensor("Hvv")
    assert _maxrel(r1, S1) < 1e-12
    assert _maxrel(r2, S2) < 1e-12
    assert _maxrel(hvv, R.intermediates(f, V, t1, t2)["Hvv"]) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_cc2_tracks_oracle(ccsd, precision):
    o, v, naux = 6, 21, 40
    s, f, fock = _sys(o, v, naux, 405, 0.05, 0.01)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=6, tol=0.0, method="cc2")
    kw = dict(precision=ccsd.PREC_SPLIT, split_min_flops=0.0) if precision == "split" else {}
    tol = 1e-9 if precision == "split" else 1e-11
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, tol=0.0, method=ccsd.METHOD_CC2, **kw) as cc:
        st, it, nrm = cc.iterate(6)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert it == 6
    assert abs(e - ref["energy"]) < tol
    assert max(np.max(np.abs(t1 - ref["t1"])), np.max(np.abs(t2 - ref["t2"]))) < 10 * tol


def test_cc2_converges_and_differs_from_ccsd(ccsd):
    o, v, naux = 4, 12, 30
    s, f, fock = _sys(o, v, naux, 406, 0.05, 0.0)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=100, tol=1e-11, method="cc2")
    assert ref["converged"]
    with ccsd.CCSD(o, v, s.eps, B=s.B, tol=1e-11, max_iter=100, method=ccsd.METHOD_CC2) as cc:
        st, it, nrm = cc.iterate(100)
        e_cc2 = cc.energy()
    assert st == 0
    assert abs(e_cc2 - ref["energy"]) < 1e-10
    with ccsd.CCSD(o, v, s.eps, B=s.B, tol=1e-11, max_iter=100) as cc:
        cc.iterate(100)
        e_ccsd = cc.energy()
    assert abs(e_ccsd - e_cc2) > 1e-8


def test_cc2_needs_df_factors(ccsd):
    o, v = 2, 3
    s, f, fock = _sys(o, v, 5, 407, 0.3, 0.0)
    with pytest.raises(ccsd.CCSDError):
        ccsd.CCSD(o, v, s.eps, V=R.full_integrals(s.B), method=ccsd.METHOD_CC2)
