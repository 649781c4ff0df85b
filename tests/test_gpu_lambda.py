"""GPU parity of the Lambda equations and the one-body density against the CPU oracle.

The library evaluates the Lambda residual as the adjoint of its residual plan; the oracle
differentiates its Appendix-A residual (``oracle.lambda_ref``). Both are dL/dt of the same
Lagrangian, so they agree to rounding: residuals within 1e-12 of max(1, max|R|), converged
multipliers within 1e-8, densities within 1e-10.
"""
import numpy as np
import pytest

from oracle import ccsd_ref as R
from oracle import lambda_ref as L
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
    (3, 5, 7, 501, 0.3, 0.1),
    (5, 13, 20, 502, 0.2, 0.05),
    (7, 23, 40, 503, 0.1, 0.02),
    (2, 4, 6, 504, 0.3, 0.0),
])
def test_lambda_residual_matches_oracle(ccsd, o, v, naux, seed, scale, fs):
    s, f, fock = _sys(o, v, naux, seed, scale, fs)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 2, scale=0.1)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock) as cc:
        cc.set_amplitudes(t1, t2)
        r1, r2 = cc.lambda_residual(l1, l2)
        g = cc.density()
        gs = cc.density(symmetrize=True)
    assert _maxrel(r1, R1) < 1e-12
    assert _maxrel(r2, R2) < 1e-12
    want = L.density(t1, t2, l1, l2)
    assert _maxrel(g, want) < 1e-12
    assert _maxrel(gs, L.density(t1, t2, l1, l2, symmetrize=True)) < 1e-12


@pytest.mark.parametrize("vblock", [1, 2, 3])
def test_blocked_vovv_terms_match_oracle(ccsd, vblock):
    """<ak||cd> unpacked a few rows a at a time (vovv_block; large systems take about 1 GB of rows
    per block): the H^{ak}_{ci} term of the residual and its adjoint in the Lambda residual run
    over several blocks, including a short last one, and still match the oracle."""
    o, v, naux, seed = 5, 13, 20, 507
    s, f, fock = _sys(o, v, naux, seed, 0.2, 0.05)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 2, scale=0.1)
    S1, S2 = R.residual(f, V, t1, t2)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    # with vblock 2 also no permuted copy of any integral block (each use permutes it)
    extra = dict(permute_cache_limit=-1.0) if vblock == 2 else {}
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, vovv_block=vblock, **extra) as cc:
        r1, r2 = cc.residual(t1, t2)
        cc.set_amplitudes(t1, t2)
        q1, q2 = cc.lambda_residual(l1, l2)
    assert _maxrel(r1, S1) < 1e-12 and _maxrel(r2, S2) < 1e-12
    assert _maxrel(q1, R1) < 1e-12 and _maxrel(q2, R2) < 1e-12


@pytest.mark.parametrize("o,v,naux,seed,vblock", [(5, 13, 20, 508, 0), (4, 40, 30, 509, 7), (7, 23, 40, 510, 0)])
def test_split_lambda_residual_matches_oracle(ccsd, o, v, naux, seed, vblock):
    """The Lambda residual in split precision with every GEMM on the tensor cores (8 digits of
    5 bits): its ladder adjoint runs against the digits of <ab||cd> cut at creation, read as
    the conjugates of the rows it needs (<ab||cd> = conj <cd||ab>). The digits' relative error
    ~2^-38 per product puts the residual within 1e-10 of the oracle's."""
    s, f, fock = _sys(o, v, naux, seed, 0.2, 0.02)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 2, scale=0.1)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, precision=ccsd.PREC_SPLIT, split_min_flops=0.0,
                   vovv_block=vblock) as cc:
        cc.set_amplitudes(t1, t2)
        r1, r2 = cc.lambda_residual(l1, l2)
        again = cc.lambda_residual(l1, l2)
    assert _maxrel(r1, R1) < 1e-10 and _maxrel(r2, R2) < 1e-10
    assert np.array_equal(again[0], r1) and np.array_equal(again[1], r2)


def test_split_lambda_iterations_track_fp64(ccsd):
    """Eight Lambda iterations (CUDA graph replay) in split precision against the FP64 ones."""
    o, v, naux = 5, 17, 30
    s, f, fock = _sys(o, v, naux, 511, 0.05, 0.0)
    out = {}
    for prec in ("fp64", "split"):
        kw = dict(precision=ccsd.PREC_SPLIT, split_min_flops=0.0) if prec == "split" else {}
        with ccsd.CCSD(o, v, s.eps, B=s.B, tol=0.0, **kw) as cc:
            cc.iterate(10)
            st, it, nrm = cc.lambda_iterate(8)
            out[prec] = cc.get_lambda()
        assert it == 8
    d = max(np.max(np.abs(out["split"][0] - out["fp64"][0])), np.max(np.abs(out["split"][1] - out["fp64"][1])))
    assert d < 1e-9


def test_lambda_converges_to_the_oracle(ccsd):
    o, v, naux = 4, 10, 24
    s, f, fock = _sys(o, v, naux, 505, 0.05, 0.0)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=100, tol=1e-12)
    lam = L.solve_lambda(f, V, ref["t1"], ref["t2"], max_iter=100, tol=1e-12)
    assert ref["converged"] and lam["converged"]
    with ccsd.CCSD(o, v, s.eps, B=s.B, tol=1e-12, max_iter=100) as cc:
        st, it, nrm = cc.iterate(100)
        assert st == 0
        st, it, nrm = cc.lambda_iterate(100)
        assert st == 0
        l1, l2 = cc.get_lambda()
        g = cc.density()
    assert max(np.max(np.abs(l1 - lam["l1"])), np.max(np.abs(l2 - lam["l2"]))) < 1e-8
    assert np.max(np.abs(g - L.density(ref["t1"], ref["t2"], lam["l1"], lam["l2"]))) < 1e-10
    assert abs(np.trace(g)) < 1e-10


def test_lambda_needs_ccsd_with_stored_integrals(ccsd):
    o, v = 3, 5
    s, f, fock = _sys(o, v, 8, 506, 0.3, 0.0)
    with ccsd.CCSD(o, v, s.eps, B=s.B, method=ccsd.METHOD_CC2) as cc:
        with pytest.raises(ccsd.CCSDError):
            cc.lambda_iterate(1)
    with ccsd.CCSD(o, v, s.eps, B=s.B, store_w=0) as cc:
        with pytest.raises(ccsd.CCSDError):
            cc.lambda_residual()
