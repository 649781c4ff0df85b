"""GPU parity of the perturbative triples corrections (ccsd_triples) against the CPU oracle.

The three energies and the per-pair contributions are compared with
``oracle.triples_ref`` on the same seeded amplitudes: the full oracle at small
sizes, its per-pair form at sizes where o^3 v^3 arrays do not fit, and sampled
pairs at the o20/v120 workload's full size. The arithmetic is FP64 on both sides
in a different summation order, so the bar is 1e-11 relative on every energy
and per-pair term. Batches of 1, 2 and as many triples as fit must agree. In a
split-precision context the six products that make W (e- and m-terms) are split
GEMMs with 8 digits of 5 bits, one per term and batch of k: each product carries a
relative error of at most ~2^-38 of its row and column scales, and the energies,
quadratic in W, are held to 1e-9 relative. In both modes the fifth-order terms Z, Y
and t1's determinant are formed in double-single arithmetic (~2^-47 relative), well
inside the 1e-11 bar on the energies they enter.
"""
import numpy as np
import pytest

from oracle import ccsd_ref as R
from oracle import triples_ref as T3
from paper_2103_08473_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("+T", "(T)", "-T")


@pytest.fixture(scope="module")
def ccsd():
    from paper_2103_08473_gb300 import build, ccsd as mod
    mod.load(build.build())
    return mod


def _case(o, v, naux, seed, scale, fock_scale):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    fock = None
    if fock_scale:
        fock = f + inputs.random_hermitian(o + v, seed + 500, scale=fock_scale)
        f = fock
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    return s, f, fock, t1, t2


def _close(got, ref, tol=1e-11):
    return abs(got - ref) <= tol * max(abs(ref), 1e-8)


@pytest.mark.parametrize("o,v,naux,seed,scale,fs", [
    (3, 3, 6, 301, 0.4, 0.05),      # one triple, one virtual triple
    (4, 9, 18, 302, 0.3, 0.05),
    (6, 17, 30, 303, 0.2, 0.02),
    (5, 24, 40, 304, 0.2, 0.0),     # diagonal Fock: no f_ov part
])
@pytest.mark.parametrize("max_batch", [1, 2, 0])
def test_triples_match_oracle(ccsd, o, v, naux, seed, scale, fs, max_batch):
    s, f, fock, t1, t2 = _case(o, v, naux, seed, scale, fs)
    ref = T3.corrections(f, R.integrals(s.B, o), t1, t2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock) as cc:
        cc.set_amplitudes(t1, t2)
        got = cc.triples(max_batch=max_batch)
    for key in KEYS:
        assert _close(got[key], ref[key]), (key, got[key], ref[key])


def test_pair_terms_match_oracle_pairs(ccsd):
    o, v = 7, 29
    s, f, fock, t1, t2 = _case(o, v, 40, 305, 0.2, 0.03)
    V = {k: R.antisym_block(s.B, o, k) for k in ("oovv", "ooov", "vovv")}
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock) as cc:
        cc.set_amplitudes(t1, t2)
        got, pt = cc.triples(max_batch=3, pair_terms=True)
    total = np.zeros(3)
    for i in range(o):
        for j in range(o):
            if i < j:
                ref = T3.pair_contributions(f, V, t1, t2, i, j)
                for m in range(3):
                    assert _close(pt[i, j, m], ref[m]), (i, j, m)
                total += ref
            else:
                assert np.all(pt[i, j] == 0.0)
    for m, key in enumerate(KEYS):
        assert _close(got[key], total[m])
        assert _close(got[key], np.sum(pt[..., m]), 1e-13)


def test_batch_sizes_agree(ccsd):
    o, v = 8, 20
    s, f, fock, t1, t2 = _case(o, v, 30, 306, 0.2, 0.02)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock) as cc:
        cc.set_amplitudes(t1, t2)
        runs = [cc.triples(max_batch=b) for b in (1, 2, 5, 0)]
        again = cc.triples(max_batch=2)
    assert again == runs[1]                      # reproducible run to run
    for r in runs[1:]:
        for key in KEYS:
            assert _close(r[key], runs[0][key], 1e-13)


@pytest.mark.parametrize("o,v", [(2, 8), (5, 2), (1, 4)])
def test_no_triples_give_zero(ccsd, o, v):
    s, f, fock, t1, t2 = _case(o, v, 10, 307, 0.3, 0.0)
    with ccsd.CCSD(o, v, s.eps, B=s.B) as cc:
        cc.set_amplitudes(t1, t2)
        got, pt = cc.triples(pair_terms=True)
    assert got == {"+T": 0.0, "(T)": 0.0, "-T": 0.0}
    assert np.all(pt == 0.0)


def test_bad_arguments(ccsd):
    s, f, fock, t1, t2 = _case(3, 4, 6, 308, 0.3, 0.0)
    with ccsd.CCSD(3, 4, s.eps, B=s.B) as cc:
        with pytest.raises(ccsd.CCSDError):
            cc.triples(max_batch=-1)


@pytest.mark.parametrize("o,v,naux,seed,fs", [(4, 9, 18, 311, 0.05), (6, 33, 40, 312, 0.02)])
def test_split_triples_match_oracle(ccsd, o, v, naux, seed, fs):
    s, f, fock, t1, t2 = _case(o, v, naux, seed, 0.2, fs)
    V = {k: R.antisym_block(s.B, o, k) for k in ("oovv", "ooov", "vovv")}
    ref = sum(T3.pair_contributions(f, V, t1, t2, i, j) for i in range(o) for j in range(i + 1, o))
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, precision=ccsd.PREC_SPLIT) as cc:
        cc.set_amplitudes(t1, t2)
        got = cc.triples(max_batch=2)
        launches = cc.query("triples_launches")
        batches = cc.query("triples_batches")
        whole = cc.triples(max_batch=0)
        single = cc.triples(max_batch=1)
    for m, key in enumerate(KEYS):
        assert _close(got[key], ref[m], 1e-9), (key, got[key], ref[m])
    # split mode: per batch of k one tensor-core GEMM for each of the three e-terms and the
    # three m-terms, the energy kernel and its accumulation (after 16 launches that cut the digits,
    # one that packs t2 and four that make the double-single copies for the energy kernel)
    assert launches == 21 + 8 * batches
    # the batch's k run along the rows of the GEMM operands: the grouping does not change W
    for r in (whole, single):
        for key in KEYS:
            assert _close(r[key], got[key], 1e-13), (key, r[key], got[key])


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_o20_v120_sampled_pairs(ccsd, precision):
    """The o20/v120 workload at full size: MP2 doubles from the context, random singles;
    pairs whose triples the per-pair oracle evaluates in seconds."""
    s = inputs.make_config("o20v120")
    o, v = s.o, s.v
    f = R.fock_matrix(s.eps)
    t1, _ = inputs.random_amplitudes(o, v, 309, scale=0.01)
    kw = {"precision": ccsd.PREC_SPLIT} if precision == "split" else {}
    tol = 1e-9 if precision == "split" else 1e-11
    with ccsd.CCSD(o, v, s.eps, B=s.B, **kw) as cc:
        _, t2 = cc.get_amplitudes()
        cc.set_amplitudes(t1, t2)
        got, pt = cc.triples(pair_terms=True)
    V = {k: R.antisym_block(s.B, o, k) for k in ("oovv", "ooov", "vovv")}
    for i, j in ((17, 18), (0, 18), (5, 17), (18, 19)):
        ref = T3.pair_contributions(f, V, t1, t2, i, j)
        for m in range(3):
            assert _close(pt[i, j, m], ref[m], tol), (i, j, m, pt[i, j, m], ref[m])
    assert got["+T"] < 0.0
