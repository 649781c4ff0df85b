"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every case compares element by element on the same seeded inputs. Sizes span
several GEMM tiles with ragged tails (odd o, v not multiples of 8/32/64). The
FP64 bar: |S_gpu - S_oracle| <= 1e-12 * max(1, max|S|) element-wise for
residuals and intermediates; |dE| <= 1e-10 Eh and amplitudes within 1e-9
max-abs after iterating.
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


def _sys(o, v, naux, seed, scale=0.05, fock_scale=0.0):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    fock = None
    if fock_scale:
        fock = f + inputs.random_hermitian(o + v, seed + 500, scale=fock_scale)
        f = fock
    return s, f, fock


def _maxrel(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


RES_CASES = [
    (3, 5, 7, 101, 0.3, 0.1),
    (5, 13, 20, 102, 0.2, 0.05),
    (7, 37, 50, 103, 0.1, 0.02),
    (10, 30, 120, 1, 0.05, 0.0),   # the 10/30/120 workload's shapes
    (11, 70, 90, 104, 0.05, 0.01),
]


@pytest.mark.parametrize("o,v,naux,seed,scale,fs", RES_CASES)
@pytest.mark.parametrize("complex_4m", [0, 1], ids=["3M", "4M"])
def test_residual_matches_oracle(ccsd, o, v, naux, seed, scale, fs, complex_4m):
    s, f, fock = _sys(o, v, naux, seed, scale, fs)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    parts = {}
    S1, S2 = R.residual(f, V, t1, t2, parts=parts)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, complex_4m=complex_4m) as cc:
        r1, r2 = cc.residual(t1, t2)
        assert _maxrel(r1, S1) < 1e-12
        assert _maxrel(r2, S2) < 1e-12
        # intermediates of the same evaluation
        lad = R.ladder(V["vvvv"], parts["tau"])
        ref = dict(tau=parts["tau"], Hvv=parts["Hvv"], Gvv=parts["Gvv"], Hoo=parts["Hoo"], Goo=parts["Goo"],
                   Hov=parts["Hov"], Hvoov=parts["Hvoov"].transpose(3, 0, 1, 2), C=parts["C"], A=parts["A"],
                   ladder=lad)
        for name, want in ref.items():
            got = cc.get_tensor(name)
            assert _maxrel(got, want) < 1e-12, name


def test_full_integral_input_matches_df_input(ccsd):
    o, v, naux = 4, 9, 11
    s, f, fock = _sys(o, v, naux, 105, 0.3, 0.05)
    Vf = R.full_integrals(s.B)
    t1, t2 = inputs.random_amplitudes(o, v, 106, scale=0.1)
    S1, S2 = R.residual(f, R.blocks_from_full(Vf, o), t1, t2)
    with ccsd.CCSD(o, v, s.eps, V=Vf, fock=fock) as cc:
        r1, r2 = cc.residual(t1, t2)
    assert _maxrel(r1, S1) < 1e-12 and _maxrel(r2, S2) < 1e-12


def test_mp2_guess_and_energy(ccsd):
    s = inputs.make_config("o10v30")
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, s.o)
    t1, t2 = R.mp2_guess(f, V, s.o, s.v)
    with ccsd.CCSD(s.o, s.v, s.eps, B=s.B) as cc:
        g1, g2 = cc.get_amplitudes()
        e = cc.energy()
    assert np.max(np.abs(g2 - t2)) < 1e-13 and np.max(np.abs(g1 - t1)) < 1e-13
    assert abs(e - R.energy(f, V, t1, t2)) < 1e-12


def test_c1_converges_to_oracle(ccsd):
    """10/30/120 workload: converge to 1e-10; |dE| <= 1e-10 Eh, amplitudes within 1e-9."""
    s = inputs.make_config("o10v30")
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, s.o)
    ref = R.solve(f, V, s.o, s.v, max_iter=60, tol=1e-10)
    assert ref["converged"]
    with ccsd.CCSD(s.o, s.v, s.eps, B=s.B, tol=1e-10) as cc:
        st, it, nrm = cc.iterate(60)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert st == ccsd.OK and nrm <= 1e-10
    assert abs(it - ref["iterations"]) <= 1
    assert abs(e - ref["energy"]) < 1e-10
    assert max(np.max(np.abs(t1 - ref["t1"])), np.max(np.abs(t2 - ref["t2"]))) < 1e-9


@pytest.mark.parametrize("diis", [0, 8])
def test_fixed_iterations_track_oracle(ccsd, diis):
    o, v, naux = 6, 21, 40
    s, f, fock = _sys(o, v, naux, 107, 0.05, 0.01)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=6, tol=0.0, diis_dim=diis)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, diis_dim=diis, tol=0.0) as cc:
        st, it, nrm = cc.iterate(6)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert st == ccsd.ERR_NOT_CONVERGED and it == 6
    assert abs(e - ref["energy"]) < 1e-10
    assert np.max(np.abs(t2 - ref["t2"])) < 1e-9 and np.max(np.abs(t1 - ref["t1"])) < 1e-9


def test_checkpoint_resume_bitwise(ccsd):
    o, v, naux = 5, 17, 30
    s, f, fock = _sys(o, v, naux, 108)
    with ccsd.CCSD(o, v, s.eps, B=s.B, diis_dim=0, tol=0.0) as a:
        a.iterate(6)
        ta = a.get_amplitudes()
    with ccsd.CCSD(o, v, s.eps, B=s.B, diis_dim=0, tol=0.0) as b:
        b.iterate(3)
        mid = b.get_amplitudes()
    with ccsd.CCSD(o, v, s.eps, B=s.B, diis_dim=0, tol=0.0) as c:
        c.set_amplitudes(*mid)
        c.iterate(3)
        tc = c.get_amplitudes()
    assert np.array_equal(ta[0], tc[0]) and np.array_equal(ta[1], tc[1])


def test_overflow_is_reported_as_divergence(ccsd):
    o, v, naux = 3, 6, 8
    s, f, fock = _sys(o, v, naux, 109)
    t1, t2 = inputs.random_amplitudes(o, v, 110, scale=0.1)
    t1[0, 0] = 1e300
    with ccsd.CCSD(o, v, s.eps, B=s.B) as cc:
        cc.set_amplitudes(t1, t2)
        st, it, nrm = cc.iterate(5)
        g1, g2 = cc.get_amplitudes()
    assert st == ccsd.ERR_DIVERGED and it == 1
    assert np.array_equal(g1, t1) and np.array_equal(g2, t2)


def test_device_buffers_through_torch(ccsd):
    torch = pytest.importorskip("torch")
    o, v, naux = 4, 10, 16
    s, f, fock = _sys(o, v, naux, 111, 0.2)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, 112, scale=0.1)
    S1, S2 = R.residual(f, V, t1, t2)
    stream = torch.cuda.current_stream()
    with ccsd.CCSD(o, v, s.eps, B=s.B, stream=stream.cuda_stream) as cc:
        d1 = torch.from_numpy(t1).cuda()
        d2 = torch.from_numpy(t2).cuda()
        r1, r2 = cc.residual(d1, d2)
        torch.cuda.synchronize()
    assert _maxrel(r1.cpu().numpy(), S1) < 1e-12 and _maxrel(r2.cpu().numpy(), S2) < 1e-12


def test_full_size_o20_v120_residual_and_iterations(ccsd):
    """The benchmarked workload (o20/v120/naux400, FP64, packed <ab||cd>): MP2 guess, the
    residual at it element by element, and two level-shifted iterations, against the oracle."""
    s = inputs.make_config("o20v120")
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, s.o)
    t1, t2 = R.mp2_guess(f, V, s.o, s.v, shift=20.0)
    S1, S2 = R.residual(f, V, t1, t2)
    with ccsd.CCSD(s.o, s.v, s.eps, B=s.B, level_shift=20.0, tol=0.0) as cc:
        g1, g2 = cc.get_amplitudes()
        assert _maxrel(g2, t2) < 1e-12 and _maxrel(g1, t1) < 1e-12
        r1, r2 = cc.residual()
        assert _maxrel(r1, S1) < 1e-12 and _maxrel(r2, S2) < 1e-12
        e_mp2 = cc.energy()
        assert abs(e_mp2 - R.energy(f, V, t1, t2)) < 1e-10
        st, it, nrm = cc.iterate(2)
        e2 = cc.energy()
        h1, h2 = cc.get_amplitudes()
    ref = R.solve(f, V, s.o, s.v, max_iter=2, tol=0.0, shift=20.0)
    assert abs(e2 - ref["energy"]) < 1e-10
    assert np.max(np.abs(h2 - ref["t2"])) < 1e-9 and np.max(np.abs(h1 - ref["t1"])) < 1e-9


@pytest.mark.parametrize("o,v,naux,seed,blk", [(5, 17, 23, 301, 3), (7, 37, 50, 302, 0), (4, 9, 11, 303, 1)])
def test_df_ladder_without_stored_w_matches_oracle(ccsd, o, v, naux, seed, blk):
    """store_w = 0: <ab||cd> is rebuilt from B^Q in blocks of a inside each ladder evaluation."""
    s, f, fock = _sys(o, v, naux, seed, 0.1, 0.02)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    S1, S2 = R.residual(f, V, t1, t2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, store_w=0, df_block=blk) as cc:
        r1, r2 = cc.residual(t1, t2)
        lad = cc.get_tensor("ladder")
        st, it, nrm = cc.iterate(3)
        e = cc.energy()
    assert _maxrel(r1, S1) < 1e-12 and _maxrel(r2, S2) < 1e-12
    assert _maxrel(lad, R.ladder(V["vvvv"], R.tau(t1, t2))) < 1e-12
    ref = R.solve(f, V, o, v, max_iter=3, tol=0.0)
    assert abs(e - ref["energy"]) < 1e-10


@pytest.mark.parametrize("o,v", [(1, 4), (3, 1), (2, 2), (1, 1)])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_degenerate_shapes_match_oracle(ccsd, o, v, precision):
    """No (i<j) pair (o = 1), no (a<b) pair (v = 1), one pair of each: the doubles vanish or
    shrink to single pairs; residual, a few iterations and the energy still follow the oracle."""
    s, f, fock = _sys(o, v, 5, 300 + 10 * o + v, scale=0.3, fock_scale=0.1)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, 7, scale=0.1)
    S1, S2 = R.residual(f, V, t1, t2)
    kw = dict(precision=ccsd.PREC_SPLIT, split_min_flops=0.0) if precision == "split" else {}
    tol = 1e-10 if precision == "split" else 1e-12
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, tol=0.0, **kw) as cc:
        r1, r2 = cc.residual(t1, t2)       # the context keeps its own (MP2) amplitudes
        assert _maxrel(r1, S1) < tol and _maxrel(r2, S2) < tol
        ref = R.solve(f, V, o, v, max_iter=3, tol=0.0)
        st, it, nrm = cc.iterate(3)
        assert it == 3
        assert abs(cc.energy() - ref["energy"]) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_integral_blocks_permuted_at_each_use_match_oracle(ccsd, precision):
    """permute_cache_limit < 0: no permuted copy of any integral block is kept (the path large
    systems take for blocks over 2 GiB); each contraction permutes them into the plan's scratch.
    Residual, three iterations and the energy still follow the oracle, and the context holds
    no cached copies."""
    o, v, naux = 5, 14, 30
    s, f, fock = _sys(o, v, naux, 134, 0.2, 0.05)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, 135, scale=0.1)
    S1, S2 = R.residual(f, V, t1, t2)
    kw = dict(precision=ccsd.PREC_SPLIT, split_min_flops=0.0) if precision == "split" else {}
    tol = 1e-10 if precision == "split" else 1e-12
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, tol=0.0, permute_cache_limit=-1.0, **kw) as cc:
        assert cc.query("plan_cached_bytes") == 0.0
        r1, r2 = cc.residual(t1, t2)
        st, it, nrm = cc.iterate(3)
        e = cc.energy()
    assert _maxrel(r1, S1) < tol and _maxrel(r2, S2) < tol
    ref = R.solve(f, V, o, v, max_iter=3, tol=0.0)
    assert it == 3 and abs(e - ref["energy"]) < (1e-9 if precision == "split" else 1e-11)


@pytest.mark.parametrize("o,v,naux,seed", [(3, 5, 7, 131), (5, 14, 30, 132), (6, 21, 40, 133)])
def test_ccd_residual_is_the_doubles_residual_at_zero_singles(ccsd, o, v, naux, seed):
    """The CCD plan (no t1 terms, no C^{kb}_{ij}, no singles): at random amplitudes with a nonzero
    t1 it returns S1 = 0 and the Appendix-A doubles residual of the oracle at t1 = 0, with a
    non-diagonal Fock matrix (its off-diagonal occupied-virtual block feeds only the t1 terms)."""
    s, f, fock = _sys(o, v, naux, seed, 0.2, 0.05)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.1)
    _, S2 = R.residual(f, V, np.zeros_like(t1), t2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, method=ccsd.METHOD_CCD) as cc:
        r1, r2 = cc.residual(t1, t2)
    assert np.max(np.abs(r1)) == 0.0
    assert _maxrel(r2, S2) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_ccd_tracks_oracle(ccsd, precision):
    """CCD (method = CCD): t1 stays exactly zero, and fixed iterations and the energy follow the
    oracle's CCD (the doubles equations with T1 = 0)."""
    o, v, naux = 6, 21, 40
    s, f, fock = _sys(o, v, naux, 109, 0.05, 0.01)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=5, tol=0.0, method="ccd")
    kw = dict(precision=ccsd.PREC_SPLIT, split_min_flops=0.0) if precision == "split" else {}
    tol = 1e-9 if precision == "split" else 1e-11
    with ccsd.CCSD(o, v, s.eps, B=s.B, fock=fock, tol=0.0, method=ccsd.METHOD_CCD, **kw) as cc:
        st, it, nrm = cc.iterate(5)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert it == 5
    assert np.max(np.abs(t1)) == 0.0
    assert abs(e - ref["energy"]) < tol
    assert np.max(np.abs(t2 - ref["t2"])) < 10 * tol
