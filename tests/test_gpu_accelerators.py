"""GPU parity of the subspace accelerators (DIIS and CROP) with a non-canonical reference, and
of the growth check of the iterations, through the C ABI against the CPU oracle.

Non-canonical reference: a Fock matrix with off-diagonal occupied-occupied and virtual-virtual
blocks (random unitary rotations within the occupied and within the virtual spinors, as for
the open-shell references of the paper's discussion, whose working equations do not need a
diagonal Fock operator). The denominators are taken from the real diagonal of the Fock matrix
(the "recomputed spinor energies"); the off-diagonal parts stay in the residual. Bars as for
the other FP64 tests: |dE| <= 1e-10 Eh, amplitudes within 1e-9 max-abs.
"""
import warnings

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


def _rotated(o, v, naux, seed, scale):
    """(system, canonical Fock, rotated B, rotated Fock) with unitaries within occ and vir."""
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    n = o + v
    U = np.zeros((n, n), complex)
    U[:o, :o] = inputs.random_unitary(o, seed + 1)
    U[o:, o:] = inputs.random_unitary(v, seed + 2)
    Bp = np.ascontiguousarray(np.einsum("pi,Xpq,qj->Xij", U.conj(), s.B, U, optimize=True))
    fp = U.conj().T @ f @ U
    fp = 0.5 * (fp + fp.conj().T)
    return s, f, Bp, fp


@pytest.mark.parametrize("accel,dim", [("diis", 8), ("crop", 3), ("crop", 2)])
def test_fixed_iterations_track_oracle_with_rotated_reference(ccsd, accel, dim):
    o, v, naux = 6, 21, 40
    s, f, Bp, fp = _rotated(o, v, naux, 701, 0.05)
    assert np.max(np.abs(fp[:o, :o] - np.diag(np.diag(fp[:o, :o])))) > 1e-2
    V = R.integrals(Bp, o)
    ref = R.solve(fp, V, o, v, max_iter=8, tol=0.0, diis_dim=dim, accelerator=accel)
    code = ccsd.ACCEL_CROP if accel == "crop" else ccsd.ACCEL_DIIS
    with ccsd.CCSD(o, v, s.eps, B=Bp, fock=fp, diis_dim=dim, accelerator=code, tol=0.0) as cc:
        st, it, nrm = cc.iterate(8)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert st == ccsd.ERR_NOT_CONVERGED and it == 8
    assert abs(e - ref["energy"]) < 1e-10
    assert max(np.max(np.abs(t1 - ref["t1"])), np.max(np.abs(t2 - ref["t2"]))) < 1e-9
    assert abs(nrm - ref["norm"]) < 1e-9 * max(1.0, ref["norm"])


@pytest.mark.parametrize("accel,dim", [("diis", 8), ("crop", 3)])
def test_rotated_reference_converges_to_the_canonical_energy(ccsd, accel, dim):
    """Unitary invariance on the GPU: the non-canonical solve reaches the canonical oracle
    energy, although its denominators (the rotated diagonal) and path differ."""
    o, v, naux = 5, 17, 30
    s, f, Bp, fp = _rotated(o, v, naux, 702, 0.05)
    ref = R.solve(f, R.integrals(s.B, o), o, v, max_iter=200, tol=1e-12)
    assert ref["converged"]
    code = ccsd.ACCEL_CROP if accel == "crop" else ccsd.ACCEL_DIIS
    with ccsd.CCSD(o, v, s.eps, B=Bp, fock=fp, diis_dim=dim, accelerator=code, tol=1e-12) as cc:
        st, it, nrm = cc.iterate(200)
        e = cc.energy()
    assert st == ccsd.OK
    assert abs(e - ref["energy"]) < 1e-10


def test_crop_converges_to_the_oracle_on_the_10_30_120_workload(ccsd):
    s = inputs.make_config("o10v30")
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, s.o)
    ref = R.solve(f, V, s.o, s.v, max_iter=80, tol=1e-10, diis_dim=3, accelerator="crop")
    dref = R.solve(f, V, s.o, s.v, max_iter=80, tol=1e-10)
    assert ref["converged"] and dref["converged"]
    with ccsd.CCSD(s.o, s.v, s.eps, B=s.B, tol=1e-10, diis_dim=3, accelerator=ccsd.ACCEL_CROP) as cc:
        st, it, nrm = cc.iterate(80)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert st == ccsd.OK and abs(it - ref["iterations"]) <= 1
    assert abs(e - ref["energy"]) < 1e-10 and abs(e - dref["energy"]) < 1e-10
    assert max(np.max(np.abs(t1 - dref["t1"])), np.max(np.abs(t2 - dref["t2"]))) < 1e-9


def test_crop_split_precision_tracks_fp64(ccsd):
    o, v, naux = 6, 21, 40
    s, f, Bp, fp = _rotated(o, v, naux, 703, 0.05)
    V = R.integrals(Bp, o)
    ref = R.solve(fp, V, o, v, max_iter=8, tol=0.0, diis_dim=3, accelerator="crop")
    with ccsd.CCSD(o, v, s.eps, B=Bp, fock=fp, diis_dim=3, accelerator=ccsd.ACCEL_CROP, tol=0.0,
                   precision=ccsd.PREC_SPLIT, split_min_flops=0.0) as cc:
        cc.iterate(8)
        e = cc.energy()
        t1, t2 = cc.get_amplitudes()
    assert abs(e - ref["energy"]) < 1e-9
    assert max(np.max(np.abs(t1 - ref["t1"])), np.max(np.abs(t2 - ref["t2"]))) < 1e-9


def test_lambda_with_crop_reaches_the_diis_multipliers(ccsd):
    o, v, naux = 4, 10, 24
    s = inputs.make_system(o, v, naux, 505, scale=0.05)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=100, tol=1e-12)
    lam = L.solve_lambda(f, V, ref["t1"], ref["t2"], max_iter=100, tol=1e-12)
    assert lam["converged"]
    with ccsd.CCSD(o, v, s.eps, B=s.B, tol=1e-12, max_iter=100, diis_dim=3, accelerator=ccsd.ACCEL_CROP) as cc:
        assert cc.iterate(100)[0] == ccsd.OK
        st, it, nrm = cc.lambda_iterate(100)
        assert st == ccsd.OK
        l1, l2 = cc.get_lambda()
    assert max(np.max(np.abs(l1 - lam["l1"])), np.max(np.abs(l2 - lam["l2"]))) < 1e-8


def _slow_divergence():
    """A system on which undamped Jacobi (no DIIS, no shift) diverges slowly: the update norm
    rises steadily by ~20% per iteration before it explodes."""
    o, v, naux = 4, 12, 30
    s = inputs.make_system(o, v, naux, 5, scale=0.15)
    return s, R.fock_matrix(s.eps), R.integrals(s.B, o)


@pytest.mark.parametrize("iters,factor", [(8, 20.0), (12, 50.0)])
def test_sustained_growth_is_reported_as_divergence(ccsd, iters, factor):
    s, f, V = _slow_divergence()
    o, v = s.o, s.v
    norms, traj = [], []

    def keep(it, t1, t2, n):
        norms.append(n)
        traj.append((t1.copy(), t2.copy()))

    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        R.solve(f, V, o, v, max_iter=60, tol=0.0, diis_dim=0, callback=keep)
    k = ccsd.divergence_index(norms, iters, factor)
    assert 0 < k < 40 and np.all(np.isfinite(norms[:k]))
    with ccsd.CCSD(o, v, s.eps, B=s.B, diis_dim=0, tol=0.0, diverge_iters=iters, diverge_factor=factor) as cc:
        st, it, nrm = cc.iterate(60)
        t1, t2 = cc.get_amplitudes()
        # the growth record runs across calls: one more call stops after one iteration
        st2, it2, _ = cc.iterate(5)
    assert st == ccsd.ERR_DIVERGED and it == k
    assert abs(nrm - norms[k - 1]) < 1e-9 * norms[k - 1]
    assert max(np.max(np.abs(t1 - traj[k - 1][0])), np.max(np.abs(t2 - traj[k - 1][1]))) < 1e-9
    assert st2 == ccsd.ERR_DIVERGED and it2 == 1


def test_growth_check_off_runs_to_the_cap(ccsd):
    s, f, V = _slow_divergence()
    with ccsd.CCSD(s.o, s.v, s.eps, B=s.B, diis_dim=0, tol=0.0, diverge_iters=0) as cc:
        st, it, nrm = cc.iterate(30)
    assert st == ccsd.ERR_NOT_CONVERGED and it == 30 and np.isfinite(nrm)
