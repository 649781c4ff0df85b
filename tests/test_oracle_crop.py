"""Pins for the oracle's CROP accelerator (Sec. "Coupled cluster implementation" names CROP,
Ziolkowski et al. 2008, as the lighter-memory alternative to DIIS).

What fixes CROP independently of its own code:
  * on a linear problem b - A x = 0 with A symmetric, the optimal residual of CROP with only
    three vectors is, at every iteration, the minimal residual over the Krylov subspace
    K_n(A, b) (CROP is then the conjugate residual method): computed here by an explicit
    least-squares solve over a QR basis of K_n. DIIS with an unbounded subspace gives the
    same residuals (it is GMRES there); DIIS truncated to three vectors does not, and neither
    does CROP with its write-back of the optimal vector removed;
  * on converging CCSD cases it reaches the fixed point of DIIS and of plain Jacobi, where
    the determinant-space projections vanish;
  * its coefficients are the constrained least-squares minimiser over the residuals it holds.
"""
import numpy as np
import pytest

from oracle import brute_force as BF
from oracle import ccsd_ref as R
from paper_2103_08473_gb300 import inputs


def _linear_problem(n, seed, symmetric=True):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / np.sqrt(n)
    if symmetric:
        M = 0.5 * (M + M.T)
    A = np.eye(n) + 0.6 * M / np.max(np.abs(np.linalg.eigvals(M)))
    b = rng.standard_normal(n)
    return A, b


def _as_amplitudes(x):
    """A vector as t1 of a one-occupied system (no unique doubles)."""
    v = len(x)
    return x.reshape(1, v).astype(np.complex128), np.zeros((1, 1, v, v), np.complex128)


def _krylov_min_residuals(A, b, nmax):
    """min over x in K_k(A, b) of |b - A x| for k = 1..nmax, by least squares on a QR basis."""
    out = []
    K = [b]
    for k in range(1, nmax + 1):
        Q, _ = np.linalg.qr(np.array(K).T)
        y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        out.append(np.linalg.norm(b - A @ Q @ y))
        K.append(A @ K[-1])
    return np.array(out)


def _crop_residual_norms(A, b, nit, m, writeback=True):
    acc = R.CROP(m)
    x = np.zeros_like(b)
    norms = []
    for it in range(nit + 1):
        r = b - A @ x
        t1, t2 = _as_amplitudes(x)
        e1, e2 = _as_amplitudes(r)
        if writeback:
            n1, _ = acc.step(t1, t2, e1, e2)
        else:  # planted: keep the raw trial vectors (DIIS storage) instead of the optimal ones
            acc.x.append((t1, t2))
            acc.r.append((e1, e2))
            c = acc.coefficients() if len(acc.x) >= 2 else np.ones(1)
            xo = sum(ci * xi[0] for ci, xi in zip(c, acc.x))
            ro = sum(ci * ri[0] for ci, ri in zip(c, acc.r))
            if len(acc.x) > m:
                acc.x.pop(0)
                acc.r.pop(0)
            n1 = xo + ro
            acc_r = ro
        if it >= 1:
            norms.append(np.linalg.norm(acc.r[-1][0] if writeback else acc_r))
        x = np.real(n1.ravel())
    return np.array(norms)


def _diis_residual_norms(A, b, nit, m):
    d = R.DIIS(m)
    x = np.zeros_like(b)
    norms = []
    for it in range(nit + 1):
        r = b - A @ x
        t1, t2 = _as_amplitudes(x + r)
        e1, e2 = _as_amplitudes(r)
        d.push(t1, t2, e1, e2)
        if len(d.t) >= 2:
            c = d.coefficients()
            norms.append(np.linalg.norm(sum(ci * ei for ci, ei in zip(c, d.e))))
            x = np.real(d.extrapolate()[0].ravel())
        else:
            x = np.real(t1.ravel())
    return np.array(norms)


@pytest.mark.parametrize("n,seed", [(40, 1), (60, 2)])
def test_crop3_is_the_minimal_krylov_residual_on_symmetric_linear_problems(n, seed):
    A, b = _linear_problem(n, seed)
    nit = 12
    want = _krylov_min_residuals(A, b, nit)
    crop = _crop_residual_norms(A, b, nit, 3)
    np.testing.assert_allclose(crop, want, rtol=1e-8, atol=1e-12 * np.linalg.norm(b))
    full = _diis_residual_norms(A, b, nit, 50)
    np.testing.assert_allclose(full, want, rtol=1e-8, atol=1e-12 * np.linalg.norm(b))


def test_truncated_diis_and_crop_without_writeback_are_not_minimal():
    """Sensitivity: with three raw vectors (DIIS(3), or CROP with the write-back of the
    optimal vector planted out) the residuals leave the Krylov minimum after three steps."""
    A, b = _linear_problem(40, 1)
    nit = 10
    want = _krylov_min_residuals(A, b, nit)
    d3 = _diis_residual_norms(A, b, nit, 3)
    raw = _crop_residual_norms(A, b, nit, 3, writeback=False)
    assert np.max(np.abs(d3[4:] / want[4:] - 1)) > 1e-3
    assert np.max(np.abs(raw[4:] / want[4:] - 1)) > 1e-3


def test_crop3_differs_from_the_krylov_minimum_without_symmetry():
    """The three-vector recurrence rests on the symmetry of A: a nonsymmetric A breaks it."""
    A, b = _linear_problem(40, 3, symmetric=False)
    want = _krylov_min_residuals(A, b, 10)
    crop = _crop_residual_norms(A, b, 10, 3)
    assert np.max(np.abs(crop[4:] / want[4:] - 1)) > 1e-4


def _system(o, v, naux, seed, scale, fock_offdiag=0.0):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    if fock_offdiag:
        f = f + inputs.random_hermitian(o + v, seed + 100, scale=fock_offdiag)
    Vf = R.full_integrals(s.B)
    return s, f, Vf, R.blocks_from_full(Vf, o)


@pytest.mark.parametrize("o,v,naux,seed,scale,offdiag,shift",
                         [(2, 4, 6, 93, 0.3, 0.05, 0.0), (3, 4, 6, 94, 0.3, 0.05, 0.0),
                          (4, 12, 30, 95, 0.05, 0.0, 0.0), (4, 12, 30, 96, 0.05, 0.02, 2.0)])
def test_crop_reaches_the_diis_and_jacobi_fixed_point(o, v, naux, seed, scale, offdiag, shift):
    s, f, Vf, V = _system(o, v, naux, seed, scale, offdiag)
    ref = R.solve(f, V, o, v, max_iter=400, tol=1e-13, shift=shift)
    jac = R.solve(f, V, o, v, max_iter=2000, tol=1e-13, diis_dim=0, shift=shift)
    assert ref["converged"] and jac["converged"]
    for m in (2, 3, 4):
        cr = R.solve(f, V, o, v, max_iter=400, tol=1e-13, diis_dim=m, accelerator="crop", shift=shift)
        assert cr["converged"], (m, cr["iterations"], cr["norm"])
        for other in (ref, jac):
            assert abs(cr["energy"] - other["energy"]) < 1e-10
            assert np.max(np.abs(cr["t2"] - other["t2"])) < 1e-9
            assert np.max(np.abs(cr["t1"] - other["t1"])) < 1e-9
    if BF.n_determinants(o, v) <= 500:
        _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, cr["t1"], cr["t2"])
        assert max(np.max(np.abs(S1b)), np.max(np.abs(S2b))) < 1e-10


def test_crop_needs_fewer_iterations_than_jacobi():
    o, v, naux, seed = 4, 12, 30, 95
    s, f, Vf, V = _system(o, v, naux, seed, 0.05)
    jac = R.solve(f, V, o, v, max_iter=2000, tol=1e-12, diis_dim=0)
    cr = R.solve(f, V, o, v, max_iter=400, tol=1e-12, diis_dim=3, accelerator="crop")
    assert cr["converged"] and cr["iterations"] < jac["iterations"]


def test_crop_coefficients_minimise_the_error_norm_over_its_optimal_vectors():
    """After several steps the stored residuals are optimal combinations, not raw ones; the
    next coefficients still minimise |sum_i c_i r_i|^2 over sum_i c_i = 1 (independent
    least squares in the null space of the constraint)."""
    o, v = 3, 5
    acc = R.CROP(3)
    for k in range(7):
        t1, t2 = inputs.random_amplitudes(o, v, 300 + k)
        e1, e2 = inputs.random_amplitudes(o, v, 400 + k, scale=0.3)
        acc.step(t1, t2, e1, e2)
    assert len(acc.r) == 3
    E = np.array([R.CROP._flat(*r) for r in acc.r]).T
    Er = np.vstack([E.real, E.imag])
    m = E.shape[1]
    c0 = np.full(m, 1.0 / m)
    null = np.linalg.svd(np.ones((1, m)))[2][1:].T
    y = np.linalg.lstsq(Er @ null, -Er @ c0, rcond=None)[0]
    np.testing.assert_allclose(acc.coefficients(), c0 + null @ y, rtol=1e-9, atol=1e-11)


def test_two_vector_crop_is_not_the_krylov_minimum():
    """The subspace size counts the new trial vector: CROP with two vectors (one previous optimum
    and the new trial) is steepest-descent-like and leaves the Krylov minimum, while three
    vectors (the conjugate residual recurrence) stay on it."""
    A, b = _linear_problem(40, 1)
    want = _krylov_min_residuals(A, b, 10)
    two = _crop_residual_norms(A, b, 10, 2)
    assert np.max(np.abs(two[3:] / want[3:] - 1)) > 1e-3
