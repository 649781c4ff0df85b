"""Pins for the Lambda and density oracle (appendices "Working equations for CCSD lambda
equations" and "Working equations for Lagrange 1-body density matrix").

The oracle's Lambda residual is the derivative of the coupled-cluster Lagrangian
E(t) + sum_mu lambda_mu S_mu(t) with respect to the amplitudes. It is compared with
  * <0| (1 + Lambda) [H_bar, tau_nu] |0> in the determinant space, at random complex
    amplitudes and multipliers with a non-diagonal Fock matrix,
  * for two electrons, where CCSD is exact, the full-CI left eigenvector of H_bar:
    <Psi| exp(T) / <Psi| exp(T) |0>, against the converged lambda.
The density blocks are compared with <0| (1 + Lambda) exp(-T) a+_q a_p exp(T) |0> less
the reference occupation (reading r20), and their trace is zero for any amplitudes.
Planted mistakes (the conjugate derivative, the derivative without the unique-amplitude
sum, the occupied block as printed) fail a pin.
"""
import numpy as np
import pytest

from oracle import brute_force as BF
from oracle import ccsd_ref as R
from oracle import lambda_ref as L
import lambda_adjoint as LA
from paper_2103_08473_gb300 import inputs


def _system(o, v, naux, seed, scale, fock_offdiag=0.0):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    if fock_offdiag:
        f = f + inputs.random_hermitian(o + v, seed + 100, scale=fock_offdiag)
    Vf = R.full_integrals(s.B)
    return s, f, Vf, R.blocks_from_full(Vf, o)


CASES = [(2, 3, 5, 11), (2, 5, 6, 12), (3, 4, 6, 13), (3, 5, 7, 14), (4, 4, 8, 15)]


@pytest.mark.parametrize("o,v,naux,seed", CASES)
def test_lambda_residual_matches_brute_force(o, v, naux, seed):
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 200, scale=0.3)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 300, scale=0.3)
    R1b, R2b = BF.Space(o, v).lagrangian_gradient(f, Vf, t1, t2, l1, l2)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    scale = max(np.max(np.abs(R2b)), 1.0)
    assert np.max(np.abs(R1 - R1b)) < 1e-12 * scale
    assert np.max(np.abs(R2 - R2b)) < 1e-12 * scale


def test_lambda_driver_terms():
    """At lambda = 0 the residual is dE/dt: <ij||ab> for the doubles (the printed V^{ij}_{ab})
    and f_ia + sum_jb <ij||ab> t^b_j for the singles."""
    o, v = 3, 5
    s, f, Vf, V = _system(o, v, 7, 21, scale=0.5, fock_offdiag=0.2)
    t1, t2 = inputs.random_amplitudes(o, v, 22, scale=0.3)
    z1, z2 = np.zeros((o, v), complex), np.zeros((o, o, v, v), complex)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, z1, z2)
    np.testing.assert_allclose(R2, V["oovv"], atol=1e-14)
    np.testing.assert_allclose(R1, f[:o, o:] + np.einsum("ijab,jb->ia", V["oovv"], t1), atol=1e-14)


@pytest.mark.parametrize("v,naux,seed", [(4, 6, 31), (6, 9, 32)])
def test_two_electron_lambda_is_the_full_ci_left_vector(v, naux, seed):
    o = 2
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.3)
    cc = R.solve(f, V, o, v, max_iter=200, tol=1e-13)
    assert cc["converged"]
    lam = L.solve_lambda(f, V, cc["t1"], cc["t2"], max_iter=200, tol=1e-13)
    assert lam["converged"]
    l1b, l2b = BF.Space(o, v).fci_left_lambda(f, Vf, cc["t1"], cc["t2"])
    assert np.max(np.abs(l2b)) > 1e-3
    np.testing.assert_allclose(lam["l1"], l1b, atol=1e-10)
    np.testing.assert_allclose(lam["l2"], l2b, atol=1e-10)


@pytest.mark.parametrize("o,v,naux,seed", CASES[2:])
def test_density_matches_brute_force(o, v, naux, seed):
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.5)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 400, scale=0.3)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 500, scale=0.3)
    gb = BF.Space(o, v).density(t1, t2, l1, l2).T     # <a+_q a_p>
    gb[:o, :o] -= np.eye(o)
    g = L.density(t1, t2, l1, l2)
    np.testing.assert_allclose(g, gb, atol=1e-13)
    assert abs(np.trace(g)) < 1e-13                   # the number of electrons is conserved
    gs = L.density(t1, t2, l1, l2, symmetrize=True)
    np.testing.assert_allclose(gs, gs.conj().T, atol=1e-15)


def test_pins_catch_planted_mistakes(monkeypatch):
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 41, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 42, scale=0.3)
    l1, l2 = inputs.random_amplitudes(o, v, 43, scale=0.3)
    sp = BF.Space(o, v)
    R1b, R2b = sp.lagrangian_gradient(f, Vf, t1, t2, l1, l2)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    assert np.max(np.abs(np.conj(R1) - R1b)) > 1e-3            # the conjugate derivative
    G = R2 / 4.0                                                # no sum over the four positions
    assert np.max(np.abs(G - R2b)) > 1e-3
    # the occupied density block exactly as printed (not transposed)
    g = L.density(t1, t2, l1, l2)
    gb = sp.density(t1, t2, l1, l2).T
    gb[:o, :o] -= np.eye(o)
    assert np.max(np.abs(g[:o, :o].T - gb[:o, :o])) > 1e-3


@pytest.mark.parametrize("o,v,naux,seed", [(3, 5, 7, 51), (4, 6, 9, 52), (5, 7, 10, 53)])
def test_explicit_adjoint_equals_the_derivative(o, v, naux, seed):
    """The term-by-term adjoint of the Appendix-A residual (the device contraction list) equals the
    differentiated Lagrangian."""
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.5, fock_offdiag=0.2)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 600, scale=0.3)
    l1, l2 = inputs.random_amplitudes(o, v, seed + 700, scale=0.3)
    R1, R2 = L.lagrangian_gradient(f, V, t1, t2, l1, l2)
    E1, E2 = LA.lagrangian_gradient_explicit(f, V, t1, t2, l1, l2)
    scale = max(np.max(np.abs(R2)), 1.0)
    assert np.max(np.abs(E1 - R1)) < 1e-12 * scale
    assert np.max(np.abs(E2 - R2)) < 1e-12 * scale
