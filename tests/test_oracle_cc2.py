"""Pins for the CC2 oracle (appendix "Working equations for CC2 amplitude equations").

None of these re-types the appendix. The CC2 residuals are compared with what
defines the model in the determinant space:
  * S^{ab}_{ij} = <ijab| exp(-T1) H exp(T1) + [F, T2] |0> and S^a_i the CCSD singles
    projection <ia| exp(-T) H exp(T) |0>, at random complex amplitudes with a
    non-diagonal complex Fock matrix,
  * with the singles at zero and canonical orbitals the doubles equation is the
    first-order one, so the MP2 amplitudes are its fixed point,
  * the converged energy is invariant under unitary rotations within the occupied
    and within the virtual spinors,
and each printed S2 term dropped must break the brute-force agreement.
"""
import numpy as np
import pytest

from oracle import brute_force as BF
from oracle import ccsd_ref as R
from paper_2103_08473_gb300 import inputs


def _system(o, v, naux, seed, scale, fock_offdiag=0.0):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    if fock_offdiag:
        f = f + inputs.random_hermitian(o + v, seed + 100, scale=fock_offdiag)
    Vf = R.full_integrals(s.B)
    return s, f, Vf, R.blocks_from_full(Vf, o)


def _brute_cc2(f, Vf, o, v, t1, t2):
    sp = BF.Space(o, v)
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    T1 = sp.cluster_operator(t1, np.zeros((o, o, v, v)))
    T2 = sp.cluster_operator(np.zeros((o, v)), t2)
    F = np.einsum("pq,pqxy->xy", f, sp.E)
    ket = sp.expm_nilpotent(-T1) @ H @ sp.expm_nilpotent(T1) @ sp.ref + (F @ T2 - T2 @ F) @ sp.ref
    Evo = sp.E[o:, :o]
    doubles = np.einsum("aixz,bjzy,y->ijabx", Evo, Evo, sp.ref, optimize=True)
    S2 = np.einsum("ijabx,x->ijab", doubles, ket, optimize=True)
    _, _, S1, _ = sp.projections(f, Vf, t1, t2)
    return S1, S2


CASES = [(2, 3, 5, 11), (2, 5, 6, 12), (3, 4, 6, 13), (3, 5, 7, 14), (4, 4, 8, 15)]


@pytest.mark.parametrize("o,v,naux,seed", CASES)
def test_cc2_residual_matches_brute_force(o, v, naux, seed):
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 200, scale=0.3)
    S1b, S2b = _brute_cc2(f, Vf, o, v, t1, t2)
    S1, S2 = R.residual_cc2(f, V, t1, t2)
    scale = max(np.max(np.abs(S2b)), 1.0)
    assert np.max(np.abs(S2 - S2b)) < 1e-12 * scale
    assert np.max(np.abs(S1 - S1b)) < 1e-12 * scale


@pytest.mark.parametrize("term", ["driver", "t1_abej", "t1_mbij", "t1t1_mnij", "t1t1_abef", "f_vv", "f_oo"])
def test_pin_catches_dropped_cc2_term(term):
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 31, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 231, scale=0.3)
    _, S2b = _brute_cc2(f, Vf, o, v, t1, t2)
    parts = {}
    _, S2 = R.residual_cc2(f, V, t1, t2, parts=parts)
    assert np.max(np.abs(S2 - S2b)) < 1e-12 * np.max(np.abs(S2b))
    assert np.max(np.abs(S2 - parts["S2_" + term] - S2b)) > 1e-6


def test_cc2_without_singles_has_the_mp2_fixed_point():
    o, v = 4, 9
    s = inputs.make_system(o, v, 12, 41, scale=0.3)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    e = np.real(np.diag(f))
    D = e[:o, None, None, None] + e[None, :o, None, None] - e[None, None, o:, None] - e[None, None, None, o:]
    t2 = np.conj(V["oovv"]) / D                      # <ab||ij> / (e_i + e_j - e_a - e_b)
    _, S2 = R.residual_cc2(f, V, np.zeros((o, v), complex), t2)
    assert np.max(np.abs(S2)) < 1e-14 * np.max(np.abs(t2 * D))


def _rotate(B, f, o, Uo, Uv):
    n = B.shape[1]
    U = np.zeros((n, n), complex)
    U[:o, :o] = Uo
    U[o:, o:] = Uv
    return np.einsum("pi,Xpq,qj->Xij", U.conj(), B, U, optimize=True), U.conj().T @ f @ U


def test_cc2_energy_invariant_under_rotations_and_differs_from_ccsd():
    o, v, naux, seed = 4, 10, 24, 51
    s = inputs.make_system(o, v, naux, seed, scale=0.05)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=100, tol=1e-11, method="cc2")
    assert ref["converged"]
    Bp, fp = _rotate(s.B, f, o, inputs.random_unitary(o, 8), inputs.random_unitary(v, 9))
    rot = R.solve(fp, R.integrals(Bp, o), o, v, max_iter=200, tol=1e-11, method="cc2")
    assert rot["converged"]
    assert abs(rot["energy"] - ref["energy"]) < 1e-10
    ccsd = R.solve(f, V, o, v, max_iter=100, tol=1e-11)
    assert abs(ccsd["energy"] - ref["energy"]) > 1e-8
