"""Pins for the CPU oracle: checks against results the mathematics fixes.

None of these tests re-types the Appendix-A equations. They compare the oracle with
  * brute force in the determinant space (exp(-T) H exp(T) projected on the
    reference, singles and doubles, Eq. CCSD) at random amplitudes,
  * full CI for two electrons (CCSD is exact there),
  * the MP2 closed form (first update from t = 0),
  * invariance of the converged energy under unitary rotations within the
    occupied and within the virtual spinors,
  * the real spin-restricted limit (closed-shell spatial MP2, spin adaptation),
  * structural invariants (antisymmetry, Hermiticity).
A sensitivity test drops or perturbs each term and checks that the brute-force
pin then fails, so that a dropped term, a wrong sign or a transposed operand
cannot pass unnoticed.
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


BRUTE_CASES = [(2, 3, 5, 11), (2, 4, 6, 12), (3, 4, 6, 13), (3, 5, 7, 14), (4, 4, 8, 15), (4, 5, 6, 16)]


@pytest.mark.parametrize("o,v,naux,seed", BRUTE_CASES)
def test_residual_and_energy_match_brute_force(o, v, naux, seed):
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 200, scale=0.3)
    e_ref, e_cc, S1b, S2b = BF.Space(o, v).projections(f, Vf, t1, t2)
    S1, S2 = R.residual(f, V, t1, t2)
    scale = max(np.max(np.abs(S2b)), 1.0)
    assert np.max(np.abs(S1 - S1b)) < 1e-12 * scale
    assert np.max(np.abs(S2 - S2b)) < 1e-12 * scale
    assert abs(R.energy(f, V, t1, t2) - (e_cc - e_ref)) < 1e-12 * max(abs(e_cc), 1.0)


def test_residual_zero_amplitudes_is_driver_only():
    """At t = 0 only F^{i+}_a and V^{ij+}_{ab} survive; brute force agrees."""
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 21, scale=0.5, fock_offdiag=0.2)
    z1, z2 = np.zeros((o, v), complex), np.zeros((o, o, v, v), complex)
    _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, z1, z2)
    S1, S2 = R.residual(f, V, z1, z2)
    np.testing.assert_allclose(S1, S1b, atol=1e-13)
    np.testing.assert_allclose(S2, S2b, atol=1e-13)
    np.testing.assert_allclose(S2b, np.conj(Vf[:o, :o, o:, o:]), atol=1e-13)


def _perturbations(V):
    """Plausible implementation mistakes, each applied to one term of the residual."""
    swaps = {
        "sign_vovo": lambda V: {**V, "vovo": -V["vovo"]},
        "braket_oooo": lambda V: {**V, "oooo": V["oooo"].transpose(2, 3, 0, 1).copy()},
        "conj_oovv": lambda V: {**V, "oovv": np.conj(V["oovv"])},
        "conj_vovv": lambda V: {**V, "vovv": np.conj(V["vovv"])},
        "sign_ooov": lambda V: {**V, "ooov": -V["ooov"]},
    }
    return swaps


@pytest.mark.parametrize("term", ["ring", "goo", "vt1", "gvv", "ct1", "hole", "ladder", "driver"])
def test_pin_catches_dropped_s2_term(term):
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 31, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 231, scale=0.3)
    _, _, _, S2b = BF.Space(o, v).projections(f, Vf, t1, t2)
    parts = {}
    _, S2 = R.residual(f, V, t1, t2, parts=parts)
    assert np.max(np.abs(S2 - S2b)) < 1e-12 * np.max(np.abs(S2b))
    assert np.max(np.abs((S2 - parts["S2_" + term]) - S2b)) > 1e-6
    flipped = S2 - 2 * parts["S2_" + term]
    assert np.max(np.abs(flipped - S2b)) > 1e-6


@pytest.mark.parametrize("term", ["f", "hvv", "hoo", "hov", "hf", "vovv", "ooov", "vovo"])
def test_pin_catches_dropped_s1_term(term):
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 32, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 232, scale=0.3)
    _, _, S1b, _ = BF.Space(o, v).projections(f, Vf, t1, t2)
    parts = {}
    S1, _ = R.residual(f, V, t1, t2, parts=parts)
    assert np.max(np.abs(S1 - S1b)) < 1e-12 * np.max(np.abs(S1b))
    assert np.max(np.abs((S1 - parts["S1_" + term]) - S1b)) > 1e-6


@pytest.mark.parametrize("mistake", ["conj_oovv", "conj_vovv", "sign_ooov", "sign_vovo", "braket_oooo"])
def test_pin_catches_wrong_integral_block(mistake):
    o, v = 3, 3
    s, f, Vf, V = _system(o, v, 6, 33, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 233, scale=0.3)
    _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, t1, t2)
    Vbad = _perturbations(V)[mistake](V)
    S1, S2 = R.residual(f, Vbad, t1, t2)
    assert max(np.max(np.abs(S1 - S1b)), np.max(np.abs(S2 - S2b))) > 1e-6


def test_energy_sign_and_transposed_amplitudes_are_caught():
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 34, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 234, scale=0.3)
    e_ref, e_cc, _, S2b = BF.Space(o, v).projections(f, Vf, t1, t2)
    assert abs(R.energy(f, V, t1, t2) - (e_cc - e_ref)) < 1e-12
    # t2 with (ab) and (ij) roles mixed up (t^{ij}_{ab} read as t^{ab}_{ij}) must fail
    _, S2 = R.residual(f, V, t1, -t2)
    assert np.max(np.abs(S2 - S2b)) > 1e-6


@pytest.mark.parametrize("v,naux,seed,scale", [(6, 10, 21, 0.3), (10, 12, 22, 0.2), (14, 20, 23, 0.15)])
def test_two_electron_ccsd_equals_full_ci(v, naux, seed, scale):
    o = 2
    s, f, Vf, V = _system(o, v, naux, seed, scale=scale)
    res = R.solve(f, V, o, v, max_iter=200, tol=1e-12)
    assert res["converged"]
    e_ref, e_fci = BF.Space(o, v).fci(f, Vf)
    assert abs(res["energy"] - (e_fci - e_ref)) < 1e-10


@pytest.mark.parametrize("v,naux,seed,fock_offdiag", [(6, 8, 61, 0.0), (8, 10, 62, 0.04)])
def test_two_electron_ccd_equals_doubles_ci(v, naux, seed, fock_offdiag):
    """CCD (t1 held at zero) for two electrons: T2 squared vanishes, so its energy is the
    lowest-lying root of H in the reference plus doubles space (explicit diagonalisation)."""
    o = 2
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.3, fock_offdiag=fock_offdiag)
    res = R.solve(f, V, o, v, max_iter=300, tol=1e-12, method="ccd")
    assert res["converged"] and np.max(np.abs(res["t1"])) == 0.0
    e_ref, e_cid = BF.Space(o, v).ci_doubles(f, Vf)
    assert abs(res["energy"] - (e_cid - e_ref)) < 1e-10
    # the singles matter: CCSD (= full CI for two electrons) differs
    e_ccsd = R.solve(f, V, o, v, max_iter=300, tol=1e-12)["energy"]
    assert abs(e_ccsd - res["energy"]) > 1e-8


def test_two_electron_full_ci_with_nondiagonal_fock():
    o, v = 2, 8
    s, f, Vf, V = _system(o, v, 10, 24, scale=0.25, fock_offdiag=0.05)
    res = R.solve(f, V, o, v, max_iter=300, tol=1e-12)
    assert res["converged"]
    e_ref, e_fci = BF.Space(o, v).fci(f, Vf)
    assert abs(res["energy"] - (e_fci - e_ref)) < 1e-10


@pytest.mark.parametrize("o,v,naux,seed", [(4, 12, 30, 41), (6, 18, 40, 42)])
def test_first_update_is_mp2_closed_form(o, v, naux, seed):
    s = inputs.make_system(o, v, naux, seed)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    t1, t2 = R.mp2_guess(f, V, o, v)
    # closed form from the integrals alone: E = sum_{i<j, a<b} |<ij||ab>|^2 / (e_i + e_j - e_a - e_b)
    e = s.eps
    iu, ju = np.triu_indices(o, 1)
    au, bu = np.triu_indices(v, 1)
    g = R.antisym_block(s.B, o, "oovv")[iu, ju][:, au, bu]
    den = (e[iu] + e[ju])[:, None] - (e[o + au] + e[o + bu])[None, :]
    e_mp2 = np.sum(np.abs(g) ** 2 / den)
    assert abs(R.energy(f, V, t1, t2) - e_mp2) < 1e-13 * max(1.0, abs(e_mp2))
    assert np.max(np.abs(t1)) == 0.0
    # amplitudes: t^{ab}_{ij} = <ab||ij> / D^{ab}_{ij}
    g_abij = R.antisym_block(s.B, o, "vvoo").transpose(2, 3, 0, 1)
    D = (e[:o, None, None, None] + e[None, :o, None, None] - e[None, None, o:, None] - e[None, None, None, o:])
    np.testing.assert_allclose(t2, g_abij / D, atol=1e-15)


def _rotate(B, f, o, Uo, Uv):
    n = B.shape[1]
    U = np.zeros((n, n), complex)
    U[:o, :o] = Uo
    U[o:, o:] = Uv
    Bp = np.einsum("pi,Xpq,qj->Xij", U.conj(), B, U, optimize=True)
    fp = U.conj().T @ f @ U
    return Bp, fp


@pytest.mark.parametrize("phase_only", [False, True])
def test_converged_energy_invariant_under_occupied_virtual_rotations(phase_only):
    o, v, naux, seed = 4, 12, 30, 51
    s = inputs.make_system(o, v, naux, seed, scale=0.05)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    ref = R.solve(f, V, o, v, max_iter=100, tol=1e-11)
    assert ref["converged"]
    if phase_only:
        rng = np.random.default_rng(7)
        Uo = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, o)))
        Uv = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, v)))
    else:
        Uo, Uv = inputs.random_unitary(o, 8), inputs.random_unitary(v, 9)
    Bp, fp = _rotate(s.B, f, o, Uo, Uv)
    Vp = R.integrals(Bp, o)
    rot = R.solve(fp, Vp, o, v, max_iter=200, tol=1e-11)
    assert rot["converged"]
    assert abs(rot["energy"] - ref["energy"]) < 1e-10
    if phase_only:
        # amplitudes transform like <ab||ij>: t'^{ab}_{ij} = t^{ab}_{ij} u_i u_j conj(u_a) conj(u_b)
        po, pv = np.diag(Uo), np.diag(Uv)
        t2p = ref["t2"] * po[:, None, None, None] * po[None, :, None, None] \
            * np.conj(pv)[None, None, :, None] * np.conj(pv)[None, None, None, :]
        np.testing.assert_allclose(rot["t2"], t2p, atol=1e-9)


def _spin_blocked(m_occ, m_vir, naux, seed):
    """Real closed-shell spatial DF factors and energies, expanded to spinors (iA, iB, ...)."""
    rng = np.random.default_rng(seed)
    m = m_occ + m_vir
    eo = np.sort(rng.uniform(-2.0, -0.5, m_occ))
    ev = np.sort(rng.uniform(0.3, 5.0, m_vir))
    x = 0.05 * rng.standard_normal((naux, m, m))
    Bs = 0.5 * (x + x.transpose(0, 2, 1))
    e_sp = np.concatenate([eo, ev])
    # spinor p = 2*spatial + spin
    B = np.einsum("Xpq,st->Xpsqt", Bs, np.eye(2)).reshape(naux, 2 * m, 2 * m)
    eps = np.repeat(e_sp, 2)
    return Bs, e_sp, B.astype(complex), eps


def test_real_spin_restricted_limit():
    mo, mv, naux = 3, 7, 20
    Bs, e_sp, B, eps = _spin_blocked(mo, mv, naux, 61)
    o, v = 2 * mo, 2 * mv
    f = R.fock_matrix(eps)
    V = R.integrals(B, o)
    # MP2: spinor oracle == closed-shell spatial formula sum (ia|jb)[2(ia|jb) - (ib|ja)] / D
    t1, t2 = R.mp2_guess(f, V, o, v)
    g = np.einsum("Xia,Xjb->iajb", Bs[:, :mo, mo:], Bs[:, :mo, mo:])
    D = (e_sp[:mo, None, None, None] - e_sp[None, mo:, None, None]
         + e_sp[None, None, :mo, None] - e_sp[None, None, None, mo:])
    e_rmp2 = np.sum(g * (2 * g - g.transpose(0, 3, 2, 1)) / D)
    assert abs(R.energy(f, V, t1, t2) - e_rmp2) < 1e-13
    res = R.solve(f, V, o, v, max_iter=100, tol=1e-11)
    assert res["converged"]
    t1, t2 = res["t1"], res["t2"]
    assert np.max(np.abs(t1.imag)) < 1e-14 and np.max(np.abs(t2.imag)) < 1e-14
    assert abs(res["energy"].imag) < 1e-14
    # spin structure: spin-forbidden amplitudes vanish; aa = ab - ba (spin adaptation)
    T2 = t2.real.reshape(mo, 2, mo, 2, mv, 2, mv, 2)
    T1 = t1.real.reshape(mo, 2, mv, 2)
    assert np.max(np.abs(T1[:, 0, :, 1])) < 1e-14
    assert np.max(np.abs(T2[:, 0, :, 0, :, 0, :, 1])) < 1e-14
    aa = T2[:, 0, :, 0, :, 0, :, 0]
    ab = T2[:, 0, :, 1, :, 0, :, 1]
    np.testing.assert_allclose(aa, ab - ab.transpose(0, 1, 3, 2), atol=1e-12)
    # alpha/beta symmetry of the closed shell
    np.testing.assert_allclose(T2[:, 1, :, 1, :, 1, :, 1], aa, atol=1e-12)


def test_integral_symmetries_and_residual_antisymmetry():
    o, v = 3, 5
    s, f, Vf, V = _system(o, v, 8, 71, scale=0.4, fock_offdiag=0.2)
    np.testing.assert_allclose(Vf, -Vf.transpose(1, 0, 2, 3), atol=1e-15)
    np.testing.assert_allclose(Vf, -Vf.transpose(0, 1, 3, 2), atol=1e-15)
    np.testing.assert_allclose(np.conj(Vf), Vf.transpose(2, 3, 0, 1), atol=1e-15)
    blocks = R.integrals(s.B, o)
    for k in R.BLOCKS:
        np.testing.assert_allclose(blocks[k], V[k], atol=1e-15)
    t1, t2 = inputs.random_amplitudes(o, v, 271, scale=0.3)
    _, S2 = R.residual(f, V, t1, t2)
    np.testing.assert_allclose(S2, -S2.transpose(1, 0, 2, 3), atol=1e-14)
    np.testing.assert_allclose(S2, -S2.transpose(0, 1, 3, 2), atol=1e-14)


def test_diis_reproduces_linear_extrapolation():
    """Two error vectors e1 = -e2 give c = (1/2, 1/2) exactly (Pulay)."""
    d = R.DIIS(8)
    o, v = 2, 3
    t1a, t2a = inputs.random_amplitudes(o, v, 1)
    t1b, t2b = inputs.random_amplitudes(o, v, 2)
    e1, e2 = inputs.random_amplitudes(o, v, 3)
    d.push(t1a, t2a, e1, e2)
    d.push(t1b, t2b, -e1, -e2)
    np.testing.assert_allclose(d.coefficients(), [0.5, 0.5], atol=1e-15)
    t1, t2 = d.extrapolate()
    np.testing.assert_allclose(t2, 0.5 * (t2a + t2b), atol=1e-16)


@pytest.mark.parametrize("m,pushed", [(3, 3), (5, 5), (8, 8), (8, 11)])
def test_diis_coefficients_minimise_the_error_norm(m, pushed):
    """The DIIS coefficients are the minimiser of |sum_i c_i e_i|^2 over sum_i c_i = 1 (Pulay),
    here found independently by least squares in the null space of the constraint; with more
    vectors pushed than kept, the newest `max_vec` are the ones used."""
    o, v = 3, 5
    d = R.DIIS(m)
    errs = []
    for k in range(pushed):
        t1, t2 = inputs.random_amplitudes(o, v, 100 + k)
        e1, e2 = inputs.random_amplitudes(o, v, 200 + k, scale=0.3)
        d.push(t1, t2, e1, e2)
        iu, ju = np.triu_indices(o, 1)
        au, bu = np.triu_indices(v, 1)
        uniq = e2[iu, ju][:, au, bu].ravel()
        errs.append(np.concatenate([e1.ravel(), uniq]))
    E = np.array(errs[-m:]).T                      # columns: the kept error vectors
    Er = np.vstack([E.real, E.imag])               # Re<e_i, e_j> = (Er^T Er)_ij
    c0 = np.full(m, 1.0 / m)
    null = np.linalg.svd(np.ones((1, m)))[2][1:].T  # basis of sum(c) = 0
    y = np.linalg.lstsq(Er @ null, -Er @ c0, rcond=None)[0]
    want = c0 + null @ y
    np.testing.assert_allclose(d.coefficients(), want, rtol=1e-9, atol=1e-11)


def test_sampled_ladder_elements_match_full_ladder():
    """The element-wise ladder used for full-size sampling agrees with the full einsum."""
    o, v, naux = 4, 11, 13
    s = inputs.make_system(o, v, naux, 81, scale=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 82, scale=0.2)
    full = R.ladder(R.integrals(s.B, o)["vvvv"], R.tau(t1, t2))
    rng = np.random.default_rng(3)
    idx = [tuple(int(x) for x in (rng.integers(o), rng.integers(o), rng.integers(v), rng.integers(v)))
           for _ in range(40)]
    got = R.ladder_elements(s.B, o, t1, t2, idx)
    want = np.array([full[i, j, a, b] for (i, j, a, b) in idx])
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_ladder_rows_match_full_ladder():
    """Whole (a, b) rows of the ladder formed from B^Q (used to time the oracle at sizes where
    <ab||cd> cannot be stored) agree with the full einsum ladder."""
    o, v, naux = 3, 9, 7
    s = inputs.make_system(o, v, naux, 83, scale=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, 84, scale=0.2)
    tau = R.tau(t1, t2)
    full = R.ladder(R.integrals(s.B, o)["vvvv"], tau)
    pairs = [(0, 1), (2, 7), (8, 3), (4, 4)]
    got = R.ladder_rows(s.B, o, tau, pairs)
    for n, (a, b) in enumerate(pairs):
        np.testing.assert_allclose(got[n], full[:, :, a, b], atol=1e-14)


# ---------------------------------------------------------------------------
# Level shift (keyword .LSHIFT of the input-keyword table; Sec. "Coupled cluster
# implementation": the update scales the residual by the orbital-energy denominators).
# Read as: +shift on every virtual orbital energy, in the denominators only. The shift
# changes the path of the iteration, never its fixed point S = 0.
# ---------------------------------------------------------------------------

def _hand_denominators(eps, o, shift):
    """D^a_i = e_i - e_a - shift and D^{ab}_{ij} = e_i + e_j - e_a - e_b - 2 shift, by loops."""
    v = len(eps) - o
    D1 = np.empty((o, v))
    D2 = np.empty((o, o, v, v))
    for i in range(o):
        for a in range(v):
            D1[i, a] = eps[i] - eps[o + a] - shift
            for j in range(o):
                for b in range(v):
                    D2[i, j, a, b] = eps[i] + eps[j] - eps[o + a] - eps[o + b] - 2.0 * shift
    return D1, D2


def _shifted_guess_error(oracle_guess, shift):
    """max relative distance between the oracle's shifted MP2 guess and S_bf(0) / D_hand."""
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 91, scale=0.5, fock_offdiag=0.2)
    eps = np.real(np.diag(f))
    z1, z2 = np.zeros((o, v), complex), np.zeros((o, o, v, v), complex)
    _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, z1, z2)
    D1, D2 = _hand_denominators(eps, o, shift)
    t1, t2 = oracle_guess(f, V, o, v, shift)
    want1, want2 = S1b / D1, S2b / D2
    return max(np.max(np.abs(t1 - want1)) / np.max(np.abs(want1)),
               np.max(np.abs(t2 - want2)) / np.max(np.abs(want2)))


@pytest.mark.parametrize("shift", [0.0, 0.5, 5.0, 20.0])
def test_shifted_mp2_guess_is_brute_force_driver_over_hand_denominators(shift):
    """t1 = S1(0)/(D1 - s), t2 = S2(0)/(D2 - 2s), with S(0) from the determinant space
    and D from the orbital energies by explicit loops."""
    assert _shifted_guess_error(R.mp2_guess, shift) < 1e-13


def _planted(kind):
    """The oracle's denominators with a plausible misreading of the shift planted."""
    def den(f, o, shift=0.0):
        d = np.real(np.diag(f)).astype(np.float64)
        if kind == "occupied":      # shift added to the occupied energies
            eo, ev = d[:o] + shift, d[o:]
        elif kind == "sign":        # shift subtracted from the virtual energies
            eo, ev = d[:o], d[o:] - shift
        elif kind == "once":        # doubles shifted once instead of once per virtual label
            eo, ev = d[:o], d[o:]
            D1 = eo[:, None] - ev[None, :] - shift
            D2 = (eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None]
                  - ev[None, None, None, :] - shift)
            return D1, D2
        D1 = eo[:, None] - ev[None, :]
        D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
        return D1, D2
    return den


@pytest.mark.parametrize("kind", ["occupied", "sign", "once"])
def test_shift_pin_catches_planted_misreadings(kind, monkeypatch):
    monkeypatch.setattr(R, "denominators", _planted(kind))
    assert _shifted_guess_error(R.mp2_guess, 5.0) > 1e-3


@pytest.mark.parametrize("shift", [0.5, 5.0])
def test_one_shifted_step_is_brute_force_residual_over_shifted_denominators(shift):
    """One Jacobi step from random amplitudes (no DIIS): t + S_bf(t) / D_hand(shift)."""
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 92, scale=0.5, fock_offdiag=0.2)
    t1, t2 = inputs.random_amplitudes(o, v, 292, scale=0.2)
    _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, t1, t2)
    D1, D2 = _hand_denominators(np.real(np.diag(f)), o, shift)
    res = R.solve(f, V, o, v, max_iter=1, tol=0.0, diis_dim=0, shift=shift, t_init=(t1, t2))
    np.testing.assert_allclose(res["t1"], t1 + S1b / D1, atol=1e-13)
    np.testing.assert_allclose(res["t2"], t2 + S2b / D2, atol=1e-13)


SHIFT_CASES = [(2, 4, 6, 93, 0.3, 0.05), (3, 4, 6, 94, 0.3, 0.05), (4, 12, 30, 95, 0.05, 0.0)]


@pytest.mark.parametrize("o,v,naux,seed,scale,offdiag", SHIFT_CASES)
def test_level_shift_moves_the_path_not_the_fixed_point(o, v, naux, seed, scale, offdiag):
    """Converged solves with shifts 0.5, 5 and 20 reach the unshifted fixed point (energy
    1e-10, amplitudes 1e-9). At the brute-force sizes, the shifted fixed point also zeroes
    <Phi_l| exp(-T) H exp(T) |Phi_0> in the determinant space."""
    s, f, Vf, V = _system(o, v, naux, seed, scale=scale, fock_offdiag=offdiag)
    ref = R.solve(f, V, o, v, max_iter=400, tol=1e-13)
    assert ref["converged"]
    space = BF.Space(o, v) if BF.n_determinants(o, v) <= 500 else None
    for shift in (0.5, 5.0, 20.0):
        res = R.solve(f, V, o, v, max_iter=2000, tol=1e-13, shift=shift)
        assert res["converged"], (shift, res["iterations"], res["norm"])
        assert abs(res["energy"] - ref["energy"]) < 1e-10
        assert np.max(np.abs(res["t1"] - ref["t1"])) < 1e-9
        assert np.max(np.abs(res["t2"] - ref["t2"])) < 1e-9
        if space is not None:
            _, _, S1b, S2b = space.projections(f, Vf, res["t1"], res["t2"])
            assert max(np.max(np.abs(S1b)), np.max(np.abs(S2b))) < 1e-10


def test_fixed_point_pin_catches_a_shift_leaking_into_the_residual(monkeypatch):
    """If the shift entered the residual (a shifted virtual Fock block in S) the iteration
    would converge to a different point, where the brute-force projections do not vanish."""
    o, v, naux, seed = 2, 4, 6, 93
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.3, fock_offdiag=0.05)
    shift = 5.0
    good_residual = R.residual

    def leaky(fm, Vm, t1, t2, **kw):
        g = fm.copy()
        g[o:, o:] += shift * np.eye(v)
        return good_residual(g, Vm, t1, t2, **kw)

    monkeypatch.setattr(R, "residual", leaky)
    res = R.solve(f, V, o, v, max_iter=2000, tol=1e-13, shift=shift)
    assert res["converged"]
    _, _, S1b, S2b = BF.Space(o, v).projections(f, Vf, res["t1"], res["t2"])
    assert max(np.max(np.abs(S1b)), np.max(np.abs(S2b))) > 1e-4
