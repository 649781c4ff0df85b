"""Pins for the triples oracle (appendix "Working equations for perturbative Triples").

None of these re-types the appendix. The oracle's intermediates and energies are
compared with
  * projections in the determinant space: the connected triples <T| V T2 |0>,
    the disconnected numerator <T| V T1 + F T2 |0>, and the triples part of
    exp(T1 + T2)|0>,
  * Rayleigh-Schrodinger perturbation theory (Moller-Plesset partitioning):
    E(+T) at first-order T2 is the triples part of the fourth-order energy, and
    the (T) term at second-order T1 is the singles-triples coupling of the
    fifth order,
  * the ratio 3/2 of the -T and (T) terms in a model with degenerate levels,
  * invariance under spinor phases, and the vanishing of all three terms when
    no triple excitation exists.
Sensitivity tests plant mistakes in the oracle (a dropped term, the integrals
as printed without the Hermitian-partner reading) and check that a pin fails.
"""
import numpy as np
import pytest

from oracle import brute_force as BF
from oracle import ccsd_ref as R
from oracle import triples_ref as T3
from paper_2103_08473_gb300 import inputs


def _system(o, v, naux, seed, scale, fock_offdiag=0.0):
    s = inputs.make_system(o, v, naux, seed, scale=scale)
    f = R.fock_matrix(s.eps)
    if fock_offdiag:
        f = f + inputs.random_hermitian(o + v, seed + 100, scale=fock_offdiag)
    Vf = R.full_integrals(s.B)
    return s, f, Vf, R.blocks_from_full(Vf, o)


def _project(trip, vec):
    """<ijk abc| vec> for every label, [i,j,k,a,b,c] (the triples vectors are real)."""
    return np.einsum("ijkabcx,x->ijkabc", trip, vec, optimize=True)


def _unique_sum(x):
    """Sum of x over i<j<k and a<b<c."""
    o, v = x.shape[0], x.shape[3]
    return sum(x[i, j, k, a, b, c]
               for i in range(o) for j in range(i + 1, o) for k in range(j + 1, o)
               for a in range(v) for b in range(a + 1, v) for c in range(b + 1, v))


CASES = [(3, 4, 6, 61), (3, 5, 7, 62), (4, 4, 8, 63), (4, 5, 6, 64)]


@pytest.mark.parametrize("o,v,naux,seed", CASES)
def test_connected_numerator_is_the_triples_projection(o, v, naux, seed):
    """cyclic sum of W = <ijk abc| V T2 |0> (f diagonal, so F T2 has no triples part)."""
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6)
    _, t2 = inputs.random_amplitudes(o, v, seed + 200, scale=0.3)
    sp = BF.Space(o, v)
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    T = sp.cluster_operator(np.zeros((o, v)), t2)
    Xb = _project(sp.triples(), H @ (T @ sp.ref))
    X = T3.cyclic_virtual(T3.w_intermediate(V, t2))
    assert np.max(np.abs(Xb)) > 1e-2
    np.testing.assert_allclose(X, Xb, atol=1e-13)


@pytest.mark.parametrize("o,v,naux,seed", CASES[:2])
def test_disconnected_numerator_is_the_triples_projection(o, v, naux, seed):
    """conj of the cyclic sum of Z = <ijk abc| V T1 + F T2 |0>, with an off-diagonal Fock block."""
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6, fock_offdiag=0.3)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 300, scale=0.3)
    sp = BF.Space(o, v)
    trip = sp.triples()
    fd = np.diag(np.diag(f))
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    Hd = BF.hamiltonian(BF.core_hamiltonian(fd, Vf, o), Vf, sp.E)
    T = sp.cluster_operator(t1, t2)
    T2op = sp.cluster_operator(np.zeros((o, v)), t2)
    # <T| H (T1 + T2) |0> = X + Y_d; X alone comes from the diagonal-Fock Hamiltonian
    Yb = _project(trip, H @ (T @ sp.ref)) - _project(trip, Hd @ (T2op @ sp.ref))
    Zs = T3.cyclic_virtual(T3.z_intermediate(f, V, t1, t2))
    assert np.max(np.abs(Yb)) > 1e-2
    np.testing.assert_allclose(np.conj(Zs), Yb, atol=1e-13)


@pytest.mark.parametrize("o,v,seed", [(3, 4, 71), (4, 5, 72)])
def test_y_is_the_triples_part_of_the_exponential(o, v, seed):
    t1, t2 = inputs.random_amplitudes(o, v, seed, scale=0.4)
    sp = BF.Space(o, v)
    C3 = _project(sp.triples(), sp.expm_nilpotent(sp.cluster_operator(t1, t2)) @ sp.ref)
    Ys = T3.cyclic_virtual(T3.y_intermediate(t1, t2))
    assert np.max(np.abs(C3)) > 1e-2
    np.testing.assert_allclose(Ys, C3, atol=1e-14)


def _mp_amplitudes(o, v, naux, seed, scale):
    s, f, Vf, V = _system(o, v, naux, seed, scale=scale)
    sp = BF.Space(o, v)
    H, W, psi1, psi2 = sp.moller_plesset(f, Vf)
    lvl = sp.excitation_level()
    Evo = sp.E[o:, :o]
    singles = np.einsum("aixy,y->iax", Evo, sp.ref)
    doubles = np.einsum("aixz,bjzy,y->ijabx", Evo, Evo, sp.ref, optimize=True)
    assert np.max(np.abs(psi1[lvl != 2])) < 1e-14      # first order: doubles only
    t2 = np.einsum("ijabx,x->ijab", doubles, psi1, optimize=True)
    t1 = np.einsum("iax,x->ia", singles, psi2)
    return f, V, sp, W, psi1, psi2, lvl, t1, t2


@pytest.mark.parametrize("o,v,naux,seed", [(3, 4, 6, 81), (3, 5, 7, 82), (4, 4, 6, 83)])
def test_plus_t_is_the_fourth_order_triples_energy(o, v, naux, seed):
    f, V, sp, W, psi1, psi2, lvl, t1, t2 = _mp_amplitudes(o, v, naux, seed, scale=0.6)
    psi2_t = np.where(lvl == 3, psi2, 0.0)
    e4t = np.vdot(psi1, W @ psi2_t)
    assert abs(e4t.imag) < 1e-14 and e4t.real < -1e-6
    e = T3.corrections(f, V, t1, t2)
    assert abs(e["+T"] - e4t.real) < 1e-12 * abs(e4t)


@pytest.mark.parametrize("o,v,naux,seed", [(3, 4, 6, 84), (4, 5, 6, 85)])
def test_paren_t_term_is_the_fifth_order_singles_triples_coupling(o, v, naux, seed):
    """E((T)) - E(+T) at second-order T1 and first-order T2 = Re <psi2_S| V |psi2_T>."""
    f, V, sp, W, psi1, psi2, lvl, t1, t2 = _mp_amplitudes(o, v, naux, seed, scale=0.6)
    psi2_s = np.where(lvl == 1, psi2, 0.0)
    psi2_t = np.where(lvl == 3, psi2, 0.0)
    e5st = np.vdot(psi2_s, W @ psi2_t).real
    e = T3.corrections(f, V, t1, t2)
    assert abs(e5st) > 1e-7
    assert abs((e["(T)"] - e["+T"]) - e5st) < 1e-12 * abs(e5st)


@pytest.mark.parametrize("o,v,naux,seed", [(3, 4, 6, 86), (4, 4, 8, 87)])
def test_minus_t_term_is_the_disconnected_triples_energy(o, v, naux, seed):
    """E(-T) - E(+T) = Re <C3| V T2 |0>, C3 the triples part of exp(T1 + T2)|0>."""
    s, f, Vf, V = _system(o, v, naux, seed, scale=0.6)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 400, scale=0.3)
    sp = BF.Space(o, v)
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    lvl = sp.excitation_level()
    c3 = np.where(lvl == 3, sp.expm_nilpotent(sp.cluster_operator(t1, t2)) @ sp.ref, 0.0)
    ref = np.vdot(c3, H @ (sp.cluster_operator(np.zeros((o, v)), t2) @ sp.ref)).real
    e = T3.corrections(f, V, t1, t2)
    assert abs(ref) > 1e-4
    assert abs((e["-T"] - e["+T"]) - ref) < 1e-12 * abs(ref)


def test_fifth_order_terms_agree_with_degenerate_levels():
    """With all occupied levels at e_o and all virtual ones at e_v, first-order T2 and
    small T1, the -T term over the (T) term tends to D3/D2 = 3/2: the two readings of the
    fifth-order terms have the same sign."""
    o, v = 4, 6
    s = inputs.make_system(o, v, 10, 91, scale=0.4)
    eps = np.concatenate([np.full(o, -1.0), np.full(v, 1.0)])
    f = R.fock_matrix(eps)
    V = R.integrals(s.B, o)
    t2 = np.conj(V["oovv"]) / -4.0                      # -<ab||ij> / D2, D2 = 4
    t1, _ = inputs.random_amplitudes(o, v, 92, scale=1e-4)
    e = T3.corrections(f, V, t1, t2)
    paren, minus = e["(T)"] - e["+T"], e["-T"] - e["+T"]
    assert abs(paren) > 1e-12
    assert abs(minus / paren - 1.5) < 1e-6


def test_invariant_under_spinor_phases():
    o, v = 4, 7
    s = inputs.make_system(o, v, 12, 93, scale=0.3)
    f = R.fock_matrix(s.eps) + np.pad(inputs.random_hermitian(o + v, 94, 0.05)[:o, o:], ((0, v), (o, 0)))
    f = 0.5 * (f + f.conj().T)
    t1, t2 = inputs.random_amplitudes(o, v, 95, scale=0.1)
    e0 = T3.corrections(f, R.integrals(s.B, o), t1, t2)
    u = np.exp(1j * np.random.default_rng(96).uniform(0, 2 * np.pi, o + v))
    Bp = np.conj(u)[None, :, None] * s.B * u[None, None, :]
    fp = np.conj(u)[:, None] * f * u[None, :]
    uo, uv = u[:o], u[o:]
    t1p = t1 * uo[:, None] * np.conj(uv)[None, :]
    t2p = t2 * uo[:, None, None, None] * uo[None, :, None, None] \
        * np.conj(uv)[None, None, :, None] * np.conj(uv)[None, None, None, :]
    e1 = T3.corrections(fp, R.integrals(Bp, o), t1p, t2p)
    for key in e0:
        assert abs(e1[key] - e0[key]) < 1e-13 * max(abs(e0[key]), 1e-8), key


@pytest.mark.parametrize("o,v", [(2, 5), (4, 2)])
def test_no_triples_without_three_distinct_labels(o, v):
    s = inputs.make_system(o, v, 6, 97, scale=0.5)
    t1, t2 = inputs.random_amplitudes(o, v, 98, scale=0.2)
    e = T3.corrections(R.fock_matrix(s.eps), R.integrals(s.B, o), t1, t2)
    assert all(abs(x) < 1e-25 for x in e.values())


def test_full_sum_over_36_is_the_unique_sum():
    """The cyclic sums are antisymmetric under every transposition, so 1/36 of the full sum
    equals the sum over i<j<k, a<b<c."""
    o, v = 4, 5
    s = inputs.make_system(o, v, 8, 99, scale=0.5)
    f = R.fock_matrix(s.eps)
    V = R.integrals(s.B, o)
    t1, t2 = inputs.random_amplitudes(o, v, 100, scale=0.2)
    X = T3.cyclic_virtual(T3.w_intermediate(V, t2))
    for perm in [(1, 0, 2, 3, 4, 5), (0, 2, 1, 3, 4, 5), (0, 1, 2, 4, 3, 5), (0, 1, 2, 3, 5, 4)]:
        np.testing.assert_allclose(X.transpose(perm), -X, atol=1e-15)
    D = T3.denominators(f, o)
    e = T3.corrections(f, V, t1, t2)
    assert abs(e["+T"] + _unique_sum(np.abs(X) ** 2 / D)) < 1e-13 * abs(e["+T"])


@pytest.mark.parametrize("term", ["e_i", "e_j", "e_k", "m_ij", "m_jk", "m_ki"])
def test_pin_catches_a_dropped_w_term(term):
    o, v = 3, 4
    s, f, Vf, V = _system(o, v, 6, 61, scale=0.6)
    _, t2 = inputs.random_amplitudes(o, v, 261, scale=0.3)
    sp = BF.Space(o, v)
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    Xb = _project(sp.triples(), H @ (sp.cluster_operator(np.zeros((o, v)), t2) @ sp.ref))
    parts = {}
    W = T3.w_intermediate(V, t2, parts=parts)
    assert np.max(np.abs(T3.cyclic_virtual(W) - Xb)) < 1e-13
    assert np.max(np.abs(T3.cyclic_virtual(W - parts[term]) - Xb)) > 1e-3


def test_pins_catch_the_integrals_as_printed(monkeypatch):
    """Without the Hermitian-partner reading of <ie||ab> and <jk||am>, both the projection
    pin and the phase invariance fail."""
    o, v = 3, 5
    s, f, Vf, V = _system(o, v, 7, 62, scale=0.6)
    t1, t2 = inputs.random_amplitudes(o, v, 262, scale=0.3)
    sp = BF.Space(o, v)
    H = BF.hamiltonian(BF.core_hamiltonian(f, Vf, o), Vf, sp.E)
    Xb = _project(sp.triples(), H @ (sp.cluster_operator(np.zeros((o, v)), t2) @ sp.ref))
    good = T3._blocks

    def as_printed(V, o):
        vvov, vooo, vvoo = good(V, o)
        return np.conj(vvov), np.conj(vooo), vvoo

    e0 = T3.corrections(f, V, t1, t2)
    monkeypatch.setattr(T3, "_blocks", as_printed)
    assert np.max(np.abs(T3.cyclic_virtual(T3.w_intermediate(V, t2)) - Xb)) > 1e-3
    printed = T3.corrections(f, V, t1, t2)["+T"]
    assert abs(printed - e0["+T"]) > 1e-6
    # and the printed form depends on the phases of the spinors
    u = np.exp(1j * np.random.default_rng(263).uniform(0, 2 * np.pi, o + v))
    Bp = np.conj(u)[None, :, None] * s.B * u[None, None, :]
    uo, uv = u[:o], u[o:]
    t2p = t2 * uo[:, None, None, None] * uo[None, :, None, None] \
        * np.conj(uv)[None, None, :, None] * np.conj(uv)[None, None, None, :]
    assert abs(T3.corrections(f, R.integrals(Bp, o), t1, t2p)["+T"] - printed) > 1e-6


def test_pair_contributions_sum_to_the_corrections():
    """The per-pair form (fixed occupied labels, blocks oovv/ooov/vovv only) sums to the full one."""
    o, v = 5, 6
    s, f, Vf, V = _system(o, v, 12, 101, scale=0.4, fock_offdiag=0.1)
    t1, t2 = inputs.random_amplitudes(o, v, 102, scale=0.1)
    ref = T3.corrections(f, V, t1, t2)
    small = {k: V[k] for k in ("oovv", "ooov", "vovv")}
    tot = sum(T3.pair_contributions(f, small, t1, t2, i, j) for i in range(o) for j in range(i + 1, o))
    for m, key in enumerate(("+T", "(T)", "-T")):
        assert abs(tot[m] - ref[key]) < 1e-13 * abs(ref[key]), key
