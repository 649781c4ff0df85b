"""Plain CPU oracle for the perturbative triples corrections E(+T), E((T)) and E(-T).

TEST INFRASTRUCTURE, under the same rule as ``oracle/ccsd_ref.py``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may
import it.

It follows the appendix "Working equations for perturbative Triples" in its own
order: the intermediate W (Eq. W-term), its sum over the three cyclic orders of
the virtual labels, the denominator, the fourth-order term (Eq. 4order-term),
the fifth-order term with the intermediate Z (Eqs. 5order-term and Z-term), and
the alternative fifth-order term with the intermediate Y (Eq. Y-term). As the
appendix states, the sums run over all i, j, k and a, b, c (not only i<j<k,
a<b<c), and each is divided by 36. Everything is complex128 / float64 with one
``numpy.einsum`` per printed term, no blocking and no reordering.

Tensor layout as in ``oracle/ccsd_ref.py``: V is the dict of antisymmetrised
blocks ("oovv" = <ij||ab>, "ooov" = <kl||ic>, "vovv" = <ak||cd>), f is the full
Fock matrix (occupied first), t1[i,a] = t^a_i, t2[i,j,a,b] = t^{ab}_{ij}.

Readings of the appendix (the printed equations carry no complex conjugation in
W and E(+T), and their signs do not agree with one another):

* r14 (W). The integrals <ie||ab> and <jk||am> are read as their Hermitian
  partners <ab||ie> = conj(<ie||ab>) and <am||jk> = conj(<jk||am>), which equal
  them for real spinors. Under this reading the cyclic sum of W is the
  connected triples numerator <Phi^{abc}_{ijk}| V T2 |Phi_0>. As printed it is
  not that projection, and E(+T) would change with the phases of the spinors.
* r15 (denominator, E(+T)). D^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j - e_k,
  with e the real diagonal of f (the same reading as the CCSD denominators).
  The first factor of the numerator is conjugated, so
  E(+T) = -1/36 sum |X|^2 / D <= 0. At first-order T2 this is the triples part
  of the fourth-order Moller-Plesset energy.
* r16 (E((T))). Z is read as conj(Y_d), where Y_d is the disconnected triples
  numerator <Phi^{abc}_{ijk}| V T1 + F T2 |Phi_0>: Z = <ij||ab> conj(t^c_k) +
  conj(t^{ab}_{ij}) f_kc + (cyclic in i, j, k). The term is
  <T1 Phi_0| V |T3 Phi_0> + <T2 Phi_0| F |T3 Phi_0> with t3 = -X/D, i.e.
  -1/36 sum Re[X Z] / D. The appendix prints "+" with the same D as E(+T).
  That sign would make the (T) and -T terms opposite at leading order, where
  both estimate the same singles-triples coupling. The sign taken here makes
  them agree, and it is the singles-triples term of fifth-order perturbation
  theory.
* r17 (E(-T)). The cyclic sum of Y is the triples part of exp(T1 + T2)|Phi_0>.
  It enters conjugated: +1/36 sum Re[X conj(Y)], with the printed sign and no
  denominator.
* The energies are real, and the real part of each complex sum is taken.

Each reading is pinned by ``tests/test_oracle_triples.py``. The pins compare
against projections in the determinant space, Rayleigh-Schrodinger
perturbation theory, the exponential of the cluster operator, invariance under
spinor phases, and the ratio of the two fifth-order terms in a model with
degenerate levels.
"""
from __future__ import annotations

import itertools

import numpy as np


def _blocks(V: dict, o: int):
    """<ab||ie> [a,b,i,e], <am||jk> [a,m,j,k] and <ab||ij> [a,b,i,j] from the stored blocks."""
    # <ie||ab> = -<ei||ab> = -vovv[e,i,a,b]; its Hermitian partner is the conjugate.
    vvov = -np.conj(V["vovv"]).transpose(2, 3, 1, 0)
    # <jk||am> = -<jk||ma> = -ooov[j,k,m,a]; its Hermitian partner is the conjugate.
    vooo = -np.conj(V["ooov"]).transpose(3, 2, 0, 1)
    vvoo = np.conj(V["oovv"]).transpose(2, 3, 0, 1)
    return vvov, vooo, vvoo


def w_intermediate(V: dict, t2: np.ndarray, parts: dict | None = None) -> np.ndarray:
    """W^{abc}_{ijk} of Eq. W-term (reading r14), as W[i,j,k,a,b,c]."""
    o = t2.shape[0]
    vvov, vooo, _ = _blocks(V, o)
    es = np.einsum
    terms = {
        "e_i": es("abie,jkec->ijkabc", vvov, t2),      # sum_e <ab||ie> t^{ec}_{jk}
        "e_j": es("abje,kiec->ijkabc", vvov, t2),      # sum_e <ab||je> t^{ec}_{ki}
        "e_k": es("abke,ijec->ijkabc", vvov, t2),      # sum_e <ab||ke> t^{ec}_{ij}
        "m_ij": es("amij,kmbc->ijkabc", vooo, t2),     # sum_m <am||ij> t^{bc}_{km}
        "m_jk": es("amjk,imbc->ijkabc", vooo, t2),     # sum_m <am||jk> t^{bc}_{im}
        "m_ki": es("amki,jmbc->ijkabc", vooo, t2),     # sum_m <am||ki> t^{bc}_{jm}
    }
    if parts is not None:
        parts.update(terms)
    return sum(terms.values())


def cyclic_virtual(W: np.ndarray) -> np.ndarray:
    """W^{abc} + W^{bca} + W^{cab} over the last three (virtual) axes."""
    return W + W.transpose(0, 1, 2, 4, 5, 3) + W.transpose(0, 1, 2, 5, 3, 4)


def denominators(f: np.ndarray, o: int) -> np.ndarray:
    """D^{abc}_{ijk} = e_a + e_b + e_c - e_i - e_j - e_k (reading r15), as D[i,j,k,a,b,c]."""
    e = np.real(np.diag(f))
    eo, ev = e[:o], e[o:]
    occ = eo[:, None, None] + eo[None, :, None] + eo[None, None, :]
    vir = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    return vir[None, None, None] - occ[:, :, :, None, None, None]


def z_intermediate(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
    """Z^{abc}_{ijk} of Eq. Z-term (reading r16), as Z[i,j,k,a,b,c]."""
    o = t1.shape[0]
    oovv = V["oovv"]
    fov = f[:o, o:]
    t1c, t2c = np.conj(t1), np.conj(t2)
    es = np.einsum
    return (es("ijab,kc->ijkabc", oovv, t1c) + es("ijab,kc->ijkabc", t2c, fov)
            + es("jkab,ic->ijkabc", oovv, t1c) + es("jkab,ic->ijkabc", t2c, fov)
            + es("kiab,jc->ijkabc", oovv, t1c) + es("kiab,jc->ijkabc", t2c, fov))


def y_intermediate(t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
    """Y^{abc}_{ijk} of Eq. Y-term, as Y[i,j,k,a,b,c]."""
    es = np.einsum
    t111 = es("ia,jb,kc->ijkabc", t1, t1, t1)     # t^a_i t^b_j t^c_k
    # the six orderings of (i, j, k) with their signs, as listed in Eq. Y-term
    alt = np.zeros_like(t111)
    for perm in itertools.permutations(range(3)):
        sign = 1 if sum(perm[x] > perm[y] for x in range(3) for y in range(x + 1, 3)) % 2 == 0 else -1
        alt += sign * t111.transpose(*perm, 3, 4, 5)
    return (alt / 3.0 + es("ijab,kc->ijkabc", t2, t1) + es("jkab,ic->ijkabc", t2, t1)
            + es("kiab,jc->ijkabc", t2, t1))


def corrections(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray) -> dict:
    """The three triples corrections to the CCSD energy: {"+T", "(T)", "-T"} (real)."""
    o = t1.shape[0]
    X = cyclic_virtual(w_intermediate(V, t2))
    D = denominators(f, o)
    e4 = -np.sum(np.abs(X) ** 2 / D) / 36.0                                      # Eq. 4order-term
    Zs = cyclic_virtual(z_intermediate(f, V, t1, t2))
    e5 = -np.sum(np.real(X * Zs) / D) / 36.0                                     # Eq. 5order-term
    Ys = cyclic_virtual(y_intermediate(t1, t2))
    e5m = np.sum(np.real(X * np.conj(Ys))) / 36.0                                # Eq. for E(-T)
    return {"+T": float(e4), "(T)": float(e4 + e5), "-T": float(e4 + e5m)}


def pair_contributions(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, i: int, j: int) -> np.ndarray:
    """Contributions of the triples (i, j, k), k > j, to [E(+T), E((T)), E(-T)] (i < j).

    The same equations evaluated at fixed occupied labels: W, Z and Y of one triple by the
    printed terms with i, j, k held fixed, summed over the unique a < b < c (the full sum over
    the virtual labels / 6, by antisymmetry). Needs only the blocks "oovv", "ooov" and "vovv"
    of V, so it runs at sizes where <ab||cd> cannot be formed.
    """
    o, v = t1.shape
    vvov, vooo, _ = _blocks(V, o)
    oovv, fov = V["oovv"], f[:o, o:]
    e = np.real(np.diag(f))
    es = np.einsum
    out = np.zeros(3)
    for k in range(j + 1, o):
        W = (es("abe,ec->abc", vvov[:, :, i, :], t2[j, k]) + es("abe,ec->abc", vvov[:, :, j, :], t2[k, i])
             + es("abe,ec->abc", vvov[:, :, k, :], t2[i, j])
             + es("am,mbc->abc", vooo[:, :, i, j], t2[k]) + es("am,mbc->abc", vooo[:, :, j, k], t2[i])
             + es("am,mbc->abc", vooo[:, :, k, i], t2[j]))
        X = W + W.transpose(2, 0, 1) + W.transpose(1, 2, 0)              # W^{abc} + W^{bca} + W^{cab}
        Z = np.zeros((v, v, v), complex)
        Y = np.zeros((v, v, v), complex)
        for p, q, r in ((i, j, k), (j, k, i), (k, i, j)):
            Z += es("ab,c->abc", oovv[p, q], np.conj(t1[r])) + es("ab,c->abc", np.conj(t2[p, q]), fov[r])
            Y += es("ab,c->abc", t2[p, q], t1[r])
        Zs = Z + Z.transpose(2, 0, 1) + Z.transpose(1, 2, 0)
        rows = t1[[i, j, k]]                 # 3 x v; the six signed orderings of Eq. Y-term (their
                                             # cyclic virtual sum is 3 times the same determinant)
        det = (es("a,b,c->abc", rows[0], rows[1], rows[2]) - es("a,b,c->abc", rows[1], rows[0], rows[2])
               + es("a,b,c->abc", rows[1], rows[2], rows[0]) - es("a,b,c->abc", rows[2], rows[1], rows[0])
               + es("a,b,c->abc", rows[2], rows[0], rows[1]) - es("a,b,c->abc", rows[0], rows[2], rows[1]))
        Ys = det + Y + Y.transpose(2, 0, 1) + Y.transpose(1, 2, 0)
        ev = e[o:]
        D = ev[:, None, None] + ev[None, :, None] + ev[None, None, :] - e[i] - e[j] - e[k]
        e4 = -np.sum(np.abs(X) ** 2 / D) / 6.0
        out += [e4, e4 - np.sum(np.real(X * Zs) / D) / 6.0, e4 + np.sum(np.real(X * np.conj(Ys))) / 6.0]
    return out
