"""Brute force in the N-electron determinant space: the pin for the CCSD and triples oracles.

TEST INFRASTRUCTURE ONLY (see ``oracle/ccsd_ref.py``).

This module never uses the Appendix-A working equations. It builds the
second-quantised Hamiltonian of Eq. Hamiltonian as an explicit matrix over all
C(n, N) Slater determinants, forms the similarity-transformed Hamiltonian
H_bar = exp(-T) H exp(T) of Eq. CCSD with explicit operator matrices for T1 and T2
(Eq. t_amp, with the 1/4 normalisation of T2), and projects on the reference, the
singles and the doubles. It also diagonalises H (full CI), projects on the
triple excitations, gives the Moller-Plesset perturbed wavefunctions through
second order (the pins of the triples corrections), and evaluates the Lambda
equations as <0|(1 + Lambda)[H_bar, tau]|0>, the one-body density
<0|(1 + Lambda) exp(-T) a+_p a_q exp(T)|0> and the full-CI left vector.

Conventions: spinors 0..n-1 with the N = o lowest occupied in the reference;
a determinant is a sorted tuple of occupied spinors; a+_p acting on a determinant
carries the sign (-1)^(number of occupied spinors with index < p).
E_pq = a+_p a_q; a+_p a+_q a_s a_r = E_pr E_qs - delta_qr E_ps.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def determinants(n: int, nel: int):
    dets = [tuple(c) for c in itertools.combinations(range(n), nel)]
    return dets, {d: k for k, d in enumerate(dets)}


def excitation_matrices(n: int, nel: int) -> np.ndarray:
    """E[p, q] = matrix of a+_p a_q in the determinant basis, shape (n, n, d, d)."""
    dets, index = determinants(n, nel)
    d = len(dets)
    E = np.zeros((n, n, d, d))
    for col, det in enumerate(dets):
        occ = set(det)
        for q in det:
            s1 = sum(1 for x in det if x < q)  # sign of a_q
            rem = occ - {q}
            for p in range(n):
                if p in rem:
                    continue
                s2 = sum(1 for x in rem if x < p)  # sign of a+_p
                new = tuple(sorted(rem | {p}))
                E[p, q, index[new], col] += (-1) ** (s1 + s2)
    return E


def hamiltonian(h: np.ndarray, V: np.ndarray, E: np.ndarray) -> np.ndarray:
    """H = sum_pq h_pq E_pq + 1/4 sum_pqrs <pq||rs> (E_pr E_qs - delta_qr E_ps)."""
    H = np.einsum("pq,pqxy->xy", h, E)
    M = np.einsum("pqrs,prxz->qsxz", V, E, optimize=True)
    H = H + 0.25 * np.einsum("qsxz,qszy->xy", M, E, optimize=True)
    H = H - 0.25 * np.einsum("pqqs,psxy->xy", V, E, optimize=True)
    return H


def core_hamiltonian(f: np.ndarray, V: np.ndarray, o: int) -> np.ndarray:
    """h_pq = f_pq - sum_k <pk||qk>: the one-body part that yields Fock matrix f."""
    return f - np.einsum("pkqk->pq", V[:, :o, :, :o])


class Space:
    """Determinant space of an o-electron system in n = o + v spinors."""

    def __init__(self, o: int, v: int):
        self.o, self.v, self.n = o, v, o + v
        self.E = excitation_matrices(self.n, o)
        self.dets, self.index = determinants(self.n, o)
        self.ref = np.zeros(len(self.dets))
        self.ref[self.index[tuple(range(o))]] = 1.0

    def cluster_operator(self, t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
        """T = sum_ia t^a_i E_ai + 1/4 sum_ijab t^{ab}_{ij} E_ai E_bj."""
        o = self.o
        Evo = self.E[o:, :o]  # E[a, i] = a+_a a_i
        T1 = np.einsum("ia,aixy->xy", t1, Evo)
        P = np.einsum("ijab,aixz->jbxz", t2, Evo, optimize=True)
        T2 = 0.25 * np.einsum("jbxz,bjzy->xy", P, Evo, optimize=True)
        return T1 + T2

    def expm_nilpotent(self, T: np.ndarray) -> np.ndarray:
        """exp(T) = sum_k T^k / k!, exact because T raises the excitation level."""
        out = np.eye(T.shape[0], dtype=np.complex128)
        term = np.eye(T.shape[0], dtype=np.complex128)
        for k in range(1, self.o + 2):
            term = term @ T / k
            out = out + term
        assert not np.any(term @ T), "T is not nilpotent at order o + 1"
        return out

    def projections(self, f: np.ndarray, V: np.ndarray, t1: np.ndarray, t2: np.ndarray):
        """(E_ref, <0|H_bar|0>, <ia|H_bar|0>, <ijab|H_bar|0>) with |ijab> = E_ai E_bj |0>."""
        o, v = self.o, self.v
        h = core_hamiltonian(f, V, o)
        H = hamiltonian(h, V, self.E)
        T = self.cluster_operator(t1, t2)
        ket = self.expm_nilpotent(-T) @ (H @ (self.expm_nilpotent(T) @ self.ref))
        e_ref = self.ref @ H @ self.ref
        e_cc = self.ref @ ket
        Evo = self.E[o:, :o]
        singles = np.einsum("aixy,y->iax", Evo, self.ref)  # |ia> vectors
        S1 = np.einsum("iax,x->ia", singles, ket)
        doubles = np.einsum("aixz,bjzy,y->ijabx", Evo, Evo, self.ref, optimize=True)
        S2 = np.einsum("ijabx,x->ijab", doubles, ket, optimize=True)
        return e_ref, e_cc, S1, S2

    def fci(self, f: np.ndarray, V: np.ndarray):
        """Full CI: (E_ref, eigenvalue of the state with the largest reference weight)."""
        h = core_hamiltonian(f, V, self.o)
        H = hamiltonian(h, V, self.E)
        assert np.allclose(H, H.conj().T, atol=1e-12)
        w, U = np.linalg.eigh(H)
        k = int(np.argmax(np.abs(self.ref @ U)))
        return float(np.real(self.ref @ H @ self.ref)), float(w[k])


    def ci_doubles(self, f: np.ndarray, V: np.ndarray):
        """CI in the reference and its double excitations only: (E_ref, eigenvalue of the state
        with the largest reference weight). For two electrons this is CCD (T2 squared vanishes)."""
        h = core_hamiltonian(f, V, self.o)
        H = hamiltonian(h, V, self.E)
        occ = set(range(self.o))
        keep = [k for k, d in enumerate(self.dets) if self.o - len(occ.intersection(d)) in (0, 2)]
        Hs = H[np.ix_(keep, keep)]
        ref = self.ref[keep]
        w, U = np.linalg.eigh(Hs)
        k = int(np.argmax(np.abs(ref @ U)))
        return float(np.real(self.ref @ H @ self.ref)), float(w[k])


    def triples(self) -> np.ndarray:
        """|ijk abc> = E_ai E_bj E_ck |0> for all labels, as an array [i, j, k, a, b, c, x]."""
        Evo = self.E[self.o:, :self.o]
        s1 = np.einsum("ckxy,y->ckx", Evo, self.ref)
        s2 = np.einsum("bjxz,ckz->jkbcx", Evo, s1, optimize=True)
        return np.einsum("aixz,jkbcz->ijkabcx", Evo, s2, optimize=True)

    def excitation_level(self) -> np.ndarray:
        """Number of virtual spinors occupied in each determinant."""
        return np.array([sum(1 for p in d if p >= self.o) for d in self.dets])

    def moller_plesset(self, f: np.ndarray, V: np.ndarray):
        """Rayleigh-Schrodinger perturbation theory with H0 = sum of the diagonal Fock energies
        of each determinant's spinors (f must be diagonal, so that H0 has the reference as
        eigenvector and the singles do not couple at first order).

        Returns (H, H - H0, psi1, psi2) in intermediate normalisation:
        (E0 - H0) psi1 = Q V |0>, (E0 - H0) psi2 = Q (V - E1) psi1, Q = 1 - |0><0|."""
        assert np.allclose(f, np.diag(np.diag(f))), "Moller-Plesset partitioning needs a diagonal f"
        H = hamiltonian(core_hamiltonian(f, V, self.o), V, self.E)
        e = np.real(np.diag(f))
        h0 = np.array([sum(e[p] for p in d) for d in self.dets])
        W = H - np.diag(h0)
        r = self.index[tuple(range(self.o))]
        gap = h0[r] - h0
        gap[r] = 1.0
        q = np.ones(len(self.dets))
        q[r] = 0.0
        psi1 = q * (W @ self.ref) / gap
        e1 = self.ref @ W @ self.ref
        psi2 = q * ((W - e1 * np.eye(len(self.dets))) @ psi1) / gap
        return H, W, psi1, psi2


    def excitation_vectors(self):
        """(|ia> as [i,a,x], |ijab> as [i,j,a,b,x]) with |ia> = E_ai|0>, |ijab> = E_ai E_bj|0>."""
        Evo = self.E[self.o:, :self.o]
        singles = np.einsum("aixy,y->iax", Evo, self.ref)
        doubles = np.einsum("aixz,bjzy,y->ijabx", Evo, Evo, self.ref, optimize=True)
        return singles, doubles

    def left_vector(self, l1: np.ndarray, l2: np.ndarray) -> np.ndarray:
        """<0| (1 + Lambda) as a row vector, Lambda = sum_ia l^i_a (E_ai)^+ + 1/4 sum_ijab
        l^{ij}_{ab} (E_ai E_bj)^+: 1 on the reference, lambda_mu on each |mu> (i<j, a<b)."""
        singles, doubles = self.excitation_vectors()
        return (self.ref.astype(np.complex128) + np.einsum("ia,iax->x", l1, singles)
                + 0.25 * np.einsum("ijab,ijabx->x", l2, doubles, optimize=True))

    def lagrangian_gradient(self, f, V, t1, t2, l1, l2):
        """<0| (1 + Lambda) [H_bar, tau_nu] |0> for tau_nu = E_ai and E_ai E_bj, H_bar = exp(-T) H exp(T)."""
        o = self.o
        H = hamiltonian(core_hamiltonian(f, V, o), V, self.E)
        T = self.cluster_operator(t1, t2)
        Hb = self.expm_nilpotent(-T) @ H @ self.expm_nilpotent(T)
        bra = self.left_vector(l1, l2)
        Evo = self.E[o:, :o]
        singles, doubles = self.excitation_vectors()
        w = bra @ Hb                      # <L| H_bar
        h0 = Hb @ self.ref                # H_bar |0>
        # <L| tau_nu as row vectors
        b1 = np.einsum("x,aixy->iay", bra, Evo)
        b2 = np.einsum("x,aixz,bjzy->ijaby", bra, Evo, Evo, optimize=True)
        R1 = np.einsum("x,iax->ia", w, singles) - np.einsum("iay,y->ia", b1, h0)
        R2 = np.einsum("x,ijabx->ijab", w, doubles) - np.einsum("ijaby,y->ijab", b2, h0)
        return R1, R2

    def density(self, t1, t2, l1, l2):
        """gamma_pq = <0| (1 + Lambda) exp(-T) a+_p a_q exp(T) |0>."""
        T = self.cluster_operator(t1, t2)
        bra = self.left_vector(l1, l2) @ self.expm_nilpotent(-T)
        ket = self.expm_nilpotent(T) @ self.ref
        return np.einsum("x,pqxy,y->pq", bra, self.E, ket, optimize=True)

    def fci_left_lambda(self, f, V, t1, t2):
        """For a state that CCSD describes exactly (two electrons): the left eigenvector of H_bar,
        <Psi| exp(T) / <Psi| exp(T) |0>, as (l1, l2) on the singles and doubles."""
        H = hamiltonian(core_hamiltonian(f, V, self.o), V, self.E)
        w, U = np.linalg.eigh(H)
        k = int(np.argmax(np.abs(self.ref @ U)))
        bra = np.conj(U[:, k]) @ self.expm_nilpotent(self.cluster_operator(t1, t2))
        bra = bra / (bra @ self.ref)
        singles, doubles = self.excitation_vectors()
        return np.einsum("x,iax->ia", bra, singles), np.einsum("x,ijabx->ijab", bra, doubles)


def n_determinants(o: int, v: int) -> int:
    return math.comb(o + v, o)
