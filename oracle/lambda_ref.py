"""Plain CPU oracle for the CCSD Lambda equations and the one-body density matrix.

TEST INFRASTRUCTURE, under the same rule as ``oracle/ccsd_ref.py``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.

Lambda (appendix "Working equations for CCSD lambda equations"). The appendix prints
the Lambda equations in terms of similarity-transformed-Hamiltonian intermediates and
leaves several of them to its reference (among them W^{ef}_{ag}, the bar F^j_m and
W^{ij}_{mb}). The equations have a plain definition that needs none of them. They are
the stationarity conditions of the coupled-cluster Lagrangian

    L(t, lambda) = E(t) + sum_mu lambda_mu S_mu(t)     (mu over t^a_i and t^{ab}_{ij}, i<j, a<b)

with respect to the amplitudes: R_nu = dL/dt_nu = <0| (1 + Lambda) [H_bar, tau_nu] |0>,
with Lambda = sum_mu lambda_mu tau_mu^+. Their driving terms are dE/dt. For t^{ab}_{ij}
this is V^{ij}_{ab}, the first term the appendix prints; for t^a_i it is F^a_i
+ sum_jb <ij||ab> t^b_j. This module evaluates that definition: E and S are the
oracle's Appendix-A energy and residual, and the derivative is exact reverse-mode
differentiation of those same expressions (torch autograd on the CPU, complex128). L
is a polynomial, holomorphic in t, so dL/dt is the conjugate of the gradient of Re L.
``tests/test_oracle_lambda.py`` pins it to <0|(1 + Lambda)[H_bar, tau_nu]|0> in the
determinant space. For two electrons it pins the converged lambda to the full-CI left
eigenvector.

Layout: l1[i,a] = lambda^i_a, l2[i,j,a,b] = lambda^{ij}_{ab}, antisymmetric in (i,j)
and in (a,b), like t1 and t2. R1 and R2 come in the same layout. R2 is the derivative
with respect to each unique t^{ab}_{ij}, extended antisymmetrically.

Density (appendix "Working equations for Lagrange 1-body density matrix"). The printed
blocks gamma_ij, gamma_ia, gamma_ai and gamma_ab, one einsum per printed term.

Reading r20. The printed gamma_ia = lambda^i_a, gamma_ai = t^a_i + ... and gamma_ab are
the blocks of gamma_pq = <0| (1 + Lambda) exp(-T) a+_q a_p exp(T) |0>. The printed
gamma_ij is that definition with its two labels exchanged, less the reference occupation
delta_ij. The oracle transposes the printed occupied block into the convention of the
other three, so that all four blocks are one matrix: the definition less delta_ij. For
real spinors the appendix's symmetrisation makes the two conventions agree; for complex
ones they differ. ``symmetrize`` returns the Hermitian part, the appendix's
symmetrised density.
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd_ref as R


def _torch(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128))


def lagrangian_gradient(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, l1: np.ndarray,
                        l2: np.ndarray, method: str = "ccsd"):
    """(R1[i,a], R2[i,j,a,b]) = dL/dt at (t, lambda): the Lambda-equation residuals."""
    import torch
    o = t1.shape[0]
    T1 = _torch(t1).requires_grad_(True)
    T2 = _torch(t2).requires_grad_(True)
    F = _torch(f)
    Vt = {k: _torch(x) for k, x in V.items()}
    res = R.residual_cc2 if method == "cc2" else R.residual
    S1, S2 = res(F, Vt, T1, T2)
    # E = sum_ia f_ia t^a_i + 1/4 sum_ijab <ij||ab> tau^{ab}_{ij}
    E = (F[:o, o:] * T1).sum() + 0.25 * (Vt["oovv"] * R.tau(T1, T2)).sum()
    # sum over unique mu: all (i, a), and (i<j, a<b) = 1/4 of the full antisymmetric sum
    L = E + (_torch(l1) * S1).sum() + 0.25 * (_torch(l2) * S2).sum()
    g1, g2 = torch.autograd.grad(L.real, (T1, T2))
    d1 = g1.conj().resolve_conj().numpy()
    G = g2.conj().resolve_conj().numpy()
    # t^{ab}_{ij} (i<j, a<b) sits at [i,j,a,b], -[j,i,a,b], -[i,j,b,a], [j,i,b,a]
    d2 = G - G.transpose(1, 0, 2, 3) - G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2)
    return d1, d2


def solve_lambda(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, max_iter: int = 100,
                 tol: float = 1e-10, diis_dim: int = 8, method: str = "ccsd"):
    """Iterate lambda from zero with the amplitudes' update rule: lambda <- lambda + R / D,
    D^a_i = f_ii - f_aa, D^{ab}_{ij} = f_ii + f_jj - f_aa - f_bb (R is linear in lambda with
    diagonal ~ -D), DIIS as for the amplitudes. Returns dict(l1, l2, iterations, norm, converged)."""
    o, v = t1.shape
    D1, D2 = R.denominators(f, o, 0.0)
    l1 = np.zeros((o, v), np.complex128)
    l2 = np.zeros((o, o, v, v), np.complex128)
    diis = R.DIIS(diis_dim) if diis_dim > 0 else None
    norm, it, converged = np.inf, 0, False
    for it in range(1, max_iter + 1):
        r1, r2 = lagrangian_gradient(f, V, t1, t2, l1, l2, method)
        d1, d2 = r1 / D1, r2 / D2
        norm = max(np.max(np.abs(d1), initial=0.0), np.max(np.abs(d2), initial=0.0))
        l1, l2 = l1 + d1, l2 + d2
        if diis is not None:
            diis.push(l1, l2, d1, d2)
            if it >= 2 and len(diis.t) >= 2:
                l1, l2 = diis.extrapolate()
        if norm <= tol:
            converged = True
            break
    return dict(l1=l1, l2=l2, iterations=it, norm=float(norm), converged=converged)


def density(t1: np.ndarray, t2: np.ndarray, l1: np.ndarray, l2: np.ndarray, symmetrize: bool = False):
    """The one-body density of the appendix's Lagrange density equations (reading r20), as an
    (o+v) x (o+v) matrix, occupied first: <0|(1 + Lambda) exp(-T) a+_q a_p exp(T)|0> less the
    reference occupation."""
    o, v = t1.shape
    es = lambda s, *ops: np.einsum(s, *ops, optimize=True)
    g = np.zeros((o + v, o + v), np.complex128)
    # gamma_ij = 1/2 sum_mef t^{ef}_{im} lambda^{mj}_{ef} - sum_e t^e_i lambda^j_e, transposed (r20)
    g[:o, :o] = (0.5 * es("imef,mjef->ij", t2, l2) - es("ie,je->ij", t1, l1)).T
    # gamma_ia = lambda^i_a
    g[:o, o:] = l1
    # gamma_ai = t^a_i + sum_me lambda^m_e (t^{ae}_{im} - t^e_i t^a_m)
    #            - 1/2 sum_mnef lambda^{mn}_{ef} (t^{ef}_{in} t^a_m + t^e_i t^{af}_{mn})
    g[o:, :o] = (t1.T + es("me,imae->ai", l1, t2) - es("me,ie,ma->ai", l1, t1, t1)
                 - 0.5 * es("mnef,inef,ma->ai", l2, t2, t1) - 0.5 * es("mnef,ie,mnaf->ai", l2, t1, t2))
    # gamma_ab = 1/2 sum_mne t^{ae}_{mn} lambda^{mn}_{be} + sum_m t^a_m lambda^m_b
    g[o:, o:] = 0.5 * es("mnae,mnbe->ab", t2, l2) + es("ma,mb->ab", t1, l1)
    if symmetrize:
        g = 0.5 * (g + g.conj().T)
    return g
