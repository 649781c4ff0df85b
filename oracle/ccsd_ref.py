"""Plain CPU oracle for the complex Kramers-unrestricted CCSD iteration.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The product (the CUDA library and its Python binding) never does.

Everything is complex128 / float64: the paper carries the whole coupled-cluster
calculation in complex double precision (Sec. "ExaTENSOR and TAL-SH", complex
double tensors). Each step is one ``numpy.einsum`` per printed term, in the order
and notation of Appendix A ("Working equations for CCSD amplitude equations"),
with no blocking, fusion or packing. A reader can check every line against the
appendix by eye.

Notation and readings of the paper used here:

* Integrals. ``V[p,q,r,s]`` holds V^{pq}_{rs} = <pq||rs> = <pq|rs> - <pq|sr>,
  with <pq|rs> = (pr|qs) (Eq. two_electron and the antisymmetrisation step of
  the AO-to-MO section). In Appendix A the upper pair is the bra pair; this is
  the only reading under which the last S2 term is the particle-particle ladder.
* Density fitting. (pr|qs) = sum_Q B^Q_pr B^Q_qs with B^Q Hermitian in (p, r).
* Dagger. V^{ij+}_{ab}, V^{cj+}_{ab}, F^{i+}_a denote the element-wise complex
  conjugate of the stored tensor with those labels (the "+" conjugation of the
  ExaTENSOR contraction strings), so V^{ij+}_{ab} = conj(<ij||ab>) = <ab||ij>.
* Amplitudes. t1[i,a] = t^a_i, t2[i,j,a,b] = t^{ab}_{ij}, antisymmetric in (i,j)
  and in (a,b); T2 = 1/4 sum t^{ab}_{ij} a+_a a+_b a_j a_i.
* Fock. F^p_q = f[p,q]; the residual S contains the full Fock matrix (through
  H^a_c and H^k_i), so the amplitude update is t <- t + S/D.
* Energy (not printed in the paper): E = sum_ia f_ia t^a_i
  + 1/4 sum_ijab <ij||ab> tau^{ab}_{ij}, the full conjugated contraction
  E() += V+ * T of the ExaTENSOR example.
* Spinor order: occupied first. Blocks are sliced as o = [0, o), v = [o, n).

Every function here is pinned by the CPU tests against brute force in the
determinant space (``oracle.brute_force``), full CI for two electrons, the MP2
closed form, unitary invariance and the real spin-restricted limit.
"""
from __future__ import annotations

import numpy as np

BLOCKS = ("oooo", "ooov", "oovv", "vovo", "vovv", "vvvv")


# ---------------------------------------------------------------------------
# Integrals (Eq. two_electron; AO-to-MO section: <pr||qs> = (pq|rs) - (ps|rq))
# ---------------------------------------------------------------------------

def _space(o: int, n: int, c: str) -> slice:
    return slice(0, o) if c == "o" else slice(o, n)


def coulomb_block(B: np.ndarray, P: slice, Q: slice, R: slice, S: slice) -> np.ndarray:
    """<pq|rs> = (pr|qs) = sum_Q B^Q_pr B^Q_qs over the given index ranges."""
    return np.einsum("Xpr,Xqs->pqrs", B[:, P, R], B[:, Q, S], optimize=True)


def antisym_block(B: np.ndarray, o: int, spaces: str) -> np.ndarray:
    """<pq||rs> = <pq|rs> - <pq|sr> for p,q,r,s in the spaces named by ``spaces``."""
    n = B.shape[1]
    P, Q, R, S = (_space(o, n, c) for c in spaces)
    return coulomb_block(B, P, Q, R, S) - coulomb_block(B, P, Q, S, R).transpose(0, 1, 3, 2)


def integrals(B: np.ndarray, o: int, blocks=BLOCKS) -> dict:
    """The six integral classes the residual needs (bra pair first)."""
    return {name: antisym_block(B, o, name) for name in blocks}


def full_integrals(B: np.ndarray) -> np.ndarray:
    """All of <pq||rs> over n^4 (small n only)."""
    return (np.einsum("Xpr,Xqs->pqrs", B, B, optimize=True)
            - np.einsum("Xps,Xqr->pqrs", B, B, optimize=True))


def blocks_from_full(V: np.ndarray, o: int) -> dict:
    n = V.shape[0]
    out = {}
    for name in BLOCKS:
        P, Q, R, S = (_space(o, n, c) for c in name)
        out[name] = np.ascontiguousarray(V[P, Q, R, S])
    return out


def fock_matrix(eps: np.ndarray, fock: np.ndarray | None = None) -> np.ndarray:
    """The Fock matrix: the supplied Hermitian matrix, else diag(eps)."""
    if fock is not None:
        return np.asarray(fock, dtype=np.complex128)
    return np.diag(np.asarray(eps, dtype=np.float64)).astype(np.complex128)


# ---------------------------------------------------------------------------
# Appendix A: CCSD amplitude equations
# ---------------------------------------------------------------------------

def _es(spec: str, *ops):
    """einsum over numpy arrays, or over torch tensors (the Lambda oracle differentiates these
    same equations with torch's autograd); the arithmetic is the same either way."""
    if type(ops[0]).__module__.split(".")[0] == "torch":
        import torch
        return torch.einsum(spec, *ops)
    return np.einsum(spec, *ops, optimize=True)


def _perm(x, axes):
    """Axes permutation of a numpy array or a torch tensor."""
    return x.permute(*axes) if type(x).__module__.split(".")[0] == "torch" else x.transpose(*axes)


def p_minus(x: np.ndarray, ax1: int, ax2: int) -> np.ndarray:
    """P^-_{pq} f(p,q) = f(p,q) - f(q,p), acting on axes ax1, ax2."""
    return x - x.swapaxes(ax1, ax2)


def tau(t1: np.ndarray, t2: np.ndarray) -> np.ndarray:
    """tau^{ab}_{ij} = t^{ab}_{ij} + P^-_ij (t^a_i t^b_j)."""
    return t2 + p_minus(_es("ia,jb->ijab", t1, t1), 0, 1)


def intermediates(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray) -> dict:
    """H^a_c, G^a_c, H^k_i, G^k_i, H^k_c, H^{ak}_{ci}, C^{kb}_{ij}, A^{kl}_{ij} (Appendix A)."""
    o = t1.shape[0]
    foo, fvv, fov = f[:o, :o], f[o:, o:], f[:o, o:]
    oooo, ooov, oovv = V["oooo"], V["ooov"], V["oovv"]
    vovo, vovv = V["vovo"], V["vovv"]
    ta = tau(t1, t2)
    es = _es

    # H^a_c = F^a_c + 1/2 sum_kld V^{kl}_{cd} tau^{da}_{kl}
    Hvv = fvv + 0.5 * es("klcd,klda->ac", oovv, ta)
    # G^a_c = H^a_c + sum_kd V^{ak}_{cd} t^d_k - sum_k F^k_c t^a_k
    Gvv = Hvv + es("akcd,kd->ac", vovv, t1) - es("kc,ka->ac", fov, t1)
    # H^k_i = -F^k_i + 1/2 sum_lcd V^{kl}_{cd} tau^{cd}_{li}
    Hoo = -foo + 0.5 * es("klcd,licd->ki", oovv, ta)
    # G^k_i = H^k_i - sum_lc V^{kl}_{ic} t^c_l - sum_c F^k_c t^c_i
    Goo = Hoo - es("klic,lc->ki", ooov, t1) - es("kc,ic->ki", fov, t1)
    # H^k_c = F^k_c + sum_ld V^{kl}_{cd} t^d_l
    Hov = fov + es("klcd,ld->kc", oovv, t1)
    # H^{ak}_{ci} = V^{ak}_{ci} + sum_d V^{ak}_{cd} t^d_i - sum_l V^{kl}_{ic} t^a_l
    #             + sum_ld V^{kl}_{cd} (1/2 t^{ad}_{li} + t^a_l t^d_i)
    Hvoov = (vovo
             + es("akcd,id->akci", vovv, t1)
             - es("klic,la->akci", ooov, t1)
             + es("klcd,liad->akci", oovv, 0.5 * t2 + es("la,id->liad", t1, t1)))
    # C^{kb}_{ij} = V^{ij+}_{kb} + sum_c P^-_ij (V^{bk}_{ci} t^c_j) - 1/2 sum_cd V^{bk}_{cd} tau^{cd}_{ij}
    C = (_perm(ooov.conj(), (2, 3, 0, 1))
         + p_minus(es("bkci,jc->kbij", vovo, t1), 2, 3)
         - 0.5 * es("bkcd,ijcd->kbij", vovv, ta))
    # A^{kl}_{ij} = V^{kl}_{ij} + sum_c P^-_ij (V^{kl}_{ic} t^c_j) + 1/2 sum_cd V^{kl}_{cd} tau^{cd}_{ij}
    A = (oooo
         + p_minus(es("klic,jc->klij", ooov, t1), 2, 3)
         + 0.5 * es("klcd,ijcd->klij", oovv, ta))
    return dict(tau=ta, Hvv=Hvv, Gvv=Gvv, Hoo=Hoo, Goo=Goo, Hov=Hov, Hvoov=Hvoov, C=C, A=A)


def ladder(vvvv: np.ndarray, ta: np.ndarray) -> np.ndarray:
    """Particle-particle ladder 1/2 sum_cd V^{ab}_{cd} tau^{cd}_{ij}, as [i,j,a,b]."""
    return 0.5 * _es("abcd,ijcd->ijab", vvvv, ta)


def ladder_elements(B: np.ndarray, o: int, t1: np.ndarray, t2: np.ndarray, idx) -> np.ndarray:
    """Selected elements of the ladder 1/2 sum_cd V^{ab}_{cd} tau^{cd}_{ij}, from B^Q directly.

    For each (i, j, a, b) in ``idx`` the row <ab||cd> = (ac|bd) - (ad|bc) over all c, d is
    formed from the DF factors, so no n^4 tensor is ever built (full-size sampling).
    """
    out = np.empty(len(idx), np.complex128)
    Bv = B[:, o:, o:]
    for n, (i, j, a, b) in enumerate(idx):
        coul = Bv[:, a, :].T @ Bv[:, b, :]          # (ac|bd) over (c, d)
        w = coul - coul.T                           # <ab||cd> = (ac|bd) - (ad|bc)
        ta = t2[i, j] + np.outer(t1[i], t1[j]) - np.outer(t1[j], t1[i])   # tau^{cd}_{ij}
        out[n] = 0.5 * np.sum(w * ta)
    return out


def ladder_rows(B: np.ndarray, o: int, tau: np.ndarray, pairs) -> np.ndarray:
    """The ladder 1/2 sum_cd V^{ab}_{cd} tau^{cd}_{ij} at every (i, j) for chosen (a, b).

    For each (a, b) in ``pairs`` the row <ab||cd> = (ac|bd) - (ad|bc) over all (c, d) is formed
    from the DF factors and contracted with the full tau (no n^4 tensor is built). Returns an
    array [len(pairs), o, o].
    """
    Bv = B[:, o:, o:]
    out = np.empty((len(pairs), o, o), np.complex128)
    for n, (a, b) in enumerate(pairs):
        coul = Bv[:, a, :].T @ Bv[:, b, :]          # (ac|bd) over (c, d)
        w = coul - coul.T                           # <ab||cd>
        out[n] = 0.5 * np.einsum("cd,ijcd->ij", w, tau)
    return out


def _singles_terms(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, I: dict) -> dict:
    """The printed terms of S^a_i (Appendix A), given the intermediates I."""
    o = t1.shape[0]
    fov = f[:o, o:]
    ooov, vovo, vovv = V["ooov"], V["vovo"], V["vovv"]
    ta = I["tau"]
    es = _es
    Hvv, Hoo, Hov = I["Hvv"], I["Hoo"], I["Hov"]
    t1terms = {}
    t1terms["f"] = fov.conj()                                         # F^{i+}_a
    t1terms["hvv"] = es("ac,ic->ia", Hvv, t1)                         # sum_c H^a_c t^c_i
    t1terms["hoo"] = es("ki,ka->ia", Hoo, t1)                         # sum_k H^k_i t^a_k
    t1terms["hov"] = es("kc,ikac->ia", Hov, t2)                       # sum_kc H^k_c t^{ac}_{ik}
    t1terms["hf"] = es("kc,ic,ka->ia", Hov - 2.0 * fov, t1, t1)       # sum_k (sum_c (H^k_c - 2F^k_c) t^c_i) t^a_k
    t1terms["vovv"] = 0.5 * es("akcd,ikcd->ia", vovv, ta)             # 1/2 sum_kcd V^{ak}_{cd} tau^{cd}_{ik}
    t1terms["ooov"] = 0.5 * es("klic,klca->ia", ooov, ta)             # 1/2 sum_klc V^{kl}_{ic} tau^{ca}_{kl}
    t1terms["vovo"] = -es("akci,kc->ia", vovo, t1)                    # - sum_kc V^{ak}_{ci} t^c_k
    return t1terms


def residual(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, parts: dict | None = None):
    """S^a_i and S^{ab}_{ij} of Appendix A at amplitudes (t1, t2).

    Returns (S1[i,a], S2[i,j,a,b]). If ``parts`` is a dict, the individual S2
    terms and the intermediates are stored in it (for term-wise parity tests).
    """
    o = t1.shape[0]
    fov = f[:o, o:]
    ooov, oovv, vovo, vovv = V["ooov"], V["oovv"], V["vovo"], V["vovv"]
    I = intermediates(f, V, t1, t2)
    ta = I["tau"]
    es = _es

    terms = {}
    # sum_kc P^-_ij P^-_ab (H^{ak}_{ci} t^{cb}_{jk})
    terms["ring"] = p_minus(p_minus(es("akci,jkcb->ijab", I["Hvoov"], t2), 0, 1), 2, 3)
    # sum_k P^-_ji G^k_j t^{ab}_{ik}
    terms["goo"] = p_minus(es("kj,ikab->ijab", I["Goo"], t2), 0, 1)
    # sum_c P^-_ij (V^{cj+}_{ab} t^c_i)
    terms["vt1"] = p_minus(es("cjab,ic->ijab", vovv.conj(), t1), 0, 1)
    # sum_c P^-_ab G^a_c t^{cb}_{ij}
    terms["gvv"] = p_minus(es("ac,ijcb->ijab", I["Gvv"], t2), 2, 3)
    # sum_k P^-_ab (C^{ka}_{ij} t^b_k)
    terms["ct1"] = p_minus(es("kaij,kb->ijab", I["C"], t1), 2, 3)
    # 1/2 sum_kl A^{kl}_{ij} tau^{ab}_{kl}
    terms["hole"] = 0.5 * es("klij,klab->ijab", I["A"], ta)
    # 1/2 sum_cd V^{ab}_{cd} tau^{cd}_{ij}
    terms["ladder"] = ladder(V["vvvv"], ta)
    # V^{ij+}_{ab}
    terms["driver"] = oovv.conj()
    S2 = sum(terms.values())

    t1terms = _singles_terms(f, V, t1, t2, I)
    S1 = sum(t1terms.values())
    if parts is not None:
        parts.update(I)
        parts.update({"S2_" + k: v for k, v in terms.items()})
        parts.update({"S1_" + k: v for k, v in t1terms.items()})
    return S1, S2


def residual_cc2(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, parts: dict | None = None):
    """CC2 residuals (appendix "Working equations for CC2 amplitude equations").

    S^a_i is the singles residual of Appendix A, unchanged. S^{ab}_{ij} is the CC2 doubles
    equation: the driver V^{ab}_{ij}, four terms in t1 with the CC2 intermediates W^{ab}_{ej},
    W^{mb}_{ij}, W^{mn}_{ij}, W^{ab}_{ef}, and the Fock terms in t2. The sums over m<n and
    e<f are taken as half the full sums; their summands are symmetric under m <-> n and e <-> f.
    The notation and readings are those of ``residual``: V^{pq}_{rs} = <pq||rs>, f^p_q = f[p,q].
    Returns (S1[i,a], S2[i,j,a,b]).
    """
    o = t1.shape[0]
    oooo, ooov, oovv, vovo, vovv = V["oooo"], V["ooov"], V["oovv"], V["vovo"], V["vovv"]
    fo, fv = f[:o, :o], f[o:, o:]
    es = lambda s, *ops: np.einsum(s, *ops, optimize=True)
    # the blocks with the labels of the CC2 equations
    v_abij = np.conj(oovv)                              # V^{ab}_{ij} = conj <ij||ab>, as [i,j,a,b]
    v_abej = np.conj(vovv).transpose(2, 3, 0, 1)        # V^{ab}_{ej} = conj <ej||ab>, as [a,b,e,j]
    v_mbij = np.conj(ooov).transpose(2, 3, 0, 1)        # V^{mb}_{ij} = conj <ij||mb>, as [m,b,i,j]
    v_mbej = -vovo.transpose(1, 0, 2, 3)                # V^{mb}_{ej} = -<bm||ej>, as [m,b,e,j]

    # W^{mn}_{ij} = V^{mn}_{ij} + sum_e P^-_ij t^e_j V^{mn}_{ie} + 1/4 sum_ef P^-_ij t^e_i t^f_j V^{mn}_{ef}
    w_mnij = (oooo + p_minus(es("je,mnie->mnij", t1, ooov), 2, 3)
              + 0.25 * p_minus(es("ie,jf,mnef->mnij", t1, t1, oovv), 2, 3))
    # W^{ab}_{ef} = V^{ab}_{ef} - sum_m P^-_ab t^b_m V^{am}_{ef} + 1/4 sum_mn P^-_ab t^a_m t^b_n V^{mn}_{ef}
    w_abef = (V["vvvv"] - p_minus(es("mb,amef->abef", t1, vovv), 0, 1)
              + 0.25 * p_minus(es("ma,nb,mnef->abef", t1, t1, oovv), 0, 1))
    # W^{ab}_{ej} = V^{ab}_{ej} - 1/2 sum_m P^-_ab t^a_m V^{mb}_{ej}
    w_abej = v_abej - 0.5 * p_minus(es("ma,mbej->abej", t1, v_mbej), 0, 1)
    # W^{mb}_{ij} = V^{mb}_{ij} + 1/2 sum_e P^-_ij t^e_i V^{mb}_{ej}
    w_mbij = v_mbij + 0.5 * p_minus(es("ie,mbej->mbij", t1, v_mbej), 2, 3)

    terms = {}
    terms["driver"] = v_abij                                                      # V^{ab}_{ij}
    terms["t1_abej"] = p_minus(es("ie,abej->ijab", t1, w_abej), 0, 1)             # sum_e P^-_ij t^e_i W^{ab}_{ej}
    terms["t1_mbij"] = -p_minus(es("ma,mbij->ijab", t1, w_mbij), 2, 3)            # - sum_m P^-_ab t^a_m W^{mb}_{ij}
    terms["t1t1_mnij"] = 0.5 * p_minus(es("ma,nb,mnij->ijab", t1, t1, w_mnij), 2, 3)  # sum_{m<n} P^-_ab t^a_m t^b_n W^{mn}_{ij}
    terms["t1t1_abef"] = 0.5 * p_minus(es("ie,jf,abef->ijab", t1, t1, w_abef), 0, 1)  # sum_{e<f} P^-_ij t^e_i t^f_j W^{ab}_{ef}
    terms["f_vv"] = p_minus(es("be,ijae->ijab", fv, t2), 2, 3)                    # sum_e P^-_ab f^b_e t^{ae}_{ij}
    terms["f_oo"] = -p_minus(es("mj,imab->ijab", fo, t2), 0, 1)                   # - sum_m P^-_ij f^m_j t^{ab}_{im}
    S2 = sum(terms.values())
    I = intermediates(f, V, t1, t2)
    t1terms = _singles_terms(f, V, t1, t2, I)
    S1 = sum(t1terms.values())
    if parts is not None:
        parts.update({"S2_" + k: v for k, v in terms.items()})
        parts.update({"S1_" + k: v for k, v in t1terms.items()})
    return S1, S2


def energy(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray) -> complex:
    """E = sum_ia f_ia t^a_i + 1/4 sum_ijab <ij||ab> tau^{ab}_{ij} (complex value)."""
    o = t1.shape[0]
    return complex(np.einsum("ia,ia->", f[:o, o:], t1)
                   + 0.25 * np.einsum("ijab,ijab->", V["oovv"], tau(t1, t2)))


# ---------------------------------------------------------------------------
# Denominators, update, DIIS (Sec. "Coupled cluster implementation")
# ---------------------------------------------------------------------------

def denominators(f: np.ndarray, o: int, shift: float = 0.0):
    """D^a_i = f_ii - (f_aa + shift), D^{ab}_{ij} = f_ii + f_jj - (f_aa + shift) - (f_bb + shift)."""
    d = np.real(np.diag(f)).astype(np.float64)
    eo, ev = d[:o], d[o:] + shift
    D1 = eo[:, None] - ev[None, :]
    D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return D1, D2


def mp2_guess(f: np.ndarray, V: dict, o: int, v: int, shift: float = 0.0):
    """One denominator update from t = 0: t1 = F^{i+}_a / D^a_i, t2 = <ab||ij> / D^{ab}_{ij}."""
    D1, D2 = denominators(f, o, shift)
    t1 = np.zeros((o, v), np.complex128)
    t2 = np.zeros((o, o, v, v), np.complex128)
    S1, S2 = residual(f, V, t1, t2)
    return S1 / D1, S2 / D2


def mp2_energy(f: np.ndarray, V: dict, o: int, v: int) -> complex:
    t1, t2 = mp2_guess(f, V, o, v)
    return energy(f, V, t1, t2)


def _unique_t2(x: np.ndarray) -> np.ndarray:
    o, v = x.shape[0], x.shape[2]
    iu, ju = np.triu_indices(o, 1)
    au, bu = np.triu_indices(v, 1)
    return x[iu, ju][:, au, bu]


class DIIS:
    """Pulay DIIS on the stacked unique amplitudes (t1, t2 with i<j, a<b).

    Error vector = the denominator update S/D of the iteration; B_ij = Re<e_i, e_j>;
    real coefficients from [[B, 1], [1^T, 0]] [c; lam] = [0; 1] solved by LU with
    partial pivoting; at most ``max_vec`` vectors, the oldest dropped first.
    """

    def __init__(self, max_vec: int = 8):
        self.max_vec = max_vec
        self.t: list = []
        self.e: list = []

    def push(self, t1, t2, e1, e2):
        self.t.append((t1.copy(), t2.copy()))
        self.e.append(np.concatenate([e1.ravel(), _unique_t2(e2).ravel()]))
        if len(self.t) > self.max_vec:
            self.t.pop(0)
            self.e.pop(0)

    def coefficients(self) -> np.ndarray:
        m = len(self.e)
        Bm = np.zeros((m + 1, m + 1))
        for a in range(m):
            for b in range(m):
                Bm[a, b] = np.real(np.vdot(self.e[a], self.e[b]))
        Bm[m, :m] = 1.0
        Bm[:m, m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        return np.linalg.solve(Bm, rhs)[:m]

    def extrapolate(self):
        c = self.coefficients()
        t1 = sum(ci * ti[0] for ci, ti in zip(c, self.t))
        t2 = sum(ci * ti[1] for ci, ti in zip(c, self.t))
        return t1, t2


class CROP:
    """CROP, the conjugate residual method with optimal trial vectors (Ziolkowski, Weijo,
    Jorgensen and Olsen 2008), the lighter-memory alternative to DIIS the paper names in
    Sec. "Coupled cluster implementation".

    The subspace holds the OPTIMAL vectors of the last iterations, x~_i and their residuals
    r~_i (here the preconditioned residual, the update S/D), over the unique amplitudes.
    Iteration n, with the new trial vector x^(n) and its residual r^(n):
      1. the subspace is [x~_{n-m+1}, ..., x~_{n-1}, x^(n)] with residuals likewise (m =
         ``max_vec`` vectors, the new trial vector included);
      2. real c minimises |sum_i c_i r_i|^2 subject to sum_i c_i = 1, from
         [[B, 1], [1^T, 0]] [c; lam] = [0; 1] with B_ij = Re<r_i, r_j> (as DIIS);
      3. x~^(n) = sum_i c_i x_i and r~^(n) = sum_i c_i r_i replace (x^(n), r^(n));
      4. the next trial vector is the preconditioned step from the optimum,
         x^(n+1) = x~^(n) + r~^(n).
    At most ``max_vec`` optimal vectors are kept, the oldest dropped first; the usual choice
    is 3. Before extrapolation starts (iteration < start, or a single vector) c = (1) and
    the step is the plain update.
    """

    def __init__(self, max_vec: int = 3):
        self.max_vec = max_vec
        self.x: list = []  # optimal (t1, t2)
        self.r: list = []  # their residuals (e1, e2)

    @staticmethod
    def _flat(e1, e2):
        return np.concatenate([e1.ravel(), _unique_t2(e2).ravel()])

    def coefficients(self) -> np.ndarray:
        m = len(self.r)
        flat = [self._flat(*r) for r in self.r]
        Bm = np.zeros((m + 1, m + 1))
        for a in range(m):
            for b in range(m):
                Bm[a, b] = np.real(np.vdot(flat[a], flat[b]))
        Bm[m, :m] = 1.0
        Bm[:m, m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        return np.linalg.solve(Bm, rhs)[:m]

    def step(self, t1, t2, e1, e2, extrapolate: bool = True):
        """Add the trial (t, e = S/D at t); return the next trial vector (step 4)."""
        self.x.append((t1.copy(), t2.copy()))
        self.r.append((e1.copy(), e2.copy()))
        if len(self.x) > self.max_vec:  # the subspace of step 1 holds max_vec vectors, the new one included
            self.x.pop(0)
            self.r.pop(0)
        if extrapolate and len(self.x) >= 2:
            c = self.coefficients()
            xo = (sum(ci * xi[0] for ci, xi in zip(c, self.x)), sum(ci * xi[1] for ci, xi in zip(c, self.x)))
            ro = (sum(ci * ri[0] for ci, ri in zip(c, self.r)), sum(ci * ri[1] for ci, ri in zip(c, self.r)))
            self.x[-1], self.r[-1] = xo, ro
        xo, ro = self.x[-1], self.r[-1]
        return xo[0] + ro[0], xo[1] + ro[1]


def solve(f: np.ndarray, V: dict, o: int, v: int, max_iter: int = 50, tol: float = 1e-10,
          diis_dim: int = 8, diis_start: int = 2, shift: float = 0.0, t_init=None,
          callback=None, method: str = "ccsd", accelerator: str = "diis"):
    """CCSD iterations from the MP2 guess (or ``t_init``); method="ccd" holds t1 at zero (CCD:
    the doubles equations of Appendix A with T1 = 0, the variant the paper also times);
    method="cc2" iterates the CC2 residuals (``residual_cc2``).

    Each iteration: S = residual(t); d = S/D; norm = max|d|; then
      * DIIS (accelerator="diis"): t <- t + d; if the iteration number is >= diis_start with
        >= 2 stored vectors, t <- sum_i c_i t_i;
      * CROP (accelerator="crop", ``diis_dim`` optimal vectors): t <- x~ + r~ (class CROP),
        extrapolating from iteration diis_start on;
      * neither (diis_dim = 0): t <- t + d.
    Stops when norm <= tol. Returns dict(t1, t2, energy, iterations, norm, converged).
    """
    D1, D2 = denominators(f, o, shift)
    if t_init is None:
        t1, t2 = mp2_guess(f, V, o, v, shift)
    else:
        t1, t2 = (np.array(x, dtype=np.complex128) for x in t_init)
    if method == "ccd":
        t1 = np.zeros_like(t1)
    elif method not in ("ccsd", "cc2"):
        raise ValueError("method must be 'ccsd', 'ccd' or 'cc2'")
    res = residual_cc2 if method == "cc2" else residual
    if accelerator not in ("diis", "crop"):
        raise ValueError("accelerator must be 'diis' or 'crop'")
    diis = DIIS(diis_dim) if diis_dim > 0 and accelerator == "diis" else None
    crop = CROP(diis_dim) if diis_dim > 0 and accelerator == "crop" else None
    norm = np.inf
    it = 0
    converged = False
    for it in range(1, max_iter + 1):
        S1, S2 = res(f, V, t1, t2)
        d1, d2 = S1 / D1, S2 / D2
        if method == "ccd":
            d1 = np.zeros_like(d1)
        norm = max(np.max(np.abs(d1), initial=0.0), np.max(np.abs(d2), initial=0.0))
        if crop is not None:
            t1, t2 = crop.step(t1, t2, d1, d2, extrapolate=it >= diis_start)
        else:
            t1, t2 = t1 + d1, t2 + d2
        if diis is not None:
            diis.push(t1, t2, d1, d2)
            if it >= diis_start and len(diis.t) >= 2:
                t1, t2 = diis.extrapolate()
        if callback is not None:
            callback(it, t1, t2, norm)
        if not np.isfinite(norm):
            break
        if norm <= tol:
            converged = True
            break
    return dict(t1=t1, t2=t2, energy=energy(f, V, t1, t2), iterations=it, norm=float(norm),
                converged=converged)
