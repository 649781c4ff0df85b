"""Development aid of the Lambda tests (not part of the oracle): the derivative of the CCSD
Lagrangian written out as the explicit adjoint of the Appendix-A residual, term by term in
reverse order, the contraction list a device Lambda residual runs. ``test_oracle_lambda.py``
checks it against the oracle's definition (``oracle.lambda_ref.lagrangian_gradient``, exact
reverse-mode differentiation of the oracle's energy and residual); the GPU parity tests compare
the device with that definition, never with this list.
"""
from __future__ import annotations

import numpy as np

from oracle import ccsd_ref as R


def lagrangian_gradient_explicit(f: np.ndarray, V: dict, t1: np.ndarray, t2: np.ndarray, l1: np.ndarray,
                                 l2: np.ndarray):
    """The same dL/dt as ``oracle.lambda_ref.lagrangian_gradient`` (CCSD), written out as the
    adjoint of the Appendix-A residual, term by term in reverse order: every forward contraction
    gives one transposed contraction per amplitude-dependent factor."""
    o, v = t1.shape
    foo, fvv, fov = f[:o, :o], f[o:, o:], f[:o, o:]
    oooo, ooov, oovv, vovo, vovv, vvvv = (V[k] for k in ("oooo", "ooov", "oovv", "vovo", "vovv", "vvvv"))
    es = lambda s, *ops: np.einsum(s, *ops, optimize=True)
    pm = R.p_minus
    I = R.intermediates(f, V, t1, t2)
    ta, Hvv, Gvv, Hoo, Goo, Hov, Hvoov, C, A = (I[k] for k in ("tau", "Hvv", "Gvv", "Hoo", "Goo", "Hov",
                                                               "Hvoov", "C", "A"))
    t1b = np.zeros_like(t1)
    t2b = np.zeros_like(t2)
    taub = np.zeros_like(t2)
    # energy: E = sum f_ia t^a_i + 1/4 sum <ij||ab> tau^{ab}_{ij}
    t1b += fov
    taub += 0.25 * oovv
    # S2 terms, weighted by 1/4 l2 (unique doubles); an antisymmetriser's adjoint on l2 gives 2 per P^-
    Hvoovb = es("ijab,jkcb->akci", l2, t2)                          # ring
    t2b += es("ijab,akci->jkcb", l2, Hvoov)
    Goob = 0.5 * es("ijab,ikab->kj", l2, t2)                        # goo
    t2b += 0.5 * es("ijab,kj->ikab", l2, Goo)
    t1b += 0.5 * es("ijab,cjab->ic", l2, vovv.conj())               # vt1
    Gvvb = 0.5 * es("ijab,ijcb->ac", l2, t2)                        # gvv
    t2b += 0.5 * es("ijab,ac->ijcb", l2, Gvv)
    Cb = 0.5 * es("ijab,kb->kaij", l2, t1)                          # ct1
    t1b += 0.5 * es("ijab,kaij->kb", l2, C)
    Ab = 0.125 * es("ijab,klab->klij", l2, ta)                      # hole
    taub += 0.125 * es("ijab,klij->klab", l2, A)
    taub += 0.125 * es("ijab,abcd->ijcd", l2, vvvv)                 # ladder: lambda . <ab||cd>
    # S1 terms, weighted by l1
    Hvvb = es("ia,ic->ac", l1, t1)                                  # hvv
    t1b += es("ia,ac->ic", l1, Hvv)
    Hoob = es("ia,ka->ki", l1, t1)                                  # hoo
    t1b += es("ia,ki->ka", l1, Hoo)
    Hovb = es("ia,ikac->kc", l1, t2)                                # hov
    t2b += es("ia,kc->ikac", l1, Hov)
    Y = Hov - 2.0 * fov                                             # hf
    Hovb += es("ia,ic,ka->kc", l1, t1, t1)
    t1b += es("ia,kc,ka->ic", l1, Y, t1) + es("ia,kc,ic->ka", l1, Y, t1)
    taub += 0.5 * es("ia,akcd->ikcd", l1, vovv)                     # vovv
    taub += 0.5 * es("ia,klic->klca", l1, ooov)                     # ooov
    t1b -= es("ia,akci->kc", l1, vovo)                              # vovo
    # intermediates, in reverse order of their definitions
    taub += 0.5 * es("klij,klcd->ijcd", Ab, oovv)                   # A
    t1b += es("klij,klic->jc", pm(Ab, 2, 3), ooov)
    taub -= 0.5 * es("kbij,bkcd->ijcd", Cb, vovv)                   # C
    t1b += es("kbij,bkci->jc", pm(Cb, 2, 3), vovo)
    t1b += es("akci,akcd->id", Hvoovb, vovv) - es("akci,klic->la", Hvoovb, ooov)   # H^{ak}_{ci}
    Xb = es("akci,klcd->liad", Hvoovb, oovv)
    t2b += 0.5 * Xb                                                 # X = 1/2 t2 + t1 t1
    t1b += es("liad,id->la", Xb, t1) + es("liad,la->id", Xb, t1)
    t1b += es("kc,klcd->ld", Hovb, oovv)                            # H^k_c
    Hoob += Goob                                                    # G^k_i
    t1b -= es("ki,klic->lc", Goob, ooov) + es("ki,kc->ic", Goob, fov)
    taub += 0.5 * es("ki,klcd->licd", Hoob, oovv)                   # H^k_i
    Hvvb += Gvvb                                                    # G^a_c
    t1b += es("ac,akcd->kd", Gvvb, vovv) - es("ac,kc->ka", Gvvb, fov)
    taub += 0.5 * es("ac,klcd->klda", Hvvb, oovv)                   # H^a_c
    t2b += taub                                                     # tau = t2 + P^-_ij t1 t1
    zb = pm(taub, 0, 1)
    t1b += es("ijab,jb->ia", zb, t1) + es("ijab,ia->jb", zb, t1)
    G = t2b
    return t1b, G - G.transpose(1, 0, 2, 3) - G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2)
