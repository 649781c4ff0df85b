"""Batched systems (ccsd_batch_*) and the measured tile autotuner.

A batch runs every system's own iteration (same kernels, same order) inside one
fork/join CUDA graph, so each system's energy must equal the energy of the same
system solved alone, and the converged oracle energy within 1e-10 Eh.
"""
import numpy as np
import pytest

from oracle import ccsd_ref as R
from paper_2103_08473_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(4, 16, 48, 1101), (6, 23, 69, 1102), (5, 17, 51, 1103), (8, 31, 93, 1104), (3, 19, 57, 1105),
          (7, 12, 36, 1106)]


@pytest.fixture(scope="module")
def ccsd():
    from paper_2103_08473_gb300 import build, ccsd as mod
    mod.load(build.build())
    return mod


def test_batch_matches_single_solves_and_oracle(ccsd):
    systems = [inputs.make_system(o, v, naux, seed) for (o, v, naux, seed) in SHAPES]
    with ccsd.Batch([(s.o, s.v, s.eps, s.B) for s in systems], tol=1e-10, max_iter=80) as b:
        st, its, norms, sts = b.iterate()
        eb = b.energies()
        t1b, t2b = b.get_amplitudes(3)
    assert st == ccsd.OK and all(x == ccsd.OK for x in sts)
    for k, s in enumerate(systems):
        with ccsd.CCSD(s.o, s.v, s.eps, B=s.B, tol=1e-10) as cc:
            st1, it1, _ = cc.iterate(80)
            e1 = cc.energy()
            if k == 3:
                t1s, t2s = cc.get_amplitudes()
        assert st1 == ccsd.OK and it1 == its[k]
        assert abs(eb[k] - e1) < 1e-12
        f = R.fock_matrix(s.eps)
        ref = R.solve(f, R.integrals(s.B, s.o), s.o, s.v, max_iter=80, tol=1e-10)
        assert ref["converged"] and abs(eb[k] - ref["energy"]) < 1e-10
    assert np.max(np.abs(t2b - t2s)) < 1e-12 and np.max(np.abs(t1b - t1s)) < 1e-12


def test_batch_reports_per_system_status(ccsd):
    systems = [inputs.make_system(o, v, naux, seed) for (o, v, naux, seed) in SHAPES[:3]]
    with ccsd.Batch([(s.o, s.v, s.eps, s.B) for s in systems], tol=1e-10) as b:
        st, its, norms, sts = b.iterate(2)
    assert st == ccsd.ERR_NOT_CONVERGED
    assert its == [2, 2, 2] and all(x == ccsd.ERR_NOT_CONVERGED for x in sts)


def test_autotuned_plan_gives_the_same_residual(ccsd):
    o, v, naux, seed = 9, 41, 60, 1201
    s = inputs.make_system(o, v, naux, seed)
    t1, t2 = inputs.random_amplitudes(o, v, seed + 1, scale=0.05)
    with ccsd.CCSD(o, v, s.eps, B=s.B) as a:
        r1, r2 = a.residual(t1, t2)
    with ccsd.CCSD(o, v, s.eps, B=s.B, autotune=1) as b:
        q1, q2 = b.residual(t1, t2)
    assert np.max(np.abs(q2 - r2)) < 1e-12 * max(1.0, np.max(np.abs(r2)))
    assert np.max(np.abs(q1 - r1)) < 1e-12 * max(1.0, np.max(np.abs(r1)))
