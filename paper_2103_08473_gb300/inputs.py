"""Seeded synthetic inputs for the complex CCSD engine and for its CPU oracle.

This module only draws random numbers and lays them out; it holds none of the
CCSD arithmetic, so both the CUDA path's tests and the oracle's tests can use
it without sharing any of the method.

The system recipe follows the synthetic density-fitting configurations:

* orbital energies: occupied uniform in [-2, -0.5], virtual uniform in [0.3, 5],
  each sorted ascending, occupied spinors first;
* DF factors B^Q_pr: Z = 0.05 (x + i y)/sqrt(2) with x, y standard normal drawn
  in C order over (naux, n, n), then B^Q = (Z^Q + Z^Q^H)/2 (Hermitian in p, r).

Draw order is fixed: eps_occ, eps_vir, x, y, all from
``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Named workloads (o occupied spinors, v virtual spinors, naux DF functions, seed).
CONFIGS = {
    "o10v30": dict(o=10, v=30, naux=120, seed=1),
    "o20v120": dict(o=20, v=120, naux=400, seed=2),
    "o40v240": dict(o=40, v=240, naux=800, seed=3),
    "o60v400": dict(o=60, v=400, naux=1200, seed=5),
}


@dataclass
class System:
    o: int
    v: int
    naux: int
    eps: np.ndarray  # (n,) float64, occupied first
    B: np.ndarray  # (naux, n, n) complex128, Hermitian in the last two indices
    fock: np.ndarray | None = None  # (n, n) complex128 Hermitian, or None = diag(eps)

    @property
    def n(self) -> int:
        return self.o + self.v


def make_system(o: int, v: int, naux: int, seed: int, scale: float = 0.05,
                eps_occ=(-2.0, -0.5), eps_vir=(0.3, 5.0)) -> System:
    """Draw one synthetic Kramers-unrestricted system (see the module docstring)."""
    rng = np.random.default_rng(seed)
    eo = np.sort(rng.uniform(eps_occ[0], eps_occ[1], size=o))
    ev = np.sort(rng.uniform(eps_vir[0], eps_vir[1], size=v))
    n = o + v
    x = rng.standard_normal((naux, n, n))
    y = rng.standard_normal((naux, n, n))
    z = scale * (x + 1j * y) / np.sqrt(2.0)
    B = 0.5 * (z + np.conj(np.transpose(z, (0, 2, 1))))
    return System(o=o, v=v, naux=naux, eps=np.concatenate([eo, ev]), B=np.ascontiguousarray(B))


def make_config(name: str) -> System:
    c = CONFIGS[name]
    return make_system(c["o"], c["v"], c["naux"], c["seed"])


def batch_shapes(nsys: int = 64, seed: int = 4, o_range=(4, 16), v_range=(16, 64)):
    """(o_k, v_k, naux_k = 3 v_k, seed_k = 1000 + k) for the batched workload."""
    rng = np.random.default_rng(seed)
    os_ = rng.integers(o_range[0], o_range[1] + 1, size=nsys)
    vs_ = rng.integers(v_range[0], v_range[1] + 1, size=nsys)
    return [(int(os_[k]), int(vs_[k]), int(3 * vs_[k]), 1000 + k) for k in range(nsys)]


def make_batch(nsys: int = 64, seed: int = 4):
    return [make_system(o, v, naux, s) for (o, v, naux, s) in batch_shapes(nsys, seed)]


def random_amplitudes(o: int, v: int, seed: int, scale: float = 0.05):
    """Random complex t1[i,a] and t2[i,j,a,b] antisymmetric in (i,j) and in (a,b)."""
    rng = np.random.default_rng(seed)
    t1 = scale * (rng.standard_normal((o, v)) + 1j * rng.standard_normal((o, v)))
    r = scale * (rng.standard_normal((o, o, v, v)) + 1j * rng.standard_normal((o, o, v, v)))
    t2 = r - r.transpose(1, 0, 2, 3)
    t2 = t2 - t2.transpose(0, 1, 3, 2)
    return np.ascontiguousarray(t1), np.ascontiguousarray(0.5 * t2)


def random_hermitian(n: int, seed: int, scale: float = 0.05) -> np.ndarray:
    rng = np.random.default_rng(seed)
    m = scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return 0.5 * (m + m.conj().T)


def random_unitary(n: int, seed: int) -> np.ndarray:
    """Haar-like random unitary from the QR of a complex Gaussian matrix."""
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(m)
    d = np.diag(r)
    return q * (d / np.abs(d))
