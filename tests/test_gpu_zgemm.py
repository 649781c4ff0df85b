"""The engine's complex GEMM (ccsd_zgemm) against numpy, for every tile configuration,
transpose/conjugate flag, ragged shapes and the split-K path (fixed-order reduction)."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_2103_08473_gb300 import build, ccsd
    ccsd.load(build.build())
    return torch, ccsd


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _op(x, trans, conj):
    y = x.T if trans else x
    return np.conj(y) if conj else y


@pytest.mark.parametrize("cfg", list(range(7)))
@pytest.mark.parametrize("M,N,K", [(20, 77, 45), (67, 130, 9), (190, 33, 301), (5, 3, 700)])
def test_zgemm_configs(env, cfg, M, N, K):
    torch, ccsd = env
    rng = np.random.default_rng(cfg * 1000 + M + N + K)
    for tA, cA, tB, cB in [(0, 0, 0, 0), (1, 1, 0, 0), (0, 0, 1, 1), (1, 0, 1, 0), (0, 1, 0, 1)]:
        a = _rand(rng, *((K, M) if tA else (M, K)))
        b = _rand(rng, *((N, K) if tB else (K, N)))
        c0 = _rand(rng, M, N)
        alpha, beta = 0.7 - 0.2j, -0.3 + 0.5j
        want = alpha * (_op(a, tA, cA) @ _op(b, tB, cB)) + beta * c0
        da, db, dc = (torch.from_numpy(x).cuda() for x in (a, b, c0))
        ccsd.zgemm(da, db, dc, alpha, beta, bool(tA), bool(cA), bool(tB), bool(cB), cfg=cfg)
        got = dc.cpu().numpy()
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want))) * np.sqrt(K)


@pytest.mark.parametrize("M,N,K", [(20, 20, 288000 // 16), (7, 11, 5000), (120, 20, 4800)])
def test_zgemm_split_k_is_exact_and_deterministic(env, M, N, K):
    torch, ccsd = env
    rng = np.random.default_rng(M * N)
    a, b = _rand(rng, M, K), _rand(rng, K, N)
    want = a @ b
    ws = torch.empty(64 * 1024 * 1024 // 16, dtype=torch.complex128, device="cuda")
    outs = []
    for _ in range(2):
        dc = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
        ccsd.zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc, workspace=ws)
        outs.append(dc.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0] - want)) <= 1e-13 * np.max(np.abs(want)) * np.sqrt(K)
    # without a workspace the same product comes out of the unsplit path
    dc = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc)
    assert np.max(np.abs(dc.cpu().numpy() - want)) <= 1e-13 * np.max(np.abs(want)) * np.sqrt(K)


def test_zgemm_rejects_bad_arguments(env):
    torch, ccsd = env
    x = torch.zeros((2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(ccsd.CCSDError):
        ccsd.zgemm(x, x, x, cfg=9)
