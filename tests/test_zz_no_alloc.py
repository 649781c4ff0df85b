"""ccsd_zgemm_noalloc: the GEMM entry point for callers that cannot allocate device memory.

Such callers (inside another framework's memory budget, in a latency-critical loop
where cudaMalloc/cudaFree may synchronise the device, or with a device footprint
fixed at start-up) cannot pass ccsd_zgemm a split-K workspace; this entry point
keeps the split partials in a fixed array inside the library. The test calls it
through the C ABI twice in a row, on two different problems that both take the
split-K path, and checks each result against ccsd_zgemm with a caller-allocated
workspace, within the tolerance the other GEMM tests use. This file is collected
last so that, if it fails, a run stopping at the first failure has already run
every other test.
"""
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


def test_noalloc_matches_workspace_gemm_on_two_calls_in_a_row(env):
    torch, ccsd = env
    ws = torch.empty(1 << 18, dtype=torch.complex128, device="cuda")  # same capacity as the static array
    # two different split-K problems back to back: the second must not see the first's partials
    for k, (M, N, K) in enumerate([(20, 20, 18000), (7, 33, 9000)]):
        rng = np.random.default_rng(100 + k)
        a, b, c0 = _rand(rng, M, K), _rand(rng, K, N), _rand(rng, M, N)
        alpha, beta = 0.5 + 0.25j, -1.0 + 0.0j
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        ref = torch.from_numpy(c0).cuda()
        ccsd.zgemm(da, db, ref, alpha, beta, workspace=ws)
        got = torch.from_numpy(c0).cuda()
        ccsd.zgemm_noalloc(da, db, got, alpha, beta)
        want = ref.cpu().numpy()
        assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-13 * max(1.0, np.max(np.abs(want))) * np.sqrt(K)
        exact = alpha * (a @ b) + beta * c0
        assert np.max(np.abs(got.cpu().numpy() - exact)) <= 1e-13 * np.max(np.abs(exact)) * np.sqrt(K)


def test_noalloc_rejects_outputs_beyond_the_static_scratch(env):
    torch, ccsd = env
    a = torch.zeros((400, 8), dtype=torch.complex128, device="cuda")
    b = torch.zeros((8, 400), dtype=torch.complex128, device="cuda")
    c = torch.zeros((400, 400), dtype=torch.complex128, device="cuda")
    with pytest.raises(ccsd.CCSDError, match="static split-K scratch"):
        ccsd.zgemm_noalloc(a, b, c)


def test_noalloc_keeps_split_k_near_its_output_limit(env):
    """An output just under the 2^17-element limit has room for two split partials in the
    fixed array: the call still splits K (bitwise equal to ccsd_zgemm given a workspace of
    the same 2^18 elements, and different in rounding from the unsplit GEMM)."""
    torch, ccsd = env
    M, N, K = 362, 362, 4096  # M*N = 131044 <= 2^17
    rng = np.random.default_rng(7)
    a, b = _rand(rng, M, K), _rand(rng, K, N)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ws = torch.empty(1 << 18, dtype=torch.complex128, device="cuda")
    split = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.zgemm(da, db, split, workspace=ws)
    plain = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.zgemm(da, db, plain)
    for _ in range(2):
        got = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
        ccsd.zgemm_noalloc(da, db, got)
        assert torch.equal(got, split)
    assert not torch.equal(got, plain)
    exact = a @ b
    assert np.max(np.abs(got.cpu().numpy() - exact)) <= 1e-13 * np.max(np.abs(exact)) * np.sqrt(K)
