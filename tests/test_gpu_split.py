"""Split-precision complex GEMM on tcgen05 (ccsd_split_zgemm) and its accumulation probe.

The probe checks the premise of the scheme: integer-valued digit products summed
in the FP32 tensor-memory accumulator are exact while every partial sum stays
below 2^24. The GEMM is checked against numpy complex128 (and the FP64 DMMA
GEMM) with the error bound of the digit count: ~2^(-bits*slices) relative.
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


@pytest.mark.parametrize("kind,lim,K", [(0, 16, 4096), (0, 16, 1000), (1, 128, 512), (1, 100, 200)])
def test_probe_integer_accumulation_is_exact(env, kind, lim, K):
    torch, ccsd = env
    rng = np.random.default_rng(kind * 7 + K)
    M, N = 200, 130
    a = rng.integers(-lim, lim + 1, size=(M, K)).astype(np.float64)
    b = rng.integers(-lim, lim + 1, size=(N, K)).astype(np.float64)
    assert K * lim * lim < 2 ** 24
    want = (a.astype(np.int64) @ b.astype(np.int64).T).astype(np.float64)
    got = ccsd.split_probe(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), kind=kind).cpu().numpy()
    assert np.array_equal(got, want)


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("kind,bits,slices,tol", [(0, 4, 11, 2e-12), (0, 4, 6, 2e-6), (1, 7, 7, 2e-13), (1, 6, 5, 3e-8),
                                                  (0, 5, 9, 2e-12), (0, 5, 6, 6e-8), (0, 5, 8, 6e-11)])
def test_split_zgemm_matches_complex128(env, kind, bits, slices, tol):
    torch, ccsd = env
    rng = np.random.default_rng(slices * 10 + kind)
    M, N, K = 300, 200, 1000
    a, b, c0 = _rand(rng, M, K), _rand(rng, K, N), _rand(rng, M, N)
    alpha, beta = 0.75 - 0.5j, 0.25 + 1.0j
    want = alpha * (a @ b) + beta * c0
    dc = torch.from_numpy(c0).cuda()
    ccsd.split_zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc, alpha, beta, kind=kind, bits=bits,
                     slices=slices)
    err = np.max(np.abs(dc.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < tol, err


@pytest.mark.parametrize("kind,bits,slices,tol", [(0, 5, 9, 1e-9), (0, 4, 11, 1e-9), (1, 8, 5, 1e-9)])
def test_split_zgemm_first_digit_at_its_bound(env, kind, bits, slices, tol):
    """Rows whose largest entry sits just below a power of two (and exactly on one): the
    first digit then takes its largest magnitude, which must still be exact in the type."""
    torch, ccsd = env
    rng = np.random.default_rng(bits * 100 + slices)
    M, N, K = 150, 140, 520
    top = 1.0 - 2.0 ** -45
    a = rng.choice([top, -top, 0.5, -0.75, top / 2, 2.0 ** -20], size=(M, K)) * (2.0 ** rng.integers(-6, 6, (M, 1)))
    a = a + 1j * rng.choice([top, -top, 0.0, 0.25], size=(M, K)) * (2.0 ** rng.integers(-6, 6, (M, 1)))
    b = rng.choice([-top, top, 1.0, -0.5, 0.0], size=(K, N)) + 1j * rng.choice([top, -1.0, 0.125], size=(K, N))
    want = a @ b
    dc = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.split_zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc, 1.0, 0.0, kind=kind, bits=bits,
                     slices=slices)
    err = np.max(np.abs(dc.cpu().numpy() - want) / np.max(np.abs(want), axis=1, keepdims=True))
    assert err < tol, err


@pytest.mark.parametrize("tA,cA,tB,cB", [(0, 0, 1, 0), (1, 1, 0, 0), (0, 1, 1, 1), (1, 0, 0, 1)])
def test_split_zgemm_transpose_and_conjugate(env, tA, cA, tB, cB):
    torch, ccsd = env
    rng = np.random.default_rng(tA * 8 + cA * 4 + tB * 2 + cB)
    M, N, K = 131, 257, 300
    a = _rand(rng, *((K, M) if tA else (M, K)))
    b = _rand(rng, *((N, K) if tB else (K, N)))
    opa = (a.T if tA else a)
    opa = np.conj(opa) if cA else opa
    opb = (b.T if tB else b)
    opb = np.conj(opb) if cB else opb
    want = opa @ opb
    dc = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.split_zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc, 1.0, 0.0, bool(tA), bool(cA),
                     bool(tB), bool(cB))
    assert np.max(np.abs(dc.cpu().numpy() - want)) / np.max(np.abs(want)) < 2e-12


def test_split_zgemm_ladder_shape_matches_fp64_path(env):
    """The ladder GEMM of the o20/v120 workload: M = 190 (i<j), N = K = 7140 (a<b, c<d)."""
    torch, ccsd = env
    rng = np.random.default_rng(5)
    M, N, K = 190, 7140, 7140
    a = torch.from_numpy(_rand(rng, M, K) * 0.01).cuda()
    b = torch.from_numpy(_rand(rng, N, K) * 0.03).cuda()
    ref = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.zgemm(a, b, ref, transB=True)
    out = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    ccsd.split_zgemm(a, b, out, transB=True)
    err = (out - ref).abs().max().item() / ref.abs().max().item()
    assert err < 2e-12, err


def test_bounded_wait_gives_up_and_the_device_stays_usable(env):
    """The producer of a small split GEMM issues no copies: the MMA issuer's ~2 ms wait runs
    out, the kernel reports it and returns; the next split GEMM on the device is correct."""
    torch, ccsd = env
    st, msg = ccsd.split_wait_selftest()
    assert st == ccsd.ERR_TIMEOUT, msg
    rng = np.random.default_rng(11)
    a, b = _rand(rng, 64, 96), _rand(rng, 96, 80)
    dc = torch.zeros((64, 80), dtype=torch.complex128, device="cuda")
    ccsd.split_zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc)
    want = a @ b
    assert np.max(np.abs(dc.cpu().numpy() - want)) / np.max(np.abs(want)) < 2e-12


@pytest.mark.parametrize("M,N,K,slices,conjA,conjB,beta", [
    (20, 3000, 120, 8, 0, 0, 0.0),     # the short side as the 32-wide tiles, output transposed
    (3000, 40, 64, 8, 1, 0, 0.5 - 1j),  # no swap, conj(A), beta applied in the epilogue
    (300, 200, 512, 7, 0, 1, 1.0),    # four K blocks, the longest K the short-K kernel takes
    (130, 33, 1, 8, 1, 1, 0.0),       # K = 1, ragged tiles on both sides
])
def test_short_k_kernel_matches_complex128(env, M, N, K, slices, conjA, conjB, beta):
    """GEMMs of at most four K blocks with at most eight digit levels run on the short-K kernel
    (every level its own accumulator in tensor memory, one store per output)."""
    torch, ccsd = env
    rng = np.random.default_rng(M + N + K)
    a, b, c0 = _rand(rng, M, K), _rand(rng, N, K), _rand(rng, M, N)
    alpha = 0.5 + 0.25j
    opa = np.conj(a) if conjA else a
    opb = np.conj(b) if conjB else b
    want = alpha * (opa @ opb.T) + beta * c0
    dc = torch.from_numpy(c0).cuda()
    ccsd.split_zgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), dc, alpha, beta, conjA=bool(conjA),
                     transB=True, conjB=bool(conjB), bits=5, slices=slices)
    err = np.max(np.abs(dc.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < (2e-10 if slices == 8 else 6e-9), err


def test_split_zgemm_k_split_filling_whole_waves(env):
    """224 output tiles (1.5 waves of the GPU's SMs) and 32 K blocks: K is split in two so that
    the CTAs fill whole waves; the partial products are summed in a fixed order."""
    torch, ccsd = env
    rng = np.random.default_rng(224)
    M, N, K = 14 * 128, 16 * 128, 32 * 128
    a = torch.from_numpy(_rand(rng, M, K)).cuda()
    b = torch.from_numpy(_rand(rng, N, K)).cuda()
    c0 = _rand(rng, M, N)
    outs = []
    for _ in range(2):
        dc = torch.from_numpy(c0).cuda()
        ccsd.split_zgemm(a, b, dc, 1.0, -0.5, transB=True, bits=5, slices=8)
        outs.append(dc.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    want = a.cpu().numpy() @ b.cpu().numpy().T - 0.5 * c0
    assert np.max(np.abs(outs[0] - want)) / np.max(np.abs(want)) < 2e-10


@pytest.mark.parametrize("M,N,K,tA,cA,tB,cB", [(190, 1500, 1000, 0, 0, 1, 0), (190, 3000, 3000, 0, 0, 1, 1),
                                              (40, 1500, 1000, 1, 1, 0, 0), (40, 900, 2000, 0, 1, 1, 0),
                                              (100, 1500, 700, 0, 0, 0, 0)])
def test_split_zgemm_short_m_on_the_narrow_tile_side(env, M, N, K, tA, cA, tB, cB):
    """A short M (the occupied pairs of the ladder, 190 at o20/v120) goes to the BN side of the
    main kernel (96- or 64-wide tiles, output stored transposed), with and without K split;
    the result is the same GEMM to the digit bound."""
    torch, ccsd = env
    rng = np.random.default_rng(M * 7 + N + K)
    a = _rand(rng, *((K, M) if tA else (M, K)))
    b = _rand(rng, *((N, K) if tB else (K, N)))
    c0 = _rand(rng, M, N)
    oa = (a.T if tA else a)
    ob = (b.T if tB else b)
    oa = oa.conj() if cA else oa
    ob = ob.conj() if cB else ob
    alpha, beta = 0.5 + 0.25j, -0.75 + 0.5j
    want = alpha * (oa @ ob) + beta * c0
    dc = torch.from_numpy(c0).cuda()
    ccsd.split_zgemm(torch.from_numpy(np.ascontiguousarray(a)).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda(),
                     dc, alpha, beta, transA=bool(tA), conjA=bool(cA), transB=bool(tB), conjB=bool(cB), bits=5,
                     slices=8)
    got = dc.cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err < 6e-11, err
    # run to run bitwise
    dc2 = torch.from_numpy(c0).cuda()
    ccsd.split_zgemm(torch.from_numpy(np.ascontiguousarray(a)).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda(),
                     dc2, alpha, beta, transA=bool(tA), conjA=bool(cA), transB=bool(tB), conjB=bool(cB), bits=5,
                     slices=8)
    assert torch.equal(dc, dc2)


@pytest.mark.parametrize("M,N,K,tB,cB,kind", [(190, 3000, 3000, 1, 0, 0), (2000, 200, 1500, 1, 1, 0),
                                              (2000, 200, 6000, 0, 0, 0), (1000, 500, 1200, 1, 0, 0),
                                              (1000, 500, 1200, 0, 1, 1), (150, 2500, 2000, 1, 1, 0)])
def test_split_zgemm_cluster_pairs_share_the_long_operand(env, M, N, K, tB, cB, kind):
    """Two N tiles (or four) of one M tile and K range run as a cluster of two CTAs that each
    multicast one part (real or imaginary) of the shared 128-row digit tile into both; the
    product, with and without K split, swapped or not, is the same GEMM to the digit bound and
    the same bits from run to run."""
    torch, ccsd = env
    bits, slices = (5, 8) if kind == 0 else (8, 5)
    d = ccsd.split_describe(M, N, K, kind=kind, bits=bits, slices=slices)
    assert d["short_k"] == 0 and d["cluster"] == 2, d
    rng = np.random.default_rng(M + 3 * N + 7 * K + kind)
    a = _rand(rng, M, K)
    b = _rand(rng, *((N, K) if tB else (K, N)))
    c0 = _rand(rng, M, N)
    ob = b.T if tB else b
    ob = ob.conj() if cB else ob
    alpha, beta = 0.5 - 0.25j, 0.75 + 0.5j
    want = alpha * (a @ ob) + beta * c0
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    outs = []
    for _ in range(2):
        dc = torch.from_numpy(c0).cuda()
        ccsd.split_zgemm(da, db, dc, alpha, beta, transB=bool(tB), conjB=bool(cB), kind=kind, bits=bits, slices=slices)
        outs.append(dc)
    assert torch.equal(outs[0], outs[1])
    err = np.max(np.abs(outs[0].cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < (6e-11 if kind == 0 else 2e-10), err
