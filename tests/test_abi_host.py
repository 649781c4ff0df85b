"""Host-side checks of the C ABI (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/ccsd.h declares; argument errors are reported as status codes before
any device work.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_08473_gb300 import build, ccsd
    path = build.build()
    return ccsd.load(path)


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ccsd_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ccsd_create", "ccsd_residual", "ccsd_iterate", "ccsd_energy", "ccsd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2103_08473_gb300 import ccsd
    bound = {name for name, _, _ in ccsd.SIGNATURES}
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in bound, f"{name} has no binding signature"


def test_default_opts(lib):
    from paper_2103_08473_gb300 import ccsd
    o = ccsd.default_opts()
    assert o.max_iter == 50 and o.diis_dim == 8 and o.diis_start == 2 and o.tol == 1e-10 and o.store_w == 1
    assert o.split_min_flops == 1e8 and o.precision == 0
    assert o.slices == 0 and o.digit_bits == 0 and o.complex_4m == 0 and o.method == ccsd.METHOD_CCSD
    assert o.accelerator == ccsd.ACCEL_DIIS and o.diverge_iters == 8 and o.diverge_factor == 1e3
    assert o.vovv_block == 0 and o.permute_cache_limit == 0.0


def _create(lib, o, v, eps, B, naux, opts=None):
    from paper_2103_08473_gb300 import ccsd
    h = C.c_void_p()
    st = lib.ccsd_create(o, v, eps.ctypes.data_as(C.c_void_p) if eps is not None else None, None, 0,
                         B.ctypes.data_as(C.c_void_p) if B is not None else None, naux,
                         C.byref(opts) if opts is not None else None, C.byref(h))
    return st, h


@pytest.mark.parametrize("case", ["o0", "v0", "naux0", "null_eps", "null_ints", "nonhermitian", "diis17", "bits6", "bits_x_slices", "method3", "accel2", "diverge_neg", "diverge_factor", "vovv_block_neg"])
def test_create_rejects_bad_arguments(lib, case):
    from paper_2103_08473_gb300 import ccsd, inputs
    s = inputs.make_system(2, 3, 4, seed=1)
    eps, B, o, v, naux = s.eps, s.B.copy(), 2, 3, 4
    opts = None
    if case == "o0":
        o = 0
    elif case == "v0":
        v = 0
    elif case == "naux0":
        naux = 0
    elif case == "null_eps":
        eps = None
    elif case == "null_ints":
        B = None
    elif case == "nonhermitian":
        B[1, 0, 2] += 1e-6
    elif case == "diis17":
        opts = ccsd.default_opts(diis_dim=17)
    elif case == "bits6":  # e4m3 holds every integer digit only up to 16: at most 5 bits
        opts = ccsd.default_opts(precision=ccsd.PREC_SPLIT, digit_bits=6)
    elif case == "method3":
        opts = ccsd.default_opts(method=3)
    elif case == "accel2":
        opts = ccsd.default_opts(accelerator=2)
    elif case == "diverge_neg":
        opts = ccsd.default_opts(diverge_iters=-1)
    elif case == "diverge_factor":
        opts = ccsd.default_opts(diverge_factor=0.5)
    elif case == "vovv_block_neg":
        opts = ccsd.default_opts(vovv_block=-1)
    elif case == "bits_x_slices":
        opts = ccsd.default_opts(precision=ccsd.PREC_SPLIT, digit_bits=5, slices=12)
    st, h = _create(lib, o, v, eps, B, naux, opts)
    assert st == ccsd.ERR_ARG
    assert not h.value
    assert len(lib.ccsd_last_error(None)) > 0


def test_cc2_rejects_full_integrals_before_device_work(lib):
    """CC2 is built on the T1-dressed DF factors: full integrals are refused up front."""
    from paper_2103_08473_gb300 import ccsd, inputs
    o, v = 2, 3
    s = inputs.make_system(o, v, 4, seed=1)
    Vf = np.ascontiguousarray(np.zeros((o + v,) * 4, np.complex128))
    h = C.c_void_p()
    opts = ccsd.default_opts(method=ccsd.METHOD_CC2)
    st = lib.ccsd_create(o, v, s.eps.ctypes.data_as(C.c_void_p), None, ccsd.INT_FULL,
                         Vf.ctypes.data_as(C.c_void_p), 0, C.byref(opts), C.byref(h))
    assert st == ccsd.ERR_UNSUPPORTED
    assert not h.value
    assert b"DF" in lib.ccsd_last_error(None)


def test_null_context_calls_return_arg_error(lib):
    from paper_2103_08473_gb300 import ccsd
    assert lib.ccsd_iterate(None, 1, None, None) == ccsd.ERR_ARG
    assert lib.ccsd_energy(None, None) == ccsd.ERR_ARG
    out = (C.c_double * 3)()
    assert lib.ccsd_triples(None, 0, out, None) == ccsd.ERR_ARG
    assert lib.ccsd_lambda_iterate(None, 1, None, None) == ccsd.ERR_ARG
    assert lib.ccsd_lambda_residual(None, None, None, None, None, 0) == ccsd.ERR_ARG
    assert lib.ccsd_get_lambda(None, None, None, 0) == ccsd.ERR_ARG
    assert lib.ccsd_density(None, None, 0) == ccsd.ERR_ARG
    lib.ccsd_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2103_08473_gb300 import ccsd
    with pytest.raises(OSError):
        ccsd.load(str(tmp_path / "missing.so"))


def test_divergence_rule_on_synthetic_norm_sequences(lib):
    """The growth rule the iterations apply (ccsd_divergence_index), on host sequences."""
    from paper_2103_08473_gb300 import ccsd
    # converging, and converging with DIIS-like bumps: never
    assert ccsd.divergence_index(np.geomspace(1.0, 1e-12, 60)) == 0
    bumpy = [(1.8 if k % 2 else 1.0) * 0.5 ** (k // 2) for k in range(40)]  # up, down, up, ...
    assert ccsd.divergence_index(bumpy, iters=2, factor=1.5) == 0
    assert ccsd.divergence_index(bumpy, iters=1, factor=1.5) == 2
    # steady growth by 3x per iteration from norm 1: the run reaches 8 increases at index 9,
    # and 3^8 > 1e3 there
    grow = 3.0 ** np.arange(20)
    assert ccsd.divergence_index(grow, iters=8, factor=1e3) == 9
    # slow growth: eight increases, but not by the factor yet; the first index with
    # 1.5^r > 1e3 is r = 18
    slow = 1.5 ** np.arange(30)
    assert ccsd.divergence_index(slow, iters=8, factor=1e3) == 19
    # a drop restarts the run (and its base)
    seq = list(3.0 ** np.arange(7)) + [0.5] + list(0.5 * 3.0 ** np.arange(1, 10))
    assert ccsd.divergence_index(seq, iters=8, factor=1e3) == 16  # 0.5 at index 8 (1-based), then 8 rises
    # off, empty, non-finite, and bad arguments
    assert ccsd.divergence_index(grow, iters=0) == 0
    assert ccsd.divergence_index([], iters=8) == 0
    assert ccsd.divergence_index([1.0, 2.0, float("nan"), 1e9], iters=1, factor=1.0) == 2
    assert lib.ccsd_divergence_index(None, 3, 8, 1e3) == -1


def test_gemm_entry_points_refuse_bad_arguments_before_device_work(lib):
    """ccsd_zgemm, ccsd_zgemm_noalloc and ccsd_split_zgemm check sizes, pointers, the tile shape,
    the precision and (no-alloc) the static scratch limit on the host and return a status with a
    message; none of these calls reaches the device."""
    from paper_2103_08473_gb300 import ccsd
    z = ccsd.ccsd_z
    one, zero = z(1.0, 0.0), z(0.0, 0.0)
    p = C.c_void_p(16)  # never dereferenced: every call below is refused first
    # ccsd_zgemm: negative size, NULL operand, tile shape out of range, precision not built
    assert lib.ccsd_zgemm(0, 0, 0, 0, 0, -1, 4, 4, one, p, 4, p, 4, zero, p, 4, None, 0, 0, None) == ccsd.ERR_ARG
    assert lib.ccsd_zgemm(0, 0, 0, 0, 0, 4, 4, 4, one, None, 4, p, 4, zero, p, 4, None, 0, 0, None) == ccsd.ERR_ARG
    assert lib.ccsd_zgemm(0, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, p, 4, None, 0, 7, None) == ccsd.ERR_ARG
    assert lib.ccsd_zgemm(1, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, p, 4, None, 0, 0, None) == ccsd.ERR_UNSUPPORTED
    # ccsd_zgemm_noalloc: the same checks, and an output beyond the static scratch (M*N <= 2^17)
    assert lib.ccsd_zgemm_noalloc(0, 0, 0, 0, 0, 4, 4, -1, one, p, 4, p, 4, zero, p, 4, 0, None) == ccsd.ERR_ARG
    assert lib.ccsd_zgemm_noalloc(0, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, None, 4, 0, None) == ccsd.ERR_ARG
    assert lib.ccsd_zgemm_noalloc(1, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, p, 4, 0, None) == ccsd.ERR_UNSUPPORTED
    big = 1 << 9  # 512 x 512 = 2^18 > 2^17
    assert lib.ccsd_zgemm_noalloc(0, 0, 0, 0, 0, big, big, 4, one, p, 4, p, 4, zero, p, big, 0, None) == ccsd.ERR_ARG
    assert "exceeds the limit" in lib.ccsd_last_error(None).decode()
    # ccsd_split_zgemm: digit configuration, sizes, workspace
    assert lib.ccsd_split_zgemm(0, 6, 8, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, p, 4, p, 1 << 30, None) == ccsd.ERR_ARG
    assert lib.ccsd_split_zgemm(0, 5, 8, 0, 0, 0, 0, 4, 4, 0, one, p, 4, p, 4, zero, p, 4, p, 1 << 30, None) == ccsd.ERR_ARG
    need = lib.ccsd_split_workspace(0, 5, 8, 4, 4, 4)
    assert need > 0
    assert lib.ccsd_split_zgemm(0, 5, 8, 0, 0, 0, 0, 4, 4, 4, one, p, 4, p, 4, zero, p, 4, p, need - 1, None) == ccsd.ERR_ARG
    assert "workspace needs" in lib.ccsd_last_error(None).decode()
