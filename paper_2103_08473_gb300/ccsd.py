"""ctypes binding of libccsd (include/ccsd.h): argument marshalling only.

Every step of the CCSD iteration runs in the CUDA library; this module converts
numpy arrays / torch CUDA tensors to pointers and status codes to exceptions.
There is no CPU fallback: if libccsd.so is missing or cannot be loaded, every
entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libccsd.so")

STATUS = {0: "CCSD_OK", 1: "CCSD_ERR_ARG", 2: "CCSD_ERR_OOM", 3: "CCSD_ERR_CUDA", 4: "CCSD_ERR_NOT_CONVERGED",
          5: "CCSD_ERR_DIVERGED", 6: "CCSD_ERR_TIMEOUT", 7: "CCSD_ERR_UNSUPPORTED"}
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
INT_DF, INT_FULL = 0, 1
PREC_FP64, PREC_SPLIT = 0, 1
METHOD_CCSD, METHOD_CCD, METHOD_CC2 = 0, 1, 2
ACCEL_DIIS, ACCEL_CROP = 0, 1


class ccsd_z(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class ccsd_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("tol", C.c_double), ("norm", C.c_int), ("diis_dim", C.c_int),
                ("diis_start", C.c_int), ("level_shift", C.c_double), ("precision", C.c_int),
                ("slices", C.c_int), ("store_w", C.c_int), ("profile", C.c_int), ("stream", C.c_void_p),
                ("split_min_flops", C.c_double), ("df_block", C.c_int), ("autotune", C.c_int),
                ("digit_bits", C.c_int), ("complex_4m", C.c_int), ("split_budget", C.c_double),
                ("method", C.c_int), ("accelerator", C.c_int), ("diverge_iters", C.c_int),
                ("diverge_factor", C.c_double), ("vovv_block", C.c_int), ("permute_cache_limit", C.c_double)]


class CCSDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every entry point declared in include/ccsd.h
_P = C.c_void_p
SIGNATURES = [
    ("ccsd_default_opts", None, [C.POINTER(ccsd_opts)]),
    ("ccsd_create", C.c_int, [C.c_int, C.c_int, _P, _P, C.c_int, _P, C.c_int, C.POINTER(ccsd_opts), C.POINTER(_P)]),
    ("ccsd_residual", C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    ("ccsd_iterate", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ccsd_divergence_index", C.c_int, [_P, C.c_int, C.c_int, C.c_double]),
    ("ccsd_energy", C.c_int, [_P, C.POINTER(ccsd_z)]),
    ("ccsd_triples", C.c_int, [_P, C.c_int, _P, _P]),
    ("ccsd_lambda_residual", C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    ("ccsd_lambda_iterate", C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ccsd_get_lambda", C.c_int, [_P, _P, _P, C.c_int]),
    ("ccsd_density", C.c_int, [_P, _P, C.c_int]),
    ("ccsd_get_amplitudes", C.c_int, [_P, _P, _P, C.c_int]),
    ("ccsd_set_amplitudes", C.c_int, [_P, _P, _P, C.c_int]),
    ("ccsd_get_tensor", C.c_int, [_P, C.c_char_p, _P, C.c_size_t, C.c_int]),
    ("ccsd_timings", C.c_int, [_P, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
    ("ccsd_query", C.c_int, [_P, C.c_char_p, C.POINTER(C.c_double)]),
    ("ccsd_zgemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong,
                             ccsd_z, _P, C.c_longlong, _P, C.c_longlong, ccsd_z, _P, C.c_longlong, _P, C.c_size_t,
                             C.c_int, _P]),
    ("ccsd_zgemm_noalloc", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_longlong,
                                     C.c_longlong, ccsd_z, _P, C.c_longlong, _P, C.c_longlong, ccsd_z, _P,
                                     C.c_longlong, C.c_int, _P]),
    ("ccsd_split_workspace", C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong]),
    ("ccsd_split_zgemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_longlong,
                                   C.c_longlong, C.c_longlong, ccsd_z, _P, C.c_longlong, _P, C.c_longlong, ccsd_z, _P,
                                   C.c_longlong, _P, C.c_size_t, _P]),
    ("ccsd_split_describe", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, _P]),
    ("ccsd_split_probe", C.c_int, [C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, _P, _P, _P, _P, C.c_size_t,
                                   _P]),
    ("ccsd_split_wait_selftest", C.c_int, [_P]),
    ("ccsd_batch_create", C.c_int, [C.c_int, _P, _P, _P, _P, _P, C.POINTER(ccsd_opts), C.POINTER(_P)]),
    ("ccsd_batch_iterate", C.c_int, [_P, C.c_int, _P, _P, _P]),
    ("ccsd_batch_energy", C.c_int, [_P, _P]),
    ("ccsd_batch_get_amplitudes", C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    ("ccsd_batch_last_error", C.c_char_p, [_P]),
    ("ccsd_batch_destroy", None, [_P]),
    ("ccsd_last_error", C.c_char_p, [_P]),
    ("ccsd_destroy", None, [_P]),
]


def load(path: str | None = None):
    """Load libccsd.so (raises OSError if it is missing: there is no fallback).

    With no argument the in-tree library is loaded once and cached; an explicit
    path is always loaded afresh.
    """
    global _lib
    if path is None and _lib is not None:
        return _lib
    target = LIB_PATH if path is None else path
    if not os.path.exists(target):
        raise OSError(f"libccsd.so not found at {target}; run __graft_entry__.build() first")
    lib = C.CDLL(target)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None or os.path.abspath(target) == LIB_PATH:
        _lib = lib
    return lib


def default_opts(**kw) -> ccsd_opts:
    lib = load()
    o = ccsd_opts()
    lib.ccsd_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            o.stream = C.c_void_p(v if isinstance(v, int) else getattr(v, "cuda_stream", 0))
        else:
            setattr(o, k, v)
    return o


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.complex128):
    """(pointer, on_device, keepalive) of a numpy array or torch CUDA tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("torch tensors must be contiguous CUDA tensors")
        return C.c_void_p(x.data_ptr()), 1, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), 0, a


class CCSD:
    """One CCSD problem on the GPU (wraps a ccsd_ctx)."""

    def __init__(self, o, v, eps, B=None, V=None, fock=None, **opts):
        lib = load()
        self.o, self.v = int(o), int(v)
        self.n = self.o + self.v
        self._opts = default_opts(**opts)
        eps_a = np.ascontiguousarray(eps, dtype=np.float64)
        if eps_a.shape != (self.n,):
            raise ValueError("eps must have o + v entries")
        if (B is None) == (V is None):
            raise ValueError("give exactly one of B (DF factors) or V (full integrals)")
        if B is not None:
            ints = np.ascontiguousarray(B, dtype=np.complex128)
            kind, naux = INT_DF, ints.shape[0]
            if ints.shape != (naux, self.n, self.n):
                raise ValueError("B must be (naux, n, n)")
        else:
            ints = np.ascontiguousarray(V, dtype=np.complex128)
            kind, naux = INT_FULL, 0
            if ints.shape != (self.n,) * 4:
                raise ValueError("V must be (n, n, n, n)")
        fk = None if fock is None else np.ascontiguousarray(fock, dtype=np.complex128)
        h = C.c_void_p()
        st = lib.ccsd_create(self.o, self.v, eps_a.ctypes.data_as(C.c_void_p),
                             None if fk is None else fk.ctypes.data_as(C.c_void_p), kind,
                             ints.ctypes.data_as(C.c_void_p), naux, C.byref(self._opts), C.byref(h))
        if st != OK:
            raise CCSDError(st, lib.ccsd_last_error(None).decode())
        self._h = h
        self._lib = lib

    # -- helpers
    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise CCSDError(st, self._lib.ccsd_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ccsd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shapes(self):
        return (self.o, self.v), (self.o, self.o, self.v, self.v)

    # -- ABI calls
    def residual(self, t1=None, t2=None, out=None):
        """(S1, S2) of Appendix A at (t1, t2) (numpy -> numpy, torch CUDA -> torch CUDA)."""
        s1, s2 = self.shapes
        dev = t1 is not None and _is_torch(t1)
        if out is None:
            if dev:
                import torch
                out = (torch.empty(s1, dtype=torch.complex128, device=t1.device),
                       torch.empty(s2, dtype=torch.complex128, device=t1.device))
            else:
                out = (np.empty(s1, np.complex128), np.empty(s2, np.complex128))
        p1, d1, k1 = _ptr(t1)
        p2, d2, k2 = _ptr(t2)
        q1, e1, _ = _ptr(out[0]) if _is_torch(out[0]) else (out[0].ctypes.data_as(C.c_void_p), 0, None)
        q2, e2, _ = _ptr(out[1]) if _is_torch(out[1]) else (out[1].ctypes.data_as(C.c_void_p), 0, None)
        on_dev = 1 if (d1 or e1) else 0
        if t1 is not None and (d1 != e1 or d2 != e2 or d1 != d2):
            raise ValueError("inputs and outputs must all be host arrays or all CUDA tensors")
        self._check(self._lib.ccsd_residual(self._h, p1, p2, q1, q2, on_dev))
        return out

    def iterate(self, max_iter=0):
        """Run iterations; returns (status, iterations, norm). Raises on CUDA/arg errors."""
        it = C.c_int(0)
        nrm = C.c_double(0.0)
        st = self._lib.ccsd_iterate(self._h, int(max_iter), C.byref(it), C.byref(nrm))
        self._check(st, allow=(ERR_NOT_CONVERGED, ERR_DIVERGED))
        return st, it.value, nrm.value

    def energy(self) -> complex:
        e = ccsd_z()
        self._check(self._lib.ccsd_energy(self._h, C.byref(e)))
        return complex(e.re, e.im)

    def triples(self, max_batch=0, pair_terms=False):
        """Triples corrections {"+T", "(T)", "-T"} at the current amplitudes; with pair_terms,
        also the (o, o, 3) array of each pair's contributions."""
        out = np.zeros(3)
        pt = np.zeros((self.o, self.o, 3)) if pair_terms else None
        self._check(self._lib.ccsd_triples(self._h, int(max_batch), out.ctypes.data_as(C.c_void_p),
                                           pt.ctypes.data_as(C.c_void_p) if pt is not None else None))
        e = {"+T": float(out[0]), "(T)": float(out[1]), "-T": float(out[2])}
        return (e, pt) if pair_terms else e

    def lambda_residual(self, l1=None, l2=None):
        """(R1, R2) of the Lambda equations at (l1, l2), which become the context's multipliers;
        with none given, at the context's own."""
        s1, s2 = self.shapes
        r1, r2 = np.empty(s1, np.complex128), np.empty(s2, np.complex128)
        a1 = None if l1 is None else np.ascontiguousarray(l1, dtype=np.complex128)
        a2 = None if l2 is None else np.ascontiguousarray(l2, dtype=np.complex128)
        self._check(self._lib.ccsd_lambda_residual(
            self._h, None if a1 is None else a1.ctypes.data_as(C.c_void_p),
            None if a2 is None else a2.ctypes.data_as(C.c_void_p),
            r1.ctypes.data_as(C.c_void_p), r2.ctypes.data_as(C.c_void_p), 0))
        return r1, r2

    def lambda_iterate(self, max_iter=0):
        """Iterate the Lambda equations; returns (status, iterations, norm)."""
        it = C.c_int(0)
        nrm = C.c_double(0.0)
        st = self._lib.ccsd_lambda_iterate(self._h, int(max_iter), C.byref(it), C.byref(nrm))
        self._check(st, allow=(ERR_NOT_CONVERGED, ERR_DIVERGED))
        return st, it.value, nrm.value

    def get_lambda(self):
        s1, s2 = self.shapes
        l1, l2 = np.empty(s1, np.complex128), np.empty(s2, np.complex128)
        self._check(self._lib.ccsd_get_lambda(self._h, l1.ctypes.data_as(C.c_void_p),
                                              l2.ctypes.data_as(C.c_void_p), 0))
        return l1, l2

    def density(self, symmetrize=False):
        """The one-body density (n x n, occupied first), less the reference occupation."""
        g = np.empty((self.n, self.n), np.complex128)
        self._check(self._lib.ccsd_density(self._h, g.ctypes.data_as(C.c_void_p), int(bool(symmetrize))))
        return g

    def get_amplitudes(self, out=None):
        s1, s2 = self.shapes
        if out is None:
            out = (np.empty(s1, np.complex128), np.empty(s2, np.complex128))
        p1, d1, _ = _ptr(out[0]) if _is_torch(out[0]) else (out[0].ctypes.data_as(C.c_void_p), 0, None)
        p2, d2, _ = _ptr(out[1]) if _is_torch(out[1]) else (out[1].ctypes.data_as(C.c_void_p), 0, None)
        self._check(self._lib.ccsd_get_amplitudes(self._h, p1, p2, d1))
        return out

    def set_amplitudes(self, t1, t2):
        p1, d1, k1 = _ptr(t1)
        p2, d2, k2 = _ptr(t2)
        self._check(self._lib.ccsd_set_amplitudes(self._h, p1, p2, d1))

    def get_tensor(self, name):
        o, v = self.o, self.v
        shapes = {"tau": (o, o, v, v), "Hvv": (v, v), "Gvv": (v, v), "Hoo": (o, o), "Goo": (o, o),
                  "Hov": (o, v), "Hvoov": (o, v, o, v), "C": (o, v, o, o), "A": (o, o, o, o),
                  "ladder": (o, o, v, v)}
        out = np.empty(shapes[name], np.complex128)
        self._check(self._lib.ccsd_get_tensor(self._h, name.encode(), out.ctypes.data_as(C.c_void_p), out.size, 0))
        return out

    def timings(self):
        """[(op name, average ms)] since the previous call (needs profile=1); resets the averages."""
        n = C.c_int(0)
        self._check(self._lib.ccsd_timings(self._h, None, None, 0, C.byref(n)))
        if n.value == 0:
            return []
        names = (C.c_char_p * n.value)()
        ms = (C.c_double * n.value)()
        self._check(self._lib.ccsd_timings(self._h, names, ms, n.value, C.byref(n)))
        return [(names[k].decode(), ms[k]) for k in range(n.value)]

    def query(self, key):
        val = C.c_double(0.0)
        self._check(self._lib.ccsd_query(self._h, key.encode(), C.byref(val)))
        return val.value



def divergence_index(norms, iters=8, factor=1e3) -> int:
    """ccsd_divergence_index: 1-based index of the norm at which the iterations would report
    sustained growth, 0 if none."""
    lib = load()
    a = np.ascontiguousarray(norms, dtype=np.float64)
    r = lib.ccsd_divergence_index(a.ctypes.data_as(C.c_void_p), len(a), int(iters), float(factor))
    if r < 0:
        raise CCSDError(ERR_ARG, "bad norm sequence")
    return r


def zgemm(a, b, c, alpha=1.0, beta=0.0, transA=False, conjA=False, transB=False, conjB=False,
          precision=PREC_FP64, workspace=None, cfg=-1, stream=None):
    """c = alpha opA(a) opB(b) + beta c on row-major torch CUDA complex128 matrices (c in place)."""
    lib = load()
    M, N = c.shape
    K = a.shape[0] if transA else a.shape[1]
    ws_ptr, ws_n = (None, 0) if workspace is None else (_ptr(workspace)[0], workspace.numel())
    strm = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    al, be = complex(alpha), complex(beta)
    st = lib.ccsd_zgemm(int(precision), int(transA), int(conjA), int(transB), int(conjB), M, N, K,
                        ccsd_z(al.real, al.imag), _ptr(a)[0], a.stride(0), _ptr(b)[0], b.stride(0),
                        ccsd_z(be.real, be.imag), _ptr(c)[0], c.stride(0), ws_ptr, ws_n, int(cfg), strm)
    if st != OK:
        raise CCSDError(st, lib.ccsd_last_error(None).decode())
    return c


def zgemm_noalloc(a, b, c, alpha=1.0, beta=0.0, transA=False, conjA=False, transB=False, conjB=False,
                  precision=PREC_FP64, cfg=-1, stream=None):
    """ccsd_zgemm_noalloc: like zgemm, with the split-K partials in the library's fixed device array
    (for callers that cannot allocate device memory). c is updated in place."""
    lib = load()
    M, N = c.shape
    K = a.shape[0] if transA else a.shape[1]
    strm = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    al, be = complex(alpha), complex(beta)
    st = lib.ccsd_zgemm_noalloc(int(precision), int(transA), int(conjA), int(transB), int(conjB), M, N, K,
                                ccsd_z(al.real, al.imag), _ptr(a)[0], a.stride(0), _ptr(b)[0], b.stride(0),
                                ccsd_z(be.real, be.imag), _ptr(c)[0], c.stride(0), int(cfg), strm)
    if st != OK:
        raise CCSDError(st, lib.ccsd_last_error(None).decode())
    return c


SPLIT_E4M3, SPLIT_BF16 = 0, 1


def split_zgemm(a, b, c, alpha=1.0, beta=0.0, transA=False, conjA=False, transB=False, conjB=False,
                kind=SPLIT_E4M3, bits=5, slices=9, stream=None):
    """ccsd_split_zgemm on row-major torch CUDA complex128 matrices (c updated in place)."""
    import torch
    lib = load()
    M, N = c.shape
    K = a.shape[0] if transA else a.shape[1]
    need = lib.ccsd_split_workspace(kind, bits, slices, M, N, K)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=c.device)
    strm = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    al, be = complex(alpha), complex(beta)
    st = lib.ccsd_split_zgemm(kind, bits, slices, int(transA), int(conjA), int(transB), int(conjB), M, N, K,
                              ccsd_z(al.real, al.imag), _ptr(a)[0], a.stride(0), _ptr(b)[0], b.stride(0),
                              ccsd_z(be.real, be.imag), _ptr(c)[0], c.stride(0), C.c_void_p(ws.data_ptr()), need,
                              strm)
    if st != OK:
        raise CCSDError(st, lib.ccsd_last_error(None).decode())
    return c


def split_describe(M, N, K, kind=SPLIT_E4M3, bits=5, slices=8):
    """ccsd_split_describe: how ccsd_split_zgemm runs an M x N x K product, as a dict."""
    lib = load()
    out = (C.c_int * 6)()
    st = lib.ccsd_split_describe(kind, bits, slices, M, N, K, C.cast(out, C.c_void_p))
    if st != OK:
        raise CCSDError(st, lib.ccsd_last_error(None).decode())
    return {"short_k": out[0], "swap": out[1], "tile_n": out[2], "cluster": out[3], "ksplits": out[4],
            "tiles": out[5]}


def split_probe(a, b, kind=SPLIT_E4M3):
    """ccsd_split_probe on torch CUDA float64 integer-valued matrices a (M x K), b (N x K)."""
    import torch
    lib = load()
    M, K = a.shape
    N = b.shape[0]
    need = lib.ccsd_split_workspace(kind, 8 if kind == SPLIT_BF16 else 4, 1, M, N, K)
    ws = torch.empty(need, dtype=torch.uint8, device=a.device)
    out = torch.empty((M, N), dtype=torch.float64, device=a.device)
    st = lib.ccsd_split_probe(kind, M, N, K, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                              C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()), need, None)
    if st != OK:
        raise CCSDError(st, lib.ccsd_last_error(None).decode())
    return out


def split_wait_selftest(stream=None):
    """ccsd_split_wait_selftest: returns (status, message); TIMEOUT is the intended outcome."""
    lib = load()
    st = lib.ccsd_split_wait_selftest(None if stream is None else C.c_void_p(stream))
    return st, lib.ccsd_last_error(None).decode()


class Batch:
    """Many independent systems iterated together (wraps a ccsd_batch)."""

    def __init__(self, systems, **opts):
        """systems: list of (o, v, eps, B) with B of shape (naux, n, n)."""
        lib = load()
        self._lib = lib
        self.nsys = len(systems)
        self.shapes = [(int(o), int(v)) for (o, v, _, _) in systems]
        self._eps = [np.ascontiguousarray(e, dtype=np.float64) for (_, _, e, _) in systems]
        self._B = [np.ascontiguousarray(b, dtype=np.complex128) for (_, _, _, b) in systems]
        oa = (C.c_int * self.nsys)(*[s[0] for s in self.shapes])
        va = (C.c_int * self.nsys)(*[s[1] for s in self.shapes])
        na = (C.c_int * self.nsys)(*[b.shape[0] for b in self._B])
        ep = (C.c_void_p * self.nsys)(*[e.ctypes.data for e in self._eps])
        bp = (C.c_void_p * self.nsys)(*[b.ctypes.data for b in self._B])
        self._opts = default_opts(**opts)
        h = C.c_void_p()
        st = lib.ccsd_batch_create(self.nsys, oa, va, ep, bp, na, C.byref(self._opts), C.byref(h))
        if st != OK:
            raise CCSDError(st, lib.ccsd_last_error(None).decode())
        self._h = h

    def iterate(self, max_iter=0):
        it = (C.c_int * self.nsys)()
        nrm = (C.c_double * self.nsys)()
        sts = (C.c_int * self.nsys)()
        st = self._lib.ccsd_batch_iterate(self._h, int(max_iter), it, nrm, sts)
        if st not in (OK, ERR_NOT_CONVERGED):
            raise CCSDError(st, self._lib.ccsd_batch_last_error(self._h).decode())
        return st, list(it), list(nrm), list(sts)

    def energies(self):
        e = (ccsd_z * self.nsys)()
        st = self._lib.ccsd_batch_energy(self._h, e)
        if st != OK:
            raise CCSDError(st, self._lib.ccsd_batch_last_error(self._h).decode())
        return [complex(x.re, x.im) for x in e]

    def get_amplitudes(self, k):
        o, v = self.shapes[k]
        t1, t2 = np.empty((o, v), np.complex128), np.empty((o, o, v, v), np.complex128)
        st = self._lib.ccsd_batch_get_amplitudes(self._h, int(k), t1.ctypes.data_as(C.c_void_p),
                                                 t2.ctypes.data_as(C.c_void_p), 0)
        if st != OK:
            raise CCSDError(st, self._lib.ccsd_batch_last_error(self._h).decode())
        return t1, t2

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ccsd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
