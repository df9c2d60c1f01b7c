"""Thin ctypes binding of libgbhegv (C-ABI in include/gbhegv.h).

Argument marshalling only: every numerical step runs in the CUDA library.
PyTorch provides device memory (tensors, workspace) and streams.  If the
library is missing this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libgbhegv.so")

GBHE_EWORKSPACE = -101
GBHE_ECUDA = -102
GBHE_ETIMEOUT = -103
GBHE_ENONFINITE = -104
GBHE_ENOTCONV = -105


class GbheError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__("%s failed: %d (%s)" % (fn, code, status_string(code)))


class _Cplx(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIBPATH):
            raise RuntimeError("libgbhegv.so not built (run __graft_entry__.build() or "
                               "python paper_1207_1773_gb300/build.py)")
        lib = ctypes.CDLL(_LIBPATH)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        sig = {
            "gbhe_create": ([ctypes.POINTER(P), I], I),
            "gbhe_destroy": ([P], I),
            "gbhe_workspace_size": ([P, I, I, I, ctypes.POINTER(S)], I),
            "gbhe_set_workspace": ([P, P, S], I),
            "gbhe_get_status": ([P, P], I),
            "gbhe_sync_status": ([P, P], I),
            "gbhe_crt_tables": ([P, P, P, P, P, P, P], I),
            "gbhe_default_nb": ([I], I),
            "gbhe_potrf": ([P, I, P, I, P], I),
            "gbhe_hegst": ([P, I, P, I, P, I, P], I),
            "gbhe_he2hb": ([P, I, I, P, I, P, P, P], I),
            "gbhe_hb2st_sizes": ([I, I, ctypes.POINTER(S), ctypes.POINTER(S)], I),
            "gbhe_hb2st": ([P, I, I, P, I, P, P, P, P, P], I),
            "gbhe_stedc": ([P, I, P, P, I, I, P, P, I, P], I),
            "gbhe_unmtr_2stage": ([P, I, I, I, P, I, P, P, P, P, I, P, I, P], I),
            "gbhe_trsm_lh": ([P, I, I, P, I, P, I, P], I),
            "gbhe_hegv": ([P, I, I, P, I, P, I, I, I, P, P, I, P], I),
            "gbhe_hegv_onestage": ([P, I, P, I, P, I, I, I, P, P, I, P], I),
            "gbhe_status_string": ([I], ctypes.c_char_p),
            "gbhe_zgemm": ([P, I, I, I, I, I, _Cplx, P, I, P, I, _Cplx, P, I, I, P], I),
            "gbhe_crt_workspace_size": ([I, I, I, I, ctypes.POINTER(S)], I),
            "gbhe_set_gemm_engine": ([P, I], I),
            "gbhe_set_crt_block": ([P, I], I),
            "gbhe_gemm_crt": ([P, I, I, I, I, I, I, _Cplx, P, I, P, I, _Cplx, P, I, I, P], I),
            "gbhe_launch_count": ([], ctypes.c_ulonglong),
            "gbhe_profile_enable": ([I], I),
            "gbhe_profile_read": ([I, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I),
            "gbhe_probe_fp64_peaks": ([I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I),
            "gbhe_zgemm_static": ([I, I, I, I, I, _Cplx, P, I, P, I, _Cplx, P, I, I, P], I),
            "gbhe_batched_plan": ([I, I, P, P], I),
            "gbhe_hegv_adjoint": ([P, I, I, I, P, P, I, P, P, I, ctypes.c_double, P, I, P, I, P], I),
            "gbhe_hegv_batched": ([P, P, I, I, P, P, P, P, P, P, P, P, P, P, P, P], I),
            "gbhe_nb_rule_pick": ([I, P, P, P, I, I, ctypes.POINTER(I)], I),
            "gbhe_set_nb_rule": ([P, I, P, P, P], I),
            "gbhe_resolve_nb": ([P, I, I, ctypes.POINTER(I)], I),
            "gbhe_wait_selftest": ([P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def library_path() -> str:
    return _LIBPATH


def exported_symbols():
    return [n for n in ("gbhe_create", "gbhe_destroy", "gbhe_workspace_size", "gbhe_set_workspace",
                        "gbhe_get_status", "gbhe_default_nb", "gbhe_potrf", "gbhe_hegst", "gbhe_he2hb",
                        "gbhe_hb2st_sizes", "gbhe_hb2st", "gbhe_stedc", "gbhe_unmtr_2stage",
                        "gbhe_trsm_lh", "gbhe_hegv", "gbhe_hegv_onestage", "gbhe_status_string",
                        "gbhe_zgemm", "gbhe_launch_count", "gbhe_profile_enable", "gbhe_profile_read",
                        "gbhe_probe_fp64_peaks", "gbhe_crt_workspace_size", "gbhe_gemm_crt",
                        "gbhe_set_gemm_engine", "gbhe_zgemm_static", "gbhe_set_crt_block",
                        "gbhe_batched_plan", "gbhe_hegv_batched", "gbhe_hegv_adjoint",
                        "gbhe_nb_rule_pick", "gbhe_set_nb_rule", "gbhe_resolve_nb", "gbhe_wait_selftest",
                        "gbhe_sync_status", "gbhe_crt_tables")]


def status_string(code: int) -> str:
    return _load().gbhe_status_string(int(code)).decode()


def _check(fn, rc):
    if rc != 0:
        raise GbheError(fn, rc)


def _ptr(t):
    """Device address of a CUDA tensor (None gives NULL).  Host tensors are
    refused: the library would read their addresses as device memory."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("gbhegv takes CUDA tensors only (got a %s tensor)" % t.device.type)
    return ctypes.c_void_p(t.data_ptr())


C128, F64 = torch.complex128, torch.float64


def _square(*ts):
    """All are n x n matrices with one n; returns n."""
    n = ts[0].shape[0] if ts[0].dim() == 2 else -1
    for t in ts:
        if t.dim() != 2 or t.shape[0] != n or t.shape[1] != n:
            raise ValueError("gbhegv: expected %d x %d matrices, got %s" % (n, n, tuple(t.shape)))
    return n


def _block(t, n, m, name):
    """t holds an n x m column-major block (at least)."""
    if t.dim() != 2 or t.shape[0] != n or t.shape[1] < m:
        raise ValueError("gbhegv: %s must be %d x %d, got %s" % (name, n, m, tuple(t.shape)))


def _gemm_dims(opA, opB, A, B, C):
    """(m, n, k) of C = op(A) op(B) + C with every operand's stored shape
    checked against them: the C-ABI sees only pointers and leading dimensions,
    so an operand too small for (opA, opB, m, n, k) would be read past its end."""
    if opA not in OPS or opB not in ("N", "T", "C"):
        raise ValueError("gbhegv: operand modes %r, %r" % (opA, opB))
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t.dim() != 2:
            raise ValueError("gbhegv: %s must be a matrix, got %s" % (name, tuple(t.shape)))
    m, n = C.shape
    k = A.shape[1] if opA in ("N", "H") else A.shape[0]
    want_a = (m, k) if opA in ("N", "H") else (k, m)
    want_b = (k, n) if opB == "N" else (n, k)
    if tuple(A.shape) != want_a or (opA == "H" and m != k):
        raise ValueError("gbhegv: op%s(A) must be %d x %d for C %d x %d, A is %s"
                         % (opA, m, k, m, n, tuple(A.shape)))
    if tuple(B.shape) != want_b:
        raise ValueError("gbhegv: op%s(B) must be %d x %d for C %d x %d, B is %s"
                         % (opB, k, n, m, n, tuple(B.shape)))
    return m, n, k


def _want(dtype, device, *ts):
    """Every tensor is a CUDA tensor of `dtype` on `device` (the library reads
    each as that element type on the handle's device)."""
    for t in ts:
        if not t.is_cuda:
            raise ValueError("gbhegv takes CUDA tensors only (got a %s tensor)" % t.device.type)
        if t.dtype != dtype:
            raise TypeError("gbhegv: expected %s, got %s" % (dtype, t.dtype))
        if t.device != device:
            raise ValueError("gbhegv: tensors on %s and %s" % (device, t.device))


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _cuda_device(device):
    """torch.device of a CUDA device with its index (None: the current one)."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    if dev.type != "cuda":
        raise ValueError("gbhegv runs on CUDA devices only")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    return dev


class Handle:
    """A library handle on one device plus a torch-allocated workspace."""

    def __init__(self, device=None):
        dev = _cuda_device(device)
        self.device = dev
        lib = _load()
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check("gbhe_create", lib.gbhe_create(ctypes.byref(h), dev.index or 0))
        self.h = h
        self.work = None
        self.work_bytes = 0

    def close(self):
        if self.h:
            _load().gbhe_destroy(self.h)
            self.h = None
            self.work = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_size(self, n, nb=0, m=None):
        m = n if m is None else m
        b = ctypes.c_size_t()
        _check("gbhe_workspace_size", _load().gbhe_workspace_size(self.h, int(n), int(nb), int(m), ctypes.byref(b)))
        return int(b.value)

    def ensure_workspace(self, n, nb=0, m=None):
        return self.ensure_bytes(self.workspace_size(n, nb, m))

    def ensure_bytes(self, need):
        if self.work is None or self.work_bytes < need:
            self.work = None
            torch.cuda.synchronize(self.device)
            self.work = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.work_bytes = need
            _check("gbhe_set_workspace", _load().gbhe_set_workspace(self.h, _ptr(self.work), ctypes.c_size_t(need)))
        return self.work

    def status(self):
        return int(_load().gbhe_get_status(self.h, _stream(self.device)))

    def set_nb_rule(self, rule):
        """Install a band-width rule, a list of (n_max, frac_max, nb) entries
        (empty: the default band width everywhere)."""
        cnt, nm, fm, nbs = _rule_arrays(rule)
        _check("gbhe_set_nb_rule", _load().gbhe_set_nb_rule(self.h, cnt, nm, fm, nbs))

    def resolve_nb(self, n, m=None):
        """The band width nb = 0 selects on this handle for order n and m pairs."""
        m = n if m is None else m
        out = ctypes.c_int()
        _check("gbhe_resolve_nb", _load().gbhe_resolve_nb(self.h, int(n), int(m), ctypes.byref(out)))
        return out.value


def _rule_arrays(rule):
    rule = list(rule)
    k = max(len(rule), 1)
    nm = (ctypes.c_int * k)(*[int(e[0]) for e in rule])
    fm = (ctypes.c_double * k)(*[float(e[1]) for e in rule])
    nbs = (ctypes.c_int * k)(*[int(e[2]) for e in rule])
    return len(rule), nm, fm, nbs


def nb_rule_pick(rule, n, m=None):
    """Band width a rule of (n_max, frac_max, nb) entries gives for order n and
    m selected pairs (host-only; the same lookup nb = 0 does on a handle)."""
    m = n if m is None else m
    cnt, nm, fm, nbs = _rule_arrays(rule)
    out = ctypes.c_int()
    _check("gbhe_nb_rule_pick", _load().gbhe_nb_rule_pick(cnt, nm, fm, nbs, int(n), int(m), ctypes.byref(out)))
    return out.value


_handles = {}


def handle(device=None) -> Handle:
    dev = _cuda_device(device)
    key = dev.index
    if key not in _handles:
        _handles[key] = Handle(dev)
    return _handles[key]


def _ld(t):
    """Leading dimension of a column-major 2-D tensor (a transposed row-major view)."""
    if t.dim() == 1:
        return max(t.shape[0], 1)
    if t.stride(0) != 1:
        raise ValueError("matrices must be column-major (use t.t().contiguous().t() or torch_colmajor)")
    return max(t.stride(1), t.shape[0], 1)


def colmajor(x, device=None, dtype=None):
    """Column-major copy of a numpy array or tensor on the device."""
    t = torch.as_tensor(x)
    if dtype is not None:
        t = t.to(dtype)
    if device is not None:
        t = t.to(device)
    if t.dim() == 2:
        return t.t().contiguous().t()
    return t.contiguous()


def _sync_status(h, fn):
    st = h.status()
    if st != 0:
        raise GbheError(fn, st)


# ----------------------------------------------------------------- stages
def potrf(B, check=True):
    h = handle(B.device)
    _want(C128, B.device, B)
    n = _square(B)
    h.ensure_workspace(n)
    _check("gbhe_potrf", _load().gbhe_potrf(h.h, n, _ptr(B), _ld(B), _stream(B.device)))
    return h.status() if check else 0


def hegst(A, L):
    h = handle(A.device)
    _want(C128, A.device, A, L)
    n = _square(A, L)
    h.ensure_workspace(n)
    _check("gbhe_hegst", _load().gbhe_hegst(h.h, n, _ptr(A), _ld(A), _ptr(L), _ld(L), _stream(A.device)))


def he2hb(A, nb):
    """Returns (T1, tau1); A is overwritten by band + V1."""
    h = handle(A.device)
    _want(C128, A.device, A)
    n = _square(A)
    h.ensure_workspace(n, nb)
    npan = max((n + nb - 1) // nb, 1)
    T1 = torch.zeros(npan * nb * nb, dtype=torch.complex128, device=A.device)
    tau1 = torch.zeros(max(n, 1), dtype=torch.complex128, device=A.device)
    _check("gbhe_he2hb", _load().gbhe_he2hb(h.h, n, nb, _ptr(A), _ld(A), _ptr(T1), _ptr(tau1), _stream(A.device)))
    _sync_status(h, "gbhe_he2hb")
    return T1, tau1


def hb2st_sizes(n, nb):
    v, t = ctypes.c_size_t(), ctypes.c_size_t()
    _check("gbhe_hb2st_sizes", _load().gbhe_hb2st_sizes(n, nb, ctypes.byref(v), ctypes.byref(t)))
    return int(v.value), int(t.value)


def hb2st(A, nb):
    """Returns (d, e, V2, tau2) from the lower band of A."""
    h = handle(A.device)
    _want(C128, A.device, A)
    n = _square(A)
    h.ensure_workspace(n, nb)
    nv, nt = hb2st_sizes(n, nb)
    d = torch.zeros(max(n, 1), dtype=torch.float64, device=A.device)
    e = torch.zeros(max(n, 1), dtype=torch.float64, device=A.device)
    V2 = torch.zeros(max(nv, 1), dtype=torch.complex128, device=A.device)
    tau2 = torch.zeros(max(nt, 1), dtype=torch.complex128, device=A.device)
    _check("gbhe_hb2st", _load().gbhe_hb2st(h.h, n, nb, _ptr(A), _ld(A), _ptr(d), _ptr(e), _ptr(V2), _ptr(tau2),
                                            _stream(A.device)))
    _sync_status(h, "gbhe_hb2st")
    return d[:n], e[:max(n - 1, 0)], V2, tau2


def stedc(d, e, il=1, iu=None):
    """Eigenpairs il..iu of the real symmetric tridiagonal (d, e): (w, Z)."""
    h = handle(d.device)
    _want(F64, d.device, d, e)
    n = d.shape[0]
    iu = n if iu is None else iu
    m = iu - il + 1
    h.ensure_workspace(n, 0, m)
    w = torch.zeros(max(m, 1), dtype=torch.float64, device=d.device)
    Z = torch.zeros((max(m, 1), n), dtype=torch.float64, device=d.device).t()
    e_ = e if e.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=d.device)
    _check("gbhe_stedc", _load().gbhe_stedc(h.h, n, _ptr(d), _ptr(e_), il, iu, _ptr(w), _ptr(Z), max(n, 1),
                                            _stream(d.device)))
    _sync_status(h, "gbhe_stedc")
    return w[:m], Z[:, :m]


def unmtr_2stage(nb, A, T1, V2, tau2, Z):
    h = handle(A.device)
    _want(C128, A.device, A, T1, V2, tau2)
    _want(F64, A.device, Z)
    n, m = Z.shape
    if _square(A) != n:
        raise ValueError("gbhegv: Z must have %d rows, got %d" % (A.shape[0], n))
    h.ensure_workspace(n, nb, m)
    X = torch.zeros((max(m, 1), n), dtype=torch.complex128, device=A.device).t()
    _check("gbhe_unmtr_2stage", _load().gbhe_unmtr_2stage(h.h, n, nb, m, _ptr(A), _ld(A), _ptr(T1), _ptr(V2),
                                                          _ptr(tau2), _ptr(Z), _ld(Z), _ptr(X), max(n, 1),
                                                          _stream(A.device)))
    _sync_status(h, "gbhe_unmtr_2stage")
    return X[:, :m]


def trsm_lh(L, X):
    h = handle(L.device)
    _want(C128, L.device, L, X)
    n, m = X.shape
    if _square(L) != n:
        raise ValueError("gbhegv: X must have %d rows, got %d" % (L.shape[0], n))
    h.ensure_workspace(n, 0, m)
    _check("gbhe_trsm_lh", _load().gbhe_trsm_lh(h.h, n, m, _ptr(L), _ld(L), _ptr(X), _ld(X), _stream(L.device)))


PROF_CLASSES = {"zgemm": 0, "dgemm": 1, "panel": 2, "chase": 3, "q2": 4, "stedc": 5, "hemv": 6, "crt": 7,
                "crt_prep": 8, "crt_mma": 9, "crt_rec": 10}


def crt_tables():
    """The tensor-core FP64 engine's tables (host-only): dict of p, W, M as
    Python ints (W and M joined from their 32-bit words), the signed limb
    weights k13, k26, k39 and frac as the float32 values the device uses."""
    k = 16
    p = (ctypes.c_int * k)()
    W = (ctypes.c_uint * (4 * k))()
    M = (ctypes.c_uint * 4)()
    k13, k26, k39 = (ctypes.c_int * k)(), (ctypes.c_int * k)(), (ctypes.c_int * k)()
    frac = (ctypes.c_float * k)()
    nmod = _load().gbhe_crt_tables(p, W, M, k13, k26, k39, frac)
    if nmod != k:
        raise RuntimeError("unexpected number of moduli %d" % nmod)

    def join(words):
        return sum(int(x) << (32 * i) for i, x in enumerate(words))

    return {"p": list(p), "W": [join(W[4 * l:4 * l + 4]) for l in range(k)], "M": join(M[:]),
            "k13": list(k13), "k26": list(k26), "k39": list(k39), "frac": list(frac)}


def wait_selftest(device=None):
    """Run the bounded-wait self-test on the handle of `device` and return the
    status it leaves (GBHE_ETIMEOUT = -103 when the wait expired as designed;
    the status is cleared)."""
    h = handle(device)
    _check("gbhe_wait_selftest", _load().gbhe_wait_selftest(h.h, _stream(h.device)))
    return h.status()


def launch_count() -> int:
    return int(_load().gbhe_launch_count())


def profile_enable(on=True):
    _check("gbhe_profile_enable", _load().gbhe_profile_enable(int(bool(on))))


def profile_read():
    """Per kernel class: dict(launches, flops, bytes, ms)."""
    out = {}
    for name, cls in PROF_CLASSES.items():
        L, F, B, M = ctypes.c_ulonglong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check("gbhe_profile_read", _load().gbhe_profile_read(cls, ctypes.byref(L), ctypes.byref(F),
                                                              ctypes.byref(B), ctypes.byref(M)))
        out[name] = {"launches": int(L.value), "flops": F.value, "bytes": B.value, "ms": M.value}
    return out


def probe_fp64_peaks(device=0):
    """Live FP64 peaks (TFLOP/s): (DFMA pipe, DMMA m16n8k4 tensor pipe)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check("gbhe_probe_fp64_peaks", _load().gbhe_probe_fp64_peaks(int(device), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


OPS = {"N": 0, "T": 1, "C": 2, "H": 3}
ENGINES = {"dmma": 0, "crt": 1}


def set_engine(name, device=None):
    """Engine of the FP64 level-3 products: 'crt' (FP16 tensor cores, exact
    modular arithmetic; default) or 'dmma' (FP64 tensor pipe only)."""
    h = handle(device)
    _check("gbhe_set_gemm_engine", _load().gbhe_set_gemm_engine(h.h, ENGINES[name]))
    h.engine = name


def set_crt_block(block=16384, device=None):
    """Largest block of one tensor-core GEMM call (128..16384); smaller blocks
    need less workspace and run slower."""
    h = handle(device)
    _check("gbhe_set_crt_block", _load().gbhe_set_crt_block(h.h, int(block)))


def zgemm(opA, opB, A, B, C, alpha=1.0, beta=0.0, lower=False):
    """C = alpha op(A) op(B) + beta C through the library's GEMM engine (in place)."""
    _want(C128, C.device, A, B, C)
    m, n, k = _gemm_dims(opA, opB, A, B, C)
    h = handle(C.device)
    h.ensure_workspace(max(m, n, k), 1, 1)
    a, b = complex(alpha), complex(beta)
    _check("gbhe_zgemm", _load().gbhe_zgemm(h.h, OPS[opA], OPS[opB], m, n, k, _Cplx(a.real, a.imag), _ptr(A),
                                            _ld(A), _ptr(B), _ld(B), _Cplx(b.real, b.imag), _ptr(C), _ld(C),
                                            int(bool(lower)), _stream(C.device)))
    return C


def zgemm_static(opA, opB, A, B, C, alpha=1.0, beta=0.0, lower=False):
    """C = alpha op(A) op(B) + beta C on the DMMA GEMM with split-K scratch in
    the library's static array (no handle, no workspace), in place.  Calls
    must not overlap in time on one device; m * n <= 2**18."""
    _want(C128, C.device, A, B, C)
    m, n, k = _gemm_dims(opA, opB, A, B, C)
    a, b = complex(alpha), complex(beta)
    with torch.cuda.device(C.device):
        _check("gbhe_zgemm_static",
               _load().gbhe_zgemm_static(OPS[opA], OPS[opB], m, n, k, _Cplx(a.real, a.imag), _ptr(A), _ld(A),
                                         _ptr(B), _ld(B), _Cplx(b.real, b.imag), _ptr(C), _ld(C),
                                         int(bool(lower)), _stream(C.device)))
    return C


def gemm_crt(opA, opB, A, B, C, alpha=1.0, beta=0.0, lower=False):
    """C = alpha op(A) op(B) + beta C computed exactly-modularly on the FP16
    tensor cores (complex128 or float64 operands), in place."""
    if C.dtype not in (C128, F64):
        raise TypeError("gbhegv: expected complex128 or float64, got %s" % C.dtype)
    _want(C.dtype, C.device, A, B, C)
    cplx = 1 if C.dtype == torch.complex128 else 0
    m, n, k = _gemm_dims(opA, opB, A, B, C)
    h = handle(C.device)
    need = ctypes.c_size_t()
    _check("gbhe_crt_workspace_size", _load().gbhe_crt_workspace_size(m, n, k, cplx, ctypes.byref(need)))
    h.ensure_bytes(h.workspace_size(1) + int(need.value) + 4096)
    a, b = complex(alpha), complex(beta)
    _check("gbhe_gemm_crt", _load().gbhe_gemm_crt(h.h, cplx, OPS[opA], OPS[opB], m, n, k, _Cplx(a.real, a.imag),
                                                  _ptr(A), _ld(A), _ptr(B), _ld(B), _Cplx(b.real, b.imag), _ptr(C),
                                                  _ld(C), int(bool(lower)), _stream(C.device)))
    return C


def hegv_adjoint(w_all, X_all, il, iu, gw, gX, delta):
    """dL/dA and dL/dB (n x n Hermitian, column-major) of the eigenpairs
    il..iu from the whole decomposition (w_all, X_all) and the cotangents
    gw (m) and gX (n x m); see gbhe_hegv_adjoint."""
    _want(F64, X_all.device, w_all, gw)
    _want(C128, X_all.device, X_all, gX)
    n = _square(X_all)
    if not (1 <= il <= iu <= n):
        raise ValueError("gbhegv: need 1 <= il <= iu <= n = %d, got il=%d iu=%d" % (n, il, iu))
    m = iu - il + 1
    if w_all.numel() < n:
        raise ValueError("gbhegv: w_all holds %d values, needs %d" % (w_all.numel(), n))
    if gw.numel() < m:
        raise ValueError("gbhegv: gw holds %d values, needs %d" % (gw.numel(), m))
    _block(gX, n, m, "gX")
    h = handle(X_all.device)
    h.ensure_workspace(n, 0, m)
    dA = torch.empty((n, n), dtype=torch.complex128, device=X_all.device).t()
    dB = torch.empty((n, n), dtype=torch.complex128, device=X_all.device).t()
    gw = gw.contiguous()
    _check("gbhe_hegv_adjoint", _load().gbhe_hegv_adjoint(h.h, n, il, iu, _ptr(w_all), _ptr(X_all), _ld(X_all),
                                                          _ptr(gw), _ptr(gX), _ld(gX), float(delta), _ptr(dA),
                                                          _ld(dA), _ptr(dB), _ld(dB), _stream(X_all.device)))
    return dA, dB


def _int_array(vals):
    return (ctypes.c_int * max(len(vals), 1))(*[int(v) for v in vals])


def _ptr_array(ts):
    return (ctypes.c_void_p * max(len(ts), 1))(*[_ptr(t).value for t in ts])


def batched_plan(ns, nworkers):
    """Worker index of every problem (largest first, least n^3 work so far)."""
    out = (ctypes.c_int * max(len(ns), 1))()
    _check("gbhe_batched_plan", _load().gbhe_batched_plan(int(nworkers), len(ns), _int_array(ns), out))
    return [out[i] for i in range(len(ns))]


class BatchPool:
    """Worker streams, one handle each, and their workspaces for
    hegv_batched; sized by prepare() for a set of problem shapes."""

    def __init__(self, nworkers=4, device=None):
        dev = _cuda_device(device)
        self.device = dev
        self.handles = [Handle(dev) for _ in range(nworkers)]
        self.streams = [torch.cuda.Stream(dev) for _ in range(nworkers)]

    def prepare(self, ns, nbs, ms):
        assign = batched_plan(ns, len(self.handles))
        for k, h in enumerate(self.handles):
            need = 0
            for i, a in enumerate(assign):
                if a == k:
                    need = max(need, h.workspace_size(ns[i], nbs[i], ms[i]))
            if need:
                h.ensure_bytes(need)
        return assign


def hegv_batched(pool, As, Bs, ils, ius, nbs, ws, Xs):
    """Solve every A_i x = lambda B_i x for eigenpairs il_i..iu_i on the pool's
    worker streams, ordered on the current stream (capturable).  A_i, B_i
    (overwritten), the eigenvalue vectors ws[i] and the eigenvector blocks
    Xs[i] (n_i x m_i, column-major) are caller-owned CUDA tensors."""
    cnt = len(As)
    _want(C128, pool.device, *As, *Bs, *Xs)
    _want(F64, pool.device, *ws)
    if not len(Bs) == len(Xs) == len(ws) == len(ils) == len(ius) == len(nbs) == cnt:
        raise ValueError("gbhegv: one entry per problem in every list")
    for a, b, x, w, il, iu in zip(As, Bs, Xs, ws, ils, ius):
        n = _square(a, b)
        m = max(iu - il + 1, 0)
        _block(x, n, m, "X_i")
        if w.numel() < m:
            raise ValueError("gbhegv: w_i holds %d values, needs %d" % (w.numel(), m))
    ns = [a.shape[0] for a in As]
    hs = (ctypes.c_void_p * len(pool.handles))(*[h.h.value for h in pool.handles])
    strm = (ctypes.c_void_p * len(pool.streams))(*[s.cuda_stream for s in pool.streams])
    _check("gbhe_hegv_batched", _load().gbhe_hegv_batched(
        hs, strm, len(pool.handles), cnt, _int_array(ns), _int_array(nbs), _ptr_array(As),
        _int_array([_ld(a) for a in As]), _ptr_array(Bs), _int_array([_ld(b) for b in Bs]), _int_array(ils),
        _int_array(ius), _ptr_array(ws), _ptr_array(Xs), _int_array([max(_ld(x), a.shape[0]) for x, a in zip(Xs, As)]),
        _stream(pool.device)))


def hegv(A, B, il=1, iu=None, nb=0, onestage=False, check=True):
    """Eigenpairs il..iu (1-based, inclusive) of A x = lambda B x.

    A, B: column-major complex128 CUDA tensors (lower triangles read), both
    overwritten.  Returns (w, X) with X B-orthonormal."""
    h = handle(A.device)
    _want(C128, A.device, A, B)
    n = _square(A, B)
    iu = n if iu is None else iu
    m = iu - il + 1
    nbu = nb if nb else (h.resolve_nb(n, m) if 0 <= m <= n else _load().gbhe_default_nb(n))
    h.ensure_workspace(n, nbu, m)
    w = torch.zeros(max(m, 1), dtype=torch.float64, device=A.device)
    X = torch.zeros((max(m, 1), n), dtype=torch.complex128, device=A.device).t()
    st = _stream(A.device)
    if onestage:
        rc = _load().gbhe_hegv_onestage(h.h, n, _ptr(A), _ld(A), _ptr(B), _ld(B), il, iu, _ptr(w), _ptr(X),
                                        max(n, 1), st)
        _check("gbhe_hegv_onestage", rc)
    else:
        rc = _load().gbhe_hegv(h.h, n, nbu, _ptr(A), _ld(A), _ptr(B), _ld(B), il, iu, _ptr(w), _ptr(X),
                               max(n, 1), st)
        _check("gbhe_hegv", rc)
    if check:
        _sync_status(h, "gbhe_hegv")
    return w[:m], X[:, :m]
