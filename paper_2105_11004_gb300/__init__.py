"""GB300 (sm_103a) rank-revealing leverage-score estimator -- Python binding.

A thin ctypes layer over ``liblev.so`` (the C ABI of ``include/lev.h``). The
functions keep the C names (``lev_sketch_dense``, ``lev_rrqr``, ...); they take
torch tensors, pass their device pointers and the current CUDA stream, and
translate status codes into ``LevError``. Every step of the method runs in the
library's CUDA kernels: there is no Python or CPU fallback, and importing this
package fails if ``liblev.so`` has not been built (``build.build()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB_PATH, build as build_library  # noqa: F401

LEV_OK, LEV_EINVAL, LEV_ENOMEM, LEV_ECUDA, LEV_ETIMEOUT, LEV_ERANK0 = 0, 1, 2, 3, 4, 5
LEV_FP32, LEV_TF32, LEV_BF16, LEV_BF16X3 = 0, 1, 2, 3
LEV_OMEGA_IDENTITY, LEV_SKETCH_IDENTITY, LEV_FORCE_PIVOTS, LEV_HOST_ASYNC, LEV_SKETCH_SRHT = 1, 2, 4, 8, 16
LEV_RANK_SVD, LEV_SRRQR, LEV_CSR_UNCHECKED, LEV_OMEGA_REDUCED = 32, 64, 128, 256
PRECISIONS = {"fp32": LEV_FP32, "tf32": LEV_TF32, "bf16": LEV_BF16, "bf16x3": LEV_BF16X3}

# Every symbol include/lev.h declares, with (restype, argtypes).
_c_void_p, _i64, _i32, _u32, _u64, _dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)


class lev_params(ctypes.Structure):
    _fields_ = [
        ("eps", _dbl), ("delta", _dbl), ("gamma", _dbl),
        ("s", _i64), ("m", _i64), ("k", _i64),
        ("tau", _dbl), ("seed", _u64),
        ("sketch_prec", _i32), ("final_prec", _i32), ("flags", _u32), ("srht_t", _i32),
        ("perm_in", _c_void_p), ("rank_in", _i64),
        ("row0", _i64), ("n_total", _i64), ("phi", _dbl),
    ]


_P = ctypes.POINTER
SIGNATURES = {
    "lev_create": (ctypes.c_int, [_P(_c_void_p), ctypes.c_int]),
    "lev_destroy": (ctypes.c_int, [_c_void_p]),
    "lev_last_error": (ctypes.c_char_p, []),
    "lev_workspace_bytes": (ctypes.c_int, [_c_void_p, _P(_i64)]),
    "lev_params_init": (ctypes.c_int, [_P(lev_params)]),
    "lev_resolve_sizes": (ctypes.c_int, [_P(lev_params), _i64, _i64, _P(_i64), _P(_i64), _P(_i64)]),
    "lev_prepare": (ctypes.c_int, [_c_void_p, _i64, _i64, _P(lev_params), _c_void_p]),
    "lev_exact_reference_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _dbl, _c_void_p, _P(_i64),
                                                 _c_void_p, _c_void_p]),
    "lev_exact_reference_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64, _dbl,
                                               _c_void_p, _P(_i64), _c_void_p, _c_void_p]),
    "lev_sketch_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params), _c_void_p, _c_void_p]),
    "lev_sketch_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64,
                                      _P(lev_params), _c_void_p, _c_void_p]),
    "lev_rrqr": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _dbl, _c_void_p, _c_void_p, _P(_i64), _c_void_p]),
    "lev_omega_factor": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _u64, _u32,
                                        _c_void_p, _c_void_p]),
    "lev_final_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _c_void_p, _i64, _i32, _c_void_p,
                                       _c_void_p]),
    "lev_final_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64, _c_void_p,
                                     _i64, _i32, _c_void_p, _c_void_p]),
    "lev_estimate_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params), _c_void_p,
                                          _P(_i64), _c_void_p, _c_void_p]),
    "lev_estimate_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64,
                                        _P(lev_params), _c_void_p, _P(_i64), _c_void_p, _c_void_p]),
    "lev_backward_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params), _c_void_p,
                                          _c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p,
                                          _c_void_p]),
    "lev_device_status": (ctypes.c_int, [_c_void_p, _P(_i32)]),
    "lev_exact_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params), _c_void_p, _P(_i64),
                                       _c_void_p, _c_void_p]),
    "lev_exact_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params),
                                     _c_void_p, _P(_i64), _c_void_p, _c_void_p]),
    "lev_rrqr_select": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _P(lev_params), _c_void_p, _c_void_p,
                                       _P(_i64), _c_void_p, _P(_i64), _c_void_p]),
    "lev_precondition_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _P(lev_params), _c_void_p,
                                              _P(_i64), _c_void_p, _c_void_p]),
    "lev_precondition_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64,
                                            _P(lev_params), _c_void_p, _P(_i64), _c_void_p, _c_void_p]),
    "lev_lsqr_dense": (ctypes.c_int, [_c_void_p, _c_void_p, _i64, _i64, _i64, _c_void_p, _i64, _c_void_p, _c_void_p,
                                      _i32, _dbl, _dbl, _P(_i32), _P(_dbl), _c_void_p]),
    "lev_rank_stats": (ctypes.c_int, [_c_void_p, _P(_i64), _P(_i32)]),
    "lev_lsqr_csr": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i64, _i64, _i64, _c_void_p, _i64,
                                    _c_void_p, _c_void_p, _i32, _dbl, _dbl, _P(_i32), _P(_dbl), _c_void_p]),
    "lev_set_timing": (ctypes.c_int, [_c_void_p, ctypes.c_int]),
    "lev_rrqr_timing": (ctypes.c_int, [_c_void_p, _P(ctypes.c_float), _P(ctypes.c_float)]),
    "lev_final_timing": (ctypes.c_int, [_c_void_p, _P(ctypes.c_float)]),
    "lev_rrqr_noalloc": (ctypes.c_int, [_c_void_p, _i64, _i64, _dbl, _c_void_p, _c_void_p, _P(_i64), _c_void_p]),
}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"liblev.so is not built ({LIB_PATH}); run paper_2105_11004_gb300.build.build()")
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class LevError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[lev status {code}] {msg}")
        self.code = code


def _check(rc, allow=()):
    if rc != LEV_OK and rc not in allow:
        raise LevError(rc, lib.lev_last_error().decode(errors="replace"))
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Owns one lev_handle (scratch memory, G cache) on a CUDA device."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib.lev_create(ctypes.byref(self._h), int(device)))
        self.device = int(device)

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            lib.lev_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_tls = threading.local()


def default_handle(device: int = 0) -> Handle:
    """The calling thread's handle on `device`, created on first use. A handle serves one host
    thread at a time (include/lev.h), so host threads do not share their default handles."""
    handles = getattr(_tls, "handles", None)
    if handles is None:
        handles = _tls.handles = {}
    h = handles.get(device)
    if h is None:
        h = handles[device] = Handle(device)
    return h


def make_params(s=0, m=0, k=0, tau=1e-5, seed=0, sketch_prec="fp32", final_prec="fp32", eps=0.5,
                delta=1.0 / 3.0, gamma=2.0, omega_identity=False, sketch_identity=False,
                perm_in=None, rank_in=0, host_async=False, srht_t=0, row0=0, n_total=0, rank_svd=False,
                srrqr_phi=0.0) -> lev_params:
    p = lev_params()
    _check(lib.lev_params_init(ctypes.byref(p)))
    p.eps, p.delta, p.gamma = eps, delta, gamma
    p.s, p.m, p.k, p.tau, p.seed = int(s), int(m), int(k), float(tau), int(seed)
    p.sketch_prec = PRECISIONS[sketch_prec] if isinstance(sketch_prec, str) else int(sketch_prec)
    p.final_prec = PRECISIONS[final_prec] if isinstance(final_prec, str) else int(final_prec)
    flags = 0
    if omega_identity:
        flags |= LEV_OMEGA_IDENTITY
    if sketch_identity:
        flags |= LEV_SKETCH_IDENTITY
    if host_async:
        flags |= LEV_HOST_ASYNC
    if srht_t:
        flags |= LEV_SKETCH_SRHT
        p.srht_t = int(srht_t)
    if perm_in is not None:
        flags |= LEV_FORCE_PIVOTS
        p.perm_in = perm_in.data_ptr()
        p.rank_in = int(rank_in)
    if rank_svd:
        flags |= LEV_RANK_SVD
    if srrqr_phi:
        flags |= LEV_SRRQR
        p.phi = float(srrqr_phi)
    p.flags = flags
    p.row0, p.n_total = int(row0), int(n_total)
    return p


def lev_resolve_sizes(p: lev_params, n: int, d: int):
    s, m, k = _i64(), _i64(), _i64()
    _check(lib.lev_resolve_sizes(ctypes.byref(p), n, d, ctypes.byref(s), ctypes.byref(m), ctypes.byref(k)))
    return s.value, m.value, k.value


# ---- C-ABI entry points (torch tensors in, status-checked) ----

def lev_prepare(h: Handle, n: int, d: int, p: lev_params, stream=None):
    """Build the handle's caches (bucket permutation, G, Omega) for a call with (n, d, p)."""
    _check(lib.lev_prepare(h.ptr, n, d, ctypes.byref(p), _stream(stream)))


def lev_exact_reference_dense(h: Handle, A, tau, theta, perm=None, stream=None) -> int:
    """Exact leverage scores of dense A (device) by the Gram route; returns the rank."""
    n, d = A.shape
    r = _i64()
    rc = _check(lib.lev_exact_reference_dense(h.ptr, _ptr(A), n, d, A.stride(0), float(tau), _ptr(theta),
                                              ctypes.byref(r), _ptr(perm) if perm is not None else None,
                                              _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_exact_reference_csr(h: Handle, row_ptr, col, val, n, d, tau, theta, perm=None, stream=None) -> int:
    """Exact leverage scores of CSR A (device arrays) by the Gram route; returns the rank."""
    r = _i64()
    rc = _check(lib.lev_exact_reference_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(),
                                            float(tau), _ptr(theta), ctypes.byref(r),
                                            _ptr(perm) if perm is not None else None, _stream(stream)),
                allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_sketch_dense(h: Handle, A, p: lev_params, Atilde, stream=None):
    n, d = A.shape
    _check(lib.lev_sketch_dense(h.ptr, _ptr(A), n, d, A.stride(0), ctypes.byref(p), _ptr(Atilde), _stream(stream)))


def lev_sketch_csr(h: Handle, row_ptr, col, val, n, d, p: lev_params, Atilde, stream=None):
    _check(lib.lev_sketch_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(), ctypes.byref(p),
                              _ptr(Atilde), _stream(stream)))


def lev_rrqr(h: Handle, Atilde, tau, perm, R, stream=None) -> int:
    m, d = Atilde.shape
    r = _i64()
    rc = _check(lib.lev_rrqr(h.ptr, _ptr(Atilde), m, d, float(tau), _ptr(perm), _ptr(R), ctypes.byref(r),
                             _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_rrqr_select(h: Handle, Atilde, p: lev_params, perm, R, sigma=None, stream=None):
    """Pivoted QR with p's rank rule (LEV_RANK_SVD, LEV_SRRQR): returns (rank, swaps)."""
    m, d = Atilde.shape
    r, sw = _i64(), _i64()
    rc = _check(lib.lev_rrqr_select(h.ptr, _ptr(Atilde), m, d, ctypes.byref(p), _ptr(perm), _ptr(R), ctypes.byref(r),
                                    _ptr(sigma), ctypes.byref(sw), _stream(stream)), allow=(LEV_ERANK0,))
    return (0 if rc == LEV_ERANK0 else r.value), sw.value


def lev_precondition_dense(h: Handle, A, p: lev_params, N, sigma=None, stream=None) -> int:
    """Alg. 11: N (d x d FP64, device; first k columns) = V_k Sigma_k^{-1} of the sketch; returns k."""
    n, d = A.shape
    r = _i64()
    rc = _check(lib.lev_precondition_dense(h.ptr, _ptr(A), n, d, A.stride(0), ctypes.byref(p), _ptr(N),
                                           ctypes.byref(r), _ptr(sigma), _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_precondition_csr(h: Handle, row_ptr, col, val, n, d, p: lev_params, N, sigma=None, stream=None) -> int:
    r = _i64()
    rc = _check(lib.lev_precondition_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(),
                                         ctypes.byref(p), _ptr(N), ctypes.byref(r), _ptr(sigma), _stream(stream)),
                allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_lsqr_dense(h: Handle, A, N, k, b, x, max_iter=200, atol=1e-6, btol=1e-6, stream=None):
    """LSQR on min ||A N y - b||, x = N y (device FP64); returns (iterations, residual norm estimate)."""
    n, d = A.shape
    it, rn = _i32(), _dbl()
    _check(lib.lev_lsqr_dense(h.ptr, _ptr(A), n, d, A.stride(0), _ptr(N), int(k), _ptr(b), _ptr(x), int(max_iter),
                              float(atol), float(btol), ctypes.byref(it), ctypes.byref(rn), _stream(stream)))
    return it.value, rn.value


def lev_lsqr_csr(h: Handle, row_ptr, col, val, n, d, N, k, b, x, max_iter=200, atol=1e-6, btol=1e-6, stream=None):
    """LSQR on min ||A N y - b|| for CSR A, x = N y (device FP64); returns (iterations, residual estimate)."""
    it, rn = _i32(), _dbl()
    _check(lib.lev_lsqr_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(), _ptr(N), int(k), _ptr(b),
                            _ptr(x), int(max_iter), float(atol), float(btol), ctypes.byref(it), ctypes.byref(rn),
                            _stream(stream)))
    return it.value, rn.value


def lstsq(A, b, *, s=0, m=0, tau=1e-10, seed=0, sketch_prec="bf16x3", max_iter=200, atol=1e-6, btol=1e-6,
          handle: Handle | None = None):
    """min ||A x - b|| (dense FP32 A and b on a CUDA device): Alg. 11, then LSQR on A N.
    Returns (x FP64, rank, iterations, residual norm estimate)."""
    import torch
    h = handle or default_handle(A.device.index or 0)
    n, d = A.shape
    p = make_params(s=s, m=m, k=8, tau=tau, seed=seed, sketch_prec=sketch_prec)
    N = torch.empty((d, d), dtype=torch.float64, device=A.device)
    k = lev_precondition_dense(h, A, p, N)
    x = torch.zeros(d, dtype=torch.float64, device=A.device)
    if k == 0:                                          # A~ = 0: x = 0
        return x, 0, 0, None
    it, rn = lev_lsqr_dense(h, A, N, k, b, x, max_iter=max_iter, atol=atol, btol=btol)
    return x, k, it, rn


def lev_rank_stats(h: Handle):
    """(swaps, Jacobi sweeps) of the last rank-rule call on h."""
    sw, js = _i64(), _i32()
    _check(lib.lev_rank_stats(h.ptr, ctypes.byref(sw), ctypes.byref(js)))
    return sw.value, js.value


def lev_omega_factor(h: Handle, R, perm, d_rank, d, k, seed, flags, Mfull, stream=None):
    _check(lib.lev_omega_factor(h.ptr, _ptr(R), _ptr(perm), _ptr(d_rank), d, k, int(seed), int(flags), _ptr(Mfull),
                                _stream(stream)))


def lev_final_dense(h: Handle, A, Mfull, prec, theta, stream=None):
    n, d = A.shape
    k = Mfull.shape[1]
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib.lev_final_dense(h.ptr, _ptr(A), n, d, A.stride(0), _ptr(Mfull), k, prec, _ptr(theta),
                               _stream(stream)))


def lev_final_csr(h: Handle, row_ptr, col, val, n, d, Mfull, prec, theta, stream=None):
    k = Mfull.shape[1]
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(lib.lev_final_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(), _ptr(Mfull), k, prec,
                             _ptr(theta), _stream(stream)))


def lev_estimate_dense(h: Handle, A, p: lev_params, theta, perm=None, stream=None, want_rank=True):
    n, d = A.shape
    r = _i64(-1)
    rc = _check(lib.lev_estimate_dense(h.ptr, _ptr(A), n, d, A.stride(0), ctypes.byref(p), _ptr(theta),
                                       ctypes.byref(r) if want_rank else None, _ptr(perm), _stream(stream)),
                allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_exact_dense(h: Handle, A, p: lev_params, theta, perm=None, stream=None) -> int:
    """Alg. 7 (LS-HRN-exact) on a device matrix; returns the rank."""
    n, d = A.shape
    r = _i64(-1)
    rc = _check(lib.lev_exact_dense(h.ptr, _ptr(A), n, d, A.stride(0), ctypes.byref(p), _ptr(theta),
                                    ctypes.byref(r), _ptr(perm), _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_exact_csr(h: Handle, row_ptr, col, val, n, d, p: lev_params, theta, perm=None, stream=None) -> int:
    """Alg. 7 (LS-HRN-exact) on a device CSR matrix; returns the rank."""
    r = _i64(-1)
    rc = _check(lib.lev_exact_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(), ctypes.byref(p),
                                  _ptr(theta), ctypes.byref(r), _ptr(perm), _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_estimate_csr(h: Handle, row_ptr, col, val, n, d, p: lev_params, theta, perm=None, stream=None,
                     want_rank=True):
    r = _i64(-1)
    rc = _check(lib.lev_estimate_csr(h.ptr, _ptr(row_ptr), _ptr(col), _ptr(val), n, d, col.numel(),
                                     ctypes.byref(p), _ptr(theta), ctypes.byref(r) if want_rank else None,
                                     _ptr(perm), _stream(stream)), allow=(LEV_ERANK0,))
    return 0 if rc == LEV_ERANK0 else r.value


def lev_backward_dense(h: Handle, A, p: lev_params, Atilde, perm, d_rank, R, Mfull, w, gradA, stream=None):
    n, d = A.shape
    _check(lib.lev_backward_dense(h.ptr, _ptr(A), n, d, A.stride(0), ctypes.byref(p), _ptr(Atilde), _ptr(perm),
                                  _ptr(d_rank), _ptr(R), _ptr(Mfull), _ptr(w), _ptr(gradA), _stream(stream)))


def lev_rrqr_noalloc(Atilde, tau, perm, R, stream=None, want_rank: bool = True):
    """lev_rrqr without allocation (fixed device scratch; see include/lev.h). With want_rank=False
    no rank pointer is passed: the call only enqueues the work and returns None."""
    m, d = Atilde.shape
    r = _i64()
    rc = _check(lib.lev_rrqr_noalloc(_ptr(Atilde), m, d, float(tau), _ptr(perm), _ptr(R),
                                     ctypes.byref(r) if want_rank else None, _stream(stream)),
                allow=(LEV_ERANK0,))
    if not want_rank:
        return None
    return 0 if rc == LEV_ERANK0 else r.value


def lev_workspace_bytes(h: Handle) -> int:
    """Device memory the handle holds now (scratch and caches), in bytes."""
    b = _i64()
    _check(lib.lev_workspace_bytes(h.ptr, ctypes.byref(b)))
    return b.value


def lev_set_timing(h: Handle, enable: bool = True):
    _check(lib.lev_set_timing(h.ptr, 1 if enable else 0))


def lev_rrqr_timing(h: Handle):
    """(gram_ms, factor_ms) of the last pivoted QR on h since lev_set_timing(h, True)."""
    g, f = ctypes.c_float(), ctypes.c_float()
    _check(lib.lev_rrqr_timing(h.ptr, ctypes.byref(g), ctypes.byref(f)))
    return g.value, f.value


def lev_final_timing(h: Handle) -> float:
    """Duration (ms) of the main kernel of the last tensor-core dense final pass on h since
    lev_set_timing(h, True)."""
    f = ctypes.c_float()
    _check(lib.lev_final_timing(h.ptr, ctypes.byref(f)))
    return f.value


def lev_device_status(h: Handle) -> int:
    s = _i32()
    _check(lib.lev_device_status(h.ptr, ctypes.byref(s)))
    return s.value


# ---- convenience ----

def estimate(A, *, s=0, m=0, k=0, tau=1e-5, seed=0, sketch_prec="fp32", final_prec="fp32",
             omega_identity=False, sketch_identity=False, srht_t=0, handle: Handle | None = None):
    """theta~ (n, FP32), rank, perm (d, int32) for dense FP32 A (torch, on a CUDA device)."""
    import torch
    h = handle or default_handle(A.device.index or 0)
    p = make_params(s=s, m=m, k=k, tau=tau, seed=seed, sketch_prec=sketch_prec, final_prec=final_prec,
                    omega_identity=omega_identity, sketch_identity=sketch_identity, srht_t=srht_t)
    theta = torch.empty(A.shape[0], dtype=torch.float32, device=A.device)
    perm = torch.empty(A.shape[1], dtype=torch.int32, device=A.device)
    r = lev_estimate_dense(h, A, p, theta, perm)
    return theta, r, perm


# ---- row shards (rows of one matrix split across processes; see include/lev.h) ----

def row_shard(n: int, world_size: int, rank: int):
    """(row0, rows) of block `rank` when n rows are cut into world_size contiguous blocks whose
    sizes differ by at most one (the first n mod world_size blocks take the extra row)."""
    if world_size < 1 or not 0 <= rank < world_size or n < world_size:
        raise ValueError(f"cannot cut {n} rows into {world_size} blocks (rank {rank})")
    q, rem = divmod(n, world_size)
    return rank * q + min(rank, rem), q + (1 if rank < rem else 0)


def _shard_params(p: lev_params, row0: int, n_total: int) -> lev_params:
    q = lev_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(lev_params))
    q.row0, q.n_total = int(row0), int(n_total)
    return q


def sketch_shard(h: Handle, A_local, p: lev_params, row0: int, n_total: int, Atilde, csr=None, stream=None):
    """This block's part G (S_{:,block} A_block) of the sketch (rows hashed by global index)."""
    q = _shard_params(p, row0, n_total)
    if csr is None:
        lev_sketch_dense(h, A_local, q, Atilde, stream)
    else:
        row_ptr, col, val, n, d = csr
        lev_sketch_csr(h, row_ptr, col, val, n, d, q, Atilde, stream)


def allreduce_sketch(Atilde, group=None):
    """Sum the blocks' partial sketches in place on every process: the one exchange of the
    sharded path (m x d FP32). A no-op without an initialised process group of size > 1."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if Atilde.is_cuda and dist.get_backend(group) == "gloo":    # gloo reduces host memory
            host = Atilde.cpu()
            dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
            Atilde.copy_(host)
        else:
            dist.all_reduce(Atilde, op=dist.ReduceOp.SUM, group=group)
    return Atilde


def finish_shard(h: Handle, A_local, p: lev_params, Atilde, k: int, csr=None, stream=None):
    """Pivoted QR of the summed sketch, M = R_11^{-1} Omega and the final pass over this block:
    (theta~ of the block's rows, rank, perm). Every process gets the same (perm, rank, Mfull)
    from the same summed sketch."""
    import torch
    dev = Atilde.device
    d = Atilde.shape[1]
    perm = torch.empty(d, dtype=torch.int32, device=dev)
    R = torch.empty((d, d), dtype=torch.float64, device=dev)
    r = lev_rrqr(h, Atilde, p.tau, perm, R, stream)
    n_local = A_local.shape[0] if csr is None else csr[3]
    theta = torch.zeros(n_local, dtype=torch.float32, device=dev)
    if r == 0:
        return theta, 0, perm
    d_rank = torch.tensor([r], dtype=torch.int64, device=dev)
    Mfull = torch.empty((d, k), dtype=torch.float32, device=dev)
    lev_omega_factor(h, R, perm, d_rank, d, k, p.seed, p.flags | LEV_OMEGA_REDUCED, Mfull, stream)
    if csr is None:
        lev_final_dense(h, A_local, Mfull, p.final_prec, theta, stream)
    else:
        row_ptr, col, val, n, _ = csr
        lev_final_csr(h, row_ptr, col, val, n, d, Mfull, p.final_prec, theta, stream)
    return theta, r, perm


def estimate_sharded(A_local, p: lev_params, row0: int, n_total: int, *, csr=None, group=None,
                     handle: Handle | None = None):
    """Alg. 10 on a matrix whose rows [row0, row0 + rows) live on this process: the partial
    sketch, one all-reduce of it, then the QR, M and the final pass. Returns (theta~ of the
    local rows, rank, perm); rank and perm are the same on every process.

    Dense: A_local is the block (FP32, CUDA). CSR: csr = (row_ptr, col, val, rows, d) of the block
    and A_local is None."""
    import torch
    dev = (A_local if csr is None else csr[0]).device
    h = handle or default_handle(dev.index or 0)
    n_local, d = (A_local.shape if csr is None else (csr[3], csr[4]))
    _, m, k = lev_resolve_sizes(_shard_params(p, row0, n_total), n_local, d)
    Atilde = torch.empty((m, d), dtype=torch.float32, device=dev)
    sketch_shard(h, A_local, p, row0, n_total, Atilde, csr)
    allreduce_sketch(Atilde, group)
    return finish_shard(h, A_local, p, Atilde, k, csr)


def forward_state(A, p: lev_params, handle: Handle | None = None):
    """Run the estimator stage by stage and keep every intermediate the backward needs.

    Returns (theta, state) where state holds Atilde, perm, d_rank (device), rank, R, Mfull.
    """
    import torch
    h = handle or default_handle(A.device.index or 0)
    n, d = A.shape
    s, m, k = lev_resolve_sizes(p, n, d)
    dev = A.device
    Atilde = torch.empty((m, d), dtype=torch.float32, device=dev)
    perm = torch.empty(d, dtype=torch.int32, device=dev)
    R = torch.empty((d, d), dtype=torch.float64, device=dev)
    Mfull = torch.empty((d, k), dtype=torch.float32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    lev_sketch_dense(h, A, p, Atilde)
    r = lev_rrqr(h, Atilde, p.tau, perm, R)
    d_rank = torch.tensor([r], dtype=torch.int64, device=dev)
    lev_omega_factor(h, R, perm, d_rank, d, k, p.seed, p.flags | LEV_OMEGA_REDUCED, Mfull)
    lev_final_dense(h, A, Mfull, p.final_prec, theta)
    return theta, dict(Atilde=Atilde, perm=perm, d_rank=d_rank, rank=r, R=R, Mfull=Mfull, handle=h)


def _autograd_class():
    import torch

    class LevScore(torch.autograd.Function):
        """theta~ = LevScore.apply(A, params); backward gives dL/dA through lev_backward_dense."""

        @staticmethod
        def forward(ctx, A, p):
            theta, st = forward_state(A, p)
            ctx.p = p
            ctx.st = st
            ctx.save_for_backward(A)
            return theta

        @staticmethod
        def backward(ctx, grad_theta):
            (A,) = ctx.saved_tensors
            st = ctx.st
            gradA = torch.empty(A.shape, dtype=torch.float32, device=A.device)
            lev_backward_dense(st["handle"], A, ctx.p, st["Atilde"], st["perm"], st["d_rank"], st["R"],
                               st["Mfull"], grad_theta.contiguous().float(), gradA)
            return gradA, None

    return LevScore


class _LazyAutograd:
    _cls = None

    def apply(self, A, p):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _autograd_class()
        return _LazyAutograd._cls.apply(A, p)


LevScore = _LazyAutograd()
