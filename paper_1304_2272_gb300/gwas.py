"""Thin ctypes binding of the C ABI in ``include/gwas.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all steps of the GLS path run in the CUDA library
``libgwas_gb300.so``. Array arguments may be numpy arrays (host memory), torch
tensors (host or device; their ``data_ptr()`` is passed) or raw integer addresses.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libgwas_gb300.so"

GWAS_OK = 0
GWAS_ERR_ARG = 1
GWAS_ERR_NOT_SPD = 2
GWAS_ERR_CUDA = 3
GWAS_ERR_OOM = 4
GWAS_ERR_TIMEOUT = 5
GWAS_ERR_STATE = 6
GWAS_ERR_UNSUPPORTED = 7
GWAS_ERR_TOO_LARGE = 8
STATUS_NAMES = {0: "GWAS_OK", 1: "GWAS_ERR_ARG", 2: "GWAS_ERR_NOT_SPD", 3: "GWAS_ERR_CUDA",
                4: "GWAS_ERR_OOM", 5: "GWAS_ERR_TIMEOUT", 6: "GWAS_ERR_STATE",
                7: "GWAS_ERR_UNSUPPORTED", 8: "GWAS_ERR_TOO_LARGE"}

GWAS_PREC_FP64 = 0
GWAS_PREC_MIXED = 1


class gwas_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("m_blk", ctypes.c_int), ("n_limbs", ctypes.c_int),
                ("tile_cfg", ctypes.c_int), ("device", ctypes.c_int), ("timing", ctypes.c_int),
                ("use_graph", ctypes.c_int)]


class gwas_stats(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_int64), ("snps", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("trsm_launches", ctypes.c_int64),
                ("trsm_ms", ctypes.c_double), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("factor_ms", ctypes.c_double),
                ("factor_launches", ctypes.c_int64), ("factor_upload_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class gwas_tune(ctypes.Structure):
    _fields_ = [("tile_cfg", ctypes.c_int), ("m_blk", ctypes.c_int64),
                ("ms_per_snp", ctypes.c_double), ("snps_per_s", ctypes.c_double),
                ("candidates", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class gwas_reml_result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("loglik", "dl_dh", "dl_dsigma2", "sigma2_hat",
                                                "yPy", "logdet_M", "logdet_A", "sigma2")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GwasError(RuntimeError):
    def __init__(self, status: int, message: str, index: int = -1):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.index = index


_ctx_p = ctypes.c_void_p
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double

# name -> (restype, argtypes): one line per declaration of include/gwas.h
SIGNATURES = {
    "gwas_default_opts": (None, [ctypes.POINTER(gwas_opts)]),
    "gwas_init": (_int, [_i64, _int, _int, ctypes.POINTER(gwas_opts), ctypes.POINTER(_ctx_p)]),
    "gwas_factor": (_int, [_ctx_p, _vp, _int, _dbl, _dbl, _vp, _vp]),
    "gwas_solve_block": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp]),
    "gwas_solve_block_device": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp]),
    "gwas_solve_block_cov_device": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gwas_solve_block_packed": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gwas_solve_block_packed_device": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gwas_solve_all": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp]),
    "gwas_sync": (_int, [_ctx_p, _int]),
    "gwas_wait_block": (_int, [_ctx_p, _i64, _int]),
    "gwas_host_alloc": (_int, [ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "gwas_host_free": (_int, [_vp]),
    "gwas_finalize": (_int, [_ctx_p]),
    "gwas_last_error": (ctypes.c_char_p, [_ctx_p]),
    "gwas_error_index": (_i64, [_ctx_p]),
    "gwas_get_stats": (_int, [_ctx_p, ctypes.POINTER(gwas_stats)]),
    "gwas_reset_stats": (_int, [_ctx_p]),
    "gwas_stream": (_vp, [_ctx_p]),
    "gwas_solve_block_noalloc": (_int, [_i64, _int, _int, _vp, _i64, _vp, _vp, _vp, _vp, _vp,
                                        _i64, _vp, _vp, _vp, _vp]),
    "gwas_set_tile_cfg": (_int, [_ctx_p, _int]),
    "gwas_selftest_wait": (_int, [_int, _int, ctypes.POINTER(_dbl)]),
    "gwas_fp64_fma_rate": (_int, [_int, ctypes.POINTER(_dbl)]),
    "gwas_reml": (_int, [_ctx_p, _vp, _dbl, _dbl, _vp, _vp, _int, _int,
                         ctypes.POINTER(gwas_reml_result)]),
    "gwas_solve_block_grad_device": (_int, [_ctx_p, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gwas_autotune": (_int, [_ctx_p, _vp, _i64, _int, ctypes.POINTER(gwas_tune)]),
    "gwas_batch_init": (_int, [_int, ctypes.POINTER(_i64), _int, _int, ctypes.POINTER(gwas_opts),
                               ctypes.POINTER(_ctx_p)]),
    "gwas_batch_factor": (_int, [_ctx_p, _int, _vp, _int, _dbl, _dbl, _vp, _vp]),
    "gwas_batch_solve_device": (_int, [_ctx_p, ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp)]),
    "gwas_batch_sync": (_int, [_ctx_p, _int]),
    "gwas_batch_get_stats": (_int, [_ctx_p, ctypes.POINTER(gwas_stats)]),
    "gwas_batch_reset_stats": (_int, [_ctx_p]),
    "gwas_batch_finalize": (_int, [_ctx_p]),
    "gwas_batch_last_error": (ctypes.c_char_p, [_ctx_p]),
    "gwas_batch_stream": (_vp, [_ctx_p]),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists() or os.environ.get("GWAS_FORCE_BUILD"):
        if not build_if_missing:
            raise OSError(f"{LIB_PATH} is missing: run paper_1304_2272_gb300.build.build()")
        from .build import build
        build()
    lib = ctypes.CDLL(str(LIB_PATH))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _addr(x) -> int | None:
    """Raw address of a numpy array, torch tensor, ctypes buffer or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot pass {type(x).__name__} as a pointer")


def _check(ctx, st: int):
    if st != GWAS_OK:
        lib = load()
        msg = lib.gwas_last_error(ctx).decode() if ctx else ""
        idx = lib.gwas_error_index(ctx) if ctx else -1
        raise GwasError(st, msg, idx)


def _require(x, dtype, name: str, order: str = "F"):
    if isinstance(x, np.ndarray):
        if x.dtype != dtype:
            raise TypeError(f"{name} must be {np.dtype(dtype).name}, got {x.dtype}")
        ok = x.flags.f_contiguous if order == "F" else x.flags.c_contiguous
        if not ok and x.ndim > 1:
            raise ValueError(f"{name} must be contiguous in {order}-order")
    return x


_TORCH_DTYPES = {np.int8: "torch.int8", np.uint8: "torch.uint8", np.float64: "torch.float64"}


def _require_dev(x, dtype, name: str, device: int | None = None):
    """A device buffer passed as a tensor must have the C ABI's element type, be
    contiguous, live in device memory and (when `device` is given) on that device. Host
    arrays are refused; raw addresses and None pass through unchecked."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        raise TypeError(f"{name} must be a device tensor, got a host numpy array")
    if hasattr(x, "is_contiguous") and hasattr(x, "dtype"):
        if str(x.dtype) != _TORCH_DTYPES[dtype]:
            raise TypeError(f"{name} must be {_TORCH_DTYPES[dtype]}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if getattr(x, "is_cuda", True) is False:
            raise ValueError(f"{name} must be in device memory")
        if device is not None and x.device.index != device:
            raise ValueError(f"{name} is on cuda:{x.device.index}, the call runs on cuda:{device}")
    return x


def _outs_dev(b, wald, status):
    _require_dev(b, np.float64, "b")
    _require_dev(wald, np.float64, "wald")
    _require_dev(status, np.uint8, "status")


# ---- entry points (same names as the C ABI) -----------------------------------
def gwas_default_opts() -> gwas_opts:
    o = gwas_opts()
    load().gwas_default_opts(ctypes.byref(o))
    return o


def gwas_init(n: int, p: int, t: int = 1, opts: gwas_opts | None = None, **kw):
    """Create a context; keyword arguments override fields of the default options."""
    lib = load()
    o = opts if opts is not None else gwas_default_opts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    ctx = _ctx_p()
    st = lib.gwas_init(int(n), int(p), int(t), ctypes.byref(o), ctypes.byref(ctx))
    if st != GWAS_OK:
        raise GwasError(st, "gwas_init failed")
    return ctx


def gwas_factor(ctx, M_or_Phi, is_phi: bool, h: float, sigma2: float, XL, Y) -> None:
    for a, nm in ((M_or_Phi, "M_or_Phi"), (XL, "XL"), (Y, "Y")):
        _require(a, np.float64, nm)
    _check(ctx, load().gwas_factor(ctx, _addr(M_or_Phi), int(bool(is_phi)), float(h),
                                   float(sigma2), _addr(XL), _addr(Y)))


def gwas_solve_block(ctx, X, mb: int, b, wald, status) -> None:
    _require(X, np.int8, "X")
    _check(ctx, load().gwas_solve_block(ctx, _addr(X), int(mb), _addr(b), _addr(wald),
                                        _addr(status)))


def gwas_solve_block_device(ctx, X, mb: int, b, wald, status) -> None:
    _require_dev(X, np.int8, "X")
    _outs_dev(b, wald, status)
    _check(ctx, load().gwas_solve_block_device(ctx, _addr(X), int(mb), _addr(b), _addr(wald),
                                               _addr(status)))


# 2-bit call -> dosage tables: calls that are dosages (3 = missing), and SNP-major PLINK
# .bed calls (00 two copies of the first allele, 01 missing, 10 one copy, 11 none).
CODE_DOSAGE = (0, 1, 2, -1)
CODE_PLINK_BED = (2, -1, 1, 0)


def _code(code) -> ctypes.Array:
    vals = [int(v) for v in code]
    if len(vals) != 4 or any(v < -128 or v > 127 for v in vals):
        raise ValueError("code: four int8 dosages, one per 2-bit call")
    return (ctypes.c_int8 * 4)(*vals)


def gwas_solve_block_packed(ctx, Xp, mb: int, code, b, wald, status) -> None:
    """Xp: HOST uint8 array of mb columns of ceil(n/4) bytes (F-order ceil(n/4) x mb)."""
    _require(Xp, np.uint8, "Xp")
    _check(ctx, load().gwas_solve_block_packed(ctx, _addr(Xp), int(mb), _code(code), _addr(b),
                                               _addr(wald), _addr(status)))


def gwas_solve_block_packed_device(ctx, Xp, mb: int, code, b, wald, status) -> None:
    _require_dev(Xp, np.uint8, "Xp")
    _outs_dev(b, wald, status)
    _check(ctx, load().gwas_solve_block_packed_device(ctx, _addr(Xp), int(mb), _code(code),
                                                      _addr(b), _addr(wald), _addr(status)))


def gwas_solve_block_cov_device(ctx, X, mb: int, b, wald, status, cov) -> None:
    _require_dev(X, np.int8, "X")
    _outs_dev(b, wald, status)
    _require_dev(cov, np.float64, "cov")
    _check(ctx, load().gwas_solve_block_cov_device(ctx, _addr(X), int(mb), _addr(b), _addr(wald),
                                                   _addr(status), _addr(cov)))


def gwas_solve_all(ctx, X, m: int, b, wald, status) -> None:
    _require(X, np.int8, "X")
    _check(ctx, load().gwas_solve_all(ctx, _addr(X), int(m), _addr(b), _addr(wald),
                                      _addr(status)))


def gwas_sync(ctx, timeout_ms: int = -1) -> None:
    _check(ctx, load().gwas_sync(ctx, int(timeout_ms)))


def gwas_wait_block(ctx, block: int, timeout_ms: int = -1) -> None:
    _check(ctx, load().gwas_wait_block(ctx, int(block), int(timeout_ms)))


def gwas_host_alloc(nbytes: int) -> int:
    """Address of nbytes of page-locked host memory (free with gwas_host_free)."""
    p = _vp()
    st = load().gwas_host_alloc(int(nbytes), ctypes.byref(p))
    if st != GWAS_OK:
        raise GwasError(st, "gwas_host_alloc failed")
    return int(p.value or 0)


def gwas_host_free(addr: int) -> None:
    load().gwas_host_free(addr)


def gwas_finalize(ctx) -> None:
    if ctx:
        load().gwas_finalize(ctx)


def gwas_last_error(ctx) -> str:
    return load().gwas_last_error(ctx).decode()


def gwas_error_index(ctx) -> int:
    return int(load().gwas_error_index(ctx))


def gwas_get_stats(ctx) -> dict:
    s = gwas_stats()
    _check(ctx, load().gwas_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def gwas_reset_stats(ctx) -> None:
    _check(ctx, load().gwas_reset_stats(ctx))


def gwas_stream(ctx) -> int:
    return int(load().gwas_stream(ctx) or 0)


def gwas_solve_block_noalloc(n: int, p: int, t: int, Linv, ld_linv: int, XLbar, Ybar, S_TL,
                             bbar_T, X, mb: int, b, wald, status, stream=None) -> None:
    """Allocation-free FP64 block solve on caller-provided device buffers.

    For callers that must not allocate GPU memory at call time (memory already held by
    another allocator, or a serving loop that cannot afford cudaMalloc). All arrays are
    device memory on the current device; see include/gwas.h for layouts and the 16 MiB
    scratch limit (GWAS_ERR_TOO_LARGE beyond it). Tensors must be contiguous, of the C ABI's
    element type and on the current device (TypeError / ValueError otherwise). ``stream``
    is a torch.cuda.Stream or a cudaStream_t address (None = the default stream). Returns
    once the work is queued.
    """
    bufs = (Linv, XLbar, Ybar, S_TL, bbar_T, X, b, wald, status)
    dev = None
    if any(hasattr(x, "is_cuda") for x in bufs):
        import torch
        dev = torch.cuda.current_device()
    for x, nm in ((Linv, "Linv"), (XLbar, "XLbar"), (Ybar, "Ybar"), (S_TL, "S_TL"),
                  (bbar_T, "bbar_T"), (b, "b"), (wald, "wald")):
        _require_dev(x, np.float64, nm, dev)
    _require_dev(X, np.int8, "X", dev)
    _require_dev(status, np.uint8, "status", dev)
    stream = getattr(stream, "cuda_stream", stream)  # a torch.cuda.Stream or an address
    st = load().gwas_solve_block_noalloc(
        int(n), int(p), int(t), _addr(Linv), int(ld_linv), _addr(XLbar), _addr(Ybar),
        _addr(S_TL), _addr(bbar_T), _addr(X), int(mb), _addr(b), _addr(wald), _addr(status),
        stream)
    if st != GWAS_OK:
        raise GwasError(st, "gwas_solve_block_noalloc failed")


def gwas_reml(ctx, Phi, h: float, sigma2: float, XL, Y, pheno: int = 0,
              profile: bool = False) -> dict:
    """REML log-likelihood and its gradient (see include/gwas.h); Phi is the full matrix."""
    for a, nm in ((Phi, "Phi"), (XL, "XL"), (Y, "Y")):
        _require(a, np.float64, nm)
    out = gwas_reml_result()
    _check(ctx, load().gwas_reml(ctx, _addr(Phi), float(h), float(sigma2), _addr(XL), _addr(Y),
                                 int(pheno), int(bool(profile)), ctypes.byref(out)))
    return out.as_dict()


def gwas_solve_block_grad_device(ctx, X, mb: int, b, wald, status, dbdh) -> None:
    _require_dev(X, np.int8, "X")
    _outs_dev(b, wald, status)
    _require_dev(dbdh, np.float64, "dbdh")
    _check(ctx, load().gwas_solve_block_grad_device(ctx, _addr(X), int(mb), _addr(b), _addr(wald),
                                                    _addr(status), _addr(dbdh)))


def gwas_selftest_wait(device: int = 0, timeout_ms: int = 200) -> tuple[int, float]:
    """Run the bounded-wait self-test; returns (status, waited_ms)."""
    w = _dbl(0.0)
    st = load().gwas_selftest_wait(int(device), int(timeout_ms), ctypes.byref(w))
    return st, w.value


def gwas_fp64_fma_rate(device: int = 0) -> float:
    """Measured FP64 multiply-add rate of the device in TFLOP/s (the FP64 roofline)."""
    r = _dbl(0.0)
    st = load().gwas_fp64_fma_rate(int(device), ctypes.byref(r))
    if st != GWAS_OK:
        raise GwasError(st, "gwas_fp64_fma_rate failed")
    return r.value


def gwas_set_tile_cfg(ctx, tile_cfg: int) -> None:
    _check(ctx, load().gwas_set_tile_cfg(ctx, int(tile_cfg)))


def gwas_autotune(ctx, X=None, mb_max: int = 0, reps: int = 3) -> dict:
    """Time the candidate tile configurations and block sizes on a factored context,
    keep the fastest on it and return {tile_cfg, m_blk, ms_per_snp, snps_per_s, ...}."""
    out = gwas_tune()
    _check(ctx, load().gwas_autotune(ctx, _addr(X), int(mb_max), int(reps), ctypes.byref(out)))
    return out.as_dict()


# ---- batches of cohorts -------------------------------------------------------------
def _bcheck(batch, st: int):
    if st != GWAS_OK:
        msg = load().gwas_batch_last_error(batch).decode() if batch else ""
        raise GwasError(st, msg)


def gwas_batch_init(n, p: int, t: int = 1, opts: gwas_opts | None = None, **kw):
    """Create a batch of len(n) cohorts; keyword arguments override default options."""
    lib = load()
    o = opts if opts is not None else gwas_default_opts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    arr = (_i64 * len(n))(*[int(v) for v in n])
    b = _ctx_p()
    st = lib.gwas_batch_init(len(n), arr, int(p), int(t), ctypes.byref(o), ctypes.byref(b))
    if st != GWAS_OK:
        raise GwasError(st, "gwas_batch_init failed")
    return b


def gwas_batch_factor(batch, cohort: int, M_or_Phi, is_phi: bool, h: float, sigma2: float,
                      XL, Y) -> None:
    for a, nm in ((M_or_Phi, "M_or_Phi"), (XL, "XL"), (Y, "Y")):
        _require(a, np.float64, nm)
    _bcheck(batch, load().gwas_batch_factor(batch, int(cohort), _addr(M_or_Phi), int(bool(is_phi)),
                                            float(h), float(sigma2), _addr(XL), _addr(Y)))


def _ptr_array(items):
    return (_vp * len(items))(*[_addr(x) for x in items])


def gwas_batch_solve_device(batch, X, mb, b, wald, status) -> None:
    """X, b, wald, status: sequences of device arrays (one per cohort); mb: SNP counts."""
    n = len(X)
    for k in range(n):
        _require_dev(X[k], np.int8, f"X[{k}]")
        _outs_dev(b[k], wald[k] if wald is not None else None, status[k])
    mbs = (_i64 * n)(*[int(v) for v in mb])
    w = _ptr_array(wald) if wald is not None else None
    _bcheck(batch, load().gwas_batch_solve_device(batch, _ptr_array(X), mbs, _ptr_array(b), w,
                                                  _ptr_array(status)))


def gwas_batch_sync(batch, timeout_ms: int = -1) -> None:
    _bcheck(batch, load().gwas_batch_sync(batch, int(timeout_ms)))


def gwas_batch_get_stats(batch) -> dict:
    s = gwas_stats()
    _bcheck(batch, load().gwas_batch_get_stats(batch, ctypes.byref(s)))
    return s.as_dict()


def gwas_batch_reset_stats(batch) -> None:
    _bcheck(batch, load().gwas_batch_reset_stats(batch))


def gwas_batch_finalize(batch) -> None:
    if batch:
        load().gwas_batch_finalize(batch)


def gwas_batch_last_error(batch) -> str:
    return load().gwas_batch_last_error(batch).decode()


def gwas_batch_stream(batch) -> int:
    return int(load().gwas_batch_stream(batch) or 0)


# ---- convenience wrapper (still marshalling only) --------------------------------
class GLS:
    """One cohort: ``GLS(n, p, t).factor(phi, h, sigma2, XL, Y).solve(X)``."""

    def __init__(self, n: int, p: int = 4, t: int = 1, **opts):
        self.n, self.p, self.t = int(n), int(p), int(t)
        self.ctx = gwas_init(n, p, t, **opts)

    def factor(self, M_or_Phi, h=None, sigma2=None, XL=None, Y=None, is_phi=True):
        Y = np.asfortranarray(np.asarray(Y, dtype=np.float64).reshape(self.n, -1))
        XL = np.asfortranarray(np.asarray(XL, dtype=np.float64).reshape(self.n, -1))
        A = np.asfortranarray(np.asarray(M_or_Phi, dtype=np.float64))
        gwas_factor(self.ctx, A, is_phi, 0.0 if h is None else h,
                    1.0 if sigma2 is None else sigma2, XL, Y)
        return self

    def solve(self, X):
        """b (m x t x p), wald (m x t), status (m) for host dosages X (n x m int8)."""
        X = np.asfortranarray(np.asarray(X, dtype=np.int8))
        m = X.shape[1]
        b = np.empty((m, self.t, self.p), dtype=np.float64)
        wald = np.empty((m, self.t), dtype=np.float64)
        status = np.empty(m, dtype=np.uint8)
        if m:
            gwas_solve_all(self.ctx, X, m, b, wald, status)
        return b, wald, status

    def stats(self) -> dict:
        return gwas_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            gwas_finalize(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
