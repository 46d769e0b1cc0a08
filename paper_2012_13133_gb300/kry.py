"""Thin ctypes binding of the Kryging C ABI (``include/kry.h``).

Argument marshalling only: every step of the hot path runs in ``libkry.so``.
Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed through);
host outputs are NumPy arrays.  Importing this module loads the library and
fails loudly if it has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkry.so")

KRY_OK, KRY_EINVAL, KRY_ENOMEM, KRY_ENOTPSD, KRY_ENOCONV, KRY_ENAN, KRY_ETIMEOUT, KRY_ECUDA, KRY_EUNSUPPORTED = range(9)
STATUS_NAMES = ["KRY_OK", "KRY_EINVAL", "KRY_ENOMEM", "KRY_ENOTPSD", "KRY_ENOCONV", "KRY_ENAN", "KRY_ETIMEOUT",
                "KRY_ECUDA", "KRY_EUNSUPPORTED"]
KRY_F32, KRY_F64 = 0, 1
KRY_AUTO = 2   # kry_opts only: FP32 where it resolves K, FP64 for the other settings


class KryError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class kry_grid(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("dx1", C.c_double), ("dx2", C.c_double)]


class kry_cov(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("range", C.c_double), ("nu", C.c_double), ("tau2", C.c_double),
                ("aniso_angle", C.c_double), ("aniso_ratio", C.c_double)]


class kry_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("nprobe", C.c_int32), ("nsteps", C.c_int32), ("seed", C.c_uint64),
                ("rtol", C.c_double), ("maxit", C.c_int32), ("reorth", C.c_int32), ("precond", C.c_int32)]


_P = C.c_void_p
_DP = C.POINTER(C.c_double)


class kry_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n1", C.c_int32), ("n2", C.c_int32), ("mask", C.c_void_p), ("y", C.c_void_p),
                ("X", C.c_void_p), ("ncov", C.c_int32), ("cov", kry_cov), ("opts", kry_opts),
                ("loglik", C.c_void_p), ("logdet", C.c_void_p), ("beta", C.c_void_p),
                ("target_cells", C.c_void_p), ("target_X", C.c_void_p), ("mean", C.c_void_p)]


KRY_REQ_LOGLIK, KRY_REQ_KRIGE = 0, 1
# name -> (restype, argtypes)
SIGNATURES = {
    "kry_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "kry_destroy": (None, [_P]),
    "kry_last_error": (C.c_char_p, [_P]),
    "kry_set_mask": (C.c_int, [_P, C.POINTER(kry_grid), _P, C.POINTER(C.c_int64)]),
    "kry_set_sites": (C.c_int, [_P, C.POINTER(kry_grid), _P, C.c_int64]),
    "kry_mask_interior": (C.c_int, [_P, _DP]),
    "kry_promoted": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "kry_embed_eigs": (C.c_int, [_P, C.POINTER(kry_cov), C.c_int, C.POINTER(_P), _DP]),
    "kry_embed_free": (None, [_P]),
    "kry_matvec": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int64]),
    "kry_matvec_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int64]),
    "kry_logdet": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, _DP, _DP, _DP]),
    "kry_solve": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int64, C.c_double, C.c_int32,
                            C.POINTER(C.c_int32), _DP]),
    "kry_solve_pre": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int64, C.c_double, C.c_int32,
                                C.POINTER(C.c_int32), _DP]),
    "kry_profile_loglik": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(kry_cov), C.c_int32, C.POINTER(kry_opts),
                                     _DP, _DP, _DP, _DP]),
    "kry_krige": (C.c_int, [_P, C.POINTER(kry_cov), C.POINTER(kry_opts), _P, _P, C.c_int32, _P, _P, C.c_int64,
                            _P, _P, C.c_int64, _P, _P, _P, _DP]),
    "kry_loglik_krige": (C.c_int, [_P, C.POINTER(kry_cov), C.POINTER(kry_opts), _P, _P, C.c_int32, _P, _P,
                                   C.c_int64, _P, _P, C.c_int64, _P, _P, _P, _DP, _DP, _DP, _DP]),
    "kry_sample": (C.c_int, [_P, C.POINTER(kry_cov), C.c_int32, C.c_int32, _P, _P]),
    "kry_sample_size": (C.c_int, [_P, C.POINTER(kry_cov), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "kry_server_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int32, C.c_int64]),
    "kry_server_submit": (C.c_int, [_P, C.POINTER(kry_request), C.POINTER(C.c_uint64)]),
    "kry_server_wait": (C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(C.c_int), _DP, C.POINTER(C.c_int32),
                                  C.c_char_p, C.c_int32]),
    "kry_server_queued": (C.c_int64, [_P]),
    "kry_server_destroy": (None, [_P]),
    "kry_autotune": (C.c_int, [_P, _P, C.c_int32, _DP, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]),
    "kry_set_schedule": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "kry_profile_enable": (C.c_int, [_P, C.c_int]),
    "kry_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _DP]),
    "kry_launch_count": (C.c_uint64, []),
    "kry_bccb_logdet": (C.c_int, [_P, C.POINTER(kry_cov), _DP, _DP]),
    "kry_genhybr": (C.c_int, [_P, C.POINTER(kry_cov), _P, C.c_int32, _P, _DP, _DP, _DP, _DP, _DP, _DP, _P]),
    "kry_genhybr_prec": (C.c_int, [_P, C.POINTER(kry_cov), C.c_int, C.c_int32, _P, C.c_int32, _P, _DP, _DP, _DP, _DP,
                                   _DP, _DP, _P]),
    "kry_bootstrap_var": (C.c_int, [_P, C.POINTER(kry_cov), C.POINTER(kry_opts), C.c_int32, C.c_int32, C.c_int32,
                                    _P, _P, _P, C.c_int64, _P]),
}


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2012_13133_gb300.build.build_library() "
                           "(the Kryging path has no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def lib():
    return _lib


def launch_count() -> int:
    """Kernels launched by libkry.so in this process so far."""
    return int(_lib.kry_launch_count())


def _ptr(t):
    """Device pointer of a tensor the library reads as a dense array.  The
    library takes plain device pointers, so host tensors and strided views must
    never reach it (a host address handed to a kernel is not an error the
    library could detect)."""
    if t is None:
        return None
    if t.device.type != "cuda":
        raise ValueError(f"tensor passed to libkry must be a CUDA tensor (got device {t.device})")
    if not t.is_contiguous():
        raise ValueError("tensor passed to libkry must be contiguous (call .contiguous())")
    return C.c_void_p(t.data_ptr())


def _dev(*specs):
    """Device pointers of tensors, each given as (tensor, dtypes, numel, name), after checking them
    against what the C ABI will read: the dtype (one of ``dtypes``, torch dtype names such as
    "float64") and the element count.  The library sees only a pointer and the sizes it is given,
    so a wrong dtype or a short buffer would be read out of bounds rather than reported.  All
    dtypes and sizes are checked before any device check; None stays None."""
    for t, dtypes, numel, name in specs:
        if t is None:
            continue
        dt = str(t.dtype).replace("torch.", "")
        if dt not in dtypes:
            raise ValueError(f"{name}: expected dtype {' or '.join(dtypes)}, got {dt}")
        if t.numel() != numel:
            raise ValueError(f"{name}: expected {numel} elements, got {t.numel()} (shape {tuple(t.shape)})")
    ptrs = tuple(_ptr(t) for t, _, _, _ in specs)
    return ptrs if len(ptrs) > 1 else ptrs[0]


def _vec_dtype(prec):
    return ("float32",) if prec == KRY_F32 else ("float64",)


F64, I64 = ("float64",), ("int64",)


def _np_dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def make_cov(cov) -> kry_cov:
    """Accepts a kry_cov, or any object with sigma2, range, nu, tau2 (and optional angle, ratio)."""
    if isinstance(cov, kry_cov):
        return cov
    return kry_cov(float(cov.sigma2), float(cov.range), float(cov.nu), float(cov.tau2),
                   float(getattr(cov, "angle", 0.0)), float(getattr(cov, "ratio", 1.0)))


@dataclass
class Opts:
    prec: int = KRY_F32
    nprobe: int = 16
    nsteps: int = 50
    seed: int = 0
    rtol: float = 1e-6
    maxit: int = 5000
    reorth: int = 0   # 1: partial reorthogonalisation of the Lanczos basis
    precond: int = 0  # 1: CG preconditioned by the torus inverse (clustered gaps); 2: automatic

    def c(self) -> kry_opts:
        return kry_opts(self.prec, self.nprobe, self.nsteps, self.seed, self.rtol, self.maxit, self.reorth,
                        self.precond)


class Embed:
    def __init__(self, ctx, handle, min_over_max, prec):
        self.ctx, self.handle, self.min_over_max, self.prec = ctx, handle, min_over_max, prec
        ctx._embeds.add(self)

    def free(self):
        if self.handle:
            _lib.kry_embed_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """One library context on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        st = _lib.kry_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st != KRY_OK:
            raise KryError(st, "kry_create failed")
        self.h = h
        self.p = 0
        self.n1 = self.n2 = 0
        self._embeds = weakref.WeakSet()

    def close(self):
        if getattr(self, "h", None):
            for e in list(self._embeds):
                e.free()
            _lib.kry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != KRY_OK and st not in allow:
            raise KryError(st, _lib.kry_last_error(self.h).decode())
        return st

    # -- observation pattern
    def set_mask(self, mask, dx1=None, dx2=None) -> int:
        """mask: torch uint8 CUDA tensor (n1, n2), nonzero = observed."""
        n1, n2 = mask.shape
        g = kry_grid(n1, n2, 1.0 / n1 if dx1 is None else dx1, 1.0 / n2 if dx2 is None else dx2)
        p = C.c_int64()
        m = _dev((mask.contiguous(), ("uint8", "bool"), n1 * n2, "mask"))
        self._check(_lib.kry_set_mask(self.h, C.byref(g), m, C.byref(p)))
        self.p, self.n1, self.n2 = int(p.value), n1, n2
        return self.p

    def mask_interior(self) -> float:
        """Share of the observed cells whose four grid neighbours are observed (kry_mask_interior)."""
        v = C.c_double()
        self._check(_lib.kry_mask_interior(self.h, C.byref(v)))
        return v.value

    def promoted(self) -> int:
        """Covariance settings asked for in FP32 that ran in FP64 for their conditioning (kry_promoted)."""
        v = C.c_int64()
        self._check(_lib.kry_promoted(self.h, C.byref(v)))
        return v.value

    def set_sites(self, sites, n1, n2, dx1=None, dx2=None) -> int:
        """Irregular observation sites: sites is a torch float64 CUDA tensor (p, 2) of coordinates in the
        domain of the n1 x n2 latent grid (the unit square by default); the Wendland mapping matrix A
        is built on the device.  Returns p."""
        p = int(sites.shape[0])
        g = kry_grid(n1, n2, 1.0 / n1 if dx1 is None else dx1, 1.0 / n2 if dx2 is None else dx2)
        s = _dev((sites.contiguous(), F64, 2 * p, "sites"))
        self._check(_lib.kry_set_sites(self.h, C.byref(g), s, p))
        self.p, self.n1, self.n2 = p, n1, n2
        return self.p

    # -- embedding
    def embed(self, cov, prec=KRY_F32) -> Embed:
        c = make_cov(cov)
        e = C.c_void_p()
        r = C.c_double()
        self._check(_lib.kry_embed_eigs(self.h, C.byref(c), prec, C.byref(e), C.byref(r)))
        return Embed(self, e, r.value, prec)

    # -- matvec
    def matvec(self, emb: Embed, v, out=None):
        """v: (nvec, p) or (p,) CUDA tensor (float32 for KRY_F32, float64 for KRY_F64)."""
        squeeze = v.dim() == 1
        V = (v.reshape(1, -1) if squeeze else v).contiguous()
        if V.dim() != 2 or V.shape[1] != self.p:
            raise ValueError(f"v: expected (nvec, {self.p}) or ({self.p},), got {tuple(v.shape)}")
        if out is None:
            out = self.torch.empty(V.shape, dtype=V.dtype, device=V.device)
        n = V.shape[0] * self.p
        pv, po = _dev((V, _vec_dtype(emb.prec), n, "v"), (out, _vec_dtype(emb.prec), n, "out"))
        self._check(_lib.kry_matvec(self.h, emb.handle, pv, po, V.shape[0], self.p))
        return out.reshape(-1) if squeeze else out

    def logdet(self, emb: Embed, nprobe: int, nsteps: int, seed: int, reorth: int = 0):
        ld, se = C.c_double(), C.c_double()
        per = np.zeros(nprobe)
        self._check(_lib.kry_logdet(self.h, emb.handle, nprobe, nsteps, C.c_uint64(seed), reorth, C.byref(ld),
                                    C.byref(se), _np_dp(per)))
        return ld.value, se.value, per

    def solve(self, emb: Embed, B, rtol=1e-8, maxit=5000, X=None, precond=False):
        """B: (nrhs, p) float64 CUDA tensor.  Returns (X, iters, relres, status).  precond: CG
        preconditioned by the torus inverse (kry_solve_pre)."""
        squeeze = B.dim() == 1
        Bm = (B.reshape(1, -1) if squeeze else B).contiguous()
        if X is None:
            X = self.torch.empty(Bm.shape, dtype=Bm.dtype, device=Bm.device)
        it, rr = C.c_int32(), C.c_double()
        n = Bm.shape[0] * self.p
        pb, px = _dev((Bm, F64, n, "B"), (X, F64, n, "X"))
        fn = _lib.kry_solve_pre if precond else _lib.kry_solve
        st = self._check(fn(self.h, emb.handle, pb, px, Bm.shape[0], self.p, rtol, maxit, C.byref(it),
                            C.byref(rr)), allow=(KRY_ENOCONV,))
        return (X.reshape(-1) if squeeze else X), it.value, rr.value, st

    def profile_loglik(self, y, X, thetas, opts: Opts):
        """y: (p,) float64 CUDA; X: (ncov, p) float64 CUDA (column-major p x ncov)."""
        y, X = y.contiguous(), X.contiguous()
        ncov = X.shape[0]
        n = len(thetas)
        arr = (kry_cov * n)(*[make_cov(t) for t in thetas])
        ll, beta, ld, se = np.zeros(n), np.zeros(n * ncov), np.zeros(n), np.zeros(n)
        o = opts.c()
        py, pX = _dev((y, F64, self.p, "y"), (X, F64, ncov * self.p, "X"))
        st = self._check(_lib.kry_profile_loglik(self.h, py, pX, ncov, arr, n, C.byref(o), _np_dp(ll),
                                                 _np_dp(beta), _np_dp(ld), _np_dp(se)), allow=(KRY_ENOCONV,))
        return dict(loglik=ll, beta=beta.reshape(n, ncov), logdet=ld, logdet_se=se, status=st)

    def krige(self, cov, opts: Opts, y, X, cells=None, Xc=None, sites=None, Xs=None, variances=False):
        """cells: (ncell,) int64 CUDA; Xc: (ncov, ncell) float64; sites: (nsite, 2) float64; Xs: (ncov, nsite)."""
        torch = self.torch
        y, X = y.contiguous(), X.contiguous()
        cells, Xc, sites, Xs = (None if t is None else t.contiguous() for t in (cells, Xc, sites, Xs))
        ncov = X.shape[0]
        ncell = 0 if cells is None else cells.shape[0]
        nsite = 0 if sites is None else sites.shape[0]
        dev = y.device
        mc = torch.empty(ncell, dtype=torch.float64, device=dev) if ncell else None
        ms = torch.empty(nsite, dtype=torch.float64, device=dev) if nsite else None
        vc = torch.empty(ncell, dtype=torch.float64, device=dev) if (ncell and variances) else None
        beta = np.zeros(ncov)
        c = make_cov(cov)
        o = opts.c()
        a = self._krige_args(y, X, ncov, cells, Xc, ncell, sites, Xs, nsite)
        st = self._check(_lib.kry_krige(self.h, C.byref(c), C.byref(o), a[0], a[1], ncov, a[2], a[3],
                                        ncell, a[4], a[5], nsite, _ptr(mc), _ptr(ms), _ptr(vc),
                                        _np_dp(beta)), allow=(KRY_ENOCONV,))
        return dict(mean_cells=mc, mean_sites=ms, var_cells=vc, beta=beta, status=st)

    def _krige_args(self, y, X, ncov, cells, Xc, ncell, sites, Xs, nsite, *more):
        """Checked device pointers of the kriging inputs: y (p,), X (ncov, p), cells (ncell,) int64,
        Xc (ncov, ncell), sites (nsite, 2), Xs (ncov, nsite), all float64 but cells; then those of
        the further (tensor, dtypes, numel, name) specs."""
        return _dev((y, F64, self.p, "y"), (X, F64, ncov * self.p, "X"), (cells, I64, ncell, "cells"),
                    (Xc, F64, ncov * ncell, "Xc"), (sites, F64, 2 * nsite, "sites"), (Xs, F64, ncov * nsite, "Xs"),
                    *more)

    def autotune(self, emb: Embed, nvec: int):
        """Time the feasible matvec schedules for batches of nvec; keep the fastest."""
        ms = C.c_double()
        g, c, ppb = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(_lib.kry_autotune(self.h, emb.handle, nvec, C.byref(ms), C.byref(g), C.byref(c), C.byref(ppb)))
        return dict(ms=ms.value, rows_per_block=g.value, cols_per_block=c.value, pairs_per_batch=ppb.value)

    def set_schedule(self, emb: Embed, nvec: int, rows_per_block=0, cols_per_block=0, pairs_per_batch=0):
        self._check(_lib.kry_set_schedule(self.h, emb.handle, nvec, rows_per_block, cols_per_block,
                                          pairs_per_batch))

    def profile_enable(self, on=True):
        self._check(_lib.kry_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, prec=KRY_F32):
        c, v, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._check(_lib.kry_profile_read(self.h, prec, C.byref(c), C.byref(v), C.byref(ms)))
        return dict(calls=c.value, vectors=v.value, ms=ms.value)

    def loglik_krige(self, cov, opts: Opts, y, X, cells=None, Xc=None, sites=None, Xs=None, variances=False,
                     mean_cells=None):
        """Profile log-likelihood and kriging means for one covariance setting (one shared solve)."""
        torch = self.torch
        y, X = y.contiguous(), X.contiguous()
        cells, Xc, sites, Xs = (None if t is None else t.contiguous() for t in (cells, Xc, sites, Xs))
        ncov = X.shape[0]
        ncell = 0 if cells is None else cells.shape[0]
        nsite = 0 if sites is None else sites.shape[0]
        dev = y.device
        mc = mean_cells if mean_cells is not None else (
            torch.empty(ncell, dtype=torch.float64, device=dev) if ncell else None)
        ms = torch.empty(nsite, dtype=torch.float64, device=dev) if nsite else None
        vc = torch.empty(ncell, dtype=torch.float64, device=dev) if (ncell and variances) else None
        ll, beta, ld, se = C.c_double(), np.zeros(ncov), C.c_double(), C.c_double()
        c = make_cov(cov)
        o = opts.c()
        a = self._krige_args(y, X, ncov, cells, Xc, ncell, sites, Xs, nsite, (mc, F64, ncell, "mean_cells"))
        pmc = a[6]
        st = self._check(_lib.kry_loglik_krige(self.h, C.byref(c), C.byref(o), a[0], a[1], ncov, a[2],
                                               a[3], ncell, a[4], a[5], nsite, pmc, _ptr(ms),
                                               _ptr(vc), C.byref(ll), _np_dp(beta), C.byref(ld), C.byref(se)),
                         allow=(KRY_ENOCONV,))
        return dict(loglik=ll.value, beta=beta, logdet=ld.value, logdet_se=se.value, mean_cells=mc, mean_sites=ms,
                    var_cells=vc, status=st)

    def sample_size(self, cov):
        m1, m2 = C.c_int32(), C.c_int32()
        st = self._check(_lib.kry_sample_size(self.h, C.byref(make_cov(cov)), C.byref(m1), C.byref(m2)),
                         allow=(KRY_ENOTPSD,))
        return m1.value, m2.value, st

    def sample(self, cov, M1, M2, xi):
        """xi: (2, M1, M2) float64 CUDA normals.  Returns the (n1, n2) float64 field."""
        out = self.torch.empty((self.n1, self.n2), dtype=self.torch.float64, device=xi.device)
        pxi = _dev((xi.contiguous(), F64, 2 * M1 * M2, "xi"))
        self._check(_lib.kry_sample(self.h, C.byref(make_cov(cov)), M1, M2, pxi, _ptr(out)))
        return out

    def bootstrap_var(self, cov, opts: Opts, xi, eps, cells):
        """Parametric-bootstrap kriging MSE at grid cells.  xi: (nrep, 2, M1, M2) float64 CUDA white
        noise, eps: (nrep, p) float64 CUDA, cells: (ncell,) int64 CUDA.  Returns (var, status)."""
        xi, eps, cells = xi.contiguous(), eps.contiguous(), cells.contiguous()
        if xi.dim() != 4 or xi.shape[1] != 2:
            raise ValueError(f"xi: expected (nrep, 2, M1, M2), got {tuple(xi.shape)}")
        nrep, _, M1, M2 = xi.shape
        var = self.torch.empty(cells.shape[0], dtype=self.torch.float64, device=xi.device)
        pxi, peps, pc = _dev((xi, F64, nrep * 2 * M1 * M2, "xi"), (eps, F64, nrep * self.p, "eps"),
                             (cells, I64, cells.numel(), "cells"))
        st = self._check(_lib.kry_bootstrap_var(self.h, C.byref(make_cov(cov)), C.byref(opts.c()), nrep, M1, M2,
                                                pxi, peps, pc, cells.shape[0], _ptr(var)),
                         allow=(KRY_ENOCONV,))
        return var, st

    def genhybr(self, cov, b, k, want_x=True, gradient=False, prec=KRY_F64, reorth=0):
        """genHyBR with k genGK steps.  b: (p,) float64 CUDA = y - X beta.  Returns dict(x (n1 x n2
        float64 CUDA or None), alphas, betas (k+1 each), z2, psi2, pl, and with gradient=True
        grad (d pl / d lambda^2, d range, d lambda_e^2) and psi (p,) float64 CUDA).  prec=KRY_F32:
        FP32 Krylov vectors and matvec, FP64 scalars; reorth=1: reorthogonalised bidiagonalization
        (kry_genhybr_prec)."""
        b = b.contiguous()
        x = self.torch.empty((self.n1, self.n2), dtype=self.torch.float64, device=b.device) if want_x else None
        psi = self.torch.empty_like(b) if gradient else None
        grad = np.zeros(3) if gradient else None
        al, be = np.zeros(k + 1), np.zeros(k + 1)
        z2, psi2, pl = C.c_double(), C.c_double(), C.c_double()
        pb = _dev((b, F64, self.p, "b"))
        self._check(_lib.kry_genhybr_prec(self.h, C.byref(make_cov(cov)), prec, reorth, pb, k, _ptr(x), _np_dp(al),
                                          _np_dp(be), C.byref(z2), C.byref(psi2), C.byref(pl), _np_dp(grad),
                                          _ptr(psi)))
        return dict(x=x, alphas=al, betas=be, z2=z2.value, psi2=psi2.value, pl=pl.value, grad=grad, psi=psi)

    def bccb_logdet(self, cov, derivative=True):
        """BCCB approximation of log det Sigma (no nugget) on the mask's grid and its range
        derivative (None when derivative=False)."""
        ld, dl = C.c_double(), C.c_double()
        self._check(_lib.kry_bccb_logdet(self.h, C.byref(make_cov(cov)), C.byref(ld),
                                         C.byref(dl) if derivative else None))
        return ld.value, (dl.value if derivative else None)


def _np_ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Server:
    """Continuous-batching server of the library (host buffers in, host buffers out)."""

    def __init__(self, device: int = 0, nslots: int = 4, mem_budget_bytes: int = 64 << 30):
        h = C.c_void_p()
        st = _lib.kry_server_create(C.byref(h), device, nslots, int(mem_budget_bytes))
        if st != KRY_OK:
            raise KryError(st, "kry_server_create failed")
        self.h = h
        self._live = {}

    def submit(self, kind, mask, y, X, cov, opts: Opts, target_cells=None, target_X=None) -> int:
        """mask: (n1, n2) bool/uint8; y: (p,) float64; X: (ncov, p) float64 (column-major p x ncov);
        target_cells: (nt,) int64 unobserved cells and target_X: (ncov, nt) for kriging."""
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        y = np.ascontiguousarray(y, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        ncov = X.shape[0]
        # the library reads p values of y and X, and N - p of the kriging targets, from the mask alone
        p = int(np.count_nonzero(m))
        if m.ndim != 2 or y.size != p or X.ndim != 2 or X.size != ncov * p:
            raise ValueError(f"request: mask (n1, n2) with p = {p} observed cells needs y ({p},) and X (ncov, {p}); "
                             f"got mask {m.shape}, y {y.shape}, X {X.shape}")
        if kind == KRY_REQ_KRIGE:
            nt = m.size - p
            if target_cells is None or target_X is None or np.size(target_cells) != nt or \
                    np.size(target_X) != ncov * nt:
                raise ValueError(f"kriging request: target_cells ({nt},) and target_X (ncov, {nt}) are required "
                                 "(every unobserved cell)")
        out = dict(loglik=np.zeros(1), logdet=np.zeros(1), beta=np.zeros(ncov))
        keep = [m, y, X]
        r = kry_request()
        r.kind = kind
        r.n1, r.n2 = m.shape
        r.mask, r.y, r.X, r.ncov = _np_ptr(m), _np_ptr(y), _np_ptr(X), ncov
        r.cov = make_cov(cov)
        r.opts = opts.c()
        r.loglik, r.logdet, r.beta = _np_ptr(out["loglik"]), _np_ptr(out["logdet"]), _np_ptr(out["beta"])
        if kind == KRY_REQ_KRIGE:
            tc = np.ascontiguousarray(target_cells, dtype=np.int64)
            tX = np.ascontiguousarray(target_X, dtype=np.float64)
            out["mean"] = np.zeros(tc.shape[0])
            keep += [tc, tX]
            r.target_cells, r.target_X, r.mean = _np_ptr(tc), _np_ptr(tX), _np_ptr(out["mean"])
        t = C.c_uint64()
        st = _lib.kry_server_submit(self.h, C.byref(r), C.byref(t))
        if st != KRY_OK:
            raise KryError(st, "kry_server_submit refused the request")
        self._live[t.value] = (keep, out, r)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 600.0):
        rs, lat, slot = C.c_int(), C.c_double(), C.c_int32()
        err = C.create_string_buffer(512)
        st = _lib.kry_server_wait(self.h, ticket, timeout_s, C.byref(rs), C.byref(lat), C.byref(slot), err, 512)
        if st != KRY_OK:
            raise KryError(st, f"wait on ticket {ticket}")
        keep, out, _ = self._live.pop(ticket)
        res = {k: (v[0] if k in ("loglik", "logdet") else v) for k, v in out.items()}
        res.update(status=rs.value, latency_ms=lat.value, slot=slot.value, error=err.value.decode())
        return res

    def queued(self) -> int:
        return int(_lib.kry_server_queued(self.h))

    def close(self):
        if getattr(self, "h", None):
            _lib.kry_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
