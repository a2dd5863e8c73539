"""Thin ctypes binding of the C ABI in include/hodlr.h (argument marshalling only).

Every arithmetic step runs in the CUDA library; this module only allocates the device
workspace with PyTorch, passes pointers / the current CUDA stream, and converts outputs.
Loading fails loudly when the compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HODLR_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ENOTPD", -4: "ENUMERIC", -5: "ETIMEOUT", -6: "ENOTIMPL",
          -7: "ECUDA"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
WHICH = {"K": 0, "sigma2": 1, "ell": 2, "kappa": 3, "tau2": 4}

_LIB = None


class HodlrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hodlr error {ERRORS.get(code, code)}: {msg}")
        self.code = code


class Model(C.Structure):
    _fields_ = [("dim", C.c_int), ("grid", C.c_int * 2), ("nvar", C.c_int), ("nu", C.c_double),
                ("precision", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("leaf", C.c_int), ("rank_or_cap", C.c_int), ("oversample", C.c_int), ("tol", C.c_double),
                ("seed", C.c_uint64), ("guard", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "hodlr_workspace_size": (C.c_size_t, [C.POINTER(Model), C.POINTER(Opts)]),
    "hodlr_plan": (C.c_int, [C.POINTER(Model), C.POINTER(Opts), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "hodlr_create": (C.c_int, [C.POINTER(_P), C.POINTER(Model), C.POINTER(Opts), _P, _P, C.c_size_t]),
    "hodlr_build": (C.c_int, [_P, _D, _D]),
    "hodlr_nll": (C.c_int, [_P, _D, _P, _D]),
    "hodlr_grad": (C.c_int, [_P, _D, _P, _D]),
    "hodlr_grad_adjoint": (C.c_int, [_P, _D, _P, _D]),
    "hodlr_fisher": (C.c_int, [_P, _D, _D]),
    "hodlr_eval": (C.c_int, [_P, _D, _P, _D, _D, _D]),
    "hodlr_batch_nll_grad": (C.c_int, [C.POINTER(_P), C.c_int, _D, C.POINTER(_P), _D, _D]),
    "hodlr_perm": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "hodlr_dims": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "hodlr_ranks": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "hodlr_get_pivots": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "hodlr_set_pivots": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "hodlr_apply": (C.c_int, [_P, _D, C.c_int, _P, _P, C.c_int]),
    "hodlr_probe": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "hodlr_densify": (C.c_int, [_P, C.c_int, _P]),
    "hodlr_solve": (C.c_int, [_P, _P, _P]),
    "hodlr_matvec": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "hodlr_logdet": (C.c_int, [_P, _D]),
    "hodlr_traces": (C.c_int, [_P, _D, _D]),
    "hodlr_logdet_levels": (C.c_int, [_P, _D]),
    "hodlr_debug_level": (C.c_int, [_P, C.c_int, C.c_int, _D, C.c_int64, C.POINTER(C.c_int32)]),
    "hodlr_napply": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "hodlr_profile": (C.c_int, [_P, C.c_int]),
    "hodlr_profile_read": (C.c_int, [_P, _D]),
    "hodlr_autotune": (C.c_int, [_P, C.c_int]),
    "hodlr_autotune_table": (C.c_int, [C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_int)]),
    "hodlr_autotune_clear": (C.c_int, []),
    "hodlr_kernel_count": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "hodlr_reset_kernel_count": (C.c_int, [_P]),
    "hodlr_debug_wait_limit": (C.c_int, [C.c_int]),
    "hodlr_peak": (C.c_int, [C.c_int, _D]),
    "hodlr_dgemm_slices": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, C.c_longlong, C.c_longlong, C.c_int,
                                     _P, C.c_longlong, C.c_longlong, C.c_int, C.c_int, C.c_double, C.c_double, _P,
                                     C.c_longlong, C.c_longlong, _P, C.c_size_t, _P]),
    "hodlr_dgemm_slices_plan": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "hodlr_apply_static": (C.c_int, [C.c_int, C.c_double, _D, _P, _P, C.c_int, _P]),
    "hodlr_last_error": (C.c_char_p, [_P]),
    "hodlr_destroy": (None, [_P]),
}


def load(build_if_missing: bool = True):
    """Load libhodlr.so (building it in-tree first if needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path}")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(_D)


class Hodlr:
    """One HODLR likelihood context on the current CUDA device and stream."""

    def __init__(self, dim, G, nvar, nu, precision="fp64", leaf=64, cap=24, oversample=0, tol=0.0, seed=1,
                 device="cuda", guard=0.0):
        import torch
        self.torch = torch
        self.lib = load()
        self.model = Model(dim, (C.c_int * 2)(G, G if dim == 2 else 1), nvar, float(nu), PRECISION[precision])
        self.opts = Opts(leaf, cap, oversample, float(tol), int(seed), float(guard))
        nbytes = self.lib.hodlr_workspace_size(C.byref(self.model), C.byref(self.opts))
        if nbytes == 0:
            raise HodlrError(-1, "bad model or options")
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.stream = torch.cuda.current_stream(self.device)
        h = _P()
        rc = self.lib.hodlr_create(C.byref(h), C.byref(self.model), C.byref(self.opts),
                                   _P(self.stream.cuda_stream), _P(aligned), nbytes)
        if rc != HODLR_OK:
            raise HodlrError(rc, "hodlr_create failed")
        self.h = h
        d = np.zeros(6, dtype=np.int64)
        self._check(self.lib.hodlr_dims(self.h, d.ctypes.data_as(C.POINTER(C.c_int64))))
        self.N, self.tau, self.leaf, self.c, self.cap, self.nleaves = (int(v) for v in d)
        self.workspace_bytes = nbytes

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.hodlr_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _check(self, rc):
        if rc != HODLR_OK:
            msg = self.lib.hodlr_last_error(self.h)
            raise HodlrError(rc, msg.decode() if msg else "")

    @staticmethod
    def _theta(theta):
        return np.ascontiguousarray(theta, dtype=np.float64)

    def _dev(self, x):
        t = self.torch
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(np.asarray(x, dtype=np.float64))
        return x.to(device=self.device, dtype=t.float64).contiguous()

    # ------------------------------------------------------------------ main calls
    def build(self, theta):
        th = self._theta(theta)
        self._check(self.lib.hodlr_build(self.h, _dp(th), None))

    def nll(self, theta, y):
        th, yd, out = self._theta(theta), self._dev(y), np.zeros(1)
        self._check(self.lib.hodlr_nll(self.h, _dp(th), _P(yd.data_ptr()), _dp(out)))
        return float(out[0])

    def grad(self, theta, y):
        th, yd, out = self._theta(theta), self._dev(y), np.zeros(4)
        self._check(self.lib.hodlr_grad(self.h, _dp(th), _P(yd.data_ptr()), _dp(out)))
        return out

    def grad_adjoint(self, theta, y):
        """The gradient by reverse mode through the factorization (hodlr_grad_adjoint)."""
        th, yd, out = self._theta(theta), self._dev(y), np.zeros(4)
        self._check(self.lib.hodlr_grad_adjoint(self.h, _dp(th), _P(yd.data_ptr()), _dp(out)))
        return out

    def nll_grad(self, theta, y):
        """NLL and its gradient in one call (one build, one factorization)."""
        th, yd = self._theta(theta), self._dev(y)
        f, g = np.zeros(1), np.zeros(4)
        self._check(self.lib.hodlr_eval(self.h, _dp(th), _P(yd.data_ptr()), _dp(f), _dp(g), None))
        return float(f[0]), g

    def fisher(self, theta):
        th, out = self._theta(theta), np.zeros(16)
        self._check(self.lib.hodlr_fisher(self.h, _dp(th), _dp(out)))
        return out.reshape(4, 4)

    def eval(self, theta, y):
        th, yd = self._theta(theta), self._dev(y)
        f, g, F = np.zeros(1), np.zeros(4), np.zeros(16)
        self._check(self.lib.hodlr_eval(self.h, _dp(th), _P(yd.data_ptr()), _dp(f), _dp(g), _dp(F)))
        return float(f[0]), g, F.reshape(4, 4)

    # ------------------------------------------------------------------ inspection
    def perm(self):
        p = np.zeros(self.N, dtype=np.int64)
        self._check(self.lib.hodlr_perm(self.h, p.ctypes.data_as(C.POINTER(C.c_int64))))
        return p

    def ranks(self):
        r = np.zeros((1 << self.tau) - 1, dtype=np.int32)
        self._check(self.lib.hodlr_ranks(self.h, r.ctypes.data_as(C.POINTER(C.c_int32))))
        return [r[(1 << (l - 1)) - 1:(1 << l) - 1].tolist() for l in range(1, self.tau + 1)]

    def get_pivots(self):
        p = np.zeros(((1 << self.tau) - 1) * self.c, dtype=np.int32)
        self._check(self.lib.hodlr_get_pivots(self.h, p.ctypes.data_as(C.POINTER(C.c_int32))))
        return p

    def set_pivots(self, piv):
        if piv is None:
            self._check(self.lib.hodlr_set_pivots(self.h, None))
            return
        p = np.ascontiguousarray(piv, dtype=np.int32)
        self._check(self.lib.hodlr_set_pivots(self.h, p.ctypes.data_as(C.POINTER(C.c_int32))))

    def pivots_from_sets(self, sets):
        """Flatten per-level, per-pair pivot lists (oracle layout) into the C layout."""
        out = np.full(((1 << self.tau) - 1) * self.c, -1, dtype=np.int32)
        k = 0
        for lvl in sets:
            for J in lvl:
                J = np.asarray(J, dtype=np.int32)
                out[k * self.c:k * self.c + J.size] = J
                k += 1
        return out

    def apply(self, theta, which, X):
        th = self._theta(theta)
        Xd = self._dev(X)
        if Xd.dim() == 1:
            Xd = Xd[:, None]
        Xc = Xd.t().contiguous()          # column-major N x q
        q = Xc.shape[0]
        Yc = self.torch.empty_like(Xc)
        self._check(self.lib.hodlr_apply(self.h, _dp(th), WHICH[which], _P(Xc.data_ptr()), _P(Yc.data_ptr()), q))
        return Yc.t()

    def probe(self, level, ncols):
        out = self.torch.empty((ncols, self.N), dtype=self.torch.float64, device=self.device)
        self._check(self.lib.hodlr_probe(self.h, level, ncols, _P(out.data_ptr())))
        return out.t()

    def densify(self, which="K"):
        out = self.torch.empty((self.N, self.N), dtype=self.torch.float64, device=self.device)
        self._check(self.lib.hodlr_densify(self.h, WHICH[which], _P(out.data_ptr())))
        return out.t()        # column-major buffer -> row-major view of the same matrix

    def solve(self, b):
        bd = self._dev(b)
        x = self.torch.empty_like(bd)
        self._check(self.lib.hodlr_solve(self.h, _P(bd.data_ptr()), _P(x.data_ptr())))
        return x

    def matvec(self, X, which=0):
        """K~ X (which 0 or "K") or K~_j X (1..4 or the parameter's name) of the last build;
        X: N or N x ncols (natural order, any device); returns a device tensor of X's shape."""
        w = WHICH.get(which, which)
        Xd = self._dev(X)
        cols = 1 if Xd.dim() == 1 else Xd.shape[1]
        Xc = Xd.reshape(-1, cols).t().contiguous()        # column-major N x ncols
        Y = self.torch.empty_like(Xc)
        self._check(self.lib.hodlr_matvec(self.h, int(w), _P(Xc.data_ptr()), _P(Y.data_ptr()), int(cols)))
        return Y.t().reshape(Xd.shape)

    def logdet(self):
        out = np.zeros(1)
        self._check(self.lib.hodlr_logdet(self.h, _dp(out)))
        return float(out[0])

    def debug_level(self, what, level):
        n = self.N * self.cap if what <= 1 else (1 << (level - 1)) * self.cap * self.cap
        out = np.zeros(max(n, 1))
        wl = C.c_int32(0)
        self._check(self.lib.hodlr_debug_level(self.h, what, level, _dp(out), n, C.byref(wl)))
        w = wl.value
        if what <= 1:
            return out[:self.N * w].reshape(w, self.N).T
        return out[:(1 << (level - 1)) * w * w].reshape(-1, w, w).transpose(0, 2, 1)

    def logdet_levels(self):
        out = np.zeros(self.tau + 1)
        self._check(self.lib.hodlr_logdet_levels(self.h, _dp(out)))
        return out

    def traces(self):
        t, f = np.zeros(3), np.zeros(9)
        self._check(self.lib.hodlr_traces(self.h, _dp(t), _dp(f)))
        return t, f.reshape(3, 3)

    def napply(self):
        v = np.zeros(1, dtype=np.int64)
        self._check(self.lib.hodlr_napply(self.h, v.ctypes.data_as(C.POINTER(C.c_int64))))
        return int(v[0])

    def autotune(self, enable=True):
        """Tile autotuner for this context's digit-slice products (hodlr_autotune)."""
        self._check(self.lib.hodlr_autotune(self.h, int(bool(enable))))

    def profile(self, enable):
        self._check(self.lib.hodlr_profile(self.h, int(bool(enable))))

    FAMILIES = ("gemm_kernel", "sgemm_large_kernel", "gemm_df_kernel", "gemv_kernel", "tf32x3_gemm_kernel",
                "oz_mma_kernel", "oz_atb_kernel", "oz_ab_kernel")

    def profile_read(self):
        out = np.zeros(4 + 4 * len(self.FAMILIES))
        self._check(self.lib.hodlr_profile_read(self.h, _dp(out)))
        fam = {name: {"ms": float(out[4 + 4 * v]), "flops": float(out[5 + 4 * v]), "launches": int(out[6 + 4 * v]),
                      "bytes": float(out[7 + 4 * v])}
               for v, name in enumerate(self.FAMILIES)}
        return {"ms": float(out[0]), "launches": int(out[1]), "flops": float(out[2]), "bytes": float(out[3]),
                "families": fam}

    def kernel_count(self, reset=False):
        v = np.zeros(1, dtype=np.int64)
        self._check(self.lib.hodlr_kernel_count(self.h, v.ctypes.data_as(C.POINTER(C.c_int64))))
        if reset:
            self.lib.hodlr_reset_kernel_count(self.h)
        return int(v[0])


def autotune_table():
    """The autotuner's remembered plans, one dict per product shape."""
    import numpy as np
    lib = load()
    n = C.c_int(0)
    if lib.hodlr_autotune_table(None, 0, C.byref(n)) != 0:
        raise HodlrError(-1, "hodlr_autotune_table")
    out = np.zeros((max(n.value, 1), 13), dtype=np.int64)
    if lib.hodlr_autotune_table(out.ctypes.data_as(C.POINTER(C.c_int64)), out.shape[0], C.byref(n)) != 0:
        raise HodlrError(-1, "hodlr_autotune_table")
    keys = ("M", "N", "K", "batch", "tA", "tB", "A_shared", "B_shared", "bmap", "beta_mode", "path", "tile", "cprx")
    return [dict(zip(keys, (int(v) for v in row))) for row in out[:n.value]]


def from_workload(w, device="cuda", precision=None):
    """Context for a synth.Workload-like object (fields dim, G, nvar, nu, leaf, cap, c, tol, ...)."""
    prec = precision or ("fp64" if w.precision == "fp64" else "fp32")
    return Hodlr(w.dim, w.G, w.nvar, w.nu, prec, w.leaf, w.cap, w.c - w.cap, w.tol, w.seed_probe, device,
                 guard=getattr(w, "guard", 0.0))
