"""Thin Python binding of the tensorctl C ABI (include/tensorctl.h).

Argument marshalling only: every step of the solver runs in the CUDA library
libtensorctl.so. PyTorch provides device memory and the CUDA stream. The
library is required: if it cannot be loaded, every call raises (there is no
CPU fallback).

Function names match the C entry points (tctl_setup, tctl_apply_op,
tctl_apply_precond, tctl_truncate, tctl_pcg_solve, tctl_fullgrid_solve, ...).
Canonical tensors are `CP` objects holding torch CUDA tensors: weights w
(cap,) and factors U (3, cap, n), so that U[l] is the column-major n x cap
factor matrix of mode l (column k = U[l, k, :]).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "CP", "Opts", "Stats", "TctlError", "load", "lib_path",
    "tctl_default_opts", "tctl_setup", "tctl_apply_op", "tctl_apply_precond",
    "tctl_truncate", "tctl_pcg_solve", "tctl_fullgrid_solve", "tctl_fullgrid_state",
    "tctl_solve_host", "tctl_get_eigs", "tctl_get_stats", "tctl_launch_count",
    "tctl_destroy", "tctl_last_error", "tctl_profile_enable", "tctl_profile_report",
    "Context", "EXPORTED",
]

EXPORTED = [
    "tctl_default_opts", "tctl_setup", "tctl_apply_op", "tctl_apply_precond",
    "tctl_truncate", "tctl_pcg_solve", "tctl_fullgrid_solve", "tctl_fullgrid_state",
    "tctl_solve_host", "tctl_cp_alloc", "tctl_cp_free", "tctl_get_eigs",
    "tctl_get_stats", "tctl_launch_count", "tctl_destroy", "tctl_last_error",
    "tctl_profile_enable", "tctl_profile_report", "tctl_eig1d_noalloc", "tctl_get_expsum",
    "tctl_expsum_fit", "tctl_gemm", "tctl_gemm_kr", "tctl_precond_fit", "tctl_precond_dataset",
    "tctl_mlp_model_size", "tctl_mlp_train", "tctl_mlp_grad", "tctl_mlp_forward",
    "tctl_apply_state", "tctl_map_constants", "tctl_solve_batch", "tctl_inject_wait_timeout",
    "tctl_expsum_dataset", "tctl_tune_report",
]

ERRORS = {0: "OK", -1: "E_ARG", -2: "E_COEFF", -3: "E_CUDA", -4: "E_NOMEM",
          -5: "E_RANK_CAP", -6: "E_NOT_CONVERGED", -7: "E_NAN", -8: "E_NUMERIC"}


class TctlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _CP(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("rank", ctypes.c_int), ("cap", ctypes.c_int),
                ("w", ctypes.c_void_p), ("U", ctypes.c_void_p * 3)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.c_void_p), ("n", ctypes.c_int), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("yw", ctypes.c_void_p), ("yU", ctypes.c_void_p),
                ("S", ctypes.c_int), ("uw", ctypes.c_void_p), ("uU", ctypes.c_void_p),
                ("cap", ctypes.c_int), ("st", ctypes.c_void_p), ("u_rank", ctypes.c_int),
                ("status", ctypes.c_int), ("latency_ms", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("pcg_rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("op_tol", ctypes.c_double), ("r_pre", ctypes.c_int),
                ("rank_cap", ctypes.c_int), ("precision", ctypes.c_int),
                ("basis", ctypes.c_int), ("expsum_src", ctypes.c_int),
                ("paper_end_rows", ctypes.c_int), ("eps_final", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("range_tol", ctypes.c_double),
                ("tc_gemm", ctypes.c_int), ("pre_src", ctypes.c_int), ("pre_r", ctypes.c_int),
                ("pre_model", ctypes.c_void_p), ("pre_delta_max", ctypes.c_double),
                ("workspace_mb", ctypes.c_int), ("op_model", ctypes.c_void_p),
                ("op_r", ctypes.c_int), ("op_judge", ctypes.c_double), ("tune", ctypes.c_int),
                ("tc_digits", ctypes.c_int), ("refine", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("rank_x", ctypes.c_int * 3), ("max_rank", ctypes.c_int),
                ("op_rank", ctypes.c_int), ("op_basis", ctypes.c_int * 3),
                ("pre_rank", ctypes.c_int), ("op_rel_err", ctypes.c_double),
                ("s_min", ctypes.c_double), ("s_max", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("expsum_used", ctypes.c_int), ("pre_used", ctypes.c_int),
                ("pre_delta", ctypes.c_double), ("ws_peak_mb", ctypes.c_double),
                ("ws_size_mb", ctypes.c_double), ("op_learned_err", ctypes.c_double),
                ("sinc24_err", ctypes.c_double), ("refines", ctypes.c_int),
                ("true_rel_res", ctypes.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libtensorctl.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libtensorctl.so is missing; run paper_2006_09314_gb300/build.py")
    lib = ctypes.CDLL(_build.LIB)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    PCP = ctypes.POINTER(_CP)
    sig = {
        "tctl_default_opts": (I, [ctypes.POINTER(Opts)]),
        "tctl_setup": (I, [ctypes.POINTER(P), P, I, D, D, D, ctypes.POINTER(Opts), P]),
        "tctl_apply_op": (I, [P, PCP, PCP]),
        "tctl_apply_precond": (I, [P, PCP, PCP]),
        "tctl_truncate": (I, [P, PCP, PCP, D]),
        "tctl_pcg_solve": (I, [P, PCP, PCP, ctypes.POINTER(Stats)]),
        "tctl_fullgrid_solve": (I, [P, P, P]),
        "tctl_fullgrid_state": (I, [P, P, P]),
        "tctl_solve_host": (I, [P, I, D, D, D, ctypes.POINTER(Opts), P, P, I, P, P, I,
                                ctypes.POINTER(I), ctypes.POINTER(Stats)]),
        "tctl_cp_alloc": (I, [P, I, PCP]),
        "tctl_cp_free": (None, [P, PCP]),
        "tctl_get_eigs": (I, [P, I, P, P]),
        "tctl_get_stats": (I, [P, ctypes.POINTER(Stats)]),
        "tctl_launch_count": (ctypes.c_longlong, [P]),
        "tctl_destroy": (None, [P]),
        "tctl_profile_enable": (I, [P, I]),
        "tctl_profile_report": (I, [P, ctypes.c_char_p, I]),
        "tctl_eig1d_noalloc": (I, [P, I, I, P, P, P]),
        "tctl_get_expsum": (I, [P, I, P, P, P, I, P]),
        "tctl_expsum_fit": (I, [D, D, D, D, D, P, P, I, P, P]),
        "tctl_gemm": (I, [P, I, I, I, I, I, I, D, P, I, P, I, D, P, I]),
        "tctl_gemm_kr": (I, [P, I, I, I, I, I, D, P, I, P, I, P, I, D, P, I]),
        "tctl_precond_fit": (I, [D, D, D, D, I, P, P, P]),
        "tctl_precond_dataset": (I, [I, I, ctypes.c_ulonglong, I, P, P, P]),
        "tctl_expsum_dataset": (I, [I, I, I, ctypes.c_ulonglong, I, P, P, P]),
        "tctl_mlp_model_size": (I, [I]),
        "tctl_mlp_train": (I, [I, I, P, P, I, I, ctypes.c_float, ctypes.c_ulonglong, P, P]),
        "tctl_mlp_grad": (I, [I, I, P, P, P, P, P]),
        "tctl_mlp_forward": (I, [I, I, P, P, P]),
        "tctl_apply_state": (I, [P, PCP, PCP]),
        "tctl_map_constants": (I, [D, D, P, P]),
        "tctl_solve_batch": (I, [P, I, D, P, I]),
        "tctl_inject_wait_timeout": (I, [P, I]),
        "tctl_tune_report": (I, [ctypes.c_char_p, I]),
        "tctl_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code, ctx=None):
    if code != 0:
        msg = load().tctl_last_error(ctx)
        raise TctlError(code, (msg or b"").decode())
    return code


def tctl_default_opts(**overrides) -> Opts:
    o = Opts()
    _check(load().tctl_default_opts(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class CP:
    """Canonical tensor in device memory: w (cap,), U (3, cap, n) torch float64 CUDA tensors."""

    def __init__(self, n, cap, device="cuda"):
        import torch
        self.n = int(n)
        self.cap = int(cap)
        self.rank = 0
        self.w = torch.zeros(max(cap, 1), dtype=torch.float64, device=device)
        self.U = torch.zeros((3, max(cap, 1), n), dtype=torch.float64, device=device)

    @classmethod
    def from_numpy(cls, w, U, cap=None, device="cuda"):
        import torch
        w = np.asarray(w, dtype=np.float64)
        S = w.shape[0]
        n = U[0].shape[0]
        out = cls(n, cap if cap is not None else S, device=device)
        out.w[:S] = torch.from_numpy(w).to(device)
        for l in range(3):
            out.U[l, :S, :] = torch.from_numpy(np.ascontiguousarray(U[l].T)).to(device)
        out.rank = S
        return out

    def to_numpy(self):
        r = self.rank
        w = self.w[:r].cpu().numpy().copy()
        U = [self.U[l, :r, :].cpu().numpy().T.copy() for l in range(3)]
        return w, U

    def _struct(self) -> _CP:
        s = _CP()
        for l in range(3):
            s.n[l] = self.n
        s.rank = self.rank
        s.cap = self.cap
        s.w = self.w.data_ptr()
        row = self.U.stride(0) * self.U.element_size()
        for l in range(3):
            s.U[l] = self.U.data_ptr() + l * row
        return s


def tctl_setup(coeffs, n, alpha, beta, eps_trunc, opts=None, stream=None):
    """Returns an opaque context handle (int). coeffs: (3, n+1) float64 host array."""
    lib = load()
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    if coeffs.shape != (3, n + 1):
        raise ValueError("coeffs must have shape (3, n+1)")
    ctx = ctypes.c_void_p()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if stream == 0:
        # torch's default stream is the legacy default stream; the library is built
        # with per-thread default streams, so name the legacy stream explicitly
        stream = 1  # cudaStreamLegacy
    _check(lib.tctl_setup(ctypes.byref(ctx), coeffs.ctypes.data, int(n), float(alpha),
                          float(beta), float(eps_trunc),
                          ctypes.byref(opts) if opts is not None else None,
                          ctypes.c_void_p(stream)))
    return ctx.value


def _apply(fn, ctx, x: CP, cap):
    y = CP(x.n, cap)
    s = y._struct()
    code = fn(ctx, ctypes.byref(x._struct()), ctypes.byref(s))
    y.rank = s.rank
    _check(code, ctx)
    return y


def tctl_apply_op(ctx, x: CP, cap=4096) -> CP:
    return _apply(load().tctl_apply_op, ctx, x, cap)


def tctl_apply_precond(ctx, x: CP, cap=4096) -> CP:
    return _apply(load().tctl_apply_precond, ctx, x, cap)


def tctl_apply_state(ctx, u: CP, cap=4096) -> CP:
    """y = trunc(A^-alpha u) (state recovery)."""
    return _apply(load().tctl_apply_state, ctx, u, cap)


def tctl_solve_batch(problems, eps_trunc, opts=None, workers=8, cap=4096):
    """Solve independent problems concurrently (host buffers).

    problems: list of dicts with coeffs (3, n+1), n, alpha, beta, yw (S,), yU (3 arrays n x S).
    Returns a list of dicts: uw, uU (list of 3 n x rank), status, latency_ms, stats.
    """
    import numpy as np
    keep = []
    items = (_BatchItem * len(problems))()
    stats = [Stats() for _ in problems]
    outs = []
    for i, p in enumerate(problems):
        n = int(p["n"])
        co = np.ascontiguousarray(p["coeffs"], np.float64)
        yw = np.ascontiguousarray(p["yw"], np.float64)
        S = yw.size
        yU = np.ascontiguousarray(np.stack([np.asarray(u, np.float64) for u in p["yU"]])
                                  .transpose(0, 2, 1))  # (3, S, n): column-major n x S per mode
        uw = np.zeros(cap)
        uU = np.zeros((3, cap, n))
        keep += [co, yw, yU, uw, uU]
        it = items[i]
        it.coeffs, it.n, it.alpha, it.beta = co.ctypes.data, n, float(p["alpha"]), float(p["beta"])
        it.yw, it.yU, it.S = yw.ctypes.data, yU.ctypes.data, S
        it.uw, it.uU, it.cap = uw.ctypes.data, uU.ctypes.data, cap
        it.st = ctypes.addressof(stats[i])
        outs.append((uw, uU))
    load().tctl_solve_batch(items, len(problems), eps_trunc,
                            ctypes.byref(opts) if opts is not None else None, workers)
    res = []
    for i, (uw, uU) in enumerate(outs):
        r = items[i].u_rank
        res.append({"uw": uw[:r].copy(), "uU": [uU[l, :r, :].T.copy() for l in range(3)],
                    "status": items[i].status, "latency_ms": items[i].latency_ms,
                    "stats": stats[i].as_dict()})
    return res


def tctl_map_constants(beta_p, gamma):
    """(beta, u_scale) of the paper's (beta_p, gamma) form."""
    b, sc = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().tctl_map_constants(beta_p, gamma, ctypes.byref(b), ctypes.byref(sc)))
    return b.value, sc.value


def tctl_truncate(ctx, x: CP, eps, cap=4096) -> CP:
    y = CP(x.n, cap)
    s = y._struct()
    code = load().tctl_truncate(ctx, ctypes.byref(x._struct()), ctypes.byref(s), float(eps))
    y.rank = s.rank
    _check(code, ctx)
    return y


def tctl_pcg_solve(ctx, b: CP, cap=4096, check=True):
    x = CP(b.n, cap)
    s = x._struct()
    st = Stats()
    code = load().tctl_pcg_solve(ctx, ctypes.byref(b._struct()), ctypes.byref(s), ctypes.byref(st))
    x.rank = s.rank
    if check:
        _check(code, ctx)
    return x, st.as_dict(), code


def tctl_fullgrid_solve(ctx, y):
    import torch
    u = torch.empty_like(y)
    _check(load().tctl_fullgrid_solve(ctx, y.data_ptr(), u.data_ptr()), ctx)
    return u


def tctl_fullgrid_state(ctx, u):
    import torch
    y = torch.empty_like(u)
    _check(load().tctl_fullgrid_state(ctx, u.data_ptr(), y.data_ptr()), ctx)
    return y


def tctl_solve_host(coeffs, n, alpha, beta, eps_trunc, yw, yU, opts=None, cap=4096):
    """Host-buffer one-shot solve. yU: list of three (n, S) arrays. Returns (uw, uU, stats)."""
    lib = load()
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    yw = np.ascontiguousarray(yw, dtype=np.float64)
    S = yw.shape[0]
    yUh = np.ascontiguousarray(np.stack([np.asarray(u, dtype=np.float64).T for u in yU]))  # (3,S,n)
    uw = np.zeros(cap)
    uU = np.zeros((3, cap, n))
    r = ctypes.c_int(0)
    st = Stats()
    code = lib.tctl_solve_host(coeffs.ctypes.data, int(n), float(alpha), float(beta),
                               float(eps_trunc), ctypes.byref(opts) if opts is not None else None,
                               yw.ctypes.data, yUh.ctypes.data, S, uw.ctypes.data, uU.ctypes.data,
                               cap, ctypes.byref(r), ctypes.byref(st))
    _check(code)
    k = r.value
    return uw[:k].copy(), [uU[l, :k, :].T.copy() for l in range(3)], st.as_dict()


def tctl_get_eigs(ctx, mode, n):
    lam = np.zeros(n)
    V = np.zeros((n, n), order="F")
    _check(load().tctl_get_eigs(ctx, int(mode), lam.ctypes.data, V.ctypes.data), ctx)
    return lam, np.asfortranarray(V)


def tctl_get_stats(ctx):
    st = Stats()
    _check(load().tctl_get_stats(ctx, ctypes.byref(st)), ctx)
    return st.as_dict()


def tctl_launch_count(ctx):
    return int(load().tctl_launch_count(ctx))


def tctl_gemm(ctx, digits, A, B, C=None, trans_a=False, trans_b=False, alpha=1.0, beta=0.0):
    """C = alpha op(A) op(B) + beta C on CUDA float64 tensors (row-major torch views).

    torch tensors are row-major, the library column-major: a row-major X is the
    column-major X^T, so C^T = op(B)^T op(A)^T is computed with swapped roles.
    """
    import torch
    for t in (A, B):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("A, B must be contiguous CUDA float64 tensors")
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[0] if trans_b else B.shape[1]
    if C is None:
        C = torch.zeros(m, n, dtype=torch.float64, device=A.device)
    # column-major view: C^T (n x m, ld n) = op(B)^T (n x k) op(A)^T (k x m)
    _check(load().tctl_gemm(ctx, digits, 1 if trans_b else 0, 1 if trans_a else 0, n, m, k, alpha,
                            B.data_ptr(), B.shape[1], A.data_ptr(), A.shape[1], beta,
                            C.data_ptr(), n), ctx)
    return C


def tctl_gemm_kr(ctx, digits, X, Y, B, C=None, alpha=1.0, beta=0.0):
    """C = alpha KR(X, Y)^T B + beta C on CUDA float64 tensors given as row-major views.

    X (ra, k), Y (rb, k), B (n, k) hold the columns of the column-major k x ra,
    k x rb, k x n operands as rows; C (n, ra rb) is the column-major
    (ra rb) x n result: C[j, a + ra b] = alpha sum_i X[a, i] Y[b, i] B[j, i].
    """
    import torch
    for t in (X, Y, B):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("X, Y, B must be contiguous CUDA float64 tensors")
    ra, k = X.shape
    rb, n = Y.shape[0], B.shape[0]
    if Y.shape[1] != k or B.shape[1] != k:
        raise ValueError("X, Y, B must share the contracted length")
    if C is None:
        C = torch.zeros(n, ra * rb, dtype=torch.float64, device=X.device)
    _check(load().tctl_gemm_kr(ctx, digits, k, ra, rb, n, alpha, X.data_ptr(), max(k, 1),
                               Y.data_ptr(), max(k, 1), B.data_ptr(), max(k, 1), beta,
                               C.data_ptr(), max(ra * rb, 1)), ctx)
    return C


def tctl_precond_fit(alpha, beta, s_min, s_max, r):
    """r free-node preconditioner sum: (theta, p, delta) (host only)."""
    import numpy as np
    th, p, d = np.zeros(r), np.zeros(r), ctypes.c_double(0)
    _check(load().tctl_precond_fit(alpha, beta, s_min, s_max, r, th.ctypes.data, p.ctypes.data,
                                   ctypes.byref(d)))
    return th, p, d.value


def tctl_precond_dataset(r, n, seed=1, threads=None):
    """(X (n, 4), Y (n, 2r), delta (n)) float32/float32/float64 (host only)."""
    import os
    import numpy as np
    threads = threads or len(os.sched_getaffinity(0))
    X = np.zeros((n, 4), np.float32)
    Y = np.zeros((n, 2 * r), np.float32)
    d = np.zeros(n)
    _check(load().tctl_precond_dataset(r, n, seed, threads, X.ctypes.data, Y.ctypes.data,
                                       d.ctypes.data))
    return X, Y, d


def tctl_expsum_dataset(which, r, n, seed=1, threads=None):
    """which 0 (operator g = F2/s) or 1 (preconditioner): (X (n, 4), Y (n, 2r), err (n))."""
    import os
    import numpy as np
    threads = threads or len(os.sched_getaffinity(0))
    X = np.zeros((n, 4), np.float32)
    Y = np.zeros((n, 2 * r), np.float32)
    e = np.zeros(n)
    _check(load().tctl_expsum_dataset(int(which), r, n, seed, threads, X.ctypes.data, Y.ctypes.data,
                                      e.ctypes.data))
    return X, Y, e


def tctl_mlp_train(r, X, Y, steps=3000, batch=256, lr=2e-3, seed=1):
    """Train the 4 -> 64 -> 64 -> 2r network on the GPU: (model float32 array, loss[2])."""
    import numpy as np
    X = np.ascontiguousarray(X, np.float32)
    Y = np.ascontiguousarray(Y, np.float32)
    model = np.zeros(load().tctl_mlp_model_size(r), np.float32)
    loss = np.zeros(2, np.float32)
    _check(load().tctl_mlp_train(r, X.shape[0], X.ctypes.data, Y.ctypes.data, steps, batch, lr, seed,
                                 model.ctypes.data, loss.ctypes.data))
    return model, loss


def tctl_mlp_grad(r, params, X, T):
    """(loss, grad) of one batch on the GPU (standardised X, T; float32)."""
    import numpy as np
    params = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    g = np.zeros_like(params)
    loss = np.zeros(1, np.float32)
    _check(load().tctl_mlp_grad(r, X.shape[0], params.ctypes.data, X.ctypes.data, T.ctypes.data,
                                g.ctypes.data, loss.ctypes.data))
    return float(loss[0]), g


def tctl_mlp_forward(r, model, X):
    """Raw (ln tau, ln q) for raw inputs X (n, 4) through the GPU inference kernel."""
    import numpy as np
    X = np.ascontiguousarray(X, np.float32)
    Y = np.zeros((X.shape[0], 2 * r), np.float32)
    _check(load().tctl_mlp_forward(r, X.shape[0], np.ascontiguousarray(model, np.float32).ctypes.data,
                                   X.ctypes.data, Y.ctypes.data))
    return Y


def tctl_expsum_fit(alpha, beta, s_min, s_max, tol, cap=256):
    """Fitted exp-sum of F2(s)/s on [s_min, s_max] (host only): (t, w, err)."""
    import numpy as np
    t = np.zeros(cap)
    w = np.zeros(cap)
    r = ctypes.c_int(0)
    err = ctypes.c_double(0)
    _check(load().tctl_expsum_fit(alpha, beta, s_min, s_max, tol, t.ctypes.data, w.ctypes.data, cap,
                                  ctypes.byref(r), ctypes.byref(err)))
    return t[:r.value].copy(), w[:r.value].copy(), err.value


def tctl_get_expsum(ctx, which=0):
    """(t, w, m) numpy arrays of the separable operator (which=0) or preconditioner (1)."""
    import numpy as np
    R = ctypes.c_int(0)
    load().tctl_get_expsum(ctx, which, None, None, None, 0, ctypes.byref(R))  # size query
    n = R.value
    t = np.zeros(max(n, 1))
    w = np.zeros(max(n, 1))
    m = np.zeros(max(n, 1), dtype=np.int32)
    _check(load().tctl_get_expsum(ctx, which, t.ctypes.data, w.ctypes.data, m.ctypes.data, n,
                                  ctypes.byref(R)), ctx)
    return t[:n], w[:n], m[:n]


def tctl_profile_enable(ctx, on=True):
    """on: False/0 off, True/1 per kernel, 2 per (PCG step, phase, kernel)."""
    _check(load().tctl_profile_enable(ctx, int(on)), ctx)


def tctl_profile_report(ctx):
    import json
    buf = ctypes.create_string_buffer(1 << 18)
    _check(load().tctl_profile_report(ctx, buf, len(buf)), ctx)
    return json.loads(buf.value.decode())


def tctl_eig1d_noalloc(coeffs_dev, n, lam_dev, V_dev, paper_end_rows=0, stream=None):
    """Allocation-free eigendecompositions into caller-provided device tensors.

    coeffs_dev: (3, n+1) float64 CUDA tensor; lam_dev: (3, n); V_dev: (3, n, n)
    (V_dev[l].T is the column-major eigenvector matrix of mode l).
    """
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if stream == 0:
        stream = 1  # cudaStreamLegacy (see tctl_setup)
    _check(load().tctl_eig1d_noalloc(coeffs_dev.data_ptr(), int(n), int(paper_end_rows),
                                     lam_dev.data_ptr(), V_dev.data_ptr(), ctypes.c_void_p(stream)))


def tctl_inject_wait_timeout(ctx, count=1):
    """The next `count` tensor-core GEMM launches of ctx starve a bounded wait (test hook)."""
    _check(load().tctl_inject_wait_timeout(ctx, int(count)), ctx)


def tctl_tune_report():
    """The tile autotuner's decisions so far (list of dicts)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().tctl_tune_report(buf, len(buf)))
    return json.loads(buf.value.decode())


def tctl_destroy(ctx):
    load().tctl_destroy(ctx)


def tctl_last_error(ctx=None):
    return (load().tctl_last_error(ctx) or b"").decode()


class Context:
    """Owns one tensorctl context (RAII wrapper around tctl_setup/tctl_destroy)."""

    def __init__(self, coeffs, n, alpha, beta, eps_trunc, opts=None, stream=None):
        self.n = int(n)
        self.handle = tctl_setup(coeffs, n, alpha, beta, eps_trunc, opts, stream)

    def close(self):
        if self.handle:
            tctl_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_op(self, x, cap=4096):
        return tctl_apply_op(self.handle, x, cap)

    def apply_precond(self, x, cap=4096):
        return tctl_apply_precond(self.handle, x, cap)

    def apply_state(self, u, cap=4096):
        return tctl_apply_state(self.handle, u, cap)

    def truncate(self, x, eps, cap=4096):
        return tctl_truncate(self.handle, x, eps, cap)

    def pcg_solve(self, b, cap=4096, check=True):
        return tctl_pcg_solve(self.handle, b, cap, check)

    def fullgrid_solve(self, y):
        return tctl_fullgrid_solve(self.handle, y)

    def fullgrid_state(self, u):
        return tctl_fullgrid_state(self.handle, u)

    def eigs(self, mode):
        return tctl_get_eigs(self.handle, mode, self.n)

    def stats(self):
        return tctl_get_stats(self.handle)

    def launch_count(self):
        return tctl_launch_count(self.handle)

    def gemm(self, digits, A, B, C=None, trans_a=False, trans_b=False, alpha=1.0, beta=0.0):
        return tctl_gemm(self.handle, digits, A, B, C, trans_a, trans_b, alpha, beta)

    def gemm_kr(self, digits, X, Y, B, C=None, alpha=1.0, beta=0.0):
        return tctl_gemm_kr(self.handle, digits, X, Y, B, C, alpha, beta)

    def expsum(self, which=0):
        return tctl_get_expsum(self.handle, which)

    def profile(self, on=True):
        tctl_profile_enable(self.handle, on)

    def profile_report(self):
        return tctl_profile_report(self.handle)

    def inject_wait_timeout(self, count=1):
        tctl_inject_wait_timeout(self.handle, count)
