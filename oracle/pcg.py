"""Preconditioned CG in low-rank canonical format (oracle, Appendix 2, Algorithm 1).

fun(X) is the matrix-vector product "Gen3DtimesX" of Section 3.3:
    F(A) x ~= sum_k sum_j (x)_l G_l^T ( u_l^(k) .* G_l x_l^(j) ),
with G_l = V_l^T the eigenvector rows, u^(k) the canonical factors of the
separable representation of F2 (operator) or of the preconditioner function
(Section 3.5, case (B)), applied in this order: mode products with G_l, the
Hadamard/Khatri-Rao product, mode products with G_l^T. Every new vector is
truncated by `trunc` (Appendix 1) at the lines Algorithm 1 marks.

Stopping rule (the printed integral criterion is not a norm): stop when the
recursive residual satisfies ||R|| <= rtol ||B|| (Euclidean norm over the
grid, Section 3.1 uses M = I for finite differences), at most kmax steps.
"""
from __future__ import annotations

import math

import numpy as np

from . import formats as F
from .truncation import trunc

__all__ = ["cp_apply", "pcg"]


def cp_apply(dw, dU, Vs, w, U):
    """sum_k sum_j (x)_l V_l ( d_l^(k) .* V_l^T x_l^(j) ) (the paper's G = V^T)."""
    Uh = [Vs[l].T @ U[l] for l in range(3)]
    hw, hU = F.cp_hadamard(dw, dU, w, Uh)
    return hw, [Vs[l] @ hU[l] for l in range(3)]


def pcg(op, pre, Vs, bw, bU, eps, rtol=1e-7, kmax=100, x0=None):
    """Algorithm 1. op/pre = (weights, factors) of the separable symbols in the eigenbasis.

    Returns (xw, xU, info) with info = dict(iters, rel_res, history).
    """
    n = [u.shape[0] for u in bU]
    fun = lambda w, U: cp_apply(op[0], op[1], Vs, w, U)
    precond = lambda w, U: cp_apply(pre[0], pre[1], Vs, w, U)
    bnorm = F.cp_norm(bw, bU)
    if x0 is None:
        xw, xU = F.cp_empty(n)
        rw, rU = bw, bU
    else:
        xw, xU = x0
        fw, fU = fun(xw, xU)
        rw, rU = trunc(*F.cp_axpby(1.0, bw, bU, -1.0, fw, fU), eps)
    zw, zU = trunc(*precond(rw, rU), eps)
    pw, pU = zw, zU
    hist = []
    rz = F.cp_inner(rw, rU, zw, zU)
    k = 0
    rel = F.cp_norm(rw, rU) / bnorm
    while k < kmax:
        sw, sU = trunc(*fun(pw, pU), eps)
        a = rz / F.cp_inner(pw, pU, sw, sU)
        xw, xU = trunc(*F.cp_axpby(1.0, xw, xU, a, pw, pU), eps)
        rw, rU = trunc(*F.cp_axpby(1.0, rw, rU, -a, sw, sU), eps)
        rel = F.cp_norm(rw, rU) / bnorm
        hist.append(rel)
        k += 1
        if rel <= rtol:
            break
        zw, zU = trunc(*precond(rw, rU), eps)
        rz_new = F.cp_inner(rw, rU, zw, zU)
        b = rz_new / rz
        rz = rz_new
        pw, pU = trunc(*F.cp_axpby(1.0, zw, zU, b, pw, pU), eps)
    return xw, xU, dict(iters=k, rel_res=rel, history=hist)
