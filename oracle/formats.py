"""Canonical and Tucker tensors by definition (oracle, Appendix 1).

Canonical ("CP_form"):  T = sum_k w_k u_k^(1) x u_k^(2) x u_k^(3),
stored as (w (R,), [U1 (n1,R), U2 (n2,R), U3 (n3,R)]).
Tucker: T = sum_{a,b,c} beta[a,b,c] v_a^(1) x v_b^(2) x v_c^(3),
stored as (beta (r1,r2,r3), [V1 (n1,r1), V2, V3]).

The Euclidean inner product of two canonical tensors is
<A1, A2> = sum_k sum_m c_k b_m prod_l <u_k^(l), v_m^(l)>, and their Hadamard
product is sum_k sum_m c_k b_m (x_l u_k^(l) .* v_m^(l)) with rank R1*R2.
The sum X + a P of canonical tensors is the concatenation of their terms
with weights scaled (the axpy lines of Algorithm 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "cp_full",
    "cp_inner",
    "cp_norm",
    "cp_hadamard",
    "cp_axpby",
    "cp_empty",
    "tucker_full",
    "cp_to_eigenbasis",
    "cp_from_eigenbasis",
]


def cp_full(w, U) -> np.ndarray:
    """Expand a canonical tensor to (n1, n2, n3): sum_k w_k u_k^(1) x u_k^(2) x u_k^(3)."""
    w = np.asarray(w, dtype=np.float64)
    if w.shape[0] == 0:
        return np.zeros([u.shape[0] for u in U])
    return np.einsum("k,ik,jk,lk->ijl", w, U[0], U[1], U[2], optimize=True)


def cp_inner(w1, U1, w2, U2) -> float:
    """<A1, A2> = sum_k sum_m c_k b_m prod_l <u_k^(l), v_m^(l)> (Appendix 1)."""
    w1 = np.asarray(w1, dtype=np.float64)
    w2 = np.asarray(w2, dtype=np.float64)
    total = 0.0
    B = 1024  # rows of the R1 x R2 product matrix formed at a time
    for k0 in range(0, w1.shape[0], B):
        G = np.ones((min(B, w1.shape[0] - k0), w2.shape[0]))
        for l in range(3):
            G *= U1[l][:, k0:k0 + B].T @ U2[l]
        total += float(w1[k0:k0 + B] @ G @ w2)
    return total


def cp_norm(w, U) -> float:
    """Euclidean norm of a canonical tensor.

    On grids with at most 2^18 points the tensor is expanded (cost R n^3);
    otherwise the Appendix 1 inner product is used (cost R^2 n).
    """
    if len(w) == 0:
        return 0.0
    if U[0].shape[0] * U[1].shape[0] * U[2].shape[0] <= 1 << 18:
        return float(np.linalg.norm(cp_full(w, U)))
    return float(np.sqrt(max(cp_inner(w, U, w, U), 0.0)))


def cp_hadamard(w1, U1, w2, U2):
    """Canonical Hadamard product, rank R1*R2 (Appendix 1); term (k, m) at k*R2 + m."""
    w = np.outer(w1, w2).ravel()
    U = [(U1[l][:, :, None] * U2[l][:, None, :]).reshape(U1[l].shape[0], -1) for l in range(3)]
    return w, U


def cp_axpby(a, w1, U1, b, w2, U2):
    """a*A1 + b*A2 as the concatenation of terms."""
    w = np.concatenate([a * np.asarray(w1, dtype=np.float64), b * np.asarray(w2, dtype=np.float64)])
    U = [np.concatenate([U1[l], U2[l]], axis=1) for l in range(3)]
    return w, U


def cp_empty(n):
    return np.zeros(0), [np.zeros((nl, 0)) for nl in n]


def tucker_full(core, V) -> np.ndarray:
    return np.einsum("abc,ia,jb,kc->ijk", core, V[0], V[1], V[2])


def cp_to_eigenbasis(w, U, Vs):
    """Factors of (V1^T x V2^T x V3^T) T: mode-wise V_l^T U_l."""
    return np.asarray(w, dtype=np.float64), [Vs[l].T @ U[l] for l in range(3)]


def cp_from_eigenbasis(w, Uh, Vs):
    return np.asarray(w, dtype=np.float64), [Vs[l] @ Uh[l] for l in range(3)]
