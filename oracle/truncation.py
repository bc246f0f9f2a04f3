"""Rank truncation `trunc(X, eps)` of canonical tensors (oracle, Appendix 1).

Appendix 1 truncates by the canonical-to-Tucker transform with the reduced
HOSVD (RHOSVD: truncated SVD of each side matrix U^(l) = [u_1^(l) .. u_R^(l)],
no full tensor), followed by the Tucker-to-canonical transform of the small
core (slice SVDs; canonical rank <= r^2 in 3D). The paper does not fix the
threshold semantics; the reading used here (implemented independently in the
GPU library) makes the error relative to ||X|| and exact where it can be:

  1. normalise every factor column, moving the norms into the weights;
  2. RHOSVD per mode: QR of the weighted side matrix U_l diag(|w|), SVD of R;
     keep the leading left singular vectors until the tail of the singular
     values drops to 1e-2 * eps * ||X|| / sqrt(3) (a tight, nearly lossless
     projection; ||X|| from the exact canonical inner product);
  3. Tucker core beta = sum_k w_k (x_l Q_l^T u_k^(l));
  4. HOSVD of the core with per-mode tails sum_{i>r} sigma_i^2 <= eps_B^2 ||beta||^2 / 3
     (the errors of steps 4 and 5 are orthogonal, both are exact Frobenius
     norms because the Tucker bases are orthonormal);
  5. Tucker-to-canonical: SVD of every slice beta[:, :, c]; the smallest
     singular triplets over all slices are dropped while their squared sum
     stays <= eps_C^2 ||beta||^2.

With eps_B = eps_C = eps/sqrt(2) the total relative error is at most eps
(plus the ~1e-2 eps of step 2). For Tucker output (step 5 skipped) eps_B = eps.
"""
from __future__ import annotations

import math

import numpy as np

from .formats import cp_norm

__all__ = ["trunc", "c2t", "tucker_truncate", "t2c"]


def c2t(w, U, nrm, eps_a):
    """Steps 1-3: canonical -> Tucker (orthonormal Q_l, core beta)."""
    w = np.asarray(w, dtype=np.float64)
    nu = [np.linalg.norm(u, axis=0) for u in U]
    keep = (nu[0] > 0) & (nu[1] > 0) & (nu[2] > 0) & (w != 0)
    wt = w[keep] * nu[0][keep] * nu[1][keep] * nu[2][keep]
    Ub = [U[l][:, keep] / nu[l][keep][None, :] for l in range(3)]
    Qs, Cs = [], []
    for l in range(3):
        Y = Ub[l] * np.abs(wt)[None, :]
        Q, R = np.linalg.qr(Y, mode="reduced")
        P, sv, _ = np.linalg.svd(R, full_matrices=False)
        tail = np.sqrt(np.cumsum((sv ** 2)[::-1]))[::-1]
        r = max(1, int(np.sum(tail > eps_a * nrm / math.sqrt(3.0))))
        L = Q @ P[:, :r]
        Qs.append(L)
        Cs.append(L.T @ Ub[l])
    core = np.einsum("k,ak,bk,ck->abc", wt, Cs[0], Cs[1], Cs[2], optimize=True)
    return core, Qs


def tucker_truncate(core, Qs, eps_b):
    """Step 4: HOSVD of the core with sum of per-mode tails^2 <= eps_b^2 ||core||^2."""
    tot2 = float(np.sum(core * core))
    Ws = []
    for l in range(3):
        M = np.moveaxis(core, l, 0).reshape(core.shape[l], -1)
        Uu, sv, _ = np.linalg.svd(M, full_matrices=False)
        tail2 = np.cumsum((sv ** 2)[::-1])[::-1]
        r = max(1, int(np.sum(tail2 > eps_b ** 2 * tot2 / 3.0)))
        Ws.append(Uu[:, :r])
    core = np.einsum("abc,ai,bj,ck->ijk", core, Ws[0], Ws[1], Ws[2], optimize=True)
    return core, [Qs[l] @ Ws[l] for l in range(3)]


def t2c(core, Qs, eps_c):
    """Step 5: Tucker -> canonical through SVDs of the mode-3 slices."""
    tot2 = float(np.sum(core * core))
    trip = []
    for c in range(core.shape[2]):
        a, sv, bt = np.linalg.svd(core[:, :, c], full_matrices=False)
        for i in range(sv.shape[0]):
            trip.append((sv[i], c, i, a[:, i], bt[i, :]))
    order = sorted(range(len(trip)), key=lambda j: trip[j][0])
    drop = set()
    acc = 0.0
    for j in order:
        s2 = trip[j][0] ** 2
        if acc + s2 > eps_c ** 2 * tot2:
            break
        acc += s2
        drop.add(j)
    kept = [trip[j] for j in range(len(trip)) if j not in drop]
    if not kept:
        return np.zeros(0), [np.zeros((q.shape[0], 0)) for q in Qs]
    w = np.array([t[0] for t in kept])
    U1 = Qs[0] @ np.array([t[3] for t in kept]).T
    U2 = Qs[1] @ np.array([t[4] for t in kept]).T
    U3 = Qs[2][:, [t[1] for t in kept]]
    return w, [U1, U2, U3]


def trunc(w, U, eps, output="canonical"):
    """trunc(X, eps) of Algorithm 1; returns canonical (w, U) or Tucker (core, Q)."""
    n = [u.shape[0] for u in U]
    nrm = cp_norm(w, U)
    if len(w) == 0 or nrm == 0.0:
        if output == "tucker":
            return np.zeros((0, 0, 0)), [np.zeros((nl, 0)) for nl in n]
        return np.zeros(0), [np.zeros((nl, 0)) for nl in n]
    core, Qs = c2t(w, U, nrm, 1e-2 * eps)
    if output == "tucker":
        return tucker_truncate(core, Qs, eps)
    core, Qs = tucker_truncate(core, Qs, eps / math.sqrt(2.0))
    return t2c(core, Qs, eps / math.sqrt(2.0))
