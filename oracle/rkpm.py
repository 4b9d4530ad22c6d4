"""Oracle: support neighbours and corrected RKPM shape functions, plain FP64.

Test infrastructure only (see ``oracle/__init__``).

Paper: Sec. 3.2 "RKPM", Eqs. 6-11.  A field is u(X) = sum_k phi_k(X) c_k with
    phi_k(X) = varphi_k(X) P(p_k)^T C(X)                         (Eq. 7)
    M(X) C(X) = P(X),  M(X) = sum_k varphi_k(X) P(p_k) P(p_k)^T  (Eqs. 9-10)
    P(X) = [1, x, y, z]^T (linear basis, D = 1).
The reproducing condition sum_k phi_k(X) P(p_k) = P(X) (Eq. 8) is the pin.

Readings taken where the paper is silent:
* raw kernel varphi_k: the cubic B-spline of radius a_k (unnormalised) instead
  of the paper's Gaussian (the workloads ask for it);
* neighbour rule: node k contributes at X iff ||X - p_k||^2 < a_k^2, tested in
  FP64 on the FP32-stored inputs as ((dx*dx + dy*dy) + dz*dz) < a_k*a_k with no
  fused multiply-add;
* basis origin: P_o(p) = [1, (p - o)/s] with the constant origin o = X_i and
  scale s = a_i of the evaluation point.  This is an invertible affine change of
  the paper's basis P, so phi and grad phi are identical in exact arithmetic
  (``shape_functions_at`` also evaluates the paper's literal basis for the pin).
"""
from __future__ import annotations

import numpy as np

F64 = np.float64


# ---------------------------------------------------------------- raw kernel
def cubic_bspline(q):
    """Cubic B-spline w(q), q = r / a:  2/3 - 4q^2 + 4q^3 on [0, 1/2],
    (4/3)(1 - q)^3 on (1/2, 1], zero beyond.  C^2 at q = 1/2 and q = 1."""
    q = np.asarray(q, dtype=F64)
    inner = 2.0 / 3.0 - 4.0 * q * q + 4.0 * q * q * q
    outer = (4.0 / 3.0) * (1.0 - q) ** 3
    return np.where(q <= 0.5, inner, np.where(q <= 1.0, outer, 0.0))


def cubic_bspline_dw_over_q(q):
    """w'(q) / q, finite at q = 0:  -8 + 12 q on [0, 1/2],
    -4 (1 - q)^2 / q on (1/2, 1], zero beyond."""
    q = np.asarray(q, dtype=F64)
    inner = -8.0 + 12.0 * q
    qs = np.where(q > 0.5, q, 1.0)
    outer = -4.0 * (1.0 - q) ** 2 / qs
    return np.where(q <= 0.5, inner, np.where(q <= 1.0, outer, 0.0))


# ---------------------------------------------------------------- neighbours
def neighbours(X, a, chunk=128):
    """Brute-force support neighbours N(i) = {k : ||X_i - p_k|| < a_k}.

    Nodal discretisation: every particle is both a node p_k = X_k and a
    quadrature point X_i.  ``X`` is (N, 3) float32, ``a`` (N,) float32.
    Returns CSR (ptr int64 (N+1), idx int32) with each row ascending and the
    particle itself included.  The squared distance is evaluated in FP64 from
    the FP32 inputs in the fixed order ((dx*dx + dy*dy) + dz*dz); numpy applies
    each operation separately, so no fused multiply-add enters.
    """
    X = np.asarray(X, dtype=np.float32)
    a = np.asarray(a, dtype=np.float32)
    n = X.shape[0]
    Xd = X.astype(F64)
    a2 = a.astype(F64) * a.astype(F64)
    rows, cols = [], []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        dx = Xd[s:e, None, 0] - Xd[None, :, 0]
        dy = Xd[s:e, None, 1] - Xd[None, :, 1]
        dz = Xd[s:e, None, 2] - Xd[None, :, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        r, c = np.nonzero(d2 < a2[None, :])
        rows.append(r + s)
        cols.append(c)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr, cols.astype(np.int32)


def neighbours_query(Xq, P, a):
    """Support neighbours of arbitrary query points Xq among nodes P (radius a).
    Same predicate as ``neighbours``; returns a list of index arrays."""
    Xq = np.asarray(Xq, dtype=F64)
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    a2 = np.asarray(a, dtype=np.float32).astype(F64) ** 2
    out = []
    for x in Xq:
        d = x[None, :] - Pd
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        out.append(np.nonzero(d2 < a2)[0].astype(np.int32))
    return out


# ---------------------------------------------------------------- shape functions
def _raw_kernel_and_grad(Xq, p, a):
    """varphi_k(X) = w(|X - p_k| / a_k) and its gradient in X, per pair.
    grad = (w'(q)/q) (X - p_k) / a_k^2."""
    r = Xq - p                                   # X - p_k, (m, 3)
    dist = np.sqrt(np.einsum("ij,ij->i", r, r))
    q = dist / a
    w = cubic_bspline(q)
    g = (cubic_bspline_dw_over_q(q) / (a * a))[:, None] * r
    return w, g


def shape_functions(X, a, ptr, idx):
    """Corrected RKPM shape functions at the particles themselves.

    For every pair (i, k) in the CSR (row i = evaluation point X_i, column k =
    node p_k) returns phi_k(X_i) and grad phi_k(X_i), aligned with ``idx``,
    plus the 1-norm condition number of each moment matrix M(X_i).

    Steps (Sec. 3.2, Eqs. 7, 9-10, with the shifted basis of the module note):
      P_k    = [1, (p_k - X_i)/s_i]            s_i = a_i
      M      = sum_k w_k P_k P_k^T,   dM_s = sum_k d_s w_k P_k P_k^T
      C      = M^{-1} e_0                       (P_o(X_i) = e_0)
      d_s C  = M^{-1} (e_{1+s}/s_i - dM_s C)    (derivative of M C = P_o)
      phi_k  = w_k P_k^T C
      d_s phi_k = d_s w_k P_k^T C + w_k P_k^T d_s C
    """
    X = np.asarray(X, dtype=np.float32).astype(F64)
    a = np.asarray(a, dtype=np.float32).astype(F64)
    n = X.shape[0]
    rows = np.repeat(np.arange(n), np.diff(ptr))
    cols = idx.astype(np.int64)
    Xi, pk = X[rows], X[cols]
    w, g = _raw_kernel_and_grad(Xi, pk, a[cols])
    s = a[rows]
    Pk = np.empty((rows.size, 4))
    Pk[:, 0] = 1.0
    Pk[:, 1:] = (pk - Xi) / s[:, None]
    outer = Pk[:, :, None] * Pk[:, None, :]                     # (m, 4, 4)
    starts = ptr[:-1]
    M = np.add.reduceat(w[:, None, None] * outer, starts, axis=0)
    dM = np.stack([np.add.reduceat(g[:, d, None, None] * outer, starts, axis=0)
                   for d in range(3)], axis=1)                   # (n, 3, 4, 4)
    e0 = np.zeros((n, 4, 1))
    e0[:, 0, 0] = 1.0
    C = np.linalg.solve(M, e0)[:, :, 0]                           # (n, 4)
    dC = np.empty((n, 3, 4))
    for d in range(3):
        rhs = -np.einsum("nij,nj->ni", dM[:, d], C)
        rhs[:, 1 + d] += 1.0 / a
        dC[:, d] = np.linalg.solve(M, rhs[:, :, None])[:, :, 0]
    PC = np.einsum("mj,mj->m", Pk, C[rows])
    phi = w * PC
    dphi = np.empty((3, rows.size))
    for d in range(3):
        dphi[d] = g[:, d] * PC + w * np.einsum("mj,mj->m", Pk, dC[rows, d])
    cond = np.linalg.cond(M, p=1)
    return phi, dphi, cond


def shape_functions_at(Xq, P, a, literal_basis=False, scale=None):
    """phi_k and grad phi_k at arbitrary query points, dense (Nq x K).

    Used by the pins: finite differences of phi in X, and the comparison of the
    shifted basis against the paper's literal basis P(X) = [1, x, y, z]
    (``literal_basis=True``; there C = M^{-1} P(X) and d_s P(X) = e_{1+s})."""
    Xq = np.asarray(Xq, dtype=F64)
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    ad = np.asarray(a, dtype=np.float32).astype(F64)
    nq, K = Xq.shape[0], Pd.shape[0]
    nb = neighbours_query(Xq, P, a)
    phi = np.zeros((nq, K))
    dphi = np.zeros((3, nq, K))
    for j in range(nq):
        ks = nb[j]
        x = Xq[j]
        w, g = _raw_kernel_and_grad(np.broadcast_to(x, (ks.size, 3)), Pd[ks], ad[ks])
        if literal_basis:
            o, s = np.zeros(3), 1.0
        else:
            # FP64 scale: a float32 scalar here would make 1.0 / s below a
            # float32 (NumPy 2 promotion) and round the e_{1+s}/s term
            o, s = x, (float(scale[j]) if scale is not None else 1.0)
        Pk = np.concatenate([np.ones((ks.size, 1)), (Pd[ks] - o) / s], axis=1)
        Px = np.concatenate([[1.0], (x - o) / s])
        M = (w[:, None, None] * Pk[:, :, None] * Pk[:, None, :]).sum(0)
        C = np.linalg.solve(M, Px)
        phi[j, ks] = w * (Pk @ C)
        for d in range(3):
            dM = (g[:, d, None, None] * Pk[:, :, None] * Pk[:, None, :]).sum(0)
            dP = np.zeros(4)
            dP[1 + d] = 1.0 / s
            dC = np.linalg.solve(M, dP - dM @ C)
            dphi[d, j, ks] = g[:, d] * (Pk @ C) + w * (Pk @ dC)
    return phi, dphi


def connected_components(n, ptr, idx):
    """Number of connected components of the (symmetrised) support graph.
    Equals the multiplicity of the zero eigenvalue of H_w."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components as cc
    G = sp.csr_matrix((np.ones(idx.size), idx, ptr), shape=(n, n))
    return int(cc(G, directed=True, connection="weak")[0])
