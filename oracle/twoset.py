"""Oracle: the paper's two-set RKPM discretisation, plain FP64.

Test infrastructure only (see ``oracle/__init__``).

The paper's own construction (Supp. Sec. B "RKPM construction", with the
kernel of Sec. 3.2) keeps two point sets apart:

* quadrature points X_i with volumes v_i -- a uniform grid over the object's
  bounding box with the points outside the object rejected (or, for splats,
  the given points themselves); they carry the integrals of Prop. 1 and Eq. 14;
* K kernel centres p_k, about a thousand, chosen from the quadrature points by
  farthest-point sampling so that they are spread evenly;
* the raw kernel, a Gaussian  varphi_k(X) = exp(-|X - p_k|^2 / r_k^2)  (Sec. 3.2),
  with r_k the smallest radius around p_k that reaches two other centres,
  i.e. the distance from p_k to its second-nearest other centre.

The corrected shape functions are those of Eqs. 7, 9-10 with the linear basis,
evaluated at the quadrature points; H_w (Prop. 1) and M (Eq. 14) are K x K.

Readings taken where the paper is silent:
* farthest-point sampling starts from the first point in the order given and
  breaks ties in distance towards the lowest index; distances are compared
  squared, in FP64, from the FP32-stored points, as ((dx*dx + dy*dy) + dz*dz)
  with no fused multiply-add;
* the radius is the square root of that squared distance;
* support: the paper's Gaussian never vanishes.  ``trunc = t`` cuts it at
  t r_k (node k covers X iff |X - p_k|^2 < t^2 r_k^2, the same predicate as
  the nodal path); ``trunc=None`` keeps every centre at every point.  The
  cut-off kernel differs from the full one by less than exp(-t^2) per weight;
* basis origin and scale: P_o(p) = [1, (p - X)/s] around the evaluation point X
  with one positive scale s for the cloud (an invertible affine change of the
  paper's basis: phi and grad phi are unchanged in exact arithmetic).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import lame

F64 = np.float64


def _d2(A, b):
    """Squared distances from the rows of A to the point b, FP64, fixed order."""
    dx = A[:, 0] - b[0]
    dy = A[:, 1] - b[1]
    dz = A[:, 2] - b[2]
    return (dx * dx + dy * dy) + dz * dz


# ---------------------------------------------------------------- centres
def farthest_point_sampling(X, K, start=0):
    """Indices of K points of X chosen greedily: each next point is the one
    farthest from those already chosen (Supp. Sec. B).  Returns int64 (K,) in
    the order of choice.  Ties go to the lowest index (``np.argmax`` returns
    the first maximum).  Raises ValueError when the points hold fewer than K
    distinct positions (the farthest remaining point is at distance zero)."""
    Xd = np.asarray(X, dtype=np.float32).astype(F64)
    n = Xd.shape[0]
    if not 0 < K <= n:
        raise ValueError("K must lie in 1..n")
    chosen = np.empty(K, dtype=np.int64)
    chosen[0] = start
    dist = _d2(Xd, Xd[start])                  # squared distance to the chosen set
    for j in range(1, K):
        nxt = int(np.argmax(dist))
        if dist[nxt] == 0.0:
            raise ValueError("fewer than K distinct points")
        chosen[j] = nxt
        dist = np.minimum(dist, _d2(Xd, Xd[nxt]))
    return chosen


def covering_radius(X, centres):
    """max_i min_k |X_i - p_k|: how far the farthest point is from a centre."""
    Xd = np.asarray(X, dtype=np.float32).astype(F64)
    d = np.full(Xd.shape[0], np.inf)
    for k in centres:
        d = np.minimum(d, _d2(Xd, Xd[k]))
    return float(np.sqrt(d.max()))


def radii(P):
    """r_k = distance from p_k to its second-nearest other centre: the smallest
    ball around p_k that reaches two other centres (Supp. Sec. B).  Needs K >= 3."""
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    K = Pd.shape[0]
    if K < 3:
        raise ValueError("the radius rule needs at least three centres")
    r = np.empty(K)
    for k in range(K):
        d2 = _d2(Pd, Pd[k])
        d2[k] = np.inf
        r[k] = np.sqrt(np.partition(d2, 1)[1])
    return r


# ---------------------------------------------------------------- kernel
def gaussian(d2, r):
    """varphi = exp(-d^2 / r^2) (Sec. 3.2) from the squared distance."""
    return np.exp(-np.asarray(d2, F64) / (np.asarray(r, F64) ** 2))


def covering(Xq, P, r, trunc):
    """CSR (ptr, idx) of the centres covering each quadrature point: every
    centre when ``trunc`` is None, else those with |X - p_k|^2 < trunc^2 r_k^2.
    Columns ascend in each row."""
    Xd = np.asarray(Xq, dtype=np.float32).astype(F64)
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    n, K = Xd.shape[0], Pd.shape[0]
    if trunc is None:
        ptr = np.arange(n + 1, dtype=np.int64) * K
        return ptr, np.tile(np.arange(K, dtype=np.int32), n)
    t = float(trunc)
    rr = np.asarray(r, F64)
    lim = (t * t) * (rr * rr)
    cols = [np.nonzero(_d2(Pd, x) < lim)[0].astype(np.int32) for x in Xd]
    ptr = np.zeros(n + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([c.size for c in cols])
    return ptr, (np.concatenate(cols) if cols else np.zeros(0, np.int32))


def shape_functions(Xq, P, r, trunc=None, scale=None, chunk=2048):
    """Corrected RKPM shape functions with the Gaussian kernel at the quadrature
    points (Eqs. 7, 9-10).

    Returns (ptr, idx, phi, dphi, cond): the covering CSR, phi_k(X_i) and
    grad phi_k(X_i) (3 x nnz) aligned with ``idx``, and the 1-norm condition
    number of each moment matrix.  Per quadrature point X with covering
    centres k (basis P_k = [1, (p_k - X)/s], so P_o(X) = e_0):
      w_k  = exp(-|X - p_k|^2 / r_k^2),   grad w_k = -2 w_k (X - p_k) / r_k^2
      M    = sum_k w_k P_k P_k^T,         dM_s = sum_k d_s w_k P_k P_k^T
      C    = M^{-1} e_0,                  d_s C = M^{-1}(e_{1+s}/s - dM_s C)
      phi_k = w_k P_k^T C,  d_s phi_k = d_s w_k P_k^T C + w_k P_k^T d_s C
    A point covered by fewer than four non-coplanar centres has a singular M
    and raises ``numpy.linalg.LinAlgError``."""
    Xd = np.asarray(Xq, dtype=np.float32).astype(F64)
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    rd = np.asarray(r, F64)
    s = float(np.median(rd)) if scale is None else float(scale)
    ptr, idx = covering(Xq, P, r, trunc)
    n = Xd.shape[0]
    nnz = idx.size
    phi = np.empty(nnz)
    dphi = np.empty((3, nnz))
    cond = np.empty(n)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        lo, hi = ptr[a], ptr[b]
        rows = np.repeat(np.arange(a, b), np.diff(ptr[a:b + 1]))
        cols = idx[lo:hi].astype(np.int64)
        rel = Xd[rows] - Pd[cols]                                  # X - p_k
        d2 = (rel[:, 0] * rel[:, 0] + rel[:, 1] * rel[:, 1]) + rel[:, 2] * rel[:, 2]
        rk2 = rd[cols] ** 2
        w = np.exp(-d2 / rk2)
        g = (-2.0 * w / rk2)[:, None] * rel
        Pk = np.empty((rows.size, 4))
        Pk[:, 0] = 1.0
        Pk[:, 1:] = -rel / s
        outer = Pk[:, :, None] * Pk[:, None, :]
        starts = ptr[a:b] - lo
        M = np.add.reduceat(w[:, None, None] * outer, starts, axis=0)
        dM = np.stack([np.add.reduceat(g[:, d, None, None] * outer, starts, axis=0)
                       for d in range(3)], axis=1)
        e0 = np.zeros((b - a, 4, 1))
        e0[:, 0, 0] = 1.0
        C = np.linalg.solve(M, e0)[:, :, 0]
        dC = np.empty((b - a, 3, 4))
        for d in range(3):
            rhs = -np.einsum("nij,nj->ni", dM[:, d], C)
            rhs[:, 1 + d] += 1.0 / s
            dC[:, d] = np.linalg.solve(M, rhs[:, :, None])[:, :, 0]
        loc = rows - a
        PC = np.einsum("mj,mj->m", Pk, C[loc])
        phi[lo:hi] = w * PC
        for d in range(3):
            dphi[d, lo:hi] = g[:, d] * PC + w * np.einsum("mj,mj->m", Pk, dC[loc, d])
        cond[a:b] = np.linalg.cond(M, p=1)
    return ptr, idx, phi, dphi, cond


# ---------------------------------------------------------------- H_w and M
def operators(n, K, ptr, idx, phi, dphi):
    """Phi (n x K: rows quadrature points, columns centres) and G_s = d_s Phi."""
    Phi = sp.csr_matrix((np.asarray(phi, F64), idx, ptr), shape=(n, K))
    G = [sp.csr_matrix((np.asarray(dphi[t], F64), idx, ptr), shape=(n, K)) for t in range(3)]
    return Phi, G


def assemble(n, K, ptr, idx, phi, dphi, v, E, nu, dense=False):
    """H_w = sum_s G_s^T diag(v (lambda + 4 mu)) G_s (Prop. 1) and
    M = Phi^T diag(v) Phi (Eq. 14), K x K.  E, nu scalars or per quadrature point."""
    E = np.broadcast_to(np.asarray(E, F64), (n,))
    nu = np.broadcast_to(np.asarray(nu, F64), (n,))
    lam, mu = lame(E, nu)
    v = np.broadcast_to(np.asarray(v, F64), (n,))
    Phi, G = operators(n, K, ptr, idx, phi, dphi)
    Dh = sp.diags(v * (lam + 4.0 * mu))
    H = (G[0].T @ Dh @ G[0] + G[1].T @ Dh @ G[1] + G[2].T @ Dh @ G[2]).tocsr()
    M = (Phi.T @ sp.diags(v) @ Phi).tocsr()
    if dense:
        return H.toarray(), M.toarray()
    H.sort_indices()
    M.sort_indices()
    return H, M


def rows(ks, Xq, v, P, r, trunc, E, nu, scale):
    """Rows ks of H_w (Prop. 1) and M (Eq. 14) of a two-set cloud of any size,
    from the definition evaluated only where it is non-zero: row k sums over
    the quadrature points centre k covers, each with the shape functions of
    all its covering centres.  E, nu scalars or per point.  Returns a list of
    (cols, H_row, M_row), cols ascending, FP64."""
    Xq = np.asarray(Xq, dtype=np.float32)
    n = Xq.shape[0]
    Xd = Xq.astype(F64)
    Pd = np.asarray(P, dtype=np.float32).astype(F64)
    rd = np.asarray(r, F64)
    lam, mu = lame(np.broadcast_to(np.asarray(E, F64), (n,)),
                   np.broadcast_to(np.asarray(nu, F64), (n,)))
    vd = np.broadcast_to(np.asarray(v, F64), (n,))
    out = []
    for k in ks:
        d2 = _d2(Xd, Pd[k])
        sel = np.nonzero(d2 < (float(trunc) ** 2) * (rd[k] * rd[k]))[0] if trunc else np.arange(n)
        ptr, idx, phi, dphi, _ = shape_functions(Xq[sel], P, r, trunc, scale=scale)
        rowof = np.repeat(np.arange(sel.size), np.diff(ptr))
        at_k = np.nonzero(idx == k)[0]          # one entry per selected point
        assert np.array_equal(rowof[at_k], np.arange(sel.size))
        wh = vd[sel] * (lam[sel] + 4.0 * mu[sel])
        gk = dphi[:, at_k]                      # (3, points)
        fk = phi[at_k]
        h = np.zeros(P.shape[0])
        m = np.zeros(P.shape[0])
        np.add.at(h, idx, (wh[rowof] * (gk[:, rowof] * dphi).sum(0)))
        np.add.at(m, idx, vd[sel][rowof] * fk[rowof] * phi)
        cols = np.unique(idx)
        out.append((cols, h[cols], m[cols]))
    return out


def build(Xq, v, K, E, nu, trunc=None, start=0, dense=True):
    """The whole construction in the paper's order: centres by farthest-point
    sampling of the quadrature points, radii, shape functions at the
    quadrature points, then H_w and M.  Returns (centres, r, H, M)."""
    Xq = np.asarray(Xq, dtype=np.float32)
    centres = farthest_point_sampling(Xq, K, start)
    P = Xq[centres]
    r = radii(P)
    ptr, idx, phi, dphi, _ = shape_functions(Xq, P, r, trunc)
    H, M = assemble(Xq.shape[0], K, ptr, idx, phi, dphi, v, E, nu, dense=dense)
    return centres, r, H, M
