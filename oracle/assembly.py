"""Oracle: weight-space Hessian H_w, RKPM mass matrix, Neo-Hookean potential.

Test infrastructure only (see ``oracle/__init__``).

* Prop. 1 (Sec. 3.2; proof in Supp. Sec. C):
      (H_w)_kl = int (lambda + 4 mu) grad phi_k . grad phi_l dX
               ~= sum_i v_i (lambda_i + 4 mu_i) grad phi_k(X_i) . grad phi_l(X_i)
  with the Monte-Carlo quadrature of the proof (weights v_i at X_i).
* Mass matrix (Sec. 3.2, Eq. 14): M_kl = int phi_k phi_l dX
      ~= sum_i v_i phi_k(X_i) phi_l(X_i).
  The paper's printed indices are garbled (c_k^i M_lm c_l^j); this is the
  consistent reading c^T M c = I.
* Neo-Hookean energy (Eq. 16, after Smith et al.):
      Psi(F) = 1/2 [ lbar (det F - gamma)^2 + mubar tr(F^T F) - E0 ],
      lbar = lambda + mu,  mubar = mu,  gamma = 1 + mubar / lbar,
      E0 such that Psi(I) = 0.
  E_pot(d) = sum_i v_i Psi(F_i),  F_i = I + d^T grad phi(X_i)   (Supp. Sec. C).
  Only the finite-difference pins use it.
* Lame parameters from Young's modulus and Poisson ratio (standard):
      lambda = E nu / ((1 + nu)(1 - 2 nu)),  mu = E / (2 (1 + nu)).

Density does not enter: the paper's orthogonality is the plain L2 product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

F64 = np.float64


def lame(E, nu):
    E = np.asarray(E, dtype=F64)
    nu = np.asarray(nu, dtype=F64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def _per_particle(x, n):
    x = np.asarray(x, dtype=F64)
    return np.broadcast_to(x, (n,)).copy() if x.ndim == 0 else x.astype(F64)


def gradient_operators(n, ptr, idx, phi, dphi):
    """Sparse Phi (rows = quadrature points i, cols = nodes k) and G_s = d_s Phi."""
    Phi = sp.csr_matrix((np.asarray(phi, F64), idx, ptr), shape=(n, n))
    G = [sp.csr_matrix((np.asarray(dphi[s], F64), idx, ptr), shape=(n, n))
         for s in range(3)]
    return Phi, G


def assemble(n, ptr, idx, phi, dphi, v, E, nu, dense=False):
    """H_w (Prop. 1) and the mass matrix (Eq. 14) as scipy CSR (or dense).

    H_w = sum_s G_s^T diag(v (lambda + 4 mu)) G_s,  M = Phi^T diag(v) Phi.
    E and nu are scalars (homogeneous) or per-particle arrays; the material
    is sampled at the quadrature points X_i."""
    lam, mu = lame(_per_particle(E, n), _per_particle(nu, n))
    v = _per_particle(v, n)
    Phi, G = gradient_operators(n, ptr, idx, phi, dphi)
    Dh = sp.diags(v * (lam + 4.0 * mu))
    Dm = sp.diags(v)
    H = (G[0].T @ Dh @ G[0] + G[1].T @ Dh @ G[1] + G[2].T @ Dh @ G[2]).tocsr()
    M = (Phi.T @ Dm @ Phi).tocsr()
    H.sort_indices()
    M.sort_indices()
    if dense:
        return H.toarray(), M.toarray()
    return H, M


def rows(ks, X, v, a, E, nu):
    """Rows ks of H_w (Prop. 1) and M (Eq. 14) for a cloud of any size, from the
    definition evaluated only where it is non-zero: row k sums over the
    quadrature points X_i that node k covers, each with the shape functions of
    its own covering nodes (``rkpm.shape_functions_at`` on that node set).
    Returns a list of (cols, H_row, M_row), cols ascending, FP64."""
    from . import rkpm
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    Xd = X.astype(F64)
    ad = np.asarray(a, dtype=np.float32).astype(F64)
    lam, mu = lame(_per_particle(E, n), _per_particle(nu, n))
    vd = _per_particle(v, n)
    amax = float(ad.max())
    out = []
    for k in ks:
        # quadrature points node k covers (candidates within the largest radius)
        near = np.nonzero(((Xd - Xd[k]) ** 2).sum(1) <= (amax * 1.001) ** 2)[0]
        hs, ms = {}, {}
        for i in near:
            cov = rkpm.neighbours_query(X[i:i + 1], X, a)[0]
            if k not in cov:
                continue
            phi, dphi = rkpm.shape_functions_at(X[i:i + 1], X[cov], np.asarray(a)[cov],
                                                scale=[ad[i]])
            j = int(np.nonzero(cov == k)[0][0])
            wh = vd[i] * (lam[i] + 4.0 * mu[i])
            gk = dphi[:, 0, j]
            for jj, l in enumerate(cov):
                hs[l] = hs.get(l, 0.0) + wh * float(gk @ dphi[:, 0, jj])
                ms[l] = ms.get(l, 0.0) + vd[i] * phi[0, j] * phi[0, jj]
        cols = np.array(sorted(hs), dtype=np.int64)
        out.append((cols, np.array([hs[l] for l in cols]), np.array([ms[l] for l in cols])))
    return out


def neo_hookean_psi(F, lam, mu):
    """Psi(F) of Eq. 16 for a batch of 3x3 deformation gradients F (m, 3, 3)."""
    lbar = lam + mu
    mubar = mu
    gamma = 1.0 + mubar / lbar
    E0 = lbar * (1.0 - gamma) ** 2 + 3.0 * mubar          # Psi(I) = 0
    J = np.linalg.det(F)
    trFtF = np.einsum("mij,mij->m", F, F)
    return 0.5 * (lbar * (J - gamma) ** 2 + mubar * trFtF - E0)


def deformation_gradients(d, n, ptr, idx, dphi):
    """F_i = I + d^T grad phi(X_i) for nodal displacements d (K x 3)."""
    _, G = gradient_operators(n, ptr, idx, np.zeros(idx.size), dphi)
    d = np.asarray(d, dtype=F64)
    F = np.zeros((n, 3, 3))
    for a_ in range(3):            # displacement component (row of F)
        for b in range(3):         # derivative direction (column of F)
            F[:, a_, b] = G[b] @ d[:, a_]
    F += np.eye(3)[None]
    return F


def potential(d, n, ptr, idx, dphi, v, E, nu):
    """E_pot(d) = sum_i v_i Psi(I + d^T grad phi(X_i))  (Supp. Sec. C)."""
    lam, mu = lame(_per_particle(E, n), _per_particle(nu, n))
    F = deformation_gradients(d, n, ptr, idx, dphi)
    return float(np.sum(_per_particle(v, n) * neo_hookean_psi(F, lam, mu)))
