"""Parity at the benchmark's full size: the 50,000-particle torus (k = 32) in
the launch configuration bench.py times (FP64 context, default options: FP32
phase, then FP64 to a relative residual of 1e-6).

The FP64 oracle cannot assemble and factor the whole problem in test time, so
the outputs are checked where the oracle can compute them one by one -- the
neighbour lists, shape functions and rows of H_w and M of sampled particles --
and through properties that hold at any size: the residual of every returned
mode against the exported FP64 matrices (themselves checked row by row), the
M-orthonormality of the modes, ascending eigenvalues and the constant mode.
The eigenvalues are compared with the oracle's own (the 34 lowest of its FP64
H_w and M by shift-invert Lanczos, stored by
``tests/golden/make_torus50k_eigenvalues.py``), and the modes' subspace with the
oracle's exact eigenspace through the trace bound of
``oracle.eigen.subspace_angle_bound`` on the oracle's H_w and M.

Tolerances: neighbour lists bit-exact; shape functions 1e-10 of the row's
largest |value|; matrix rows 1e-10 of the row's largest |entry|; residual
1e-6; M-orthonormality 1e-9; eigenvalues 1e-5 relative; largest M-principal
angle 1e-3 rad.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly, eigen, rkpm
from paper_2605_29318_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "torus50k_eigenvalues.txt")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torus50k():
    import torch
    from paper_2605_29318_gb300 import binding
    c = synth.torus(50000, seed=2)
    ctx = binding.Context(0, "fp64")
    ctx.rkpm_build(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (c.X, c.v, c.a)))
    ctx.assemble_hessian(None, None, c.E, c.nu)
    ev, modes, rep, st = ctx.eigenmodes(32, binding.default_opts())
    out = dict(c=c, ctx=ctx, ev=ev, modes=modes.double().cpu().numpy(), rep=rep, st=st,
               rkpm=ctx.export_rkpm(), mats=ctx.export_matrices())
    yield out
    ctx.close()


SAMPLE = np.random.default_rng(7).choice(50000, 40, replace=False)


def test_sampled_neighbours_and_shape_functions(torus50k):
    c = torus50k["c"]
    ptr, idx, phi, dphi = torus50k["rkpm"]
    for i in SAMPLE:
        nb = rkpm.neighbours_query(c.X[i:i + 1], c.X, c.a)[0]
        g = idx[ptr[i]:ptr[i + 1]]
        np.testing.assert_array_equal(g, nb)
        po, dpo = rkpm.shape_functions_at(c.X[i:i + 1], c.X[nb], c.a[nb], scale=[c.a[i]])
        s = slice(ptr[i], ptr[i + 1])
        assert np.abs(phi[s] - po[0]).max() <= 1e-10 * np.abs(po[0]).max()
        assert np.abs(dphi[:, s] - dpo[:, 0, :]).max() <= 1e-10 * np.abs(dpo[:, 0, :]).max()


def test_sampled_matrix_rows(torus50k):
    c = torus50k["c"]
    ptr, col, H, M = torus50k["mats"]
    ks = SAMPLE[:12]
    for k, (cols, h, m) in zip(ks, assembly.rows(ks, c.X, c.v, c.a, c.E, c.nu)):
        s = slice(ptr[k], ptr[k + 1])
        np.testing.assert_array_equal(col[s], cols)
        assert np.abs(H[s] - h).max() <= 1e-10 * np.abs(h).max()
        assert np.abs(M[s] - m).max() <= 1e-10 * np.abs(m).max()


def test_modes_meet_the_residual_bar(torus50k):
    assert torus50k["st"] == 0, torus50k["rep"]
    ptr, col, H, M = torus50k["mats"]
    n = ptr.size - 1
    Hs = sp.csr_matrix((H, col, ptr), shape=(n, n))
    Ms = sp.csr_matrix((M, col, ptr), shape=(n, n))
    C = torus50k["modes"]
    ev = torus50k["ev"]
    MC = Ms @ C
    R = Hs @ C - MC * ev[None, :]
    res = np.linalg.norm(R[:, 1:], axis=0) / (ev[1:] * np.linalg.norm(MC[:, 1:], axis=0))
    assert res.max() <= 1e-6, res
    assert np.all(np.diff(ev) >= 0) and ev[0] == 0.0 and ev[1] > 0
    assert np.allclose(C[:, 0], C[0, 0]) and C[0, 0] > 0
    G = C.T @ MC
    assert np.abs(G - np.eye(32)).max() < 1e-9


def test_sampled_skinning_weights(torus50k):
    """The weight fields of the 32 full-size modes at sampled points between the
    particles, against the oracle's shape functions at those points; and their
    partition of unity with the constant mode (1e-10 of max |W|)."""
    import torch
    from oracle import skinning
    c, ctx = torus50k["c"], torus50k["ctx"]
    rng = np.random.default_rng(9)
    pick = SAMPLE[:30]
    Q = (c.X[pick].astype(np.float64)
         + 0.1 * c.a[pick, None] * rng.uniform(-1, 1, (pick.size, 3))).astype(np.float32)
    C = torus50k["modes"]
    Wg = ctx.skinning_weights(torch.from_numpy(Q).cuda(),
                              torch.from_numpy(np.ascontiguousarray(C)).cuda()).cpu().numpy()
    Wo = skinning.weights(Q, c.X, c.a, C)
    assert np.abs(Wg - Wo).max() <= 1e-10 * np.abs(Wo).max()
    # the constant mode's field is constant
    assert np.abs(Wg[:, 0] - C[0, 0]).max() <= 1e-10 * abs(C[0, 0])


def _cut(lam, k, rel_gap=1e-3):
    """The largest k' <= k whose cut-off is not inside a cluster: relative gap
    (lam[k'] - lam[k'-1]) / lam[k'] at least rel_gap (degenerate pairs of the
    torus's rotational symmetry are compared as whole subspaces)."""
    for kk in range(k, 1, -1):
        if (lam[kk] - lam[kk - 1]) / lam[kk] >= rel_gap:
            return kk
    raise AssertionError("no gap in the spectrum")


def test_eigenvalues_and_subspace_match_the_oracle(torus50k):
    """The 31 non-constant eigenvalues against the oracle's (1e-5 relative):
    they are the lowest ones, none of a degenerate pair missed.  The subspace
    of the modes up to the last adequate gap against the oracle's exact
    eigenspace, bounded from the oracle's FP64 H_w and M and its eigenvalues
    (largest M-principal angle 1e-3 rad)."""
    lam = np.loadtxt(GOLDEN)[:, 1]
    ev = torus50k["ev"]
    rel = np.abs(ev[1:] - lam[1:32]) / lam[1:32]
    assert rel.max() <= 1e-5, rel
    c = torus50k["c"]
    ptr, idx = rkpm.neighbours(c.X, c.a, chunk=64)
    phi, dphi, _ = rkpm.shape_functions(c.X, c.a, ptr, idx)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    kk = _cut(lam, 32)
    ang = eigen.subspace_angle_bound(H, M, torus50k["modes"][:, :kk], lam)
    assert ang <= 1e-3, (kk, ang)
