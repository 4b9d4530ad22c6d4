"""GPU parity of the two-set discretisation (``rkpm_build_twoset``, through the
C ABI) against the FP64 oracle of ``oracle/twoset.py``.

Bars: the farthest-point centres, the radii and the covering lists are
bit-exact (integer results and FP64 values decided by the same rounded
operations); shape functions within 1e-10 of their largest magnitude in FP64
contexts (double-float arithmetic, the Gaussian from the FP64 exp), 2e-5 in
FP32 ones; H_w and M within 1e-10 / 1e-4 of their largest entry; eigenvalues
within 1e-8 relative of the oracle's dense solve (FP64).
"""
import os

import numpy as np
import pytest

from oracle import assembly, eigen, twoset
from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_SHAPE = {"fp64": 1e-10, "fp32": 2e-5}
TOL_MAT = {"fp64": 1e-10, "fp32": 1e-4}


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _build(X, v, K, trunc, prec="fp64", start=0):
    from paper_2605_29318_gb300 import binding
    ctx = binding.Context(0, prec)
    ctx.rkpm_build_twoset(_dev(X), _dev(v), K, trunc, start)
    return ctx


def _oracle(X, K, trunc, start=0):
    cen = twoset.farthest_point_sampling(X, K, start)
    P = X[cen]
    r = twoset.radii(P)
    return cen, P, r


def _shuffled_grid(m, seed):
    X, v = synth.cube_grid(m)
    perm = np.random.default_rng(seed).permutation(X.shape[0])
    return X[perm], v[perm]


CASES = [
    ("cube10", lambda: synth.cube_grid(10), 80, 3.0),
    ("cube10-shuffled", lambda: _shuffled_grid(10, 3), 80, 3.0),
    ("torus-h0.05", lambda: synth.torus_grid(0.05), 120, 3.0),
    ("cube6-untruncated", lambda: synth.cube_grid(6), 20, 0.0),
]


@pytest.mark.parametrize("name,make,K,trunc", CASES, ids=[c[0] for c in CASES])
def test_centres_radii_and_lists_are_bit_exact(name, make, K, trunc):
    X, v = make()
    ctx = _build(X, v, K, trunc)
    npt, cen, rad = ctx.twoset()
    ocen, P, orad = _oracle(X, K, trunc)
    assert npt == X.shape[0]
    assert np.array_equal(cen, ocen)
    assert np.array_equal(rad, orad)
    ptr, idx, _, _ = ctx.export_rkpm()
    optr, oidx = twoset.covering(X, P, orad, trunc if trunc > 0 else None)
    assert np.array_equal(ptr, optr) and np.array_equal(idx, oidx)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,make,K,trunc", CASES, ids=[c[0] for c in CASES])
def test_shape_functions_and_matrices_match(prec, name, make, K, trunc):
    X, v = make()
    ctx = _build(X, v, K, trunc, prec)
    _, cen, rad = ctx.twoset()
    P = X[cen]
    scale = float(np.float32(rad.max()))
    optr, oidx, ophi, odphi, _ = twoset.shape_functions(X, P, rad, trunc if trunc > 0 else None,
                                                        scale=scale)
    ptr, idx, phi, dphi = ctx.export_rkpm()
    assert np.array_equal(idx, oidx)
    tol = TOL_SHAPE[prec]
    assert np.abs(phi - ophi).max() <= tol * np.abs(ophi).max()
    assert np.abs(dphi - odphi).max() <= tol * np.abs(odphi).max()
    E, nu = 1e5, 0.45
    ctx.assemble_hessian(None, None, E, nu)
    aptr, acol, H, M = ctx.export_matrices()
    OH, OM = twoset.assemble(X.shape[0], K, optr, oidx, ophi, odphi, v, E, nu, dense=True)
    rows = np.repeat(np.arange(K), np.diff(aptr))
    tm = TOL_MAT[prec]
    # the stored diagonal of H_w is minus its row's off-diagonal sum (H 1 = 0)
    assert np.abs(H - OH[rows, acol]).max() <= tm * np.abs(OH).max()
    assert np.abs(M - OM[rows, acol]).max() <= tm * np.abs(OM).max()
    # every non-zero of the oracle is stored
    mask = np.zeros((K, K), bool)
    mask[rows, acol] = True
    assert np.abs(OM[~mask]).max(initial=0.0) == 0.0
    ctx.close()


def test_eigenmodes_match_the_dense_oracle():
    """The unit cube, 16^3 grid points, 200 centres: the lowest modes of the
    assembled K x K problem against a dense FP64 solve of the oracle's
    matrices, and the Neumann spectrum (lam + 4 mu) pi^2 {1, 1, 1, 2, 2, 2}."""
    from paper_2605_29318_gb300 import binding
    X, v = synth.cube_grid(16)
    K, E, nu = 200, 1e5, 0.45
    ctx = _build(X, v, K, 3.0)
    ctx.assemble_hessian(None, None, E, nu)
    ev, modes, rep, st = ctx.eigenmodes(8, binding.default_opts(tol=1e-8))
    assert st == 0
    _, _, OH, OM = twoset.build(X, v, K, E, nu, trunc=3.0)
    lam, _ = eigen.eigh_dense(OH, OM, 8)
    np.testing.assert_allclose(ev[1:], lam[1:], rtol=1e-8)
    lm, mu = assembly.lame(E, nu)
    rel = ev / ((lm + 4 * mu) * np.pi ** 2)
    assert np.all(np.abs(rel[1:4] - 1) < 0.02) and np.all(np.abs(rel[4:7] - 2) < 0.06)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_skinning_weights_of_a_twoset_cloud(prec):
    """W(X) = sum_k phi_k(X) c_k with the Gaussian shape functions at points off
    the grid; constant nodal values reproduce 1."""
    X, v = synth.torus_grid(0.05)
    K = 120
    ctx = _build(X, v, K, 3.0, prec)
    _, cen, rad = ctx.twoset()
    P = X[cen]
    rng = np.random.default_rng(4)
    Q = (X[rng.choice(X.shape[0], 200, replace=False)]
         + rng.uniform(-0.01, 0.01, (200, 3))).astype(np.float32)
    dt = np.float64 if prec == "fp64" else np.float32
    C = rng.standard_normal((K, 3)).astype(dt)
    W = ctx.skinning_weights(_dev(Q), _dev(C)).double().cpu().numpy()
    ptr, idx, phi, _, _ = twoset.shape_functions(Q, P, rad, 3.0,
                                                 scale=float(np.float32(rad.max())))
    Phi, _ = twoset.operators(Q.shape[0], K, ptr, idx, phi, np.zeros((3, idx.size)))
    Wo = Phi @ C.astype(np.float64)
    assert np.abs(W - Wo).max() <= TOL_SHAPE[prec] * 10 * np.abs(Wo).max()
    W1 = ctx.skinning_weights(_dev(Q), _dev(np.ones((K, 1), dt))).double().cpu().numpy()
    assert np.abs(W1 - 1).max() < (1e-12 if prec == "fp64" else 2e-5)
    ctx.close()


def test_fp32_build_in_an_fp64_context():
    """FP32 build precision (the splat benchmark's plan: FP32 shape functions and
    assembly sums, FP64 storage and eigensolver): the shape functions within
    the FP32 tolerance of the oracle's, H_w and M within 1e-4 of their largest
    entry, and the eigenvalues of the unit cube within 1e-5 of the oracle's
    dense solve, every residual (against the stored matrices) at 1e-6."""
    import scipy.sparse as sp
    from paper_2605_29318_gb300 import binding
    X, v = synth.cube_grid(16)
    K, E, nu = 200, 1e5, 0.45
    ctx = binding.Context(0, "fp64")
    ctx.set_build_precision("fp32")
    ctx.rkpm_build_twoset(_dev(X), _dev(v), K, 3.0, 0)
    _, cen, rad = ctx.twoset()
    P = X[cen]
    scale = float(np.float32(rad.max()))
    optr, oidx, ophi, odphi, _ = twoset.shape_functions(X, P, rad, 3.0, scale=scale)
    ptr, idx, phi, dphi = ctx.export_rkpm()
    assert np.array_equal(idx, oidx)
    assert np.abs(phi - ophi).max() <= TOL_SHAPE["fp32"] * np.abs(ophi).max()
    ctx.assemble_hessian(None, None, E, nu)
    aptr, acol, H, M = ctx.export_matrices()
    OH, OM = twoset.assemble(X.shape[0], K, optr, oidx, ophi, odphi, v, E, nu, dense=True)
    rows = np.repeat(np.arange(K), np.diff(aptr))
    assert np.abs(H - OH[rows, acol]).max() <= TOL_MAT["fp32"] * np.abs(OH).max()
    assert np.abs(M - OM[rows, acol]).max() <= TOL_MAT["fp32"] * np.abs(OM).max()
    ev, modes, rep, st = ctx.eigenmodes(8, binding.default_opts(tol=1e-6))
    assert st == 0
    lam, _ = eigen.eigh_dense(OH, OM, 8)
    np.testing.assert_allclose(ev[1:], lam[1:], rtol=1e-5)
    Hs = sp.csr_matrix((H, acol, aptr), shape=(K, K))
    Ms = sp.csr_matrix((M, acol, aptr), shape=(K, K))
    assert eigen.residuals(Hs, Ms, ev, modes.double().cpu().numpy())[1:].max() <= 1e-6
    ctx.close()


def test_farthest_points_beyond_shared_memory():
    """More points than the cluster keeps in shared memory: the sampling runs
    from global memory and still matches the oracle exactly."""
    X, v = synth.torus_grid(0.016)
    assert X.shape[0] > 8 * 200 * 1024 // 24
    ctx = _build(X, v, 64, 3.0)
    _, cen, rad = ctx.twoset()
    ocen, _, orad = _oracle(X, 64, 3.0)
    assert np.array_equal(cen, ocen) and np.array_equal(rad, orad)
    ctx.close()


def test_farthest_points_on_the_whole_gpu():
    """From 200,000 points on, the sampling runs on every SM at once (one block
    per SM, a grid barrier per centre): a 228,000-point torus grid, K = 300,
    matches the oracle exactly, as does the cluster form below that size."""
    X, v = synth.torus_grid(0.012)
    assert X.shape[0] > 200000
    ctx = _build(X, v, 300, 3.0)
    _, cen, rad = ctx.twoset()
    ocen, _, orad = _oracle(X, 300, 3.0)
    assert np.array_equal(cen, ocen) and np.array_equal(rad, orad)
    ctx.close()


def test_errors_are_reported():
    from paper_2605_29318_gb300 import binding
    # six distinct positions, K = 7
    X = np.repeat(synth.cube_grid(2)[0][:6], 3, axis=0)
    v = np.full(X.shape[0], 0.1, np.float32)
    with pytest.raises(binding.FreeformError) as e:
        _build(X, v, 7, 3.0)
    assert e.value.status == 1 and "distinct" in str(e.value)
    # a flat grid: every moment matrix is singular
    g = (np.arange(8, dtype=np.float32) + 0.5) / 8
    Xf = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    Xf = np.concatenate([Xf, np.zeros((Xf.shape[0], 1), np.float32)], 1).astype(np.float32)
    with pytest.raises(binding.FreeformError) as e:
        _build(Xf, np.full(Xf.shape[0], 1 / 64, np.float32), 12, 3.0)
    assert e.value.status == 4 and "quadrature point" in str(e.value)
    # argument checks
    ctx = binding.Context(0, "fp64")
    Xc, vc = synth.cube_grid(4)
    for K, trunc, start in ((3, 3.0, 0), (65, 3.0, 0), (8, -1.0, 0), (8, 3.0, 64)):
        with pytest.raises(binding.FreeformError) as e:
            ctx.rkpm_build_twoset(_dev(Xc), _dev(vc), K, trunc, start)
        assert e.value.status == 1
    ctx.close()


def test_splat_of_a_million_points():
    """The splat-like cloud (1,000,000 points from 64 anisotropic Gaussians,
    volumes from local density, E per Gaussian) through the paper's own route
    for splats, in the benchmark's configuration: the points themselves as
    quadrature points, K = 1,000 farthest-point centres, k = 64, FP64 context,
    default options.  Centres and radii bit-exact against the oracle's
    farthest-point sampling of all million points; sampled rows of H_w and M
    against the oracle's rows (1e-10 of the row's largest entry); the 63
    non-constant eigenvalues against the oracle's dense solve of its own
    matrices (stored by tests/golden/make_splat_eigenvalues.py; 1e-5
    relative); every residual recomputed in FP64 from the exported K x K
    matrices; the modes' subspace within 1e-3 rad of the exact eigenspace of
    those matrices (trace bound with the oracle's eigenvalues); the weight
    fields at sampled points against the oracle's shape functions."""
    import scipy.sparse as sp
    import torch
    from paper_2605_29318_gb300 import binding
    c = synth.gaussian_mixture(1_000_000)
    K, k = 1000, 64
    ctx = _build(c.X, c.v, K, 3.0)
    _, cen, rad = ctx.twoset()
    ocen, P, orad = _oracle(c.X, K, 3.0)
    assert np.array_equal(cen, ocen) and np.array_equal(rad, orad)
    ctx.assemble_hessian(_dev(c.E), None, 1.0, float(c.nu))
    ev, modes, rep, st = ctx.eigenmodes(k, binding.default_opts(tol=1e-6))
    assert st == 0
    ptr, col, H, M = ctx.export_matrices()
    Hs = sp.csr_matrix((H, col, ptr), shape=(K, K))
    Ms = sp.csr_matrix((M, col, ptr), shape=(K, K))
    C = modes.double().cpu().numpy()
    assert eigen.residuals(Hs, Ms, ev, C)[1:].max() <= 2e-6
    scale = float(np.float32(orad.max()))
    for kk, (cols, h, m) in zip([5, 500, 999], twoset.rows([5, 500, 999], c.X, c.v, P, orad, 3.0,
                                                           c.E, c.nu, scale)):
        s = slice(ptr[kk], ptr[kk + 1])
        np.testing.assert_array_equal(col[s], cols)
        # the stored diagonal of H_w is minus the row's off-diagonal sum
        off = col[s] != kk
        assert np.abs(H[s][off] - h[off]).max() <= 1e-10 * np.abs(h).max()
        assert abs(-H[s][off].sum() - h[~off][0]) <= 1e-9 * np.abs(h).max()
        assert np.abs(M[s] - m).max() <= 1e-10 * np.abs(m).max()
    lam = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden",
                                  "splat_eigenvalues.txt"))[:, 1]
    rel = np.abs(ev[1:] - lam[1:k]) / lam[1:k]
    assert rel.max() <= 1e-5, rel
    assert eigen.subspace_angle_bound(Hs, Ms, C, lam) <= 1e-3
    rng = np.random.default_rng(6)
    Q = c.X[rng.choice(c.n, 300, replace=False)]
    Cw = rng.standard_normal((K, 4))
    W = ctx.skinning_weights(_dev(Q), _dev(Cw)).cpu().numpy()
    qp, qi, qphi, _, _ = twoset.shape_functions(Q, P, orad, 3.0,
                                                scale=float(np.float32(orad.max())))
    Phi, _ = twoset.operators(Q.shape[0], K, qp, qi, qphi, np.zeros((3, qi.size)))
    Wo = Phi @ Cw
    assert np.abs(W - Wo).max() <= 1e-9 * np.abs(Wo).max()
    ctx.close()
    torch.cuda.synchronize()


def test_splat_with_fp32_build():
    """The benchmark's splat in the benchmark's launch configuration (FP32
    build precision, FP32 preconditioner degree 32, double-float degree 48,
    hand-over from the FP32 phase at 3e-5):
    the 63 non-constant eigenvalues within 1e-5 of the oracle's (stored by
    tests/golden/make_splat_eigenvalues.py), every residual against the stored
    matrices at 2e-6, sampled rows of H_w and M against the oracle's FP64 rows
    at 1e-4 of the row's largest entry (FP32 shape functions and tile sums),
    and the modes within 1e-3 rad of the exact eigenspace of the stored
    matrices (LAPACK's dense generalized solve)."""
    import scipy.sparse as sp
    from paper_2605_29318_gb300 import binding
    c = synth.gaussian_mixture(1_000_000)
    K, k = 1000, 64
    ctx = binding.Context(0, "fp64")
    ctx.set_build_precision("fp32")
    ctx.rkpm_build_twoset(_dev(c.X), _dev(c.v), K, 3.0, 0)
    _, cen, rad = ctx.twoset()
    ocen, P, orad = _oracle(c.X, K, 3.0)
    assert np.array_equal(cen, ocen) and np.array_equal(rad, orad)
    ctx.assemble_hessian(_dev(c.E), None, 1.0, float(c.nu))
    ev, modes, rep, st = ctx.eigenmodes(
        k, binding.default_opts(tol=1e-6, cheb_degree=32, cheb_degree_fp64=48, fp32_tol=3e-5))
    assert st == 0
    lam = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden",
                                  "splat_eigenvalues.txt"))[:, 1]
    rel = np.abs(ev[1:] - lam[1:k]) / lam[1:k]
    assert rel.max() <= 1e-5, rel
    ptr, col, H, M = ctx.export_matrices()
    Hs = sp.csr_matrix((H, col, ptr), shape=(K, K))
    Ms = sp.csr_matrix((M, col, ptr), shape=(K, K))
    C = modes.double().cpu().numpy()
    assert eigen.residuals(Hs, Ms, ev, C)[1:].max() <= 2e-6
    scale = float(np.float32(orad.max()))
    for kk, (cols, h, m) in zip([5, 500, 999], twoset.rows([5, 500, 999], c.X, c.v, P, orad, 3.0,
                                                           c.E, c.nu, scale)):
        s = slice(ptr[kk], ptr[kk + 1])
        np.testing.assert_array_equal(col[s], cols)
        off = col[s] != kk
        eh = np.abs(H[s][off] - h[off]).max() / np.abs(h).max()
        em = np.abs(M[s] - m).max() / np.abs(m).max()
        assert eh <= 1e-4 and em <= 1e-4, (kk, eh, em)
    _, V = eigen.eigh_dense(Hs, Ms, k)
    assert eigen.max_principal_angle(Ms, C, V) <= 1e-3
    ctx.close()
