"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, index or coefficient, a transposed operand) fails at least one of
them.  CPU only; sizes keep the whole file to well under a minute.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly, eigen, jacobi, rkpm
from paper_2605_29318_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cloud(n=400, seed=7, support=2.0):
    return synth.unit_cube(n, seed=seed, support=support)


def _build(c):
    ptr, idx = rkpm.neighbours(c.X, c.a)
    phi, dphi, cond = rkpm.shape_functions(c.X, c.a, ptr, idx)
    return ptr, idx, phi, dphi, cond


@pytest.fixture(scope="module")
def cube400():
    c = _cloud()
    return c, _build(c)


# ------------------------------------------------------------------ raw kernel
def test_bspline_golden_values_and_library():
    rows = [l.split() for l in open(os.path.join(GOLD, "bspline_values.txt"))
            if l.strip() and not l.startswith("#")]
    q = np.array([float(r[0]) for r in rows])
    w = np.array([float(r[1]) for r in rows])
    np.testing.assert_allclose(rkpm.cubic_bspline(q), w, rtol=0, atol=1e-15)
    # w(q) is the uniform cubic B-spline on knots -2..2 evaluated at 2q
    from scipy.interpolate import BSpline
    b3 = BSpline.basis_element([-2, -1, 0, 1, 2], extrapolate=False)
    qq = np.linspace(0, 0.999, 257)
    np.testing.assert_allclose(rkpm.cubic_bspline(qq), np.nan_to_num(b3(2 * qq)), atol=1e-14)


def test_bspline_integral_and_derivative():
    from scipy.integrate import quad
    # 3D integral: 4 pi int_0^1 w(q) q^2 dq = pi / 12
    val = 4 * np.pi * (quad(lambda q: rkpm.cubic_bspline(q) * q * q, 0, 0.5)[0]
                       + quad(lambda q: rkpm.cubic_bspline(q) * q * q, 0.5, 1)[0])
    assert abs(val - np.pi / 12) < 1e-12
    # w'(q)/q against a central difference of w
    q = np.linspace(0.01, 0.99, 99)
    h = 1e-6
    fd = (rkpm.cubic_bspline(q + h) - rkpm.cubic_bspline(q - h)) / (2 * h)
    np.testing.assert_allclose(rkpm.cubic_bspline_dw_over_q(q) * q, fd, atol=1e-8)


# ------------------------------------------------------------------ neighbours
def test_neighbours_against_kdtree():
    from scipy.spatial import cKDTree
    c = _cloud(1500, seed=3)
    ptr, idx = rkpm.neighbours(c.X, c.a)
    Xd = c.X.astype(np.float64)
    tree = cKDTree(Xd)
    a = float(c.a[0])
    lists = tree.query_ball_point(Xd, r=a)
    for i in range(c.n):
        mine = set(idx[ptr[i]:ptr[i + 1]].tolist())
        ref = set(lists[i])
        for k in mine ^ ref:      # only pairs within rounding of the radius may differ
            d = np.linalg.norm(Xd[i] - Xd[k])
            assert abs(d - a) < 1e-9 * a, (i, k, d, a)
        assert i in mine
        row = idx[ptr[i]:ptr[i + 1]]
        assert np.all(np.diff(row) > 0)


def test_neighbour_predicate_is_strict_and_asymmetric():
    # node 1 has a large support and covers point 0; node 0's small support
    # does not reach point 1; a point exactly at distance a is excluded.
    X = np.array([[0, 0, 0], [0.5, 0, 0], [1.5, 0, 0]], np.float32)
    a = np.array([0.1, 1.0, 1.0], np.float32)
    ptr, idx = rkpm.neighbours(X, a)
    rows = [idx[ptr[i]:ptr[i + 1]].tolist() for i in range(3)]
    assert rows[0] == [0, 1]
    assert rows[1] == [1]          # |x1 - x2| = 1.0 = a_2: strict, excluded
    assert rows[2] == [2]


# ------------------------------------------------------------------ shape functions
def test_reproducing_conditions(cube400):
    c, (ptr, idx, phi, dphi, _) = cube400
    rows = np.repeat(np.arange(c.n), np.diff(ptr))
    Xd = c.X.astype(np.float64)
    assert np.abs(np.bincount(rows, phi) - 1).max() < 1e-10                   # Eq. 8, P = 1
    for d in range(3):
        s = np.bincount(rows, phi * Xd[idx, d])
        assert np.abs(s - Xd[:, d]).max() < 1e-10                              # Eq. 8, P = x
        assert np.abs(np.bincount(rows, dphi[d], minlength=c.n)).max() < 1e-8  # grad of 1
        for e in range(3):
            g = np.bincount(rows, dphi[d] * Xd[idx, e])
            assert np.abs(g - (d == e)).max() < 1e-8                           # grad of x


def test_gradient_against_finite_differences(cube400):
    c, (ptr, idx, phi, dphi, _) = cube400
    pts = [0, 17, 123, 399]
    h = 1e-6
    for i in pts:
        x = c.X[i].astype(np.float64)
        ks = idx[ptr[i]:ptr[i + 1]]
        g = dphi[:, ptr[i]:ptr[i + 1]]
        scale = np.abs(g).max()
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fp, _ = rkpm.shape_functions_at((x + e)[None], c.X, c.a)
            fm, _ = rkpm.shape_functions_at((x - e)[None], c.X, c.a)
            fd = (fp[0, ks] - fm[0, ks]) / (2 * h)
            assert np.abs(fd - g[d]).max() < 1e-6 * scale


def test_shifted_basis_equals_paper_basis(cube400):
    c, (ptr, idx, phi, dphi, _) = cube400
    for i in [3, 250]:
        x = c.X[i].astype(np.float64)[None]
        p1, g1 = rkpm.shape_functions_at(x, c.X, c.a, literal_basis=True)
        ks = idx[ptr[i]:ptr[i + 1]]
        np.testing.assert_allclose(p1[0, ks], phi[ptr[i]:ptr[i + 1]], atol=1e-9)
        np.testing.assert_allclose(g1[:, 0, ks], dphi[:, ptr[i]:ptr[i + 1]],
                                   atol=1e-8 * np.abs(g1).max())


def test_vectorised_equals_loop_bruteforce():
    c = _cloud(64, seed=11, support=2.5)
    ptr, idx, phi, dphi, _ = _build(c)
    pd, gd = rkpm.shape_functions_at(c.X.astype(np.float64), c.X, c.a,
                                     scale=c.a.astype(np.float64))
    rows = np.repeat(np.arange(c.n), np.diff(ptr))
    np.testing.assert_allclose(pd[rows, idx], phi, atol=1e-12)
    np.testing.assert_allclose(gd[:, rows, idx], dphi, atol=1e-10)
    mask = np.zeros((c.n, c.n), bool)
    mask[rows, idx] = True
    assert np.all(pd[~mask] == 0)


# ------------------------------------------------------------------ Neo-Hookean / Prop. 1
def _golden_K():
    lines = [l for l in open(os.path.join(GOLD, "neohookean_rest_hessian.txt"))
             if l.strip() and not l.startswith("#")]
    i1 = lines.index("K1\n")
    i2 = lines.index("K\n")
    K1 = np.array([[float(v) for v in l.split()] for l in lines[i1 + 1:i2]])
    K = np.array([[float(v) for v in l.split()] for l in lines[i2 + 1:i2 + 10]])
    return K1, K


def test_golden_K_is_commutation_matrix():
    _, K = _golden_K()
    A = np.arange(9.0).reshape(3, 3) + 1
    np.testing.assert_array_equal(K @ A.reshape(-1), A.T.reshape(-1))


def test_neohookean_rest_hessian_and_stress_free():
    K1, K = _golden_K()
    lam, mu = assembly.lame(1e5, 0.45)
    gam = 1 + mu / (lam + mu)
    ref = mu * np.eye(9) + (lam + mu) * (2 - gam) * K1 - (lam + mu) * (1 - gam) * K
    h = 1e-4

    def psi(f):
        return assembly.neo_hookean_psi(f.reshape(1, 3, 3), lam, mu)[0]
    I = np.eye(3).reshape(-1)
    assert abs(psi(I)) < 1e-9 * lam
    Hfd = np.zeros((9, 9))
    grad = np.zeros(9)
    for a in range(9):
        ea = np.zeros(9)
        ea[a] = h
        grad[a] = (psi(I + ea) - psi(I - ea)) / (2 * h)
        for b in range(9):
            eb = np.zeros(9)
            eb[b] = h
            Hfd[a, b] = (psi(I + ea + eb) - psi(I + ea - eb) - psi(I - ea + eb)
                         + psi(I - ea - eb)) / (4 * h * h)
    assert np.abs(grad).max() < 1e-6 * lam             # rest state is stress-free
    assert np.abs(Hfd - ref).max() < 1e-5 * lam


def _fd_bilinear(f, u, w, h):
    """u^T Hess(f) w by central differences with one Richardson step."""
    def d2(t):
        return (f(t * (u + w)) - f(t * (u - w)) - f(-t * (u - w)) + f(-t * (u + w))) / (4 * t * t)
    return (4 * d2(h / 2) - d2(h)) / 3


@pytest.mark.parametrize("hetero", [False, True])
def test_prop1_against_energy_finite_differences(hetero):
    c = _cloud(64, seed=5, support=2.5)
    ptr, idx, phi, dphi, _ = _build(c)
    rng = np.random.default_rng(0)
    E = rng.uniform(1e4, 1e6, c.n) if hetero else 1e5
    nu = rng.uniform(0.2, 0.45, c.n) if hetero else 0.45
    H, _ = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, E, nu, dense=True)
    lam, mu = assembly.lame(np.broadcast_to(E, (c.n,)), np.broadcast_to(nu, (c.n,)))
    for trial in range(4):
        u = rng.standard_normal(c.n)
        w = rng.standard_normal(c.n)
        fd_total = 0.0
        for s in range(3):
            def f(dvec, s=s):
                d = np.zeros((c.n, 3))
                d[:, s] = dvec
                return assembly.potential(d, c.n, ptr, idx, dphi, c.v, E, nu)
            fd = _fd_bilinear(f, u, w, 1e-3 * float(c.a[0]))
            # per-axis block of the proof: (lam + 2 mu) d_s phi d_s phi^T + mu (other two)
            G = [sp.csr_matrix((dphi[t], idx, ptr), shape=(c.n, c.n)) for t in range(3)]
            blk = sum(((lam + 2 * mu) if t == s else mu) * c.v * (G[t] @ u) * (G[t] @ w)
                      for t in range(3)).sum()
            assert abs(fd - blk) < 1e-6 * (abs(blk) + 1e-300) + 1e-9 * abs(u @ H @ w)
            fd_total += fd
        ref = u @ H @ w
        assert abs(fd_total - ref) < 1e-6 * abs(ref)


# ------------------------------------------------------------------ H, M structure
def test_symmetry_spd_and_null_mode(cube400):
    c, (ptr, idx, phi, dphi, _) = cube400
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu, dense=True)
    scale = np.abs(H).max()
    assert np.abs(H - H.T).max() <= 1e-13 * scale
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    np.linalg.cholesky(M)                                   # M is SPD
    assert np.abs(H @ np.ones(c.n)).max() <= 1e-12 * scale  # H 1 = 0
    # partition of unity: 1^T M 1 = sum_i v_i (the total volume)
    one = np.ones(c.n)
    assert abs(one @ M @ one - c.v.astype(np.float64).sum()) < 1e-12 * c.v.sum()
    lam, _ = eigen.eigh_dense(H, M, 4)
    assert abs(lam[0]) < 1e-9 * lam[1]


def test_linear_field_energy(cube400):
    c, (ptr, idx, phi, dphi, _) = cube400
    H, _ = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, mu = assembly.lame(c.E, c.nu)
    a = np.array([0.3, -1.1, 0.7])
    cvec = c.X.astype(np.float64) @ a
    ref = (lam + 4 * mu) * (a @ a) * c.v.astype(np.float64).sum()
    assert abs(cvec @ (H @ cvec) - ref) < 1e-9 * ref


def test_invariances():
    c = _cloud(300, seed=9)
    # snap to a 2^-20 grid so that the exact transforms below stay exact in FP32
    c.X = (np.round(c.X.astype(np.float64) * 2 ** 20) / 2 ** 20).astype(np.float32)
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu, dense=True)
    lam0, _ = eigen.eigh_dense(H, M, 6)
    # exact rotation (axis cycle with a sign flip) and translation
    Xr = np.stack([-c.X[:, 1], c.X[:, 2], c.X[:, 0]], 1) + np.float32(3.25)
    c2 = synth.Cloud(Xr.astype(np.float32), c.v, c.a, c.E, c.nu, c.k)
    p2, i2, f2, g2, _ = _build(c2)
    H2, M2 = assembly.assemble(c.n, p2, i2, f2, g2, c.v, c.E, c.nu, dense=True)
    np.testing.assert_allclose(H2, H, atol=1e-9 * np.abs(H).max())
    np.testing.assert_allclose(M2, M, atol=1e-9 * np.abs(M).max())
    # general rotation: the FP32 rounding of the rotated inputs perturbs the
    # cloud by ~1e-7 of its size, so only the spectrum is compared, loosely
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    c3 = synth.Cloud((c.X.astype(np.float64) @ R.T).astype(np.float32), c.v, c.a,
                     c.E, c.nu, c.k)
    p3, i3, f3, g3, _ = _build(c3)
    H3, M3 = assembly.assemble(c.n, p3, i3, f3, g3, c.v, c.E, c.nu, dense=True)
    lam3, _ = eigen.eigh_dense(H3, M3, 6)
    np.testing.assert_allclose(lam3[1:], lam0[1:], rtol=1e-4)
    # uniform scale s: H -> s H, M -> s^3 M, eigenvalues -> eigenvalues / s^2
    s = 2.0
    c3 = synth.Cloud(c.X * np.float32(s), c.v * np.float32(s ** 3), c.a * np.float32(s),
                     c.E, c.nu, c.k)
    p3, i3, f3, g3, _ = _build(c3)
    assert np.array_equal(p3, ptr) and np.array_equal(i3, idx)
    H3, M3 = assembly.assemble(c.n, p3, i3, f3, g3, c3.v, c.E, c.nu, dense=True)
    np.testing.assert_allclose(H3, s * H, atol=1e-9 * s * np.abs(H).max())
    np.testing.assert_allclose(M3, s ** 3 * M, atol=1e-9 * s ** 3 * np.abs(M).max())
    lam3, _ = eigen.eigh_dense(H3, M3, 6)
    np.testing.assert_allclose(lam3[1:], lam0[1:] / s ** 2, rtol=1e-9)
    # Young's modulus scaling at fixed nu
    H4, _ = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, 3 * c.E, c.nu, dense=True)
    np.testing.assert_allclose(H4, 3 * H, atol=1e-12 * np.abs(H).max())
    # particle permutation
    perm = np.random.default_rng(1).permutation(c.n)
    c5 = synth.Cloud(c.X[perm], c.v[perm], c.a[perm], c.E, c.nu, c.k)
    p5, i5, f5, g5, _ = _build(c5)
    H5, M5 = assembly.assemble(c.n, p5, i5, f5, g5, c5.v, c.E, c.nu, dense=True)
    np.testing.assert_allclose(H5, H[np.ix_(perm, perm)], atol=1e-12 * np.abs(H).max())


def test_continuum_sanity_cube2k():
    """Neumann unit cube: the first non-zero eigenvalue tends to (lam + 4 mu) pi^2
    (threefold).  At 2,000 particles the discrete value is within a loose band."""
    c = synth.unit_cube(2000, seed=1)
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, _ = eigen.eigh_dense(H, M, 5)
    lm, mu = assembly.lame(c.E, c.nu)
    cont = (lm + 4 * mu) * np.pi ** 2
    assert np.all(np.abs(lam[1:4] / cont - 1) < 0.5)
    assert lam[4] > lam[3]


# ------------------------------------------------------------------ eigensolvers
def test_dense_eigensolve_against_hand_jacobi():
    c = _cloud(64, seed=5, support=2.5)
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu, dense=True)
    lam, C = eigen.eigh_dense(H, M, 8)
    wj, Cj = jacobi.generalized_jacobi(H, M)
    np.testing.assert_allclose(lam[1:], wj[1:8], rtol=1e-10)
    assert abs(lam[0]) < 1e-9 * lam[1] and abs(wj[0]) < 1e-9 * wj[1]
    np.testing.assert_allclose(C.T @ M @ C, np.eye(8), atol=1e-10)
    np.testing.assert_allclose(Cj.T @ M @ Cj, np.eye(c.n), atol=1e-9)
    assert eigen.max_principal_angle(M, C[:, 1:8], Cj[:, 1:8]) < 1e-8


def test_sparse_tier_against_dense():
    c = _cloud(1200, seed=4)
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam_d, C_d = eigen.eigh_dense(H, M, 10)
    lam_s, C_s = eigen.eigsh_sparse(H, M, 10)
    np.testing.assert_allclose(lam_s[1:], lam_d[1:], rtol=1e-9)
    assert eigen.residuals(H, M, lam_s, C_s)[1:].max() < 1e-8
    assert eigen.max_principal_angle(M, C_s, C_d) < 1e-6


def test_principal_angle_and_residual_helpers():
    rng = np.random.default_rng(3)
    n = 50
    B = rng.standard_normal((n, n))
    M = B @ B.T + n * np.eye(n)
    Q = eigen.m_orthonormalise(M, rng.standard_normal((n, 2)))
    u, v = Q[:, 0], Q[:, 1]
    for ang in [1e-6, 1e-3, 0.3]:
        A = np.cos(ang) * u + np.sin(ang) * v
        assert abs(eigen.max_principal_angle(M, u[:, None], A[:, None]) - ang) < 1e-9
    Hs = B.T @ B
    lam, C = eigen.eigh_dense(Hs, M, 3)
    assert eigen.residuals(Hs, M, lam, C).max() < 1e-10
    assert eigen.residuals(Hs, M, lam * (1 + 1e-3), C).min() > 5e-4


def test_layered_sphere_generator_and_its_linear_field_energy():
    """The four-shell sphere: E follows the shell (stiff, soft, stiff, soft from
    the centre out), and with that per-particle material a linear nodal field
    c_k = a . p_k still has the exact energy c^T H_w c = |a|^2 sum_i v_i
    (lambda_i + 4 mu_i) (gradient reproduction, Eq. 8, in Prop. 1)."""
    c = synth.layered_sphere(800, seed=3)
    r = np.sqrt((c.X.astype(np.float64) ** 2).sum(1)) / 0.5
    shell = np.minimum((r * 4).astype(int), 3)
    assert np.all(c.E[shell % 2 == 0] == np.float32(1e7))
    assert np.all(c.E[shell % 2 == 1] == np.float32(1e5))
    assert all(np.any(shell == s) for s in range(4))
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    a = np.array([0.3, -1.1, 0.7])
    cf = c.X.astype(np.float64) @ a
    lam, mu = assembly.lame(np.asarray(c.E, np.float64), float(c.nu))
    expect = float(a @ a) * float(np.sum(c.v.astype(np.float64) * (lam + 4 * mu)))
    assert abs(cf @ (H @ cf) - expect) <= 1e-10 * expect


def test_rayleigh_ritz_and_absolute_residuals():
    """Rayleigh-Ritz on a span holding exact eigenvectors returns their
    eigenvalues and vectors; on any span its Ritz values interlace from above
    (theta_j >= lam_j, Courant-Fischer).  Absolute residuals vanish on exact
    pairs (the zero eigenvalue included) and equal |delta| on a shifted one."""
    rng = np.random.default_rng(5)
    n = 40
    B = rng.standard_normal((n, n))
    M = B @ B.T + n * np.eye(n)
    G = rng.standard_normal((n, n))
    Hs = G.T @ G
    Hs[:, 0] = Hs[0, :] = 0.0          # a zero eigenvalue, as the constant mode
    lam, C = eigen.eigh_dense(Hs, M, n)
    th, Y = eigen.rayleigh_ritz(Hs, M, C[:, [3, 1, 6]] @ rng.standard_normal((3, 3)))
    np.testing.assert_allclose(th, lam[[1, 3, 6]], rtol=1e-9)
    assert eigen.max_principal_angle(M, Y, C[:, [1, 3, 6]]) < 1e-7
    th, _ = eigen.rayleigh_ritz(Hs, M, rng.standard_normal((n, 5)))
    assert np.all(th >= lam[:5] * (1 - 1e-12))
    assert eigen.absolute_residuals(Hs, M, lam[:4], C[:, :4]).max() < 1e-9 * lam[3]
    delta = 1e-3 * lam[2]
    r = eigen.absolute_residuals(Hs, M, [lam[2] + delta], C[:, [2]])
    assert abs(r[0] - delta) < 1e-9 * delta


def test_subspace_angle_bound():
    """The trace bound on the largest M-principal angle: exact eigenvectors
    give 0; rotating the last kept eigenvector by theta towards the first
    excluded one makes the bound exact (sin^2 theta (lam_k - lam_{k-1}) is the
    whole excess trace); any other perturbation stays below the bound."""
    rng = np.random.default_rng(8)
    n, k = 30, 5
    B = rng.standard_normal((n, n))
    M = B @ B.T + n * np.eye(n)
    G = rng.standard_normal((n, n))
    Hs = G.T @ G + np.eye(n)
    lam, C = eigen.eigh_dense(Hs, M, n)
    assert eigen.subspace_angle_bound(Hs, M, C[:, :k], lam) < 1e-6
    for theta in (1e-4, 1e-2, 0.3):
        Y = C[:, :k].copy()
        Y[:, k - 1] = np.cos(theta) * C[:, k - 1] + np.sin(theta) * C[:, k]
        assert abs(eigen.subspace_angle_bound(Hs, M, Y, lam) - theta) < 1e-6 * max(theta, 1e-2)
        assert abs(eigen.max_principal_angle(M, Y, C[:, :k]) - theta) < 1e-8
    for _ in range(5):
        Y = C[:, :k] + 1e-3 * rng.standard_normal((n, k)) * np.abs(C[:, :k]).max()
        true = eigen.max_principal_angle(M, Y, C[:, :k])
        assert true <= eigen.subspace_angle_bound(Hs, M, Y, lam) * (1 + 1e-9)


def test_disconnected_clouds_have_one_zero_mode_each():
    c1 = synth.unit_cube(200, seed=1)
    c2 = synth.unit_cube(200, seed=2)
    X = np.concatenate([c1.X, c2.X + np.float32(5)])
    c = synth.Cloud(X, np.concatenate([c1.v, c2.v]), np.concatenate([c1.a, c2.a]),
                    1e5, 0.45, 4)
    ptr, idx, phi, dphi, _ = _build(c)
    assert rkpm.connected_components(c.n, ptr, idx) == 2
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, _ = eigen.eigh_dense(H, M, 3)
    assert abs(lam[0]) < 1e-8 * lam[2] and abs(lam[1]) < 1e-8 * lam[2]


# ---------------------------------------------------------------- warm start
def _ws_cloud(n=300, seed=9):
    c = synth.ellipsoid_union(n, seed=seed)
    ptr, idx = rkpm.neighbours(c.X, c.a)
    return c, ptr, idx


def test_warmstart_features_invariant_under_similarity_transforms():
    from oracle import warmstart
    c, ptr, idx = _ws_cloud()
    f0 = warmstart.features(c.X, c.v, c.a, ptr, idx)
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))          # rotation or reflection
    for Qm in (Q, Q @ np.diag([1.0, 1.0, -1.0])):
        sc = 2.5
        X = (c.X.astype(np.float64) @ Qm.T) * sc + np.array([3.0, -1.0, 0.5])
        f1 = warmstart.features(X, c.v * sc ** 3, c.a * sc, ptr, idx)
        np.testing.assert_allclose(f1, f0, atol=1e-9)


def test_warmstart_features_on_a_symmetric_lattice():
    """Interior points of a cubic lattice whose support sees a symmetric
    neighbourhood have zero neighbour offset and an isotropic spread equal to
    the lattice sum over the support ball (counted by brute force)."""
    from oracle import warmstart
    g = np.arange(9, dtype=np.float64)
    X = np.stack(np.meshgrid(g * 1.0, g * 1.3, g * 0.8, indexing="ij"), -1).reshape(-1, 3)
    n = X.shape[0]
    a = np.full(n, 1.55)
    ptr, idx = rkpm.neighbours(X.astype(np.float32), a.astype(np.float32))
    f = warmstart.features(X, np.ones(n), a, ptr, idx)
    centre = int(np.argmin(((X - X.mean(0)) ** 2).sum(1)))
    np.testing.assert_allclose(f[centre, 3:6], 0.0, atol=1e-12)
    offs = [np.array([i * 1.0, j * 1.3, k * 0.8]) for i in range(-2, 3) for j in range(-2, 3)
            for k in range(-2, 3)]
    inside = np.array([o for o in offs if o @ o < 1.55 ** 2])
    var = (inside ** 2).mean(0) / 1.55 ** 2                      # per lattice axis
    # canonical axes of the box are the lattice axes, longest (y) first
    np.testing.assert_allclose(np.sort(f[centre, 6:9]), np.sort(var), rtol=1e-12)
    # variance along each lattice axis of a 9-point uniform grid: (9^2 - 1)/12 h^2
    mu, R, s2, s = warmstart.canonical_frame(X, np.ones(n))
    np.testing.assert_allclose(np.sort(s2)[::-1], np.array([1.3, 1.0, 0.8]) ** 2 * 80 / 12,
                               rtol=1e-12)


def test_warmstart_loss_special_cases():
    from oracle import warmstart
    rng = np.random.default_rng(5)
    n, m = 400, 31
    v = rng.uniform(0.5, 1.5, n)
    C = rng.standard_normal((n, m))
    Y = np.concatenate([C @ rng.standard_normal((m, m)), rng.standard_normal((n, 1))], 1)
    L, _ = warmstart.subspace_loss(Y, v, C)
    assert abs(L) < 1e-4                       # span(Y) contains span(C)
    w = v / v.sum()
    B = rng.standard_normal((n, 32))
    B -= C @ np.linalg.solve(C.T @ (w[:, None] * C), C.T @ (w[:, None] * B))
    L, _ = warmstart.subspace_loss(B, v, C)
    assert abs(L - 1.0) < 1e-9                 # W-orthogonal to span(C)
    Y = rng.standard_normal((n, 32))
    L1, _ = warmstart.subspace_loss(Y, v, C)
    Q, _ = np.linalg.qr(rng.standard_normal((32, 32)))
    T = Q * rng.uniform(0.5, 2.0, 32)           # well conditioned: the ridge stays ~1e-6
    L2, _ = warmstart.subspace_loss(Y @ T, v, C)
    assert abs(L1 - L2) < 1e-5 and 0 < L1 < 1   # depends on the span only


def test_warmstart_loss_gradient_by_finite_differences():
    from oracle import warmstart
    rng = np.random.default_rng(6)
    n, m = 200, 31
    v = rng.uniform(0.5, 1.5, n)
    C = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, 32))
    L, dY = warmstart.subspace_loss(Y, v, C)
    for _ in range(4):
        D = rng.standard_normal((n, 32))
        h = 1e-6
        fd = (warmstart.subspace_loss(Y + h * D, v, C)[0]
              - warmstart.subspace_loss(Y - h * D, v, C)[0]) / (2 * h)
        assert abs(fd - (dY * D).sum()) < 1e-5 * max(1e-3, abs(fd))


def test_warmstart_network_gradient_by_finite_differences():
    from oracle import warmstart
    c, ptr, idx = _ws_cloud(120, seed=3)
    f = warmstart.features(c.X, c.v, c.a, ptr, idx)
    # random layers 1-4 and a last layer that whitens h4 in the volume inner
    # product: the loss is then well conditioned (G = Y^T W Y ~ I), so central
    # differences resolve its derivative
    theta = warmstart.init_params(11) * 0.5
    w = c.v.astype(np.float64) / c.v.sum()
    _, cache = warmstart.forward(theta, f)
    _, S, Vt = np.linalg.svd(np.sqrt(w)[:, None] * cache["h4"], full_matrices=False)
    layers = warmstart.unpack(theta)
    layers[4] = (Vt[:32] / S[:32, None], np.zeros(32))
    theta = warmstart.pack(layers)
    rng = np.random.default_rng(7)
    C = rng.standard_normal((c.n, 31))
    L, g = warmstart.loss_and_grad(theta, f, c.v, C)
    assert g.shape == (warmstart.n_params(),) == (170784,)
    off = 0
    for i, o in warmstart.DIMS:          # one random direction per layer
        for size in (i * o, o):
            D = np.zeros_like(theta)
            D[off:off + size] = rng.standard_normal(size)
            h = 1e-7
            fd = (warmstart.loss_and_grad(theta + h * D, f, c.v, C)[0]
                  - warmstart.loss_and_grad(theta - h * D, f, c.v, C)[0]) / (2 * h)
            an = g @ D
            assert abs(fd - an) < 1e-4 * max(abs(an), 1e-3 * np.abs(g).max()), (off, fd, an)
            off += size


def test_adam_step_matches_its_definition_on_a_quadratic():
    """Adam on f(x) = 0.5 ||x - t||^2 moves every coordinate by lr on its first
    step (the bias-corrected ratio is sign(g)) and converges to t."""
    from oracle import warmstart
    t = np.array([1.0, -2.0, 0.5])
    x = np.zeros(3)
    m1 = np.zeros(3)
    m2 = np.zeros(3)
    x1, m1, m2 = warmstart.adam_step(x, x - t, m1, m2, 1, 0.1)
    np.testing.assert_allclose(x1, 0.1 * np.sign(t), rtol=1e-6)
    x = x1
    for it in range(2, 3000):
        x, m1, m2 = warmstart.adam_step(x, x - t, m1, m2, it, 0.01)
    np.testing.assert_allclose(x, t, atol=1e-3)


def test_bf16_rounding_matches_its_definition():
    """Nearest representable value with 8 significant bits, ties to even."""
    from oracle import warmstart
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, 1.0 + 2 ** -7 + 2 ** -8,
                  -3.14159, 0.0, 1e-30])
    r = warmstart.bf16_round(x)                # spacing 2^-7 on [1, 2)
    assert r[0] == 1.0
    assert r[1] == 1.0                        # 1 + 2^-8 is the midpoint of 1 and 1 + 2^-7
    assert r[2] == 1.0 + 2 ** -7              # above the midpoint
    assert r[3] == 1.0                        # below the midpoint
    assert r[4] == 1.0 + 2 ** -6              # midpoint of 1 + 2^-7 (odd) and 1 + 2^-6
    assert abs(r[5] + 3.140625) == 0.0
    assert r[6] == 0.0
    m, e = np.frexp(r[np.isfinite(r) & (r != 0)])
    assert np.all(np.abs(m * 2 ** 8 - np.round(m * 2 ** 8)) == 0)   # 8-bit significand


def test_single_rows_match_the_full_assembly():
    """assembly.rows (one row from its covering quadrature points) against the
    full sparse assembly, on a heterogeneous cloud."""
    c = synth.unit_cube(500, seed=12)
    rng = np.random.default_rng(3)
    E = rng.uniform(1e4, 1e6, c.n)
    nu = rng.uniform(0.2, 0.45, c.n)
    ptr, idx, phi, dphi, _ = _build(c)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, E, nu)
    for k, (cols, h, m) in zip([0, 77, 499], assembly.rows([0, 77, 499], c.X, c.v, c.a, E, nu)):
        np.testing.assert_array_equal(cols, H[k].indices)
        np.testing.assert_allclose(h, H[k].data, rtol=1e-9, atol=1e-12 * np.abs(H[k].data).max())
        np.testing.assert_allclose(m, M[k].toarray()[0, cols], rtol=1e-9,
                                   atol=1e-12 * np.abs(M[k].data).max())


# ---------------------------------------------------------------- skinning weights, LBS (Sec. 3.2, Eq. 1)
def _query_points(c, count, seed):
    """Particles of the cloud moved by up to a tenth of their support: points
    every support rule still covers."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(c.n, count, replace=False)
    Q = c.X[pick].astype(np.float64) + 0.1 * c.a[pick, None] * rng.uniform(-1, 1, (count, 3))
    return Q.astype(np.float32)


def test_skinning_weights_reproduce_constant_and_linear_fields():
    """W of constant nodal values is constant (partition of unity, Eq. 8) and W
    of the nodes' coordinates is the query point itself (linear reproduction):
    the skinning fields inherit RKPM's consistency at arbitrary points."""
    from oracle import skinning
    c = synth.unit_cube(300, seed=11)
    Q = _query_points(c, 40, 3)
    W1 = skinning.weights(Q, c.X, c.a, np.ones((c.n, 1)))
    assert np.abs(W1 - 1.0).max() < 1e-12
    WX = skinning.weights(Q, c.X, c.a, c.X.astype(np.float32).astype(np.float64))
    assert np.abs(WX - Q.astype(np.float64)).max() < 1e-12
    # and the fields are linear in their nodal values
    rng = np.random.default_rng(4)
    C1, C2 = rng.standard_normal((c.n, 2)), rng.standard_normal((c.n, 2))
    lhs = skinning.weights(Q, c.X, c.a, 2.0 * C1 - 3.0 * C2)
    rhs = 2.0 * skinning.weights(Q, c.X, c.a, C1) - 3.0 * skinning.weights(Q, c.X, c.a, C2)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_lbs_closed_forms():
    """Eq. 1 on closed forms: zero transforms leave X; a unit-weight field with
    Z = [A | t] moves X to X + A X + t; two fields blend their transforms."""
    from oracle import skinning
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (25, 3))
    W = rng.uniform(0, 1, (25, 2))
    assert np.array_equal(skinning.lbs(X, W, np.zeros((2, 3, 4))), X)
    A, t = rng.standard_normal((3, 3)), rng.standard_normal(3)
    Z = np.concatenate([A, t[:, None]], axis=1)[None]
    x = skinning.lbs(X, np.ones((25, 1)), Z)
    assert np.abs(x - (X + X @ A.T + t)).max() < 1e-13
    t2 = rng.standard_normal(3)
    Z2 = np.zeros((2, 3, 4))
    Z2[0, :, 3], Z2[1, :, 3] = t, t2
    x2 = skinning.lbs(X, W, Z2)
    assert np.abs(x2 - (X + W[:, :1] * t + W[:, 1:] * t2)).max() < 1e-13
