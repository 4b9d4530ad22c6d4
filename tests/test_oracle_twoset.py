"""Pins of the two-set oracle (``oracle/twoset.py``: farthest-point centres,
second-nearest-centre radii, Gaussian RKPM shape functions at grid quadrature
points, the K x K H_w and M) against what the paper and the mathematics fix:
hand-worked examples, a brute-force optimum, a library k-d tree, the
reproducing conditions (Eq. 8), finite differences, the energy of Prop. 1 and
the Neumann spectrum of the unit cube.  CPU only, a few seconds in all.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import assembly, eigen, twoset
from paper_2605_29318_gb300 import synth


def _line(xs):
    X = np.zeros((len(xs), 3), np.float32)
    X[:, 0] = xs
    return X


# ------------------------------------------------------------------ centres
def test_fps_hand_example_on_a_line():
    """Eleven points at x = 0..10, start 0.  By hand: 10 is farthest from {0};
    5 from {0, 10}; then four points tie at distance 2 (2, 3, 7, 8) and the
    lowest index, 2, wins; then 7 (distance 2); then every remaining point is
    at distance 1 and they come in index order."""
    X = _line(np.arange(11))
    got = twoset.farthest_point_sampling(X, 11)
    assert got.tolist() == [0, 10, 5, 2, 7, 1, 3, 4, 6, 8, 9]
    assert twoset.farthest_point_sampling(X, 3, start=4).tolist() == [4, 10, 0]


def test_fps_is_a_two_approximation_of_the_k_centre_optimum():
    """Greedy farthest-point selection covers the points within twice the
    best radius any K of them achieve (Gonzalez 1985); the chosen centres are
    also at least the covering radius apart.  Brute force over all subsets."""
    rng = np.random.default_rng(3)
    for trial in range(6):
        X = rng.random((10, 3)).astype(np.float32)
        K = 3
        got = twoset.farthest_point_sampling(X, K)
        assert len(set(got.tolist())) == K
        cov = twoset.covering_radius(X, got)
        best = min(twoset.covering_radius(X, S)
                   for S in itertools.combinations(range(10), K))
        assert cov <= 2.0 * best + 1e-12
        Xd = X.astype(np.float64)[got]
        sep = min(np.linalg.norm(Xd[i] - Xd[j]) for i in range(K) for j in range(i))
        assert sep >= cov - 1e-12


def test_fps_refuses_more_centres_than_distinct_points():
    X = _line([0, 1, 1, 0, 2])
    assert twoset.farthest_point_sampling(X, 3).tolist() == [0, 4, 1]
    with pytest.raises(ValueError):
        twoset.farthest_point_sampling(X, 4)


def test_fps_follows_a_permutation_of_the_points():
    rng = np.random.default_rng(5)
    X = rng.random((300, 3)).astype(np.float32)
    perm = rng.permutation(300)
    inv = np.argsort(perm)
    a = twoset.farthest_point_sampling(X, 40, start=17)
    b = twoset.farthest_point_sampling(X[perm], 40, start=int(inv[17]))
    assert np.array_equal(perm[b], a)


# ------------------------------------------------------------------ radii
def test_radii_hand_example_lattice_and_kdtree():
    # points at x = 0, 1, 3, 6: other-centre distances (1,3,6), (1,2,5), (3,2,3), (6,5,3)
    assert twoset.radii(_line([0, 1, 3, 6])).tolist() == [3.0, 2.0, 3.0, 5.0]
    # cubic lattice of spacing 1/2: every centre has at least three neighbours at 1/2
    g = np.arange(4) * 0.5
    L = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    assert np.all(twoset.radii(L) == 0.5)
    from scipy.spatial import cKDTree
    P = np.random.default_rng(1).random((200, 3)).astype(np.float32)
    d, _ = cKDTree(P.astype(np.float64)).query(P.astype(np.float64), k=3)
    np.testing.assert_allclose(twoset.radii(P), d[:, 2], rtol=1e-14)


def test_gaussian_kernel_values():
    assert twoset.gaussian(0.0, 0.3) == 1.0
    assert twoset.gaussian(0.09, 0.3) == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert twoset.gaussian(4 * 0.04, 0.2) == pytest.approx(math.exp(-4.0), rel=1e-15)


# ------------------------------------------------------------------ shape functions
@pytest.fixture(scope="module")
def cube_twoset():
    X, v = synth.cube_grid(10)
    c = twoset.farthest_point_sampling(X, 80)
    P = X[c]
    r = twoset.radii(P)
    return X, v, P, r


@pytest.mark.parametrize("trunc", [None, 3.0])
def test_reproducing_conditions(cube_twoset, trunc):
    """Eq. 8 and its gradient: sum phi_k = 1, sum phi_k p_k = X,
    sum grad phi_k = 0, sum grad phi_k p_k^T = I at every quadrature point."""
    X, v, P, r = cube_twoset
    n, K = X.shape[0], P.shape[0]
    ptr, idx, phi, dphi, cond = twoset.shape_functions(X, P, r, trunc)
    Phi, G = twoset.operators(n, K, ptr, idx, phi, dphi)
    Pd = P.astype(np.float64)
    assert np.abs(Phi @ np.ones(K) - 1).max() < 1e-12
    assert np.abs(Phi @ Pd - X.astype(np.float64)).max() < 1e-12
    for s in range(3):
        assert np.abs(G[s] @ np.ones(K)).max() < 1e-10
        for t in range(3):
            assert np.abs(G[s] @ Pd[:, t] - (s == t)).max() < 1e-10
    assert cond.max() < 1e4


def test_gradient_against_finite_differences(cube_twoset):
    """grad phi against central differences with one Richardson step, at
    points moved off the grid (the centres stay put)."""
    X, v, P, r = cube_twoset
    rng = np.random.default_rng(0)
    Q = X[rng.choice(X.shape[0], 6, replace=False)].astype(np.float64)
    Q += rng.uniform(-0.03, 0.03, Q.shape)
    Q = Q.astype(np.float32).astype(np.float64)
    _, _, _, dphi, _ = twoset.shape_functions(Q, P, r, None)
    eps = 2.0 ** -10
    for d in range(3):
        def D(e):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[:, d] += e
            Qm[:, d] -= e
            return (twoset.shape_functions(Qp, P, r, None)[2]
                    - twoset.shape_functions(Qm, P, r, None)[2]) / (2 * e)
        fd = (4 * D(eps / 2) - D(eps)) / 3
        assert np.abs(fd - dphi[d]).max() < 1e-9 * np.abs(dphi[d]).max()


def test_truncated_kernel_converges_to_the_full_gaussian(cube_twoset):
    """Cutting the Gaussian at t r_k drops raw weights below exp(-t^2): the
    shape functions approach the untruncated ones as t grows."""
    X, v, P, r = cube_twoset
    n, K = X.shape[0], P.shape[0]
    full = twoset.operators(n, K, *twoset.shape_functions(X, P, r, None)[:4])[0]
    errs = [abs(twoset.operators(n, K, *twoset.shape_functions(X, P, r, t)[:4])[0]
                - full).max() for t in (2.0, 3.0, 4.0)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4
    # a cut beyond every distance keeps every centre: identical functions
    same = twoset.shape_functions(X, P, r, 100.0)
    ref = twoset.shape_functions(X, P, r, None)
    assert np.array_equal(same[1], ref[1])
    np.testing.assert_array_equal(same[2], ref[2])


def test_degenerate_centre_sets():
    """The radius rule needs three centres; three centres cannot span the
    linear basis, so the moment matrix is singular (to rounding)."""
    X, _ = synth.cube_grid(4)
    P = X[[0, 5, 10]]
    with pytest.raises(ValueError):
        twoset.radii(P[:2])
    try:
        cond = twoset.shape_functions(X[:4], P, np.ones(3), None)[4]
        assert np.all(cond > 1e12)
    except np.linalg.LinAlgError:
        pass


# ------------------------------------------------------------------ H_w and M
def test_structure_null_mode_and_linear_energy(cube_twoset):
    X, v, P, r = cube_twoset
    n, K = X.shape[0], P.shape[0]
    sf = twoset.shape_functions(X, P, r, 3.0)
    H, M = twoset.assemble(n, K, *sf[:4], v, 1e5, 0.45, dense=True)
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()
    np.linalg.cholesky(M)
    assert np.abs(H @ np.ones(K)).max() <= 1e-11 * np.abs(H).max()
    vol = v.astype(np.float64).sum()
    assert abs(np.ones(K) @ M @ np.ones(K) - vol) < 1e-12 * vol
    lam, mu = assembly.lame(1e5, 0.45)
    a = np.array([0.4, -0.9, 1.3])
    c = P.astype(np.float64) @ a
    ref = (lam + 4 * mu) * (a @ a) * vol
    assert abs(c @ H @ c - ref) < 1e-9 * ref


def _fd_bilinear(f, u, w, h):
    def d2(t):
        return (f(t * (u + w)) - f(t * (u - w)) - f(-t * (u - w)) + f(-t * (u + w))) / (4 * t * t)
    return (4 * d2(h / 2) - d2(h)) / 3


def test_prop1_against_energy_finite_differences():
    """u^T H_w w equals the second derivative of the Neo-Hookean energy
    sum_i v_i Psi(I + d^T grad phi(X_i)) (Eq. 16, Supp. Sec. C) along nodal
    displacements d = u e_s, w e_s, summed over the three axes; per-particle
    materials."""
    X, v = synth.cube_grid(5)
    n, K = X.shape[0], 12
    P = X[twoset.farthest_point_sampling(X, K)]
    r = twoset.radii(P)
    ptr, idx, phi, dphi, _ = twoset.shape_functions(X, P, r, None)
    rng = np.random.default_rng(2)
    E = rng.uniform(1e4, 1e6, n)
    nu = rng.uniform(0.2, 0.45, n)
    H, _ = twoset.assemble(n, K, ptr, idx, phi, dphi, v, E, nu, dense=True)
    lam, mu = assembly.lame(E, nu)
    _, G = twoset.operators(n, K, ptr, idx, phi, dphi)

    def energy(d):
        F = np.empty((n, 3, 3))
        for a_ in range(3):
            for b in range(3):
                F[:, a_, b] = (b == a_) + G[b] @ d[:, a_]
        return float(np.sum(v.astype(np.float64) * assembly.neo_hookean_psi(F, lam, mu)))

    for trial in range(3):
        u = rng.standard_normal(K)
        w = rng.standard_normal(K)
        total = 0.0
        for s in range(3):
            def f(dv, s=s):
                d = np.zeros((K, 3))
                d[:, s] = dv
                return energy(d)
            total += _fd_bilinear(f, u, w, 1e-3 * float(np.median(r)))
        ref = u @ H @ w
        assert abs(total - ref) < 1e-6 * abs(ref)


def test_neumann_cube_spectrum():
    """The unit cube, 16^3 grid points, 200 centres: the lowest generalized
    eigenvalues approach the Neumann Laplacian's (lam + 4 mu) pi^2 (l^2 + m^2 + n^2):
    zero, 1 (three times), 2 (three times), 3."""
    X, v = synth.cube_grid(16)
    K = 200
    centres, r, H, M = twoset.build(X, v, K, 1e5, 0.45, trunc=3.0)
    assert centres[0] == 0 and len(set(centres.tolist())) == K
    lam, _ = eigen.eigh_dense(H, M, 8)
    lm, mu = assembly.lame(1e5, 0.45)
    rel = lam / ((lm + 4 * mu) * np.pi ** 2)
    assert abs(rel[0]) < 1e-10
    assert np.all(np.abs(rel[1:4] - 1) < 0.02)
    assert np.all(np.abs(rel[4:7] - 2) < 0.06)
    assert abs(rel[7] - 3) < 0.1


def test_translation_and_permutation_invariance():
    """Shifting every point by a dyadic vector (exact in FP32) leaves H_w and M
    unchanged; permuting the quadrature points (start mapped) permutes nothing
    in the K x K matrices."""
    rng = np.random.default_rng(4)
    X = (np.round(rng.random((400, 3)) * 2 ** 12) / 2 ** 12).astype(np.float32)
    v = np.full(400, 1 / 400, np.float32)
    c0, r0, H0, M0 = twoset.build(X, v, 30, 1e5, 0.4, trunc=3.0)
    c1, r1, H1, M1 = twoset.build(X + np.float32(0.75), v, 30, 1e5, 0.4, trunc=3.0)
    assert np.array_equal(c0, c1) and np.array_equal(r0, r1)
    np.testing.assert_allclose(H1, H0, atol=1e-10 * np.abs(H0).max())
    np.testing.assert_allclose(M1, M0, atol=1e-10 * np.abs(M0).max())
    perm = rng.permutation(400)
    inv = np.argsort(perm)
    c2, r2, H2, M2 = twoset.build(X[perm], v, 30, 1e5, 0.4, trunc=3.0, start=int(inv[0]))
    assert np.array_equal(perm[c2], c0)
    np.testing.assert_allclose(H2, H0, atol=1e-10 * np.abs(H0).max())
    np.testing.assert_allclose(M2, M0, atol=1e-10 * np.abs(M0).max())


def test_torus_grid_volume():
    """The inside grid's volume approaches the torus's 2 pi^2 R r^2."""
    vols = [synth.torus_grid(h)[1].astype(np.float64).sum() for h in (0.04, 0.02)]
    exact = 2 * math.pi ** 2 * 0.5 * 0.2 ** 2
    assert abs(vols[1] - exact) < 0.01 * exact
    assert abs(vols[1] - exact) < abs(vols[0] - exact) + 1e-3 * exact


def test_batch_generator_covers_every_particle():
    """The batch generator's support floor: every particle is covered (strict
    predicate |X_i - p_k| < a_k) by at least nine nodes, itself and its eight
    nearest, each reaching it well inside its support (factor 1.5), so every
    moment matrix of the batch is well conditioned (the oracle's 1-norm
    condition numbers stay below 1e4; a floor reaching particles at the
    support edge left one at 1.7e12 in the 256-object batch)."""
    from scipy.spatial import cKDTree
    from oracle import rkpm
    for c in synth.batch(6, seed=11, nmin=2000, nmax=6000):
        X = c.X.astype(np.float64)
        a = c.a.astype(np.float64)
        cand = cKDTree(X).query_ball_point(X, float(a.max()))
        cover = [int(np.sum(np.linalg.norm(X[cd] - X[i], axis=1) < a[cd]))
                 for i, cd in enumerate(cand)]
        assert min(cover) >= 9, c.name
        ptr, idx = rkpm.neighbours(c.X, c.a)
        _, _, cond = rkpm.shape_functions(c.X, c.a, ptr, idx)
        assert np.max(cond) < 1e4, c.name


def test_single_rows_match_the_full_assembly():
    """twoset.rows (one row from the quadrature points its centre covers)
    against the full assembly, with per-point material."""
    X, v = synth.cube_grid(10)
    K = 80
    cen = twoset.farthest_point_sampling(X, K)
    P = X[cen]
    r = twoset.radii(P)
    rng = np.random.default_rng(2)
    E = rng.uniform(1e4, 1e6, X.shape[0])
    nu = 0.4
    scale = float(np.float32(r.max()))
    ptr, idx, phi, dphi, _ = twoset.shape_functions(X, P, r, 3.0, scale=scale)
    H, M = twoset.assemble(X.shape[0], K, ptr, idx, phi, dphi, v, E, nu)
    for k, (cols, h, m) in zip([0, 33, 79], twoset.rows([0, 33, 79], X, v, P, r, 3.0, E, nu,
                                                        scale)):
        np.testing.assert_array_equal(cols, H[k].indices)
        np.testing.assert_allclose(h, H[k].data, rtol=1e-9, atol=1e-12 * np.abs(H[k].data).max())
        np.testing.assert_allclose(m, M[k].toarray()[0, cols], rtol=1e-9,
                                   atol=1e-12 * np.abs(M[k].data).max())
