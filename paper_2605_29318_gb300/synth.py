"""Seeded synthetic particle clouds (inputs only; none of the method's arithmetic).

Both the CUDA path and the FP64 oracle consume these arrays.  Every generator
is deterministic in its seed (numpy PCG64) and returns a ``Cloud`` of FP32
arrays: positions X (N, 3), quadrature volumes v (N,), support radii a (N,),
and the material (Young's modulus E, Poisson ratio nu; scalars or per particle).

The shapes stand in for the paper's meshes and Gaussian-splat objects
(Supp. Sec. B "RKPM construction": points sampled inside the object; for 3DGS
the splat centres themselves).  Support radius a_i = s * h_i with h_i = v_i^(1/3)
the local spacing, so s = 2 gives "support 2.0x spacing".
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Cloud:
    X: np.ndarray          # (N, 3) float32 positions
    v: np.ndarray          # (N,) float32 quadrature volumes
    a: np.ndarray          # (N,) float32 support radii
    E: object              # float or (N,) float32 Young's modulus
    nu: object             # float or (N,) float32 Poisson ratio
    k: int                 # number of modes asked for (constant mode included)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _finish(X, volume, support, E, nu, k, name):
    n = X.shape[0]
    v = np.full(n, volume / n, dtype=np.float64)
    h = (volume / n) ** (1.0 / 3.0)
    a = np.full(n, support * h, dtype=np.float64)
    return Cloud(X.astype(np.float32), v.astype(np.float32), a.astype(np.float32),
                 E, nu, k, name)


def unit_cube(n=2000, seed=1, support=2.0, E=1e5, nu=0.45, k=10):
    """Uniform random points in [0, 1]^3, equal volumes 1/N."""
    X = _rng(seed).random((n, 3))
    return _finish(X, 1.0, support, E, nu, k, f"cube{n}")


def _rejection(n, lo, hi, inside, rng, batch=None):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    out = []
    got = 0
    batch = batch or max(1024, 2 * n)
    while got < n:
        P = lo + (hi - lo) * rng.random((batch, 3))
        P = P[inside(P)]
        out.append(P)
        got += P.shape[0]
    return np.concatenate(out)[:n]


def torus(n=50000, R=0.5, r=0.2, seed=2, support=2.0, E=1e6, nu=0.4, k=32):
    """Solid torus (major radius R, minor r), rejection-sampled in its box."""
    def inside(P):
        rho = np.sqrt(P[:, 0] ** 2 + P[:, 1] ** 2)
        return (rho - R) ** 2 + P[:, 2] ** 2 < r * r
    X = _rejection(n, [-R - r, -R - r, -r], [R + r, R + r, r], inside, _rng(seed))
    return _finish(X, 2.0 * math.pi ** 2 * R * r * r, support, E, nu, k, f"torus{n}")


def layered_sphere(n=3000, radius=0.5, seed=6, support=2.0, E_stiff=1e7, E_soft=1e5,
                   nu=0.45, k=10):
    """The heterogeneous sphere of the paper's multi-layer demonstration: four
    concentric shells of equal thickness, stiff-soft-stiff-soft from the
    centre out (the paper states the order, not the radii or moduli: the
    shells split the radius in four, and stiff / soft are 1e7 / 1e5 Pa).
    Rejection-sampled in the ball; E per particle from its shell."""
    def inside(P):
        return (P * P).sum(1) < radius * radius
    X = _rejection(n, [-radius] * 3, [radius] * 3, inside, _rng(seed))
    c = _finish(X, 4.0 / 3.0 * math.pi * radius ** 3, support, 1.0, nu, k, f"layers{n}")
    shell = np.minimum((np.sqrt((X * X).sum(1)) / radius * 4).astype(np.int64), 3)
    c.E = np.where(shell % 2 == 0, E_stiff, E_soft).astype(np.float32)
    c.nu = np.float32(nu)
    return c


def inside_grid(lo, hi, h, inside):
    """Quadrature points of the paper's two-set construction: the centres of a
    uniform grid of spacing h over the box [lo, hi], those outside the solid
    dropped, each with volume h^3 (Supp. Sec. B samples the object's bounding
    box on a grid and rejects outside points).  Returns (X float32 (n, 3),
    v float32 (n,)); points ordered x fastest, then y, then z."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    m = np.maximum(np.ceil((hi - lo) / h - 1e-9).astype(np.int64), 1)
    axes = [lo[d] + (np.arange(m[d]) + 0.5) * h for d in range(3)]
    Z, Y, Xg = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    P = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], 1)
    P = P[inside(P)]
    return P.astype(np.float32), np.full(P.shape[0], h ** 3, dtype=np.float32)


def cube_grid(m=16):
    """The unit cube's quadrature grid: m^3 cell centres, volume 1/m^3 each."""
    return inside_grid([0, 0, 0], [1, 1, 1], 1.0 / m, lambda P: np.ones(P.shape[0], bool))


def torus_grid(h=0.02, R=0.5, r=0.2):
    """Inside grid of the solid torus of ``torus`` (exact volume 2 pi^2 R r^2)."""
    def inside(P):
        rho = np.sqrt(P[:, 0] ** 2 + P[:, 1] ** 2)
        return (rho - R) ** 2 + P[:, 2] ** 2 < r * r
    return inside_grid([-R - r, -R - r, -r], [R + r, R + r, r], h, inside)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid_union(n=20000, seed=5, n_ell=None, support=2.0, E=1e6, nu=0.4, k=16):
    """Union of 2-5 overlapping random ellipsoids (a connected blob-like solid)."""
    rng = _rng(seed)
    m = n_ell or int(rng.integers(2, 6))
    axes = 0.2 + 0.3 * rng.random((m, 3))
    rots = [_random_rotation(rng) for _ in range(m)]
    # each centre lies inside the previous ellipsoid (within its smallest
    # semi-axis), so the union is connected
    centres = [np.zeros(3)]
    for j in range(1, m):
        d = rng.normal(size=3)
        d *= axes[j - 1].min() * rng.uniform(0.3, 0.8) / np.linalg.norm(d)
        centres.append(centres[-1] + d)
    centres = np.array(centres)

    def inside(P):
        ok = np.zeros(P.shape[0], bool)
        for c, ax, Rm in zip(centres, axes, rots):
            L = (P - c) @ Rm
            ok |= ((L / ax) ** 2).sum(1) < 1.0
        return ok
    lo = (centres - axes.max(1, keepdims=True)).min(0)
    hi = (centres + axes.max(1, keepdims=True)).max(0)
    # volume by Monte Carlo on the box (input construction only)
    probe = lo + (hi - lo) * rng.random((200000, 3))
    vol = float(np.prod(hi - lo) * inside(probe).mean())
    X = _rejection(n, lo, hi, inside, rng)
    return _finish(X, vol, support, E, nu, k, f"ellipsoids{n}")


def gaussian_mixture(n=1_000_000, n_comp=64, seed=3, support=2.0, nu=0.45, k=64,
                     knn=16):
    """Splat-like cloud: a mixture of anisotropic 3D Gaussians.

    Axis scales log-uniform in [0.02, 0.3], random rotations, equal weights;
    centres placed by a random walk with step 0.7 x (sum of the two largest
    scales) so that components overlap; samples truncated at 3 sigma.  The
    volume of particle i is taken from the local density of its ``knn``
    nearest neighbours, v_i = (4/3) pi d_i^3 / knn; E is log-uniform in
    [1e4, 1e7] per component (heterogeneous material).  Supports get the
    coverage floor of ``support_floor`` (the thin outskirts of the Gaussians
    otherwise leave particles covered by fewer than four nodes)."""
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    scales = np.exp(rng.uniform(np.log(0.02), np.log(0.3), size=(n_comp, 3)))
    rots = [_random_rotation(rng) for _ in range(n_comp)]
    centres = np.zeros((n_comp, 3))
    for c in range(1, n_comp):
        two = np.sort(scales[c - 1])[-2:].sum() + np.sort(scales[c])[-2:].sum()
        d = rng.normal(size=3)
        centres[c] = centres[c - 1] + 0.35 * two * d / np.linalg.norm(d)
    Ecomp = np.exp(rng.uniform(np.log(1e4), np.log(1e7), size=n_comp))
    comp = rng.integers(0, n_comp, size=n)
    Z = rng.normal(size=(n, 3))
    bad = np.abs(Z).max(1) > 3.0
    while bad.any():
        Z[bad] = rng.normal(size=(int(bad.sum()), 3))
        bad = np.abs(Z).max(1) > 3.0
    X = np.empty((n, 3))
    for c in range(n_comp):
        sel = comp == c
        X[sel] = centres[c] + (Z[sel] * scales[c]) @ rots[c].T
    X32 = X.astype(np.float32)
    tree = cKDTree(X32.astype(np.float64))
    dist, _ = tree.query(X32.astype(np.float64), k=knn + 1)
    dk = dist[:, -1]
    v = (4.0 / 3.0) * np.pi * dk ** 3 / knn
    a = support * np.cbrt(v)
    E = Ecomp[comp].astype(np.float32)
    return Cloud(X32, v.astype(np.float32), a.astype(np.float32), E,
                 np.float32(nu), k, f"splat{n}")


def batch(n_objects=256, seed=4, nmin=2000, nmax=200000, kmin=16, kmax=48):
    """Many objects: cube / torus / ellipsoid union, random scale and rotation,
    particle counts log-uniform in [nmin, nmax], k uniform in [kmin, kmax].
    Supports get the coverage floor of ``support_floor`` with factor 1.5:
    among this many random clouds some leave a particle (a cube corner,
    typically) covered by only two or three nodes at 2.0x spacing, and a floor
    that reaches it only at the edge of the nodes' supports (factor near 1)
    leaves its moment matrix numerically singular (cond ~1e12)."""
    rng = _rng(seed)
    out = []
    for j in range(n_objects):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        k = int(rng.integers(kmin, kmax + 1))
        fam = int(rng.integers(0, 3))
        s = int(rng.integers(0, 2 ** 31 - 1))
        if fam == 0:
            c = unit_cube(n, seed=s, E=1e6, nu=0.4, k=k)
        elif fam == 1:
            c = torus(n, seed=s, E=1e6, nu=0.4, k=k)
        else:
            c = ellipsoid_union(n, seed=s, E=1e6, nu=0.4, k=k)
        scale = float(np.exp(rng.uniform(np.log(0.5), np.log(2.0))))
        Rm = _random_rotation(rng)
        c.X = ((c.X.astype(np.float64) * scale) @ Rm.T).astype(np.float32)
        c.v = (c.v.astype(np.float64) * scale ** 3).astype(np.float32)
        c.a = (c.a.astype(np.float64) * scale).astype(np.float32)
        c.a = support_floor(c.X, c.a, factor=1.5)
        c.name = f"obj{j}-{c.name}"
        out.append(c)
    return out


def warmstart_shape(seed, nmin=20000, nmax=100000, k=32):
    """One object of the warm-start corpus: a box with sides in [0.5, 1.5], a
    torus with R in [0.35, 0.6] and r in [0.12, 0.25], or a union of
    ellipsoids; random scale in [0.5, 2] and rotation; particle count
    log-uniform in [nmin, nmax].  Training shapes use seeds 10000 + i, held-out
    shapes 20000 + i."""
    rng = _rng(seed)
    n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
    fam = int(rng.integers(0, 3))
    s = int(rng.integers(0, 2 ** 31 - 1))
    if fam == 0:
        sides = 0.5 + rng.random(3)
        X = _rng(s).random((n, 3)) * sides
        c = _finish(X, float(np.prod(sides)), 2.0, 1e6, 0.4, k, f"box{n}")
    elif fam == 1:
        c = torus(n, R=float(rng.uniform(0.35, 0.6)), r=float(rng.uniform(0.12, 0.25)), seed=s,
                  E=1e6, nu=0.4, k=k)
    else:
        c = ellipsoid_union(n, seed=s, E=1e6, nu=0.4, k=k)
    scale = float(np.exp(rng.uniform(np.log(0.5), np.log(2.0))))
    Rm = _random_rotation(rng)
    c.X = ((c.X.astype(np.float64) * scale) @ Rm.T).astype(np.float32)
    c.v = (c.v.astype(np.float64) * scale ** 3).astype(np.float32)
    c.a = (c.a.astype(np.float64) * scale).astype(np.float32)
    c.a = support_floor(c.X, c.a)
    c.name = f"ws{seed}-{c.name}"
    return c


def support_floor(X, a, m=8, factor=1.0001):
    """Widen supports so that every particle is covered by its m nearest other
    particles: a_k <- max(a_k, factor d(j, k)) over every j that has k among
    its m nearest (node k covers X_j iff |X_j - p_k| < a_k).  Random sampling
    otherwise leaves the odd thin spot with too few covering nodes for the
    moment matrix.  With factor near 1 a node reaches such a particle at the
    edge of its support, where the B-spline weight is ~(4/3)(1 - 1/factor)^3;
    factor = 1.5 keeps that weight above 0.04."""
    from scipy.spatial import cKDTree
    P = np.asarray(X, np.float64)
    d, nb = cKDTree(P).query(P, k=m + 1)
    out = np.asarray(a, np.float64).copy()
    np.maximum.at(out, nb[:, 1:].ravel(), factor * d[:, 1:].ravel())
    return out.astype(np.float32)
