"""Oracle: the learned warm start -- per-particle features, the point network,
its subspace loss and the loss gradient, plain FP64.

Test infrastructure only (see ``oracle/__init__``).

The paper has no learned component on this path; it starts its LOBPCG from a
random block (Supp. Sec. B).  The warm start predicts a start block for the
same eigenproblem (Sec. 3.2, Eq. 15) from the particle cloud.  Its definition
is fixed here and restated by the CUDA library:

Features (16 per particle, canonical frame of the cloud):
  mu = sum v X / sum v,  C = sum v (X - mu)(X - mu)^T / sum v = R diag(s2) R^T
  with s2 descending; axis r_j flipped so that sum v ((X - mu) . r_j)^3 >= 0;
  s = sqrt(trace C).
  f[0:3]   R^T (X_i - mu) / s
  f[3:6]   R^T (mean_{k in N(i)} X_k - X_i) / a_i
  f[6:9]   diag(R^T C_i R) / a_i^2, C_i = mean_{k in N(i)} (X_k - m_i)(X_k - m_i)^T
  f[9]     |N(i)| / mean_j |N(j)|
  f[10]    a_i / s
  f[11]    v_i / mean_j v_j
  f[12:14] sqrt(s2[1] / s2[0]), sqrt(s2[2] / s2[0])
  f[14]    log(n) / 16
  f[15]    1
  (N(i): the support neighbours of the RKPM build, self included.)

Network (170,784 parameters, flat order W1 b1 W2 b2 W3 b3 W4 b4 W5 b5, each
W row-major [out][in]):
  h1 = relu(W1 f + b1)            16 -> 128
  h2 = relu(W2 h1 + b2)           128 -> 256
  g  = max over the particles of h2          (per channel)
  h3 = relu(W3 [h1; g] + b3)      384 -> 256
  h4 = relu(W4 h3 + b4)           256 -> 128
  y  = W5 h4 + b5                 128 -> 32

Loss (how much of the span of the m true modes C the predicted block Y
misses, in the volume-weighted inner product, W = diag(v) / sum v):
  G = Y^T W Y + eps I,  Z = Y^T W C,  K = C^T W C,
  L = 1 - trace(K^-1 Z^T G^-1 Z) / m,
  eps = 1e-6 trace(Y^T W Y) / 32 (a ridge for rank-deficient blocks),
  dL/dY = -(2/m) W (C P1 - Y P2 - e q Y),  P1 = K^-1 Z^T G^-1,
          P2 = G^-1 Z P1,  q = trace(P1 G^-1 Z),  e = 1e-6 / 32.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64

DIMS = [(16, 128), (128, 256), (384, 256), (256, 128), (128, 32)]
N_FEAT = 16
N_OUT = 32


def n_params():
    return sum(i * o + o for i, o in DIMS)


def unpack(theta):
    """Flat parameter vector -> [(W, b), ...] (views, FP64)."""
    theta = np.asarray(theta, dtype=F64)
    out, off = [], 0
    for i, o in DIMS:
        W = theta[off:off + i * o].reshape(o, i)
        off += i * o
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    assert off == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


# ---------------------------------------------------------------- features
def canonical_frame(X, v):
    """(mu, R, s2, s): volume-weighted centroid, principal axes (columns of R,
    descending variance, signs fixed by the third moment) and scale."""
    X = np.asarray(X, dtype=F64)
    v = np.asarray(v, dtype=F64)
    V = v.sum()
    mu = (v[:, None] * X).sum(0) / V
    D = X - mu
    C = (v[:, None, None] * (D[:, :, None] * D[:, None, :])).sum(0) / V
    s2, R = np.linalg.eigh(C)
    order = np.argsort(s2)[::-1]
    s2, R = s2[order], R[:, order]
    t = (v[:, None] * (D @ R) ** 3).sum(0)
    R = R * np.where(t < 0, -1.0, 1.0)[None, :]
    return mu, R, s2, np.sqrt(s2.sum())


def features(X, v, a, ptr, idx):
    """Per-particle features (n x 16, FP64) from the support neighbour lists."""
    X = np.asarray(X, dtype=F64)
    v = np.asarray(v, dtype=F64)
    a = np.asarray(a, dtype=F64)
    n = X.shape[0]
    mu, R, s2, s = canonical_frame(X, v)
    f = np.zeros((n, N_FEAT), dtype=F64)
    f[:, 0:3] = (X - mu) @ R / s
    cnt = np.diff(ptr).astype(F64)
    for i in range(n):
        nb = X[idx[ptr[i]:ptr[i + 1]]]
        m = nb.mean(0)
        f[i, 3:6] = (m - X[i]) @ R / a[i]
        D = nb - m
        Ci = D.T @ D / nb.shape[0]
        f[i, 6:9] = np.diag(R.T @ Ci @ R) / (a[i] * a[i])
    f[:, 9] = cnt / cnt.mean()
    f[:, 10] = a / s
    f[:, 11] = v / v.mean()
    f[:, 12] = np.sqrt(s2[1] / s2[0])
    f[:, 13] = np.sqrt(s2[2] / s2[0])
    f[:, 14] = np.log(n) / 16.0
    f[:, 15] = 1.0
    return f


# ---------------------------------------------------------------- network
def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as FP64: the
    storage format of the CUDA network's weights and activations."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(F64)


def forward(theta, f, store=None):
    """Returns (y, cache) for the point network on one cloud.  ``store``
    (e.g. ``bf16_round``) is applied to the features and to the activations
    h1, h3, h4 where a storage format rounds them."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5) = unpack(theta)
    st = store or (lambda a: a)
    f = st(np.asarray(f, dtype=F64))
    h1 = st(np.maximum(f @ W1.T + b1, 0.0))
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    arg = np.argmax(h2, axis=0)                 # first maximiser per channel
    g = h2[arg, np.arange(h2.shape[1])]
    z = np.concatenate([h1, np.broadcast_to(g, (h1.shape[0], g.size))], axis=1)
    h3 = st(np.maximum(z @ W3.T + b3, 0.0))
    h4 = st(np.maximum(h3 @ W4.T + b4, 0.0))
    y = h4 @ W5.T + b5
    return y, dict(f=f, h1=h1, h2=h2, arg=arg, g=g, z=z, h3=h3, h4=h4)


def subspace_loss(y, v, C):
    """(L, dL/dy) of the subspace loss above; C is n x m (any basis)."""
    y = np.asarray(y, dtype=F64)
    C = np.asarray(C, dtype=F64)
    w = np.asarray(v, dtype=F64) / np.sum(v)
    m = C.shape[1]
    WY = w[:, None] * y
    G0 = y.T @ WY
    eps = 1e-6 * np.trace(G0) / y.shape[1]
    G = G0 + eps * np.eye(y.shape[1])
    Z = WY.T @ C
    K = C.T @ (w[:, None] * C)
    Gi = np.linalg.inv(G)
    Ki = np.linalg.inv(K)
    L = 1.0 - np.trace(Ki @ Z.T @ Gi @ Z) / m
    P1 = Ki @ Z.T @ Gi                  # m x 32
    P2 = Gi @ Z @ P1                    # 32 x 32
    q = np.trace(P1 @ Gi @ Z)           # d trace(K^-1 Z^T G^-1 Z) / d eps = -q
    e = 1e-6 / y.shape[1]
    dy = -(2.0 / m) * w[:, None] * (C @ P1 - y @ P2 - e * q * y)
    return L, dy


def backward(theta, cache, dy):
    """Gradient of a scalar through the network given dL/dy; flat like theta."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5) = unpack(theta)
    h1, h2, arg, g, z, h3, h4 = (cache[k] for k in ("h1", "h2", "arg", "g", "z", "h3", "h4"))
    f = cache["f"]
    dW5 = dy.T @ h4
    db5 = dy.sum(0)
    dh4 = (dy @ W5) * (h4 > 0)
    dW4 = dh4.T @ h3
    db4 = dh4.sum(0)
    dh3 = (dh4 @ W4) * (h3 > 0)
    dW3 = dh3.T @ z
    db3 = dh3.sum(0)
    dz = dh3 @ W3
    dh1 = dz[:, :128].copy()
    dg = dz[:, 128:].sum(0)
    # max pool: the gradient of channel c goes to its maximiser (if active)
    dh2 = np.zeros_like(h2)
    ch = np.arange(h2.shape[1])
    dh2[arg, ch] = dg * (g > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(0)
    dh1 += dh2 @ W2
    dh1 *= (h1 > 0)
    dW1 = dh1.T @ f
    db1 = dh1.sum(0)
    return pack([(dW1, db1), (dW2, db2), (dW3, db3), (dW4, db4), (dW5, db5)])


def loss_and_grad(theta, f, v, C, store=None):
    y, cache = forward(theta, f, store)
    L, dy = subspace_loss(y, v, C)
    return L, backward(theta, cache, dy)


def adam_step(theta, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); returns (theta, m1, m2)."""
    m1 = beta1 * m1 + (1 - beta1) * grad
    m2 = beta2 * m2 + (1 - beta2) * grad * grad
    mh = m1 / (1 - beta1 ** t)
    vh = m2 / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2


def init_params(seed):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    layers = []
    for i, o in DIMS:
        layers.append((rng.standard_normal((o, i)) * np.sqrt(2.0 / i), np.zeros(o)))
    return pack(layers)
