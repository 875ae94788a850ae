"""Learned near-diagonal residual: MLP, training step, pair data, stencil (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Not in the paper: a small network predicts, for dense pairs closer than
`radius` dense steps, the residual between the explicit model kernel and the
M1-interpolated kernel (both from Sec. 4), scaled by N_k so its values are O(1).

  features  x = (q_1, q_2, q_3, |q|, onehot(vc) [t], onehot(v'c') [t], dE_vc, dE_v'c')
            with q the Cartesian minimum-image k - k' (orthonormal axes)
  network   z1 = W1 x + b1, h1 = gelu(z1); z2 = W2 h1 + b2, h2 = gelu(z2);
            z3 = W3 h2 + b3, h3 = gelu(z3); out = W4 h3 + b4  (2 outputs: Re, Im)
            gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2   (exact form)
  loss      mean over the batch of (out - target)^2 summed over Re, Im
  Adam      m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
            p -= lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps)

Application (a reading, see the design notes): evaluated once with each dE
input at its zone average, the network gives a translation-invariant stencil
T(delta)[vc][v'c'] = out(delta)/N_k over the near offsets; the correction is the
periodic convolution (T * psi)(k) = sum_delta T(delta) psi(k - delta).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import model as om

WIDTH = 128
LAYERS = 4


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(d_in: int, seed: int, width: int = WIDTH):
    """He-style normal init (variance 2 / fan_in), zero biases; float64 arrays."""
    rng = np.random.default_rng(seed)
    dims = [d_in, width, width, width, 2]
    params = []
    for i in range(LAYERS):
        W = rng.standard_normal((dims[i + 1], dims[i])) * np.sqrt(2.0 / dims[i])
        params.append([W, np.zeros(dims[i + 1])])
    return params


def forward(params, X):
    """Returns (out [B, 2], cache)."""
    cache = [X]
    h = X
    zs = []
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = gelu(z) if i < LAYERS - 1 else z
        cache.append(h)
    return h, (cache, zs)


def loss_and_grad_out(out, target):
    B = out.shape[0]
    d = out - target
    return float(np.sum(d * d) / B), 2.0 * d / B


def backward(params, cache_zs, dout):
    """Gradients [(dW, db)] of the loss with d(loss)/d(out) = dout."""
    cache, zs = cache_zs
    grads = [None] * LAYERS
    g = dout
    for i in range(LAYERS - 1, -1, -1):
        W, _ = params[i]
        if i < LAYERS - 1:
            g = g * gelu_grad(zs[i])
        grads[i] = [g.T @ cache[i], g.sum(axis=0)]
        g = g @ W
    return grads


def adam_update(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place (step counts from 1)."""
    for layer in range(LAYERS):
        for j in range(2):
            g = grads[layer][j]
            m[layer][j] = b1 * m[layer][j] + (1 - b1) * g
            v[layer][j] = b2 * v[layer][j] + (1 - b2) * g * g
            mh = m[layer][j] / (1 - b1 ** step)
            vh = v[layer][j] / (1 - b2 ** step)
            params[layer][j] = params[layer][j] - lr * mh / (np.sqrt(vh) + eps)


def features(qvec, tr1, tr2, dE1, dE2, t):
    """Network inputs for a batch: qvec [B, 3], tr1/tr2 transition indices [B],
    dE1/dE2 [B]  ->  X [B, 4 + 2 t + 2]."""
    B = qvec.shape[0]
    X = np.zeros((B, 6 + 2 * t))
    X[:, :3] = qvec
    X[:, 3] = np.sqrt((qvec * qvec).sum(1))
    X[np.arange(B), 4 + tr1] = 1.0
    X[np.arange(B), 4 + t + tr2] = 1.0
    X[:, 4 + 2 * t] = dE1
    X[:, 5 + 2 * t] = dE2
    return X


def near_offsets(radius: int) -> np.ndarray:
    """Integer dense offsets delta with |delta| < radius (strict), lexicographic."""
    r = radius
    return np.array([(a, b, c) for a in range(-r, r + 1) for b in range(-r, r + 1) for c in range(-r, r + 1)
                     if a * a + b * b + c * c < r * r], dtype=np.int64)


def residual_samples(I, H_exp, H_m1, kd, kd2, tr1, tr2):
    """Targets N_k (K_exp - K_M1) for the sampled (dense k, dense k', vc, v'c')
    and the matching features, from dense matrices (tiny systems)."""
    t = I.t
    rows = kd * t + tr1
    cols = kd2 * t + tr2
    target = I.Nk * (H_exp[rows, cols] - H_m1[rows, cols])
    L = I.n * I.nd
    g = I.dense.gint
    d = g[kd] - g[kd2]
    dmin = np.mod(d + L // 2, L) - L // 2
    qvec = dmin / L
    dE = I.dE
    X = features(qvec, tr1, tr2, dE[rows], dE[cols], t)
    return X, np.stack([target.real, target.imag], axis=1)


def stencil(params, I, radius: int, dE_avg: np.ndarray):
    """T(delta)[vc][v'c'] for the near offsets (complex, already / N_k),
    evaluated with each dE input at its zone average dE_avg [t]."""
    t = I.t
    L = I.n * I.nd
    offs = near_offsets(radius)
    nd_ = offs.shape[0]
    q = np.repeat(offs / L, t * t, axis=0)
    tr1 = np.tile(np.repeat(np.arange(t), t), nd_)
    tr2 = np.tile(np.tile(np.arange(t), t), nd_)
    X = features(q, tr1, tr2, dE_avg[tr1], dE_avg[tr2], t)
    out, _ = forward(params, X)
    T = (out[:, 0] + 1j * out[:, 1]).reshape(nd_, t, t) / I.Nk
    # Hermitian operator: T(delta) <- (T(delta) + T(-delta)^H) / 2
    idx = {tuple(o): i for i, o in enumerate(offs)}
    neg = np.array([idx[tuple(-o)] for o in offs])
    T = 0.5 * (T + np.conj(T[neg]).transpose(0, 2, 1))
    return offs, T


def apply_stencil_fft(I, offs, T, psi):
    """The same periodic convolution through numpy FFTs on the dense grid."""
    L = I.n * I.nd
    t = I.t
    ker = np.zeros((L, L, L, t, t), dtype=np.complex128)
    for i, d in enumerate(offs):
        ker[d[0] % L, d[1] % L, d[2] % L] += T[i]
    g = I.dense.gint
    grid = np.zeros((L, L, L, t), dtype=np.complex128)
    grid[g[:, 0], g[:, 1], g[:, 2]] = psi.reshape(I.Nk, t)
    kf = np.fft.fftn(ker, axes=(0, 1, 2))
    pf = np.fft.fftn(grid, axes=(0, 1, 2))
    conv = np.fft.ifftn(np.einsum("xyzab,xyzb->xyza", kf, pf), axes=(0, 1, 2))
    return conv[g[:, 0], g[:, 1], g[:, 2]].reshape(-1)


def apply_stencil_direct(I, offs, T, psi):
    """(T * psi)(k) = sum_delta T(delta) psi(k - delta), pair by pair (k - delta
    is the dense point at integer offset -delta from k, periodic)."""
    L = I.n * I.nd
    g = I.dense.gint
    lin = {tuple(x): i for i, x in enumerate(g)}
    P = psi.reshape(I.Nk, I.t)
    out = np.zeros_like(P)
    for i, d in enumerate(offs):
        src = np.array([lin[tuple(np.mod(gk - d, L))] for gk in g])
        out += P[src] @ T[i].T
    return out.reshape(-1)


def mean_dE(I) -> np.ndarray:
    return I.dE.reshape(I.Nk, I.t).mean(axis=0)
