"""CPU reference of the learned subspace proposal (test infrastructure only: tests/, bench.py's
CPU legs).  Plain numpy in FP64, written from the definitions; nothing here is used by the
CUDA library, and nothing from the library is used here.

Definitions (no paper counterpart; the proposal seeds the range finder of eq. SVD_Ul):
  features      per mode l: c-weighted, unit-sum 64-bin histograms of the centre coordinate
                x_{k,l} over [-cbox, cbox] and of log a_k over [la, lb] (end bins catch the rest)
  basis         Chebyshev polynomials T_0..T_63 of x/b on the cell-centre grid, orthonormalised
                in order by Gram-Schmidt (two passes): the discrete orthogonal polynomials Q_T
  network       128 -> 512 -> 512 -> 512 -> 2048, h = W a + b, GELU(h) = h Phi(h) after the hidden
                layers (erf form); operands of each product optionally rounded to BF16
  output        C (64 x 32), C[i, j] = y[i + 64 j]; proposal Q0 = Q_T C
  loss          mean over the batch of ||C C^T - G||_F^2, G = (Q_T^T Z)(Q_T^T Z)^T
  Adam          beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected
"""
import math

import numpy as np
from scipy.special import erf as _erf

DIMS = (128, 512, 512, 512, 2048)
NCHEB, NCOEF, NBIN = 64, 32, 64


def bf16(x):
    """Round FP32/FP64 values to BF16 (round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    rounding = ((b >> 16) & 1) + 0x7FFF
    r = ((b + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(centres, loga, c, cbox, la, lb):
    """(3, 128): per mode, the centre-coordinate histogram then the log-exponent histogram."""
    out = np.zeros((3, 2 * NBIN))
    tot = float(np.sum(c))
    for l in range(3):
        for col, (x, lo, hi) in enumerate(((centres[:, l], -cbox, cbox), (loga, la, lb))):
            q = np.floor((x - lo) / (hi - lo) * NBIN).astype(np.int64)
            q = np.clip(q, 0, NBIN - 1)
            h = np.zeros(NBIN)
            np.add.at(h, q, c)
            out[l, col * NBIN:(col + 1) * NBIN] = h / tot if tot > 0 else 0.0
    return out


def chebyshev_basis(n, b):
    """Q_T (n x 64): T_j(x_i / b) on x_i = -b + (i + 1/2) 2b/n, orthonormalised in order."""
    x = (-b + (np.arange(n) + 0.5) * 2.0 * b / n) / b
    T = np.zeros((n, NCHEB))
    T[:, 0] = 1.0
    T[:, 1] = x
    for j in range(2, NCHEB):
        T[:, j] = 2.0 * x * T[:, j - 1] - T[:, j - 2]
    Q = T.copy()
    for j in range(NCHEB):
        for _ in range(2):
            for i in range(j):
                Q[:, j] -= (Q[:, i] @ Q[:, j]) * Q[:, i]
        Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


def target(QT, Z):
    """G = (Q_T^T Z)(Q_T^T Z)^T for the leading basis Z (n x r)."""
    P = QT.T @ Z
    return P @ P.T


def gelu(h):
    return 0.5 * h * (1.0 + _erf(h / math.sqrt(2.0)))


def gelu_grad(h):
    return 0.5 * (1.0 + _erf(h / math.sqrt(2.0))) + h * np.exp(-0.5 * h * h) / math.sqrt(2.0 * math.pi)


def init_params(seed=0):
    """Reference initialisation (He normal, zero bias) -- any weights can be loaded instead."""
    g = np.random.default_rng(seed)
    return [(g.standard_normal((DIMS[i + 1], DIMS[i])) * math.sqrt(2.0 / DIMS[i]), np.zeros(DIMS[i + 1]))
            for i in range(4)]


def forward(params, X, round_bf16=True):
    """Returns (Y, cache): Y (B x 2048); X (B x 128)."""
    a = np.asarray(X, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(params):
        A = bf16(a) if round_bf16 else a
        Wq = bf16(W) if round_bf16 else W
        h = A @ Wq.T + b
        cache.append((a, h))
        a = h if i == len(params) - 1 else gelu(h)
    return a, cache


def loss_and_grad_output(Y, G):
    """Mean over the batch of ||C C^T - G||^2 and its gradient with respect to Y."""
    B = Y.shape[0]
    loss = 0.0
    dY = np.zeros_like(Y)
    for s in range(B):
        C = Y[s].reshape(NCOEF, NCHEB).T          # C[i, j] = y[i + 64 j]
        D = C @ C.T - G[s]
        loss += np.sum(D * D)
        dC = 4.0 * D @ C / B
        dY[s] = dC.T.reshape(-1)
    return loss / B, dY


def backward(params, cache, dY, round_bf16=True):
    """Gradients [(dW, db), ...] of the loss; products use BF16 operands like the forward."""
    grads = [None] * len(params)
    d = dY
    for i in range(len(params) - 1, -1, -1):
        W, _ = params[i]
        a, h = cache[i]
        dZ = d if i == len(params) - 1 else d * gelu_grad(h)
        dZq = bf16(dZ) if round_bf16 else dZ
        Aq = bf16(a) if round_bf16 else a
        grads[i] = (dZq.T @ Aq, dZ.sum(axis=0))
        if i > 0:
            Wq = bf16(W) if round_bf16 else W
            d = dZq @ Wq
    return grads


def adam_step(params, grads, state, lr):
    """One Adam update in place; state = dict(step, m, v) (created on first use)."""
    if not state:
        state.update(step=0, m=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
                     v=[(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
    state["step"] += 1
    t = state["step"]
    c1, c2 = 1.0 / (1.0 - 0.9 ** t), 1.0 / (1.0 - 0.999 ** t)
    for i in range(len(params)):
        for j in range(2):
            g = grads[i][j]
            m = state["m"][i][j]
            v = state["v"][i][j]
            m *= 0.9
            m += 0.1 * g
            v *= 0.999
            v += 0.001 * g * g
            params[i][j][...] -= lr * (m * c1) / (np.sqrt(v * c2) + 1e-8)
