"""FP64 oracle of the learned drift proposal (test infrastructure only).

The proposal replaces the nudging optimiser of Sec. 3.1.3 by a network that
maps a particle's state at the window start and the innovation of the window's
observations to the drifts lambda [Ns][K]; any lambda keeps the particle
weights consistent through the Girsanov factor, so the network only affects
how close the proposal lands to the observations.  Not in the paper.

Network (all convolutions circular, kernel 5, stride 2, padding 2):
    features  x0[0] = u_start,  x0[1] = (y_j - u_start(x_j)) / sigma at node j n/M, 0 elsewhere
              and at unobserved points (y_j NaN)
    conv1     2 -> C channels,  n -> n/2,   ReLU
    conv2     C -> C,           n/2 -> n/4, ReLU
    conv3     C -> C,           n/4 -> n/8, ReLU
    conv4     C -> C,           n/8 -> n/16, ReLU
    modes     F[c, 2(j-1)] = (1/P) sum_q h[c, q] sin(2 pi j q / P),
              F[c, 2(j-1)+1] = (1/P) sum_q h[c, q] cos(2 pi j q / P),   P = n/16, j = 1..K/2
    head      lambda = Wh F + bh,  F flattened channel-major to C K values
Loss: L = 1/(2B) sum_b sum_o (lambda_bo - target_bo)^2.  Adam (Kingma & Ba):
m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, p <- p - lr mhat / (sqrt(vhat) + eps).

Pinned by tests/test_oracle_convnet.py against torch's CPU conv1d (circular
padding), autograd and torch.optim.Adam in FP64, and central differences.

``operands="bf16"`` evaluates the same network with both operands of every
contraction (each convolution, the mode projection and the head, forward and
backward) rounded to BF16 first, as a BF16-operand, FP32-accumulating tensor-core
path does; the sums themselves stay FP64.  The ReLU masks, decisions on the
pre-activations, are then taken on the same BF16-operand products as such a path.
"""
from __future__ import annotations

import math

import numpy as np

KSIZE = 5
STRIDE = 2
PAD = 2
NLAYER = 4


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), through FP32 as a value held in
    FP32 memory would be: keep the top 16 bits of the FP32 pattern after adding
    0x7FFF plus the lowest kept bit."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _rounder(operands):
    if operands is None or operands == "fp64":
        return lambda a: a
    if operands == "bf16":
        return bf16_round
    raise ValueError(operands)


def init_params(C: int, K: int, Ns: int, n: int, seed: int):
    """He-style initialisation from a seeded numpy generator."""
    r = np.random.default_rng(seed)
    p = {}
    cin = 2
    for l in range(NLAYER):
        fan = cin * KSIZE
        p[f"w{l}"] = r.normal(scale=math.sqrt(2.0 / fan), size=(C, cin, KSIZE))
        p[f"b{l}"] = np.zeros(C)
        cin = C
    p["wh"] = r.normal(scale=math.sqrt(1.0 / (C * K)), size=(K * Ns, C * K))
    p["bh"] = np.zeros(K * Ns)
    return p


def features(u_start: np.ndarray, y: np.ndarray, sigma: float) -> np.ndarray:
    """x0 [B, 2, n] from the start velocities [B, n] and the window observations [M]
    (an unobserved point, y_j NaN, has innovation 0)."""
    u = np.atleast_2d(np.asarray(u_start, dtype=np.float64))
    B, n = u.shape
    y = np.asarray(y, dtype=np.float64)
    M = len(y)
    stride = n // M
    x = np.zeros((B, 2, n))
    x[:, 0] = u
    inn = (y[None, :] - u[:, ::stride]) / sigma
    x[:, 1, ::stride] = np.where(np.isnan(y)[None, :], 0.0, inn)
    return x


def conv_forward(x: np.ndarray, w: np.ndarray, b: np.ndarray, rnd=lambda a: a) -> np.ndarray:
    """out[b, co, q] = b[co] + sum_ci sum_j w[co, ci, j] x[b, ci, (2q + j - 2) mod L]."""
    B, Ci, L = x.shape
    Lo = L // STRIDE
    idx = (STRIDE * np.arange(Lo)[:, None] + np.arange(KSIZE)[None, :] - PAD) % L   # [Lo, k]
    cols = rnd(x)[:, :, idx]                                                          # [B, Ci, Lo, k]
    return np.einsum("bcqj,ocj->boq", cols, rnd(w)) + b[None, :, None]


def conv_backward(x: np.ndarray, w: np.ndarray, gout: np.ndarray, rnd=lambda a: a):
    """Gradients of conv_forward: (dx, dw, db) given dL/dout."""
    B, Ci, L = x.shape
    Lo = L // STRIDE
    idx = (STRIDE * np.arange(Lo)[:, None] + np.arange(KSIZE)[None, :] - PAD) % L
    cols = rnd(x)[:, :, idx]
    dw = np.einsum("boq,bcqj->ocj", rnd(gout), cols)
    db = gout.sum(axis=(0, 2))
    dcols = np.einsum("boq,ocj->bcqj", rnd(gout), rnd(w))
    dx = np.zeros_like(x)
    for q in range(Lo):
        for j in range(KSIZE):
            dx[:, :, idx[q, j]] += dcols[:, :, q, j]
    return dx, dw, db


def mode_matrix(P: int, K: int) -> np.ndarray:
    """S[q, 2(j-1)] = sin(2 pi j q / P) / P, S[q, 2(j-1)+1] = cos(2 pi j q / P) / P."""
    q = np.arange(P)
    S = np.empty((P, K))
    for jj in range(K // 2):
        j = jj + 1
        S[:, 2 * jj] = np.sin(2 * math.pi * j * q / P) / P
        S[:, 2 * jj + 1] = np.cos(2 * math.pi * j * q / P) / P
    return S


def forward(params, x0: np.ndarray, K: int, Ns: int, operands=None):
    """lambda [B, Ns, K] and the cache of activations."""
    rnd = _rounder(operands)
    acts = [x0]
    h = x0
    for l in range(NLAYER):
        z = conv_forward(h, params[f"w{l}"], params[f"b{l}"], rnd)
        h = np.maximum(z, 0.0)
        acts.append(h)
    B, C, P = h.shape
    S = mode_matrix(P, K)
    F = np.einsum("bcq,qk->bck", rnd(h), rnd(S)).reshape(B, C * K)
    lam = rnd(F) @ rnd(params["wh"]).T + params["bh"][None, :]
    return lam.reshape(B, Ns, K), (acts, F, S)


def loss_and_grad(params, x0: np.ndarray, target: np.ndarray, K: int, Ns: int, operands=None):
    """L = 1/(2B) sum (lambda - target)^2 and dL/dparams (manual backward)."""
    rnd = _rounder(operands)
    lam, (acts, F, S) = forward(params, x0, K, Ns, operands)
    B = x0.shape[0]
    diff = (lam - target).reshape(B, Ns * K)
    L = 0.5 * float(np.sum(diff * diff)) / B
    g = {}
    glam = diff / B                                   # [B, Ns K]
    g["wh"] = rnd(glam).T @ rnd(F)
    g["bh"] = glam.sum(axis=0)
    gF = (rnd(glam) @ rnd(params["wh"])).reshape(B, -1, K)      # [B, C, K]
    gh = np.einsum("bck,qk->bcq", rnd(gF), rnd(S))
    for l in reversed(range(NLAYER)):
        gz = gh * (acts[l + 1] > 0.0)
        dx, dw, db = conv_backward(acts[l], params[f"w{l}"], gz, rnd)
        g[f"w{l}"] = dw
        g[f"b{l}"] = db
        gh = dx
    return L, g


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g * g
            mhat = self.m[k] / (1 - self.b1 ** self.t)
            vhat = self.v[k] / (1 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mhat / (np.sqrt(vhat) + self.eps)
        return params
