"""FP64 oracle of the learned surrogate of the photon-field quadrature
(test infrastructure only; imported by ``tests/`` and nothing in the product).

The surrogate is the small MLP 4 -> 64 -> 64 -> 64 -> 2 with SiLU
activations that stands in for the quadrature of the resonant scattering over
the stellar blackbody photon field (Sec. 2.2, Eq. scatteringNdot and the
momentum per scattering).  Its inputs and targets are defined with the
training samples in ``pic1d_oracle.c`` (``orc_sur_point``):

    inputs  f0 = 2 log10(gamma)/G - 1, f1 = 2 s/L - 1,
            f2 = (log10 b - B_MID)/B_HALF, f3 = sign(u)
    outputs y0 ~ <mu~>  (rate-weighted mean aberrated cosine, in [-1, 1])
            y1 ~ max(ln N^, LT) - max(B, LT)  (rate relative to a closed-form
                                              baseline B)

from which the drag and rate follow as ``ln N^ = max(B, LT) + y1`` and
``F^ = gamma b N^ y0``.  LT = -30 clamps the targets; the surrogate is
scored where ln N^ > LE = -20 (below it a rate is negligible).

The tensor-core layers (W2, W3 and the activations h1, h2 that feed them)
are BF16 on the GPU; layers 1 and 4 and the biases are FP32.

Parameters are one flat vector in the layout of the C ABI (PyTorch's
Linear convention, W[out][in]): W1[64][4] b1[64] W2[64][64] b2[64] W3[64][64]
b3[64] W4[2][64] b4[2] -- 8770 values.

Loss over a batch: L = (1/B) sum_b [ m_b (y0 - t1)^2 + (y1 - t2)^2 ].
Optimiser: Adam (Kingma and Ba 2015) with bias correction.

Everything here is plain numpy in FP64, one layer at a time, written to be
checked by eye; the pins in ``tests/test_surrogate_oracle.py`` tie it to
finite differences, to PyTorch autograd and ``torch.optim.Adam`` (independent
library routines) and to invariances of the network.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = ((64, 4), (64, 64), (64, 64), (2, 64))   # (out, in) per layer
LT = -30.0          # clamp of the rate targets (ln N^)
LE = -20.0          # floor of the scored region (ln N^)
B_MID, B_HALF = -1.25, 2.75
BASE_MIX = (0.9, 0.1)  # weights of N^_rad(mu_s) and N^_rad(mu_edge) in the baseline


def offsets():
    """[(W offset, b offset)] per layer and the total parameter count."""
    out, k = [], 0
    for o, i in SIZES:
        out.append((k, k + o * i))
        k += o * i + o
    return out, k


OFFSETS, N_PARAMS = offsets()


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    Ws, bs = [], []
    for (o, i), (kw, kb) in zip(SIZES, OFFSETS):
        Ws.append(theta[kw:kw + o * i].reshape(o, i))
        bs.append(theta[kb:kb + o])
    return Ws, bs


def pack(Ws, bs):
    theta = np.zeros(N_PARAMS)
    for (o, i), (kw, kb), W, b in zip(SIZES, OFFSETS, Ws, bs):
        theta[kw:kw + o * i] = np.asarray(W).reshape(-1)
        theta[kb:kb + o] = b
    return theta


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X):
    """X: B x 4 inputs -> (Y: B x 2, cache of pre-activations and activations)."""
    Ws, bs = unpack(theta)
    h = np.asarray(X, dtype=np.float64)
    hs, zs = [h], []
    for layer in range(4):
        z = h @ Ws[layer].T + bs[layer]
        zs.append(z)
        h = silu(z) if layer < 3 else z
        hs.append(h)
    return h, (hs, zs)


def loss_grad(theta, X, T1, T2, M):
    """Mean loss over the batch and its gradient (flat, N_PARAMS)."""
    Ws, _ = unpack(theta)
    Y, (hs, zs) = forward(theta, X)
    B = Y.shape[0]
    r0 = (Y[:, 0] - T1) * M
    r1 = Y[:, 1] - T2
    loss = float(np.sum(r0 * (Y[:, 0] - T1) + r1 * r1) / B)
    dY = np.stack([2.0 * r0, 2.0 * r1], axis=1) / B
    gW, gb = [None] * 4, [None] * 4
    dz = dY
    for layer in range(3, -1, -1):
        gW[layer] = dz.T @ hs[layer]
        gb[layer] = dz.sum(axis=0)
        if layer > 0:
            dh = dz @ Ws[layer]
            dz = dh * dsilu(zs[layer - 1])
    return loss, pack(gW, gb)


def jvp_log10g(theta, X):
    """Outputs and their derivatives with respect to f0 (forward-mode)."""
    Ws, bs = unpack(theta)
    h = np.asarray(X, dtype=np.float64)
    hd = np.zeros_like(h)
    hd[:, 0] = 1.0
    for layer in range(4):
        z = h @ Ws[layer].T + bs[layer]
        zd = hd @ Ws[layer].T
        if layer < 3:
            h, hd = silu(z), dsilu(z) * zd
        else:
            h, hd = z, zd
    return h, hd


class Adam:
    """Adam with bias correction (Kingma and Ba 2015, Algorithm 1)."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def features(log10g, s_frac, b, u, log10g_max=8.0):
    """The network's inputs for given points (arrays)."""
    return np.stack([2.0 * np.asarray(log10g) / log10g_max - 1.0, 2.0 * np.asarray(s_frac) - 1.0,
                     (np.log10(b) - B_MID) / B_HALF, np.where(np.asarray(u) < 0.0, -1.0, 1.0)], axis=1)


def reconstruct(Y, base, gamma, b):
    """(F^, ln N^) from the outputs and the baseline B at each point."""
    lnN = np.maximum(base, LT) + Y[:, 1]
    F = gamma * b * np.exp(lnN) * Y[:, 0]
    return F, lnN


def drag_error(F_nn, F_q, F_abs):
    """The surrogate's drag error |F_nn - F_q| / (|F_q| + F_abs)."""
    return np.abs(F_nn - F_q) / (np.abs(F_q) + F_abs)


def bf16(x):
    """Round FP64 values to the nearest BF16 (ties to even), as FP64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_tensor_layers(theta):
    """The parameters as the GPU uses them: W2 and W3 rounded to BF16."""
    th = np.array(theta, dtype=np.float64)
    for layer in (1, 2):
        kw, kb = OFFSETS[layer]
        th[kw:kb] = bf16(th[kw:kb])
    return th


def init_uniform_bound(layer):
    """PyTorch Linear's default init bound 1/sqrt(fan_in) for a layer."""
    return 1.0 / math.sqrt(SIZES[layer][1])
