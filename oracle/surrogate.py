"""FP64 CPU oracle of the field surrogate (test infrastructure).

The surrogate predicts the far part of the pedestrian field from occupancy and
heading channels with a 4-layer convolutional network:

    A1 = relu(conv5x5(X; W1) + b1)     3 -> 32 channels
    A2 = relu(conv3x3(A1; W2) + b2)   32 -> 32
    A3 = relu(conv3x3(A2; W3) + b3)   32 -> 32
    Y  =      conv3x3(A3; W4) + b4    32 -> 1

with "valid" cross-correlations, conv(X; W)[o, y, x] = sum_{c, i, j}
W[o, c, i, j] X[c, y + i, x + j], and the loss L = 0.5 * mean((Y - T)^2).
Inputs X are per coarse cell of s x s su: [number of pedestrians, sum of
heading x, sum of heading y] / s^2.  Targets T are the cell averages of the
exact field minus its near part (contributions within Chebyshev radius rn,
optionally tapered to zero between Euclidean distances r_in and rn so that
what is left to the network is smooth), divided by a fixed scale.  Predictions are returned to su by bilinear
interpolation between coarse cell centres.

Plain NumPy: every convolution is a sum over kernel offsets of channel
contractions (np.einsum), written out.  Shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

LAYERS = [(3, 32, 5), (32, 32, 3), (32, 32, 3), (32, 1, 3)]  # (Cin, Cout, k)
HALO = sum((k - 1) // 2 for _, _, k in LAYERS)                 # 5 cells of context


def init_params(seed: int = 0):
    """Seeded random initial weights (drawn by the shared input generator)."""
    import scenegen
    ps = scenegen.surrogate_init(seed)
    assert [(W.shape[1], W.shape[0], W.shape[2]) for W, _ in ps] == LAYERS
    return ps


def conv_valid(X, W, b):
    """X [C, H, Wd], W [O, C, k, k], b [O] -> [O, H-k+1, Wd-k+1] (cross-correlation)."""
    O, C, k, _ = W.shape
    Ho, Wo = X.shape[1] - k + 1, X.shape[2] - k + 1
    Z = np.zeros((O, Ho, Wo))
    for i in range(k):
        for j in range(k):
            Z += np.einsum("oc,chw->ohw", W[:, :, i, j], X[:, i:i + Ho, j:j + Wo])
    return Z + b[:, None, None]


def forward(params, X):
    """Returns (Y, cache) for one image X [3, H, W]."""
    acts = [X]
    zs = []
    A = X
    for li, (W, b) in enumerate(params):
        Z = conv_valid(A, W, b)
        zs.append(Z)
        A = Z if li == len(params) - 1 else np.maximum(Z, 0.0)
        acts.append(A)
    return A[0], (acts, zs)


def loss_and_grad(params, X, T):
    """0.5 * mean((Y - T)^2) and its gradients with respect to every W, b."""
    Y, (acts, zs) = forward(params, X)
    n = Y.size
    L = 0.5 * np.sum((Y - T) ** 2) / n
    dA = ((Y - T) / n)[None]
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        Z = zs[li]
        dZ = dA if li == len(params) - 1 else dA * (Z > 0)
        Ain = acts[li]
        O, C, k, _ = W.shape
        Ho, Wo = dZ.shape[1], dZ.shape[2]
        dW = np.zeros_like(W)
        for i in range(k):
            for j in range(k):
                dW[:, :, i, j] = np.einsum("ohw,chw->oc", dZ, Ain[:, i:i + Ho, j:j + Wo])
        db = dZ.sum(axis=(1, 2))
        dAin = np.zeros_like(Ain)
        for i in range(k):
            for j in range(k):
                dAin[:, i:i + Ho, j:j + Wo] += np.einsum("oc,ohw->chw", W[:, :, i, j], dZ)
        grads[li] = (dW, db)
        dA = dAin
    return L, grads


def taper_weight(d, r_in, rn):
    """Weight of the near part at Euclidean distance d: 1 up to r_in, a raised
    cosine down to 0 at rn, 0 beyond; no taper (1 on the whole Chebyshev
    window) when r_in >= rn."""
    if r_in >= rn:
        return 1.0
    if d <= r_in:
        return 1.0
    if d >= rn:
        return 0.0
    return 0.5 * (1.0 + np.cos(np.pi * (d - r_in) / (rn - r_in)))


def tapered_near_field(W, H, xy, heading, rn, r_in, kP, aP, gamma, periodic_x=0, periodic_y=0,
                       alive=None):
    """[H, W]: sum over pedestrians of w(|delta|) K_P(delta; h) over the
    Chebyshev window 0 < |delta|_inf <= rn, delta = su - pedestrian, with
    K_P(delta; h) = kP d^aP (1 + gamma h.delta / d) (h the unit heading, zero
    for heading 0) and w = taper_weight.  Out-of-lattice su are dropped, or
    wrapped in periodic dimensions."""
    from math import hypot, sqrt
    dirs = [(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    F = np.zeros((H, W))
    for i in range(len(xy)):
        if alive is not None and not alive[i]:
            continue
        px, py = int(xy[i][0]), int(xy[i][1])
        hdx, hdy = dirs[int(heading[i])]
        n = sqrt(hdx * hdx + hdy * hdy)
        hx, hy = (hdx / n, hdy / n) if n else (0.0, 0.0)
        for dy in range(-rn, rn + 1):
            for dx in range(-rn, rn + 1):
                if dx == 0 and dy == 0:
                    continue
                x, y = px + dx, py + dy
                if periodic_x:
                    x %= W
                elif not 0 <= x < W:
                    continue
                if periodic_y:
                    y %= H
                elif not 0 <= y < H:
                    continue
                d = hypot(dx, dy)
                K = kP * d ** aP * (1.0 + gamma * (hx * dx + hy * dy) / d)
                F[y, x] += taper_weight(d, r_in, rn) * K
    return F


def coarse_channels(W, H, s, xy, heading, alive=None):
    """[3, H/s, W/s]: pedestrian count, sum of heading x, sum of heading y per
    s x s cell, divided by s^2."""
    from math import sqrt
    dirs = [(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]
    Hc, Wc = H // s, W // s
    X = np.zeros((3, Hc, Wc))
    for i in range(len(xy)):
        if alive is not None and not alive[i]:
            continue
        x, y = int(xy[i][0]), int(xy[i][1])
        dx, dy = dirs[int(heading[i])]
        n = sqrt(dx * dx + dy * dy)
        hx, hy = (dx / n, dy / n) if n else (0.0, 0.0)
        X[0, y // s, x // s] += 1.0
        X[1, y // s, x // s] += hx
        X[2, y // s, x // s] += hy
    return X / (s * s)


def cell_average(F, s):
    H, W = F.shape
    return F.reshape(H // s, s, W // s, s).mean(axis=(1, 3))


def upsample(Yc, s, periodic=True):
    """Bilinear interpolation from coarse cell centres to every su."""
    Hc, Wc = Yc.shape
    H, W = Hc * s, Wc * s
    out = np.zeros((H, W))
    for y in range(H):
        fy = (y + 0.5) / s - 0.5
        y0 = int(np.floor(fy))
        ty = fy - y0
        for x in range(W):
            fx = (x + 0.5) / s - 0.5
            x0 = int(np.floor(fx))
            tx = fx - x0
            v = 0.0
            for (yy, wy) in ((y0, 1 - ty), (y0 + 1, ty)):
                for (xx, wx) in ((x0, 1 - tx), (x0 + 1, tx)):
                    if periodic:
                        yy2, xx2 = yy % Hc, xx % Wc
                    else:
                        yy2, xx2 = min(max(yy, 0), Hc - 1), min(max(xx, 0), Wc - 1)
                    v += wy * wx * Yc[yy2, xx2]
            out[y, x] = v
    return out
