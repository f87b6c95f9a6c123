"""Oracle: the small convolutional network of the learned warm start (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

The paper has no network; this is the learned part added to the method: a
stack of 3x3 convolutions on the background-mesh grid (zero padding, stride
1, cross-correlation), ReLU between layers and none after the last, trained
by mean squared error on the unknown DPs.  Layout here: channels first,
x[c, j, i] for cell (i, j) (cell index k = i + n_x j).

The network maps the residual of the current guess p (b - A p), the DP
roles and offsets and the last pressure increment to a correction e of p;
the warm start takes p + s e with s minimising ||b - A (p + s e)||_2.
bf16_round gives the rounding of the bf16 tensor-core path (8 significant
bits, round half to even) so that tests can apply it at the same points.

Every function is the plain definition: the convolution is written as the
sum over the nine kernel offsets of channel-mixing products (an einsum per
offset), and the backward pass is the chain rule of that sum.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 7   # residual, inner, boundary, void, x offset, y offset, last increment
N_CHANNELS = 8   # stored channels (the last is zero)


def bf16_round(x):
    """Round to the nearest bfloat16 (8 significant bits, ties to even)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def rms(v, sel):
    """Root mean square of v over the selected DPs (0 if none)."""
    return float(np.sqrt(np.mean(v[sel] ** 2))) if sel.any() else 0.0


def scales(mesh, r, mask, dprev=None):
    """(s_r, s_d, s_out): rms of the residual and of the last increment over
    non-void DPs, and the unit of the network output: s_d when the last
    increment is nonzero, else s_r l0^2 (the Laplacian scale)."""
    fluid = mask != 0
    s_r = rms(r, fluid)
    s_d = rms(dprev, fluid) if dprev is not None else 0.0
    s_out = s_d if s_d > 0 else (s_r if s_r > 0 else 1.0) * mesh.l0 ** 2
    return s_r, s_d, s_out


def features(mesh, r, mask, pos, dprev=None):
    """Input channels (8, n_y, n_x) of the network: r / s_r, one-hot role
    (inner, boundary, void), the DP offset from its cell centre in units of
    l0, dprev / s_d and a zero channel; every non-role channel is 0 at void
    DPs.  r is the residual b - A p of the guess, dprev the last pressure
    increment.  Returns (x, (s_r, s_d, s_out))."""
    nx, ny = mesh.n[0], mesh.n[1]
    fluid = mask != 0
    s_r, s_d, s_out = scales(mesh, r, mask, dprev)
    i = np.arange(mesh.N) % nx
    j = np.arange(mesh.N) // nx
    cx = mesh.origin[0] + (i + 0.5) * mesh.l0
    cy = mesh.origin[1] + (j + 0.5) * mesh.l0
    zero = np.zeros(mesh.N)
    ch = [np.where(fluid, r / (s_r if s_r > 0 else 1.0), 0.0),
          (mask == -1).astype(float),
          (mask >= 1).astype(float),
          (mask == 0).astype(float),
          np.where(fluid, (pos[0] - cx) / mesh.l0, 0.0),
          np.where(fluid, (pos[1] - cy) / mesh.l0, 0.0),
          zero if s_d == 0 else np.where(fluid, dprev / s_d, 0.0),
          zero]
    return np.stack([c.reshape(ny, nx) for c in ch]), (s_r, s_d, s_out)


def target(p_true, p, unknown, s_out):
    """Training target and loss weight of one solve: the correction the
    guess needed, (p_true - p) / s_out, on the unknown DPs (inner and
    Neumann), and 1 / 0 weights."""
    return np.where(unknown, (p_true - p) / s_out, 0.0), unknown.astype(float)


def conv(x, w, b):
    """y[o, j, i] = b[o] + sum_{c, dj, di} w[o, c, dj, di] x[c, j+dj-1, i+di-1]."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for dj in range(3):
        for di in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, dj, di], xp[:, dj:dj + H, di:di + W])
    return y


def forward(ws, bs, x, rnd=None):
    """Activations [x, a1, ..., y]: ReLU after every layer but the last.
    rnd, if given, is applied to every hidden activation (a1 .. a_{L-1})."""
    acts = [x]
    h = x
    for li, (w, b) in enumerate(zip(ws, bs)):
        z = conv(h, w, b)
        h = np.maximum(z, 0.0) if li < len(ws) - 1 else z
        if rnd is not None and li < len(ws) - 1:
            h = rnd(h)
        acts.append(h)
    return acts


def warm_start(A, b, p, e):
    """p + s e with s = <r, A e> / <A e, A e>, r = b - A p: the point on the
    line through p along e with the smallest residual 2-norm."""
    r = b - A @ p
    Ae = A @ e
    den = float(Ae @ Ae)
    s = float(r @ Ae) / den if den > 0 else 0.0
    return p + s * e, s


def loss(y, target, weight):
    """Mean squared error over the DPs with weight 1 (inner DPs)."""
    n = max(float(weight.sum()), 1.0)
    d = (y - target) * weight
    return float((d * d).sum() / n), 2.0 * d / n


def backward(ws, bs, acts, dy):
    """Gradients (dws, dbs) of a scalar with d(scalar)/d(output) = dy."""
    L = len(ws)
    dws = [None] * L
    dbs = [None] * L
    g = dy
    for li in range(L - 1, -1, -1):
        if li < L - 1:
            g = g * (acts[li + 1] > 0.0)       # ReLU of layer li
        x = acts[li]
        C, H, W = x.shape
        xp = np.zeros((C, H + 2, W + 2))
        xp[:, 1:-1, 1:-1] = x
        dw = np.zeros_like(ws[li])
        for dj in range(3):
            for di in range(3):
                dw[:, :, dj, di] = np.einsum("ohw,chw->oc", g, xp[:, dj:dj + H, di:di + W])
        dws[li] = dw
        dbs[li] = g.sum(axis=(1, 2))
        if li > 0:
            gp = np.zeros((C, H + 2, W + 2))
            for dj in range(3):
                for di in range(3):
                    gp[:, dj:dj + H, di:di + W] += np.einsum("oc,ohw->chw", ws[li][:, :, dj, di], g)
            g = gp[:, 1:-1, 1:-1]
    return dws, dbs


def adam(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) in place; t counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1 - b1) * g
        vv *= b2
        vv += (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
