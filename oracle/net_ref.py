"""CPU reference of the learned proposal network (FP64 numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests use it to
check the GPU rasteriser, convolutions, loss and gradients.  It shares no
code with the CUDA path.

Definitions (the proposal of the build; the paper has no network):
  * map: the 12 x 9 m field rasterised at 0.2 m, H = 46 rows (y) by W = 61
    columns (x); pixel (y, x) sits at (-6 + 0.2 x, -4.5 + 0.2 y);
  * 8 input channels per pixel c, with opponents o_j, velocities u_j, ball b,
    diagonal diag = 15 m:
      0  sum_j g(|c - o_j|)                 g(r) = exp(-r^2 / (2 * 0.3^2))
      1  sum_j (u_jx / vmax) g(|c - o_j|)
      2  sum_j (u_jy / vmax) g(|c - o_j|)
      3  exp(-|c - b|^2 / (2 * 0.5^2))
      4  |c - b| / diag
      5  min_j |c - o_j| / diag  (1 without opponents)
      6  x / (L / 2)
      7  y / (W / 2)
    rounded to bfloat16 (the network's input precision);
  * layers: four 3x3 convolutions, stride 1, zero padding 1,
    8 -> 32 -> 32 -> 32 -> 1 channels, ReLU after the first three;
    activations rounded to bfloat16 after each hidden layer, the output kept
    in float32 precision (here float64);
  * loss: mean over pixels of (out - label)^2.
Weights: per layer W[ky][kx][cout][cin] (ky, kx = 0..2 for offsets -1..1)
then bias[cout], flattened in layer order (``unflatten``).
"""
from __future__ import annotations

import numpy as np

H, W = 46, 61
CIN = 8
LAYERS = [(8, 32), (32, 32), (32, 32), (32, 1)]
SIGMA_OPP, SIGMA_BALL, DIAG = 0.3, 0.5, 15.0


def n_params() -> int:
    return sum(9 * co * ci + co for ci, co in LAYERS)


def bf16(x):
    """Round float32-representable values to bfloat16 (nearest even)."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out).astype(np.float64)


def unflatten(w):
    """Flat parameter vector -> [(W[3,3,co,ci], b[co]), ...]."""
    w = np.asarray(w, np.float64)
    out, k = [], 0
    for ci, co in LAYERS:
        n = 9 * co * ci
        out.append((w[k:k + n].reshape(3, 3, co, ci), w[k + n:k + n + co]))
        k += n + co
    assert k == w.size
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([Wl.reshape(-1), bl])
                           for Wl, bl in layers])


def raster(state: dict) -> np.ndarray:
    """Input map (H, W, 8) of one state (dict with ball, opp_pos, opp_vel,
    n_opp, vmax, field_len, field_wid), bfloat16-rounded."""
    ys, xs = np.mgrid[0:H, 0:W]
    cx = -6.0 + 0.2 * xs
    cy = -4.5 + 0.2 * ys
    n = int(state["n_opp"])
    vmax = float(state["vmax"])
    out = np.zeros((H, W, 8))
    dmin = np.full((H, W), np.inf)
    for j in range(n):
        ox, oy = (float(v) for v in state["opp_pos"][j])
        ux, uy = (float(v) for v in state["opp_vel"][j])
        r2 = (cx - ox) ** 2 + (cy - oy) ** 2
        g = np.exp(-r2 / (2 * SIGMA_OPP ** 2))
        out[..., 0] += g
        out[..., 1] += ux / vmax * g
        out[..., 2] += uy / vmax * g
        dmin = np.minimum(dmin, np.sqrt(r2))
    bx, by = (float(v) for v in state["ball"])
    rb2 = (cx - bx) ** 2 + (cy - by) ** 2
    out[..., 3] = np.exp(-rb2 / (2 * SIGMA_BALL ** 2))
    out[..., 4] = np.sqrt(rb2) / DIAG
    out[..., 5] = np.where(np.isfinite(dmin), dmin / DIAG, 1.0)
    out[..., 6] = cx / (float(state["field_len"]) / 2)
    out[..., 7] = cy / (float(state["field_wid"]) / 2)
    return bf16(out)


def conv(x, Wl, bl):
    """3x3 'same' convolution of x (B, H, W, ci) with W[3,3,co,ci]."""
    B, h, w, ci = x.shape
    xp = np.zeros((B, h + 2, w + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    out = np.broadcast_to(bl, (B, h, w, Wl.shape[2])).copy()
    for ky in range(3):
        for kx in range(3):
            out += xp[:, ky:ky + h, kx:kx + w] @ Wl[ky, kx].T
    return out


def conv_grad_input(g, Wl):
    """d(loss)/dx of conv given g = d(loss)/d(out), (B, H, W, co)."""
    B, h, w, co = g.shape
    gp = np.zeros((B, h + 2, w + 2, co))
    gp[:, 1:-1, 1:-1] = g
    dx = np.zeros((B, h, w, Wl.shape[3]))
    for ky in range(3):
        for kx in range(3):
            # out(y) uses x(y + ky - 1): x(y) receives g(y - ky + 1)
            dx += gp[:, 2 - ky:2 - ky + h, 2 - kx:2 - kx + w] @ Wl[ky, kx]
    return dx


def conv_grad_weight(g, x):
    """d(loss)/dW[3,3,co,ci] and d(loss)/db of conv."""
    B, h, w, ci = x.shape
    co = g.shape[3]
    xp = np.zeros((B, h + 2, w + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dW = np.zeros((3, 3, co, ci))
    G = g.reshape(-1, co)
    for ky in range(3):
        for kx in range(3):
            dW[ky, kx] = G.T @ xp[:, ky:ky + h, kx:kx + w].reshape(-1, ci)
    return dW, G.sum(axis=0)


def forward(x, layers, round_acts=True):
    """Activations [x, a1, a2, a3] and the output (B, H, W)."""
    acts = [x]
    a = x
    for i, (Wl, bl) in enumerate(layers):
        z = conv(a, Wl, bl)
        if i < len(layers) - 1:
            a = np.maximum(z, 0.0)
            if round_acts:
                a = bf16(a)
            acts.append(a)
        else:
            out = z[..., 0]
    return acts, out


def loss_and_grads(x, labels, layers, round_grads=True):
    """Mean squared error and its gradients (list of (dW, db)), with the
    bfloat16 rounding of the GPU path (activations and the gradients that
    feed the tensor-core products) when round_grads is set."""
    acts, out = forward(x, layers, round_acts=round_grads)
    N = out.size
    diff = out - labels
    loss = float(np.mean(diff ** 2))
    g = (2.0 / N * diff)[..., None]
    if round_grads:
        g = bf16(g)
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        Wl, _ = layers[i]
        grads[i] = conv_grad_weight(g, acts[i])
        if i > 0:
            dx = conv_grad_input(g, Wl) * (acts[i] > 0)
            g = bf16(dx) if round_grads else dx
    return loss, grads
