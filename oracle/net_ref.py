"""CPU reference of the learned proposal network (FP64 numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests use it to
check the GPU rasteriser, convolutions, loss and gradients.  It shares no
code with the CUDA path.

Definitions (the learned proposal; the paper has no network):
  * map: the 12 x 9 m field rasterised at 0.2 m, H = 46 rows (y) by W = 61
    columns (x); pixel (y, x) is centred at c = ((x - 30) / 5, (y - 22.5) / 5);
  * 8 input channels per pixel, with opponents o_j, ball b, goal centre
    g = (L / 2, 0), diag = sqrt(L^2 + W^2), and the cell's four sub-points
    q = c + (+-0.05, +-0.05) (clamped into the field):
      0  sum_j exp(-|c - o_j|^2 / (2 * 0.3^2))
      1  the coarse score of the cell: the largest over the sub-points of
         the value function (Sec. 4.3: w_angle theta / pi - w_dist
         |g - q| / diag + w_margin min(m, cap)) where some kick speed is
         feasible (m > tau_safe, |q - b| >= min_pass_dist), -1.2 elsewhere
      2  |c - b| / diag
      3  the margin of the cell: the largest over the sub-points and the
         feature kick speeds of the safety margin of the pass (Sec. 4.2;
         the oracle's margin with K = 16 pass-line samples), clamped to
         [-2, 1]
      4  the largest open shot angle over the sub-points (Sec. 4.3) / pi
      5  |g - c| / diag
      6  c_x / (L / 2),  7  c_y / (W / 2)
    rounded to bfloat16 (the network's input precision);
  * layers: four 3x3 convolutions, stride 1, zero padding 1,
    8 -> 32 -> 32 -> 32 -> 1 channels, ReLU after the first three;
    activations rounded to bfloat16 after each hidden layer; the output is
    the last convolution plus input channel 1 (the coarse score: the
    network learns a correction to it), kept in float32 precision (here
    float64);
  * loss: mean over pixels of w (out - label)^2, w = 1 where the label or
    the output comes within top_band of the state's best label, low_weight
    elsewhere, times under_weight where out < label (w held constant in the
    gradient); top_band = inf and under_weight = 1 is the plain mean
    squared error.
Weights: per layer W[ky][kx][cout][cin] (ky, kx = 0..2 for offsets -1..1)
then bias[cout], flattened in layer order (``unflatten``).
"""
from __future__ import annotations

import numpy as np

H, W = 46, 61
CIN = 8
LAYERS = [(8, 32), (32, 32), (32, 32), (32, 1)]
SIGMA_OPP = 0.3


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


FEATURE_SPEEDS = (2.0, 3.5, 5.0, 6.5)
FEATURE_K = 16
SCORE_FLOOR = -1.2
SUB_OFF = 0.05
# the library's default value-function parameters
FEATURE_PARAMS = {"w_angle": 1.0, "w_dist": 1.0, "w_margin": 1.0,
                  "margin_cap": 1.0, "tau_safe": 0.0, "robot_radius": 0.09,
                  "reach_radius": 0.0, "min_pass_dist": 0.0}


def _oracle_state(state: dict, K: int):
    from . import State
    n = int(state["n_opp"])
    opp = np.concatenate(
        [np.asarray(state["opp_pos"][:n], np.float64).reshape(n, 2),
         np.asarray(state["opp_vel"][:n], np.float64).reshape(n, 2)], axis=1)
    sc = {"ball_x": state["ball"][0], "ball_y": state["ball"][1]}
    for k in ("ball_decel", "vmax", "amax", "field_len", "field_wid",
              "goal_width"):
        sc[k] = state[k]
    return State(sc, opp, K)


def pixel_centres():
    ys, xs = np.mgrid[0:H, 0:W]
    return (xs - 30.0) / 5.0, (ys - 22.5) / 5.0


def raster(state: dict, speeds=FEATURE_SPEEDS, params=None,
           with_band=False):
    """Input map (H, W, 8) of one state (dict with ball, n_opp, opp_pos,
    opp_vel, ball_decel, vmax, amax, field_len, field_wid, goal_width),
    bfloat16-rounded.  with_band: also the (H, W) distance of the cell's
    feasibility decisions from their threshold, min over the sub-points
    and speeds of |margin - tau_safe|."""
    from . import default
    prm = dict(FEATURE_PARAMS, **(params or {}))
    orc = default()
    st = _oracle_state(state, FEATURE_K)
    cx, cy = pixel_centres()
    L, Wd = float(state["field_len"]), float(state["field_wid"])
    diag = np.sqrt(L * L + Wd * Wd)
    bx, by = (float(v) for v in state["ball"])
    out = np.zeros((H, W, 8))
    band = np.full((H, W), np.inf)
    for j in range(int(state["n_opp"])):
        ox, oy = (float(v) for v in state["opp_pos"][j])
        out[..., 0] += np.exp(-((cx - ox) ** 2 + (cy - oy) ** 2)
                              / (2 * SIGMA_OPP ** 2))
    for y in range(H):
        for x in range(W):
            sbest, mbest, tbest = SCORE_FLOOR, -np.inf, 0.0
            for sub in range(4):
                qx = min(max(cx[y, x] + (SUB_OFF if sub & 1 else -SUB_OFF),
                             -L / 2), L / 2)
                qy = min(max(cy[y, x] + (SUB_OFF if sub & 2 else -SUB_OFF),
                             -Wd / 2), Wd / 2)
                ms = [orc.margin(st, (qx, qy), v, prm["reach_radius"])[0]
                      for v in speeds]
                m = max(ms)
                band[y, x] = min([band[y, x]] + [abs(mm - prm["tau_safe"])
                                                 for mm in ms])
                th = orc.shot_angle(st, (qx, qy), prm["robot_radius"]) / np.pi
                dg = np.hypot(L / 2 - qx, qy) / diag
                D = np.hypot(qx - bx, qy - by)
                if m > prm["tau_safe"] and D >= prm["min_pass_dist"]:
                    sc = (prm["w_angle"] * th - prm["w_dist"] * dg
                          + prm["w_margin"] * min(m, prm["margin_cap"]))
                    sbest = max(sbest, sc)
                mbest, tbest = max(mbest, m), max(tbest, th)
            out[y, x, 1] = sbest
            out[y, x, 3] = min(max(mbest, -2.0), 1.0)
            out[y, x, 4] = tbest
    out[..., 2] = np.hypot(cx - bx, cy - by) / diag
    out[..., 5] = np.hypot(L / 2 - cx, cy) / diag
    out[..., 6] = cx / (L / 2)
    out[..., 7] = cy / (Wd / 2)
    return (bf16(out), band) if with_band else bf16(out)


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
            out = z[..., 0] + x[..., 1]
    return acts, out


def loss_weights(out, labels, top_band=np.inf, low_weight=1.0,
                 under_weight=1.0):
    """Per-pixel weights of the loss (B, H, W)."""
    cut = labels.reshape(labels.shape[0], -1).max(axis=1) - top_band
    cut = cut[:, None, None]
    w = np.where((labels >= cut) | (out >= cut), 1.0, low_weight)
    return w * np.where(out < labels, under_weight, 1.0)


def loss_and_grads(x, labels, layers, round_grads=True, top_band=np.inf,
                   low_weight=1.0, under_weight=1.0):
    """The loss and its gradients (list of (dW, db)), with the bfloat16
    rounding of the GPU path (activations and the gradients that feed the
    tensor-core products) when round_grads is set."""
    acts, out = forward(x, layers, round_acts=round_grads)
    N = out.size
    diff = out - labels
    w = loss_weights(out, labels, top_band, low_weight, under_weight)
    loss = float(np.mean(w * diff ** 2))
    g = (2.0 / N * w * diff)[..., None]
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
