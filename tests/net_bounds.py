"""Element-wise bounds on the proposal network's GPU arithmetic against the
FP64 reference (oracle/net_ref.py), by interval propagation.

What the GPU does, layer by layer, on the same input map and weights:
  * convolutions: products of bfloat16 operands (exact in float32), summed
    in float32 by the tensor cores in an order of their own, plus the bias
    (and, at the output, the coarse-score channel) in float32;
  * hidden activations: ReLU, then rounded to bfloat16 (nearest even);
  * loss gradient 2 w (out - label) / N in float32, rounded to bfloat16;
  * input gradients: a float32 sum of bfloat16 products, masked where the
    layer's input activation is 0, rounded to bfloat16;
  * weight and bias gradients: float32 sums over every pixel of the batch.
The reference does the same in FP64 with the same bfloat16 roundings.

Every reference quantity r is carried with a bound E on |gpu - r|:
  * a float32 sum of n terms t_i: |error| <= n 2^-23 sum |t_i| (each
    addition off by at most 2^-23 of a partial sum, which covers
    round-to-nearest and truncating accumulators alike), and operands that
    are off by E contribute sum |W| E;
  * a bfloat16 rounding of a value known to lie in [lo, hi]: the GPU's
    result lies in [bf16(lo), bf16(hi)] because rounding is monotone, so
    E = max(bf16(hi) - r, r - bf16(lo)) -- zero unless the interval
    reaches a rounding boundary, one bfloat16 step when it does;
  * a ReLU mask: decided where the activation's interval stays away from 0;
    elsewhere the gradient may pass or be dropped, and both are allowed;
  * the loss weights: every weight the GPU's float32 comparisons could pick
    for an output in its interval.
The bounds are rigorous for the arithmetic above.  They are tight where
little can flip: on an integer-valued network (integer input maps, weights
and biases, pre-activations within 256) the forward pass is exact on both
sides (forward_bounds(exact=True) asserts why) and only the backward
pass's roundings remain, so a kernel that gets one tap, one channel or one
sign wrong is off by whole terms, far beyond the bounds.  With real-valued
weights every hidden activation may flip by a bfloat16 step and the flips
cascade through the layers: the bounds stay valid but grow loose.
"""
from __future__ import annotations

import numpy as np

from oracle import net_ref

U2 = 2.0 ** -23          # float32 error per addition, relative to the sum
EPS_LOSS = 8 * 2.0 ** -24  # float32 roundings of the loss gradient's factors


def bits_to_float(bits):
    return (np.asarray(bits).astype(np.uint32) << 16).view(np.float32) \
        .astype(np.float64)


def layers_as_gpu(w):
    """The network as the GPU holds it: bfloat16 weights, float32 biases."""
    return [(net_ref.bf16(Wl), np.asarray(bl, np.float32).astype(np.float64))
            for Wl, bl in net_ref.unflatten(w)]


def _round_interval(ref, lo, hi):
    """Bound of |bf16(x) - ref| for x anywhere in [lo, hi]."""
    return np.maximum(net_ref.bf16(hi) - ref, ref - net_ref.bf16(lo))


def _is_int(a):
    return np.array_equal(a, np.round(a))


def forward_bounds(x, layers, exact=False):
    """Reference activations, output and their bounds.

    Returns (acts, out, E_acts, E_out): acts = [x, a1, a2, a3] as
    net_ref.forward computes them, E_acts their element-wise bounds (E for
    x is 0: both sides read the same map), out (B, H, W) and E_out.

    exact: the input map, weights and biases are integers and every sum of
    absolute terms stays below 2^24, so every float32 partial sum is an
    integer the format holds exactly, and every pre-activation is an integer
    of magnitude at most 256, which bfloat16 holds exactly: the GPU's
    forward pass equals the reference's, E = 0 (the preconditions are
    asserted)."""
    acts, out = net_ref.forward(x, layers)
    E = [np.zeros_like(x)]
    if exact:
        assert _is_int(x)
    for i, (Wl, bl) in enumerate(layers):
        a, Ea = acts[i], E[i]
        absW = np.abs(Wl)
        n = 9 * Wl.shape[3] + 2
        z = net_ref.conv(a, Wl, bl)
        prop = net_ref.conv(Ea, absW, np.zeros_like(bl))
        mag = net_ref.conv(np.abs(a) + Ea, absW, np.abs(bl))
        if exact:
            assert _is_int(Wl) and _is_int(bl) and _is_int(z)
            assert mag.max() + np.abs(x[..., 1]).max() < 2.0 ** 24
            if i < len(layers) - 1:
                assert np.abs(z).max() <= 256
                E.append(np.zeros_like(z))
            else:
                E_out = np.zeros_like(out)
            continue
        if i < len(layers) - 1:
            dz = prop + n * U2 * mag
            lo = np.maximum(z - dz, 0.0)
            hi = np.maximum(z + dz, 0.0)
            E.append(_round_interval(acts[i + 1], lo, hi))
        else:
            skip = np.abs(x[..., 1])
            E_out = prop[..., 0] + (n + 1) * U2 * (mag[..., 0] + skip)
    return acts, out, E, E_out


def _weight_choices(out, E_out, labels, top_band, low_weight, under_weight):
    """Smallest and largest loss weight the GPU may apply per pixel."""
    B = labels.shape[0]
    smax = labels.reshape(B, -1).max(axis=1)[:, None, None]
    cut64 = smax - top_band
    # the GPU's cut: one float32 subtraction (top_band = inf: every pixel
    # is within the band on both sides)
    if np.isinf(top_band):
        cut32 = np.full_like(cut64, -np.inf)
    else:
        cut32 = (np.float32(smax) - np.float32(top_band)).astype(np.float64)
    clo, chi = np.minimum(cut64, cut32), np.maximum(cut64, cut32)
    olo, ohi = out - E_out, out + E_out
    in_possible = (labels >= clo) | (ohi >= clo)
    out_possible = (labels < chi) & (olo < chi)
    under_possible = olo < labels
    over_possible = ohi >= labels
    cand = []
    for a_ok, wa in ((in_possible, 1.0), (out_possible, low_weight)):
        for b_ok, wb in ((under_possible, under_weight), (over_possible, 1.0)):
            cand.append(np.where(a_ok & b_ok, wa * wb, np.nan))
    c = np.stack(cand)
    return np.nanmin(c, axis=0), np.nanmax(c, axis=0)


def gradient_bounds(x, labels, layers, top_band=np.inf, low_weight=1.0,
                    under_weight=1.0, exact=False):
    """Reference loss, weight and bias gradients and their element-wise
    bounds: (loss, [(dW, db)], [(E_dW, E_db)]); exact as forward_bounds."""
    acts, out, E_acts, E_out = forward_bounds(x, layers, exact)
    N = out.size
    loss, grads = net_ref.loss_and_grads(
        x, labels, layers, round_grads=True, top_band=top_band,
        low_weight=low_weight, under_weight=under_weight)
    # the loss gradient of the reference, and the GPU's range
    w_ref = net_ref.loss_weights(out, labels, top_band, low_weight,
                                 under_weight)
    g = net_ref.bf16(2.0 / N * w_ref * (out - labels))[..., None]
    wlo, whi = _weight_choices(out, E_out, labels, top_band, low_weight,
                               under_weight)
    dlo, dhi = out - E_out - labels, out + E_out - labels
    cands = np.stack([2.0 / N * wv * dv for wv in (wlo, whi)
                      for dv in (dlo, dhi)])
    glo, ghi = cands.min(axis=0), cands.max(axis=0)
    glo = glo - EPS_LOSS * np.abs(glo)
    ghi = ghi + EPS_LOSS * np.abs(ghi)
    Eg = _round_interval(g[..., 0], glo, ghi)[..., None]
    bounds = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        Wl, _ = layers[i]
        a, Ea = acts[i], E_acts[i]
        G, X = np.abs(g) + Eg, np.abs(a) + Ea
        n_pix = g.shape[0] * g.shape[1] * g.shape[2]
        full_W, full_b = net_ref.conv_grad_weight(G, X)
        ref_W, ref_b = net_ref.conv_grad_weight(np.abs(g), np.abs(a))
        E_W = (full_W - ref_W) + n_pix * U2 * full_W
        E_b = (full_b - ref_b) + n_pix * U2 * full_b
        bounds[i] = (E_W, E_b)
        if i == 0:
            break
        # the input gradient of layer i, masked by a_i > 0, in bfloat16
        absW = np.abs(Wl)
        n = 9 * Wl.shape[2]
        dx = net_ref.conv_grad_input(g, Wl)
        ddx = (net_ref.conv_grad_input(Eg, absW)
               + n * U2 * net_ref.conv_grad_input(G, absW))
        lo, hi = dx - ddx, dx + ddx
        sure_on = a - Ea > 0
        sure_off = (a == 0) & (Ea == 0)
        maybe = ~(sure_on | sure_off)
        lo = np.where(sure_on, lo, np.where(sure_off, 0.0, np.minimum(lo, 0.0)))
        hi = np.where(sure_on, hi, np.where(sure_off, 0.0, np.maximum(hi, 0.0)))
        g_new = net_ref.bf16(dx * (a > 0))
        Eg = _round_interval(g_new, lo, hi)
        assert np.all(np.isfinite(Eg)) and not np.any(maybe & ~np.isfinite(dx))
        g = g_new
    return loss, grads, bounds
