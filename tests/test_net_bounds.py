"""The element-wise bounds of tests/net_bounds.py, checked on the CPU.

The network's float32 arithmetic is emulated here in numpy -- float32
convolutions (each tap a float32 matrix product, summed in float32 in tap
order: an order of additions unlike the reference's), bfloat16 roundings
where the GPU rounds, float32 loss gradient -- and every emulated
activation, output and gradient must fall inside the bounds, for a
real-valued network and for an integer-valued one (where they are tight).
Planted mistakes on the integer network (a mirrored tap in a weight
gradient, two swapped output channels in an input gradient, a missing ReLU
mask, a flipped sign) must fall outside.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import net_ref
from paper_1909_07717_gb300 import synth
from tests import net_bounds

F32 = np.float32


def conv32(x, Wl, bl):
    """3x3 'same' convolution in float32, taps summed in order."""
    B, h, w, ci = x.shape
    xp = np.zeros((B, h + 2, w + 2, ci), F32)
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((B, h, w, Wl.shape[2]), F32)
    for ky in range(3):
        for kx in range(3):
            out = out + (xp[:, ky:ky + h, kx:kx + w] @ Wl[ky, kx].T.astype(F32))
    return out + bl.astype(F32)


def grad_input32(g, Wl):
    B, h, w, co = g.shape
    gp = np.zeros((B, h + 2, w + 2, co), F32)
    gp[:, 1:-1, 1:-1] = g
    dx = np.zeros((B, h, w, Wl.shape[3]), F32)
    for ky in range(3):
        for kx in range(3):
            dx = dx + gp[:, 2 - ky:2 - ky + h, 2 - kx:2 - kx + w] @ \
                Wl[ky, kx].astype(F32)
    return dx


def grad_weight32(g, x, wrong_tap=None):
    B, h, w, ci = x.shape
    co = g.shape[3]
    xp = np.zeros((B, h + 2, w + 2, ci), F32)
    xp[:, 1:-1, 1:-1] = x
    dW = np.zeros((3, 3, co, ci), F32)
    G = g.reshape(-1, co).astype(F32)
    for ky in range(3):
        for kx in range(3):
            sy, sx = (ky, kx) if (ky, kx) != wrong_tap else (2 - ky, 2 - kx)
            dW[ky, kx] = G.T @ xp[:, sy:sy + h, sx:sx + w].reshape(-1, ci)
    return dW, G.sum(axis=0, dtype=F32)


def emulate(x, labels, layers, top_band=np.inf, low=1.0, under=1.0,
            mistake=None):
    """The GPU's arithmetic in float32: (output, activations, grads)."""
    acts = [x.astype(F32)]
    a = acts[0]
    for i, (Wl, bl) in enumerate(layers):
        z = conv32(a, Wl, bl)
        if i < 3:
            a = net_ref.bf16(np.maximum(z, F32(0))).astype(F32)
            acts.append(a)
        else:
            out = z[..., 0] + acts[0][..., 1]
    B = labels.shape[0]
    lab = labels.astype(F32)
    smax = lab.reshape(B, -1).max(axis=1)[:, None, None]
    cut = (smax - F32(3.0e38 if np.isinf(top_band) else top_band)).astype(F32)
    d = (out - lab).astype(F32)
    w = (np.where((lab >= cut) | (out >= cut), F32(1), F32(low))
         * np.where(d < 0, F32(under), F32(1))).astype(F32)
    inv_n = F32(1.0) / F32(out.size)
    g = net_ref.bf16((F32(2) * w * d * inv_n).astype(F32)).astype(F32)[..., None]
    grads = [None] * 4
    for i in range(3, -1, -1):
        Wl, _ = layers[i]
        tap = (0, 1) if mistake == "tap" and i == 2 else None
        grads[i] = grad_weight32(g, acts[i], wrong_tap=tap)
        if i == 0:
            break
        Wuse = Wl
        if mistake == "channel" and i == 2:
            Wuse = Wl.copy()
            Wuse[:, :, [3, 4]] = Wuse[:, :, [4, 3]]
        dx = grad_input32(g, Wuse)
        if mistake != "relu" or i != 1:
            dx = dx * (acts[i] > 0)
        g = net_ref.bf16(dx).astype(F32)
        if mistake == "sign" and i == 3:
            g = -g
    return out, acts, grads


@pytest.fixture(scope="module")
def real_case():
    """Real-valued maps and weights: the bounds hold but are loose."""
    maps = net_bounds.bits_to_float(synth.net_maps(31, 3))
    rng = np.random.default_rng(32)
    labels = rng.normal(0.5, 0.3, size=(3, 46, 61))
    w = rng.normal(0.0, 0.08, size=net_ref.n_params())
    return maps, labels, net_bounds.layers_as_gpu(w)


@pytest.fixture(scope="module")
def int_case():
    """Integer maps and weights: an exact forward pass, tight bounds."""
    maps = net_bounds.bits_to_float(synth.net_maps(33, 3, integer=True))
    rng = np.random.default_rng(34)
    labels = rng.uniform(-2.0, 6.0, size=(3, 46, 61))
    layers = net_bounds.layers_as_gpu(synth.net_int_weights(35))
    return maps, labels, layers


def test_forward_inside_bounds(real_case, int_case):
    for x, _, layers in (real_case, int_case):
        exact = x is int_case[0]
        acts, out, E_acts, E_out = net_bounds.forward_bounds(x, layers, exact)
        out32, acts32, _ = emulate(x, np.zeros(out.shape), layers)
        for i in (1, 2, 3):
            assert np.all(np.abs(acts32[i] - acts[i]) <= E_acts[i]), i
        assert np.all(np.abs(out32 - out) <= E_out)
    # integer network: the emulation reproduces the reference exactly
    assert np.array_equal(out32, out) and not E_out.any()


@pytest.mark.parametrize("band,low,under", [(np.inf, 1.0, 1.0),
                                            (0.4, 0.1, 3.0)])
def test_gradients_inside_bounds(real_case, int_case, band, low, under):
    for case in (real_case, int_case):
        x, labels, layers = case
        exact = case is int_case
        loss, grads, bounds = net_bounds.gradient_bounds(
            x, labels, layers, top_band=band, low_weight=low,
            under_weight=under, exact=exact)
        _, _, g32 = emulate(x, labels, layers, band, low, under)
        for (dW, db), (eW, eb), (gW, gb) in zip(grads, bounds, g32):
            assert np.all(np.abs(gW - dW) <= eW)
            assert np.all(np.abs(gb - db) <= eb)
            if exact:
                # tight: a small fraction of each gradient
                nz = np.abs(dW) > 0
                assert np.median(eW[nz] / np.abs(dW[nz])) < 2.0 ** -7


@pytest.mark.parametrize("mistake", ["tap", "channel", "relu", "sign"])
def test_planted_mistakes_leave_the_bounds(int_case, mistake):
    x, labels, layers = int_case
    _, grads, bounds = net_bounds.gradient_bounds(x, labels, layers,
                                                  exact=True)
    _, _, g32 = emulate(x, labels, layers, mistake=mistake)
    outside = 0
    for (dW, db), (eW, eb), (gW, gb) in zip(grads, bounds, g32):
        outside += int(np.sum(np.abs(gW - dW) > eW))
        outside += int(np.sum(np.abs(gb - db) > eb))
    assert outside > 0, mistake
