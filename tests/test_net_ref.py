"""Pins of the CPU reference of the proposal network (oracle/net_ref.py).

The convolution is checked against a loop written straight from its
definition, the analytic gradients against central finite differences of
the loss, the rasteriser against closed forms, and the bfloat16 rounding
against values fixed by the format.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import net_ref


def _conv_loops(x, Wl, bl):
    B, h, w, ci = x.shape
    co = Wl.shape[2]
    out = np.zeros((B, h, w, co))
    for b in range(B):
        for y in range(h):
            for xx in range(w):
                for o in range(co):
                    acc = bl[o]
                    for ky in range(3):
                        for kx in range(3):
                            yy, xs = y + ky - 1, xx + kx - 1
                            if 0 <= yy < h and 0 <= xs < w:
                                acc += np.dot(Wl[ky, kx, o], x[b, yy, xs])
                    out[b, y, xx, o] = acc
    return out


def test_conv_matches_its_definition():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 4, 3))
    Wl = rng.normal(size=(3, 3, 2, 3))
    bl = rng.normal(size=2)
    assert np.allclose(net_ref.conv(x, Wl, bl), _conv_loops(x, Wl, bl),
                       atol=1e-12)


def _tiny_layers(rng, chans=(3, 4, 4, 1)):
    return [(rng.normal(size=(3, 3, co, ci)) * 0.3, rng.normal(size=co) * 0.1)
            for ci, co in zip(chans[:-1], chans[1:])]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    layers = _tiny_layers(rng)
    x = rng.normal(size=(2, 5, 6, 3))
    labels = rng.normal(size=(2, 5, 6))
    loss, grads = net_ref.loss_and_grads(x, labels, layers, round_grads=False)
    h = 1e-6
    for li, (Wl, bl) in enumerate(layers):
        for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (2, 1, Wl.shape[2] - 1, 0)]:
            idx = tuple(min(i, s - 1) for i, s in zip(idx, Wl.shape))
            Wp = Wl.copy()
            Wp[idx] += h
            Wm = Wl.copy()
            Wm[idx] -= h
            lp = net_ref.loss_and_grads(
                x, labels, layers[:li] + [(Wp, bl)] + layers[li + 1:],
                round_grads=False)[0]
            lm = net_ref.loss_and_grads(
                x, labels, layers[:li] + [(Wm, bl)] + layers[li + 1:],
                round_grads=False)[0]
            num = (lp - lm) / (2 * h)
            assert abs(grads[li][0][idx] - num) <= 1e-6 * max(1, abs(num))
        bp = bl.copy()
        bp[0] += h
        bm = bl.copy()
        bm[0] -= h
        num = (net_ref.loss_and_grads(x, labels, layers[:li] + [(Wl, bp)]
                                      + layers[li + 1:], round_grads=False)[0]
               - net_ref.loss_and_grads(x, labels, layers[:li] + [(Wl, bm)]
                                        + layers[li + 1:],
                                        round_grads=False)[0]) / (2 * h)
        assert abs(grads[li][1][0] - num) <= 1e-6 * max(1, abs(num))


def test_input_gradient_is_the_adjoint_of_conv():
    """<conv(x) - b, g> == <x, conv_grad_input(g)> for every x, g."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, 4, 5, 3))
    g = rng.normal(size=(1, 4, 5, 2))
    Wl = rng.normal(size=(3, 3, 2, 3))
    lhs = np.sum((net_ref.conv(x, Wl, np.zeros(2))) * g)
    rhs = np.sum(x * net_ref.conv_grad_input(g, Wl))
    assert math.isclose(lhs, rhs, rel_tol=1e-12)


def test_raster_closed_forms():
    st = {"ball": (0.0, 0.0), "n_opp": 1, "opp_pos": [(-6.0 + 0.2 * 10,
                                                         -4.5 + 0.2 * 7)],
          "opp_vel": [(3.25, 0.0)], "vmax": 3.25, "field_len": 12.0,
          "field_wid": 9.0}
    m = net_ref.raster(st)
    assert m.shape == (46, 61, 8)
    assert m[7, 10, 0] == 1.0 and m[7, 10, 1] == 1.0 and m[7, 10, 2] == 0.0
    assert m[7, 10, 5] == 0.0
    # one pixel away: exp(-0.04 / 0.18) in bfloat16
    assert m[7, 11, 0] == net_ref.bf16(math.exp(-0.04 / 0.18))
    assert m[0, 0, 6] == -1.0 and m[0, 60, 6] == 1.0
    assert m[0, 0, 7] == -1.0 and m[45, 0, 7] == 1.0
    empty = dict(st, n_opp=0)
    e = net_ref.raster(empty)
    assert np.all(e[..., 0:3] == 0) and np.all(e[..., 5] == 1.0)
    # the ball sits on pixel (22.5, 30): the nearest centres are 0.1 m away
    assert e[22, 30, 3] == net_ref.bf16(math.exp(-0.01 / 0.5))


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8,
                  -2.5, 0.0, 65504.0])
    r = net_ref.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                       # tie to even
    assert r[2] == 1.0 + 2 ** -7             # representable
    assert r[3] == 1.0 + 2 ** -6             # tie to even (up)
    assert r[4] == -2.5 and r[5] == 0.0
    assert r[6] == 65536.0


def test_parameter_layout():
    assert net_ref.n_params() == 21121
    rng = np.random.default_rng(4)
    w = rng.normal(size=net_ref.n_params())
    assert np.array_equal(net_ref.flatten(net_ref.unflatten(w)), w)
