"""Pins of the CPU reference of the proposal network (oracle/net_ref.py).

The convolution is checked against a loop written straight from its
definition, the analytic gradients against central finite differences of
the loss, the rasteriser against closed forms, and the bfloat16 rounding
against values fixed by the format.  Each check takes the reference module,
so the mutant tests can run them against copies with planted mistakes.
"""
from __future__ import annotations

import math

import numpy as np

import pytest

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


def check_conv_matches_its_definition(ref):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 4, 3))
    Wl = rng.normal(size=(3, 3, 2, 3))
    bl = rng.normal(size=2)
    assert np.allclose(ref.conv(x, Wl, bl), _conv_loops(x, Wl, bl),
                       atol=1e-12)


def _tiny_layers(rng, chans=(3, 4, 4, 1)):
    return [(rng.normal(size=(3, 3, co, ci)) * 0.3, rng.normal(size=co) * 0.1)
            for ci, co in zip(chans[:-1], chans[1:])]


def check_gradients_match_finite_differences(ref):
    rng = np.random.default_rng(2)
    layers = _tiny_layers(rng)
    x = rng.normal(size=(2, 5, 6, 3))
    labels = rng.normal(size=(2, 5, 6))
    loss, grads = ref.loss_and_grads(x, labels, layers, round_grads=False)
    h = 1e-6
    for li, (Wl, bl) in enumerate(layers):
        for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (2, 1, Wl.shape[2] - 1, 0)]:
            idx = tuple(min(i, s - 1) for i, s in zip(idx, Wl.shape))
            Wp = Wl.copy()
            Wp[idx] += h
            Wm = Wl.copy()
            Wm[idx] -= h
            lp = ref.loss_and_grads(
                x, labels, layers[:li] + [(Wp, bl)] + layers[li + 1:],
                round_grads=False)[0]
            lm = ref.loss_and_grads(
                x, labels, layers[:li] + [(Wm, bl)] + layers[li + 1:],
                round_grads=False)[0]
            num = (lp - lm) / (2 * h)
            assert abs(grads[li][0][idx] - num) <= 1e-6 * max(1, abs(num))
        bp = bl.copy()
        bp[0] += h
        bm = bl.copy()
        bm[0] -= h
        num = (ref.loss_and_grads(x, labels, layers[:li] + [(Wl, bp)]
                                      + layers[li + 1:], round_grads=False)[0]
               - ref.loss_and_grads(x, labels, layers[:li] + [(Wl, bm)]
                                        + layers[li + 1:],
                                        round_grads=False)[0]) / (2 * h)
        assert abs(grads[li][1][0] - num) <= 1e-6 * max(1, abs(num))


def check_focused_loss_gradients_match_finite_differences(ref):
    rng = np.random.default_rng(6)
    layers = _tiny_layers(rng)
    x = rng.normal(size=(2, 5, 6, 3))
    labels = rng.normal(size=(2, 5, 6))
    kw = dict(round_grads=False, top_band=0.8, low_weight=0.25,
              under_weight=3.0)
    _, out = ref.forward(x, layers, round_acts=False)
    w = ref.loss_weights(out, labels, 0.8, 0.25)
    assert (w == 1).any() and (w == 0.25).any()
    _, grads = ref.loss_and_grads(x, labels, layers, **kw)
    h = 1e-6
    Wl, bl = layers[1]
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1)]:
        Wp, Wm = Wl.copy(), Wl.copy()
        Wp[idx] += h
        Wm[idx] -= h
        lp = ref.loss_and_grads(x, labels, [layers[0], (Wp, bl)]
                                    + layers[2:], **kw)[0]
        lm = ref.loss_and_grads(x, labels, [layers[0], (Wm, bl)]
                                    + layers[2:], **kw)[0]
        num = (lp - lm) / (2 * h)
        assert abs(grads[1][0][idx] - num) <= 1e-6 * max(1, abs(num))


def check_loss_weights(ref):
    labels = np.array([[[0.0, 1.0, 0.1, 0.5]]])
    out = np.array([[[0.9, 0.0, 0.2, 0.0]]])
    # best label 1.0, band 0.2: pixels reaching 0.8 by label or output
    w = ref.loss_weights(out, labels, 0.2, 0.1)
    assert np.array_equal(w, [[[1.0, 1.0, 0.1, 0.1]]])
    # under-predictions (pixels 1 and 3) cost under_weight times more
    w = ref.loss_weights(out, labels, 0.2, 0.1, 4.0)
    assert np.array_equal(w, [[[1.0, 4.0, 0.1, 0.4]]])
    # a low weight of 1 is the plain mean squared error for any band
    rng = np.random.default_rng(7)
    layers = _tiny_layers(rng)
    x = rng.normal(size=(1, 4, 4, 3))
    lab = rng.normal(size=(1, 4, 4))
    a = ref.loss_and_grads(x, lab, layers, False, 0.3, 1.0)
    b = ref.loss_and_grads(x, lab, layers, False)
    assert a[0] == b[0]
    assert np.array_equal(ref.flatten(a[1]), ref.flatten(b[1]))


def check_input_gradient_is_the_adjoint_of_conv(ref):
    """<conv(x) - b, g> == <x, conv_grad_input(g)> for every x, g."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, 4, 5, 3))
    g = rng.normal(size=(1, 4, 5, 2))
    Wl = rng.normal(size=(3, 3, 2, 3))
    lhs = np.sum((ref.conv(x, Wl, np.zeros(2))) * g)
    rhs = np.sum(x * ref.conv_grad_input(g, Wl))
    assert math.isclose(lhs, rhs, rel_tol=1e-12)


def _state(opp, vel, ball=(0.0, 0.0)):
    return {"ball": ball, "n_opp": len(opp), "opp_pos": np.array(opp),
            "opp_vel": np.array(vel), "ball_decel": 0.5, "vmax": 3.25,
            "amax": 3.0, "field_len": 12.0, "field_wid": 9.0,
            "goal_width": 1.8}


def _sub_points(x, y):
    cx, cy = (x - 30) / 5.0, (y - 22.5) / 5.0
    return [(min(max(cx + dx, -6.0), 6.0), min(max(cy + dy, -4.5), 4.5))
            for dy in (-0.05, 0.05) for dx in (-0.05, 0.05)]


def _open_mouth(q):
    """Shot angle / pi from q with no opponents: the whole +-0.9 m mouth."""
    if q[0] >= 6.0:
        return 0.0
    return (math.atan2(0.9 - q[1], 6.0 - q[0])
            - math.atan2(-0.9 - q[1], 6.0 - q[0])) / math.pi


def check_raster_closed_forms(ref):
    bf = ref.bf16
    # density: an opponent on the centre of pixel (20, 40), c = (2, -0.5)
    m = ref.raster(_state([(2.0, -0.5)], [(0.0, 0.0)]))
    assert m.shape == (46, 61, 8)
    assert m[20, 40, 0] == 1.0
    assert m[20, 41, 0] == bf(math.exp(-0.04 / 0.18))
    # the ball sits between pixel centres (22, 30) and (23, 30), 0.1 m away
    assert m[22, 30, 2] == bf(0.1 / 15.0)

    # margin: an opponent at rest on the ball.  Along the pass line it runs
    # straight from rest (time sqrt(2 s / amax), then s / vmax + vmax /
    # (2 amax) beyond vmax^2 / (2 amax)) against the ball's (v - sqrt(v^2 -
    # 2 a s)) / a, both functions of the distance s alone.
    def t_opp(s):
        return (math.sqrt(2 * s / 3.0) if s <= 3.25 ** 2 / 6.0
                else s / 3.25 + 3.25 / 6.0)

    def t_ball(s, v):
        return (v - math.sqrt(v * v - 2 * 0.5 * s)) / 0.5

    want = -math.inf
    for q in _sub_points(40, 20):
        D = math.hypot(*q)
        for v in (2.0, 3.5, 5.0, 6.5):
            if v * v < 2 * 0.5 * D:
                continue
            want = max(want, min(t_opp(k / 16 * D) - t_ball(k / 16 * D, v)
                                 for k in range(1, 17)))
    on_ball = ref.raster(_state([(0.0, 0.0)], [(0.0, 0.0)]))
    assert on_ball[20, 40, 3] == bf(min(max(want, -2.0), 1.0))

    # no opponents: every pass is feasible with margin > 1, so the coarse
    # score is the angle and distance terms plus the capped margin 1
    e = ref.raster(_state([], []))
    assert np.all(e[..., 0] == 0)
    assert np.all(e[..., 3] == 1.0)
    qs = _sub_points(0, 22)
    assert e[22, 0, 4] == bf(max(_open_mouth(q) for q in qs))
    assert e[22, 0, 1] == bf(max(_open_mouth(q) - math.hypot(6 - q[0], q[1])
                                 / 15.0 + 1.0 for q in qs))
    # column 60 straddles the goal line: only its sub-points at x = 5.95
    # see the mouth, the others sit on the line (no shot from there)
    assert e[22, 60, 4] == bf(max(_open_mouth(q) for q in _sub_points(60, 22)))
    assert e[22, 60, 5] == bf(0.1 / 15.0)
    assert e[0, 0, 6] == -1.0 and e[0, 60, 6] == 1.0
    assert e[0, 0, 7] == -1.0 and e[45, 0, 7] == 1.0
    # a 1 m/s kick stops after 1 m: far cells get the floors
    slow = ref.raster(_state([], []), speeds=(1.0,))
    assert slow[22, 60, 3] == -2.0 and slow[22, 60, 1] == bf(-1.2)
    assert slow[22, 30, 3] == 1.0


def check_bf16_rounding(ref):
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8,
                  -2.5, 0.0, 65504.0])
    r = ref.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                       # tie to even
    assert r[2] == 1.0 + 2 ** -7             # representable
    assert r[3] == 1.0 + 2 ** -6             # tie to even (up)
    assert r[4] == -2.5 and r[5] == 0.0
    assert r[6] == 65536.0


def check_zero_network_is_the_coarse_score(ref):
    """The output adds the input's coarse-score channel to the last
    convolution: with zero weights the prediction is that channel."""
    rng = np.random.default_rng(5)
    x = ref.bf16(rng.normal(size=(2, 46, 61, 8)))
    _, out = ref.forward(x, ref.unflatten(np.zeros(ref.n_params())))
    assert np.array_equal(out, x[..., 1])


def check_parameter_layout(ref):
    assert ref.n_params() == 21121
    rng = np.random.default_rng(4)
    w = rng.normal(size=ref.n_params())
    assert np.array_equal(ref.flatten(ref.unflatten(w)), w)


CHECKS = [
    check_conv_matches_its_definition,
    check_gradients_match_finite_differences,
    check_focused_loss_gradients_match_finite_differences,
    check_loss_weights,
    check_input_gradient_is_the_adjoint_of_conv,
    check_raster_closed_forms,
    check_bf16_rounding,
    check_zero_network_is_the_coarse_score,
    check_parameter_layout,
]


@pytest.mark.parametrize("chk", CHECKS, ids=[c.__name__[6:] for c in CHECKS])
def test_pin(chk):
    chk(net_ref)
