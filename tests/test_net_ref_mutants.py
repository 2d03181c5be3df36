"""The pins of the network reference catch plausible slips.

Each case plants one mistake in a copy of ``oracle/net_ref.py`` (a dropped
ReLU, a transposed or unflipped tap, a lost bias, a halved loss gradient, a
reversed asymmetric weight, a shifted pixel grid, truncating bfloat16
rounding, ...), loads the copy as a module of the ``oracle`` package, and
runs the checks of test_net_ref.py against it: at least one must fail.
Nothing here touches the real reference or any GPU.
"""
from __future__ import annotations

import importlib.util
import os

import pytest

import oracle
from tests import test_net_ref as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "net_ref.py")

MUTANTS = [
    ("conv: taps transposed", "out += xp[:, ky:ky + h, kx:kx + w] @ Wl[ky, kx].T",
     "out += xp[:, ky:ky + h, kx:kx + w] @ Wl[kx, ky].T"),
    ("conv: bias dropped",
     "out = np.broadcast_to(bl, (B, h, w, Wl.shape[2])).copy()",
     "out = np.zeros((B, h, w, Wl.shape[2]))"),
    ("grad input: taps not flipped",
     "dx += gp[:, 2 - ky:2 - ky + h, 2 - kx:2 - kx + w] @ Wl[ky, kx]",
     "dx += gp[:, ky:ky + h, kx:kx + w] @ Wl[ky, kx]"),
    ("grad weight: bias gradient averaged", "return dW, G.sum(axis=0)",
     "return dW, G.mean(axis=0)"),
    ("forward: ReLU dropped", "a = np.maximum(z, 0.0)", "a = z"),
    ("forward: coarse-score skip dropped", "out = z[..., 0] + x[..., 1]",
     "out = z[..., 0]"),
    ("loss: gradient halved", "g = (2.0 / N * w * diff)[..., None]",
     "g = (1.0 / N * w * diff)[..., None]"),
    ("backward: ReLU mask dropped", "dx = conv_grad_input(g, Wl) * (acts[i] > 0)",
     "dx = conv_grad_input(g, Wl)"),
    ("loss weights: under-weight on over-predictions",
     "return w * np.where(out < labels, under_weight, 1.0)",
     "return w * np.where(out > labels, under_weight, 1.0)"),
    ("loss weights: band above the best", "max(axis=1) - top_band",
     "max(axis=1) + top_band"),
    ("raster: density width doubled", "SIGMA_OPP = 0.3", "SIGMA_OPP = 0.6"),
    ("raster: pixel grid shifted", "return (xs - 30.0) / 5.0, (ys - 22.5) / 5.0",
     "return (xs - 30.5) / 5.0, (ys - 22.5) / 5.0"),
    ("raster: sub-points on the centre", "SUB_OFF = 0.05", "SUB_OFF = 0.0"),
    ("raster: margin not clamped", "out[y, x, 3] = min(max(mbest, -2.0), 1.0)",
     "out[y, x, 3] = mbest"),
    ("raster: goal distance from the centre line", "out[..., 5] = np.hypot(L / 2 - cx, cy) / diag",
     "out[..., 5] = np.hypot(L / 2 - cx, 0.0) / diag"),
    ("bf16: truncation", "r = ((u + 0x7FFF + lsb) >> 16) << 16",
     "r = (u >> 16) << 16"),
]


def _load(text, tmp_path):
    path = os.path.join(tmp_path, "net_ref_mutant.py")
    with open(path, "w") as f:
        f.write(text)
    spec = importlib.util.spec_from_file_location("oracle._net_ref_mutant",
                                                  path)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert text.count(orig) >= 1, f"mutation site missing: {orig!r}"
    ref = _load(text.replace(orig, mut, 1), tmp_path)
    for chk in pins.CHECKS:
        try:
            chk(ref)
        except (AssertionError, ValueError, IndexError):
            return
    pytest.fail(f"no pin caught mutant: {name}")


def test_the_unmutated_copy_passes(tmp_path):
    ref = _load(open(SRC).read(), tmp_path)
    for chk in pins.CHECKS:
        chk(ref)
