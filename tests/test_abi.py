"""The C-ABI library builds, loads and exports what include/pps.h declares.

These run without a GPU: they only call the host-side helpers (grid,
mask size, defaults, status strings) and check that context creation
fails cleanly when no device is present.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1909_07717_gb300 import build, pps

HEADER = os.path.join(os.path.dirname(os.path.dirname(
    os.path.abspath(__file__))), "include", "pps.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pps.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pps_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "pps_search" in names and "pps_create" in names
    raw = ctypes.CDLL(pps.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    assert set(pps.EXPORTS) <= set(names)


def test_record_sizes_match_header(lib):
    assert ctypes.sizeof(pps.pps_state) == 296
    assert ctypes.sizeof(pps.pps_best) == 32
    assert ctypes.sizeof(pps.pps_grid) == 20
    assert ctypes.sizeof(pps.pps_params) == 32
    assert ctypes.sizeof(pps.pps_plan_group) == 64
    assert pps.pps_plan_group.n_items.offset == 24
    text = open(HEADER).read()
    assert f"#define PPS_MAX_OPP {pps.PPS_MAX_OPP}" in text
    assert f"#define PPS_ABI_VERSION {pps.PPS_ABI_VERSION}" in text


def test_host_helpers(lib):
    assert pps.pps_abi_version() == pps.PPS_ABI_VERSION == 2
    assert pps.pps_status_string(pps.PPS_EINVAL) == "PPS_EINVAL"
    assert pps.pps_status_string(99) == "PPS_UNKNOWN"
    p = pps.pps_default_params()
    assert (p.w_angle, p.margin_cap, p.tau_safe) == (1.0, 1.0, 0.0)
    assert abs(p.robot_radius - 0.09) < 1e-7
    g = pps.pps_grid_from_field(12.0, 9.0, 0.1)
    assert (g.nx, g.ny, g.x0, g.y0) == (121, 91, -6.0, -4.5)
    g = pps.pps_grid_from_field(12.0, 9.0, 0.05)
    assert (g.nx, g.ny) == (241, 181)
    assert pps.pps_mask_words(g, 4) == 4 * ((241 * 181 + 31) // 32)
    g = pps.pps_grid_from_field(9.0, 6.0, 0.025)
    assert (g.nx, g.ny) == (361, 241)
    for bad in [(0.0, 9.0, 0.1), (12.0, 9.0, 0.0), (12.0, 9.0, -1.0),
                (float("nan"), 9.0, 0.1), (12.0, 9.0, 1e-6)]:
        with pytest.raises(pps.PpsError):
            pps.pps_grid_from_field(*bad)


def test_running_point_host_helpers(lib):
    assert pps.pps_run_grid(12.0, 9.0, 0.1) == (61, 91)
    assert pps.pps_run_grid(9.0, 6.0, 0.05) == (91, 121)
    assert pps.pps_run_grid(12.0, 9.0, 0.025) == (241, 361)
    for bad in [(0.0, 9.0, 0.1), (12.0, 9.0, 0.0), (12.0, float("inf"), 0.1),
                (12.0, 9.0, 1e-5)]:
        with pytest.raises(pps.PpsError):
            pps.pps_run_grid(*bad)
    p = pps.pps_run_default_params()
    assert abs(p.spacing - 0.1) < 1e-7 and p.n_run == 4
    assert (p.w_goal, p.w_ball, p.w_angle, p.w_guard, p.w_avoid) == (1.0,) * 5
    assert abs(p.def_depth - 1.2) < 1e-6 and abs(p.def_width - 2.4) < 1e-6
    assert ctypes.sizeof(pps.pps_rparams) == 56
    assert pps.RBEST_DTYPE.itemsize == 96
    d = pps.pps_dpps_default_params()
    assert (d.n_dir, d.n_pow) == (128, 64) and abs(d.slide - 5 / 7) < 1e-7
    assert pps.pps_dpps_mask_words(d) == 128 * 64 // 32


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(pps.PpsError) as e:
        pps.pps_create(pps.pps_ctx_desc(max_states=4))
    assert e.value.status == pps.PPS_ECUDA
    assert "device" in pps.pps_last_error(None)
    with pytest.raises(pps.PpsError) as e:
        pps.pps_create(pps.pps_ctx_desc(max_states=0))
    assert e.value.status == pps.PPS_EINVAL


def test_weight_file_round_trip_and_checks(tmp_path):
    """The proposal weight file: magic, count, CRC-32, float32 data."""
    w = pps.init_weights(3)
    p = str(tmp_path / "w.bin")
    pps.save_net_weights(p, w)
    assert np.array_equal(pps.load_net_weights(p), w)
    raw = bytearray(open(p, "rb").read())
    raw[100] ^= 1
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="checksum"):
        pps.load_net_weights(p)
    with pytest.raises(ValueError):
        pps.save_net_weights(p, w[:-1])
    bad = w.copy()
    bad[5] = np.nan
    with pytest.raises(ValueError):
        pps.save_net_weights(p, bad)


def test_committed_weights_load():
    w = pps.load_net_weights()
    assert w.shape == (pps.PPS_NET_PARAMS,) and np.all(np.isfinite(w))
