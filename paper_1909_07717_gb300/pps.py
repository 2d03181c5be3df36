"""ctypes binding of libpps (include/pps.h): same names, marshalling only.

Every computation happens in the CUDA library; this module only converts
Python values to the C structs, calls the C entry points and turns status
codes into ``PpsError``.  PyTorch provides device memory and streams.  If
libpps.so is missing the first call raises: there is no other code path.

    from paper_1909_07717_gb300 import pps, synth
    ctx = pps.pps_create(pps.pps_ctx_desc(max_states=4096, max_opp=8))
    ...
    pps.pps_destroy(ctx)

``Searcher`` wraps a context and torch tensors for the common case.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpps.so")

PPS_ABI_VERSION = 2
PPS_MAX_OPP = 16
PPS_MAX_SPEEDS = 8
PPS_MAX_K = 4096
PPS_NOALLOC_MAX_STATES = 16384
PPS_NET_H, PPS_NET_W, PPS_NET_PARAMS = 46, 61, 21121
PPS_PROPOSE_FALLBACK = 1
PPS_PROPOSE_NO_PRUNE = 2

PPS_OK, PPS_EINVAL, PPS_ENOMEM, PPS_ECUDA, PPS_ETIMEOUT, PPS_ENOTIMPL = range(6)
PPS_DEVICE_PTRS = 1
PPS_STATE_OK, PPS_STATE_INVALID, PPS_STATE_INCONSISTENT = 0, 1, 2

c_float, c_int32, c_size_t, c_void_p = (ctypes.c_float, ctypes.c_int32,
                                        ctypes.c_size_t, ctypes.c_void_p)


class pps_state(ctypes.Structure):
    _fields_ = [("ball", c_float * 2), ("n_opp", c_int32),
                ("opp_pos", (c_float * 2) * PPS_MAX_OPP),
                ("opp_vel", (c_float * 2) * PPS_MAX_OPP),
                ("ball_decel", c_float), ("vmax", c_float), ("amax", c_float),
                ("field_len", c_float), ("field_wid", c_float),
                ("goal_width", c_float), ("K", c_int32)]


class pps_grid(ctypes.Structure):
    _fields_ = [("spacing", c_float), ("nx", c_int32), ("ny", c_int32),
                ("x0", c_float), ("y0", c_float)]


class pps_params(ctypes.Structure):
    _fields_ = [(n, c_float) for n in (
        "w_angle", "w_dist", "w_margin", "margin_cap", "tau_safe",
        "robot_radius", "reach_radius", "min_pass_dist")]


class pps_best(ctypes.Structure):
    _fields_ = [("idx", c_int32), ("ix", c_int32), ("iy", c_int32),
                ("speed_idx", c_int32), ("score", c_float),
                ("margin", c_float), ("n_feasible", c_int32),
                ("status", c_int32)]


class pps_debug_out(ctypes.Structure):
    _fields_ = [("margin", c_void_p), ("score", c_void_p), ("T", c_void_p),
                ("T_stride", c_int32), ("point_best", c_void_p)]


class pps_ctx_desc(ctypes.Structure):
    _fields_ = [("device", c_int32), ("stream", c_void_p),
                ("mem_budget_bytes", c_size_t), ("max_states", c_int32),
                ("max_points", c_int32), ("max_speeds", c_int32),
                ("max_K", c_int32), ("max_opp", c_int32)]

    def __init__(self, max_states=1, device=0, stream=None, mem_budget_bytes=0,
                 max_points=0, max_speeds=0, max_K=0, max_opp=0):
        super().__init__(device, stream, mem_budget_bytes, max_states,
                         max_points, max_speeds, max_K, max_opp)


class pps_job(ctypes.Structure):
    _fields_ = [("grid", pps_grid), ("n_speeds", c_int32),
                ("speeds", c_float * PPS_MAX_SPEEDS), ("max_opp", c_int32)]


class pps_plan_group(ctypes.Structure):
    _fields_ = [("opp_slots", c_int32), ("speed_slots", c_int32),
                ("n_states", c_int32), ("cta_threads", c_int32),
                ("sample_unroll", c_int32), ("reserved", c_int32),
                ("n_items", ctypes.c_int64), ("tuned_ms", c_float * 7)]


class pps_server_desc(ctypes.Structure):
    _fields_ = [("device", c_int32), ("n_streams", c_int32),
                ("max_batch", c_int32), ("max_queue", c_int32),
                ("pool_bytes", c_size_t), ("max_opp", c_int32),
                ("max_wait_us", c_int32), ("params", pps_params),
                ("mode", c_int32), ("topk", c_int32),
                ("net_weights", c_void_p)]


PPS_SERVE_EXACT = 0
PPS_SERVE_PROPOSAL = 1


class pps_server_result(ctypes.Structure):
    _fields_ = [("best", pps_best), ("ticket", ctypes.c_uint64),
                ("latency_ns", ctypes.c_int64), ("queue_ns", ctypes.c_int64),
                ("batch_size", c_int32), ("status", c_int32)]


class pps_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("states_per_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PPS_PLAN_AUTOTUNE = 1
PPS_PLAN_GRAPH = 2


# numpy mirrors of the record layouts (for packing batches).
STATE_DTYPE = np.dtype([("ball", "<f4", (2,)), ("n_opp", "<i4"),
                        ("opp_pos", "<f4", (PPS_MAX_OPP, 2)),
                        ("opp_vel", "<f4", (PPS_MAX_OPP, 2)),
                        ("ball_decel", "<f4"), ("vmax", "<f4"),
                        ("amax", "<f4"), ("field_len", "<f4"),
                        ("field_wid", "<f4"), ("goal_width", "<f4"),
                        ("K", "<i4")])
BEST_DTYPE = np.dtype([("idx", "<i4"), ("ix", "<i4"), ("iy", "<i4"),
                       ("speed_idx", "<i4"), ("score", "<f4"),
                       ("margin", "<f4"), ("n_feasible", "<i4"),
                       ("status", "<i4")])
assert STATE_DTYPE.itemsize == ctypes.sizeof(pps_state) == 296
assert BEST_DTYPE.itemsize == ctypes.sizeof(pps_best) == 32

# the direction x power search (pps_dpps_*)
PPS_MAX_TEAM = 16


class pps_dparams(ctypes.Structure):
    _fields_ = [("n_dir", c_int32), ("n_pow", c_int32), ("v_lo", c_float),
                ("v_hi", c_float), ("slide", c_float), ("tau_delta", c_float),
                ("delta_cap", c_float), ("w_time", c_float),
                ("w_angle", c_float), ("w_dist", c_float),
                ("w_refr", c_float), ("w_delta", c_float),
                ("robot_radius", c_float), ("reach_radius", c_float)]


DSTATE_DTYPE = np.dtype([("ball", "<f4", (2,)), ("n_team", "<i4"),
                         ("n_opp", "<i4"),
                         ("team_pos", "<f4", (PPS_MAX_TEAM, 2)),
                         ("team_vel", "<f4", (PPS_MAX_TEAM, 2)),
                         ("opp_pos", "<f4", (PPS_MAX_OPP, 2)),
                         ("opp_vel", "<f4", (PPS_MAX_OPP, 2)),
                         ("ball_decel", "<f4"), ("vmax", "<f4"),
                         ("amax", "<f4"), ("field_len", "<f4"),
                         ("field_wid", "<f4"), ("goal_width", "<f4"),
                         ("K", "<i4")])
DBEST_DTYPE = np.dtype([("idx", "<i4"), ("dir", "<i4"), ("pow", "<i4"),
                        ("receiver", "<i4"), ("score", "<f4"),
                        ("t_team", "<f4"), ("t_opp", "<f4"),
                        ("recv", "<f4", (2,)), ("n_feasible", "<i4"),
                        ("status", "<i4"), ("reserved", "<i4")])
assert DSTATE_DTYPE.itemsize == 556 and DBEST_DTYPE.itemsize == 48
PASS_QUERY_DTYPE = np.dtype([("state", "<i4"), ("receiver", "<i4"),
                             ("target", "<f4", (2,))])
PASS_POWER_DTYPE = np.dtype([("v0", "<f4"), ("v1", "<f4"), ("t_pass", "<f4"),
                             ("t_recv", "<f4"), ("clamped", "<i4"),
                             ("status", "<i4")])
SHOT_QUERY_DTYPE = np.dtype([("state", "<i4"), ("from", "<f4", (2,))])
SHOT_DTYPE = np.dtype([("theta", "<f4"), ("dir", "<f4"), ("t_line", "<f4"),
                       ("t_opp", "<f4"), ("shoot", "<i4"), ("status", "<i4")])


# running points (pps_run_*)
class pps_rparams(ctypes.Structure):
    _fields_ = [("spacing", c_float), ("w_goal", c_float),
                ("w_ball", c_float), ("w_angle", c_float),
                ("w_guard", c_float), ("w_avoid", c_float),
                ("ball_ref", c_float), ("angle_lo", c_float),
                ("angle_hi", c_float), ("angle_span", c_float),
                ("def_depth", c_float), ("def_width", c_float),
                ("guard_cap", c_float), ("n_run", c_int32)]


RBEST_DTYPE = np.dtype([("idx", "<i4", (4,)), ("score", "<f4", (4,)),
                        ("point", "<f4", (4, 2)), ("chosen", "<i4", (4,)),
                        ("avoided", "<i4"), ("nx", "<i4"), ("ny", "<i4"),
                        ("status", "<i4")])
assert RBEST_DTYPE.itemsize == 96 and ctypes.sizeof(pps_rparams) == 56

EXPORTS = ("pps_abi_version", "pps_status_string", "pps_last_error",
           "pps_default_params", "pps_grid_from_field", "pps_mask_words",
           "pps_create", "pps_destroy", "pps_search", "pps_sync", "pps_reset",
           "pps_launch_info", "pps_search_noalloc", "pps_plan_create",
           "pps_plan_destroy", "pps_plan_mask_offsets", "pps_plan_run",
           "pps_plan_groups", "pps_server_create", "pps_server_destroy",
           "pps_server_submit", "pps_server_wait", "pps_server_replay",
           "pps_server_get_stats", "pps_net_create", "pps_net_destroy",
           "pps_net_set_features", "pps_net_set_loss", "pps_net_set_weights",
           "pps_net_sync", "pps_net_selftest_timeout",
           "pps_net_get_weights", "pps_net_raster", "pps_net_forward_layers",
           "pps_net_forward", "pps_net_forward_map", "pps_net_grad",
           "pps_net_grad_map", "pps_net_set_train_kernels",
           "pps_net_train_step",
           "pps_net_labels", "pps_net_labels_grid", "pps_propose",
           "pps_propose_jobs", "pps_dpps_default_params",
           "pps_dpps_mask_words", "pps_dpps_search", "pps_pass_powers",
           "pps_shoot", "pps_run_default_params", "pps_run_grid",
           "pps_run_points")


class PpsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")


_STATUS = {PPS_OK: "PPS_OK", PPS_EINVAL: "PPS_EINVAL", PPS_ENOMEM: "PPS_ENOMEM",
           PPS_ECUDA: "PPS_ECUDA", PPS_ETIMEOUT: "PPS_ETIMEOUT",
           PPS_ENOTIMPL: "PPS_ENOTIMPL"}

_lock = threading.Lock()
_lib = None


def lib():
    """Load libpps.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_1909_07717_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            L.pps_abi_version.restype = ctypes.c_int
            L.pps_status_string.restype = ctypes.c_char_p
            L.pps_status_string.argtypes = [ctypes.c_int]
            L.pps_last_error.restype = ctypes.c_char_p
            L.pps_last_error.argtypes = [c_void_p]
            L.pps_default_params.argtypes = [P(pps_params)]
            L.pps_grid_from_field.argtypes = [c_float, c_float, c_float,
                                              P(pps_grid)]
            L.pps_mask_words.restype = c_size_t
            L.pps_mask_words.argtypes = [P(pps_grid), ctypes.c_int]
            L.pps_create.argtypes = [P(c_void_p), P(pps_ctx_desc)]
            L.pps_destroy.restype = None
            L.pps_destroy.argtypes = [c_void_p]
            L.pps_search.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                     P(pps_grid), c_void_p, ctypes.c_int,
                                     P(pps_params), c_void_p, c_void_p,
                                     P(pps_debug_out), ctypes.c_uint]
            L.pps_sync.argtypes = [c_void_p]
            L.pps_reset.argtypes = [c_void_p]
            L.pps_launch_info.argtypes = [c_void_p, P(ctypes.c_int),
                                          P(ctypes.c_int)]
            L.pps_search_noalloc.argtypes = [
                ctypes.c_int, c_void_p, ctypes.c_int, c_void_p, ctypes.c_int,
                P(pps_grid), c_void_p, ctypes.c_int, P(pps_params), c_void_p,
                c_void_p]
            L.pps_plan_create.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                          P(pps_params), ctypes.c_uint,
                                          P(c_void_p)]
            L.pps_plan_destroy.restype = None
            L.pps_plan_destroy.argtypes = [c_void_p]
            L.pps_plan_mask_offsets.argtypes = [c_void_p, c_void_p]
            L.pps_plan_run.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
            L.pps_plan_groups.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                          P(ctypes.c_int)]
            L.pps_server_create.argtypes = [P(pps_server_desc), P(c_void_p)]
            L.pps_server_destroy.restype = None
            L.pps_server_destroy.argtypes = [c_void_p]
            L.pps_server_submit.argtypes = [c_void_p, c_void_p, c_void_p,
                                            P(ctypes.c_uint64)]
            L.pps_server_wait.argtypes = [c_void_p, ctypes.c_uint64,
                                          ctypes.c_int64,
                                          P(pps_server_result), c_void_p]
            L.pps_server_replay.argtypes = [c_void_p, c_void_p, c_void_p,
                                            ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, c_void_p,
                                            P(pps_server_stats)]
            L.pps_server_get_stats.argtypes = [c_void_p, P(pps_server_stats)]
            L.pps_net_create.argtypes = [ctypes.c_int, c_void_p, ctypes.c_int,
                                         P(c_void_p)]
            L.pps_net_destroy.restype = None
            L.pps_net_destroy.argtypes = [c_void_p]
            L.pps_net_set_features.argtypes = [c_void_p, c_void_p,
                                               ctypes.c_int, P(pps_params)]
            L.pps_net_sync.argtypes = [c_void_p]
            L.pps_net_selftest_timeout.argtypes = [c_void_p, c_void_p,
                                                   ctypes.c_int]
            L.pps_net_set_loss.argtypes = [c_void_p, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_float]
            L.pps_net_set_weights.argtypes = [c_void_p, c_void_p]
            L.pps_net_get_weights.argtypes = [c_void_p, c_void_p]
            L.pps_net_raster.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                         c_void_p]
            L.pps_net_forward.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                          c_void_p]
            L.pps_net_forward_layers.argtypes = [c_void_p, c_void_p,
                                                 ctypes.c_int, c_void_p]
            L.pps_net_forward_map.argtypes = [c_void_p, c_void_p,
                                              ctypes.c_int, ctypes.c_int,
                                              c_void_p]
            L.pps_net_grad.argtypes = [c_void_p, c_void_p, c_void_p,
                                       ctypes.c_int, c_void_p,
                                       P(ctypes.c_float)]
            L.pps_net_grad_map.argtypes = [c_void_p, c_void_p, c_void_p,
                                           ctypes.c_int, c_void_p,
                                           P(ctypes.c_float)]
            L.pps_net_set_train_kernels.argtypes = [c_void_p, ctypes.c_int]
            L.pps_net_train_step.argtypes = [c_void_p, c_void_p, c_void_p,
                                             ctypes.c_int, ctypes.c_float,
                                             P(ctypes.c_float)]
            L.pps_net_labels.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                         ctypes.c_float, c_void_p]
            L.pps_net_labels_grid.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                              P(pps_grid), ctypes.c_float,
                                              c_void_p]
            L.pps_propose_jobs.argtypes = [c_void_p, c_void_p, c_void_p,
                                           c_void_p, ctypes.c_int, c_float,
                                           ctypes.c_int, P(pps_params),
                                           ctypes.c_int, ctypes.c_uint,
                                           c_void_p, c_void_p]
            L.pps_propose.argtypes = [c_void_p, c_void_p, c_void_p,
                                      ctypes.c_int, P(pps_grid), c_void_p,
                                      ctypes.c_int, P(pps_params),
                                      ctypes.c_int, ctypes.c_uint, c_void_p,
                                      c_void_p]
            L.pps_dpps_default_params.argtypes = [P(pps_dparams)]
            L.pps_dpps_mask_words.restype = c_size_t
            L.pps_dpps_mask_words.argtypes = [P(pps_dparams)]
            L.pps_dpps_search.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                          P(pps_dparams), c_void_p, c_void_p,
                                          c_void_p]
            L.pps_pass_powers.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                          c_void_p, ctypes.c_int, c_float,
                                          P(pps_dparams), c_void_p]
            L.pps_shoot.argtypes = [c_void_p, c_void_p, ctypes.c_int, c_void_p,
                                    ctypes.c_int, c_float, c_float,
                                    P(pps_dparams), c_void_p]
            L.pps_run_default_params.argtypes = [P(pps_rparams)]
            L.pps_run_grid.argtypes = [c_float, c_float, c_float,
                                       P(ctypes.c_int), P(ctypes.c_int)]
            L.pps_run_points.argtypes = [c_void_p, c_void_p, ctypes.c_int,
                                         P(pps_rparams), c_void_p, c_void_p,
                                         c_void_p, c_size_t]
            if L.pps_abi_version() != PPS_ABI_VERSION:
                raise RuntimeError("libpps ABI version mismatch")
            _lib = L
        return _lib


def _check(status, ctx=None):
    if status != PPS_OK:
        raise PpsError(status, pps_last_error(ctx))
    return status


# ------------------------------------------------------------ entry points
def pps_abi_version() -> int:
    return lib().pps_abi_version()


def pps_status_string(status: int) -> str:
    return lib().pps_status_string(status).decode()


def pps_last_error(ctx=None) -> str:
    return lib().pps_last_error(ctx).decode()


def pps_default_params() -> pps_params:
    p = pps_params()
    _check(lib().pps_default_params(ctypes.byref(p)))
    return p


def pps_grid_from_field(L: float, W: float, spacing: float) -> pps_grid:
    g = pps_grid()
    _check(lib().pps_grid_from_field(L, W, spacing, ctypes.byref(g)))
    return g


def pps_mask_words(grid: pps_grid, n_speeds: int) -> int:
    return lib().pps_mask_words(ctypes.byref(grid), n_speeds)


def pps_create(desc: pps_ctx_desc):
    ctx = c_void_p()
    _check(lib().pps_create(ctypes.byref(ctx), ctypes.byref(desc)))
    return ctx


def pps_destroy(ctx) -> None:
    lib().pps_destroy(ctx)


def pps_search(ctx, states, n_states, grid, speeds, n_speeds, params,
               out_best, out_mask, dbg=None, flags=0) -> int:
    """Buffers are raw addresses (int) or None; ``speeds`` is a host
    address of n_speeds float32; ``params`` a pps_params or None."""
    return _check(lib().pps_search(
        ctx, states, n_states, ctypes.byref(grid), speeds, n_speeds,
        ctypes.byref(params) if params is not None else None, out_best,
        out_mask, ctypes.byref(dbg) if dbg is not None else None, flags), ctx)


def pps_search_noalloc(device, stream, max_opp, states, n_states, grid,
                       speeds, n_speeds, params, out_best, out_mask) -> int:
    """No-allocation search: ``states``, ``out_best``, ``out_mask`` are
    device addresses (int); ``speeds`` a host address of n_speeds float32;
    ``stream`` a cudaStream_t handle (int) or None."""
    return _check(lib().pps_search_noalloc(
        device, stream, max_opp, states, n_states, ctypes.byref(grid), speeds,
        n_speeds, ctypes.byref(params) if params is not None else None,
        out_best, out_mask))


def pps_plan_create(ctx, jobs, n_states, params=None, flags=0):
    """``jobs``: a ctypes array of pps_job (host)."""
    plan = c_void_p()
    _check(lib().pps_plan_create(
        ctx, ctypes.addressof(jobs), n_states,
        ctypes.byref(params) if params is not None else None, flags,
        ctypes.byref(plan)), ctx)
    return plan


def pps_plan_destroy(plan) -> None:
    lib().pps_plan_destroy(plan)


def pps_plan_mask_offsets(plan, n_states, ctx=None) -> np.ndarray:
    off = np.zeros(n_states + 1, np.int64)
    _check(lib().pps_plan_mask_offsets(plan, off.ctypes.data), ctx)
    return off


def pps_plan_run(plan, states, out_best, out_mask, ctx=None) -> int:
    """Device addresses (int); out_mask may be None."""
    return _check(lib().pps_plan_run(plan, states, out_best, out_mask), ctx)


def pps_plan_groups(plan, ctx=None):
    n = ctypes.c_int()
    _check(lib().pps_plan_groups(plan, None, 0, ctypes.byref(n)), ctx)
    arr = (pps_plan_group * max(1, n.value))()
    _check(lib().pps_plan_groups(plan, ctypes.addressof(arr), n.value,
                                 ctypes.byref(n)), ctx)
    return [arr[i] for i in range(n.value)]


def pps_server_create(desc: pps_server_desc):
    srv = c_void_p()
    _check(lib().pps_server_create(ctypes.byref(desc), ctypes.byref(srv)))
    return srv


def pps_server_destroy(srv) -> None:
    lib().pps_server_destroy(srv)


def pps_server_submit(srv, state_addr, job_addr) -> int:
    """Host addresses of one pps_state and one pps_job; returns the ticket."""
    t = ctypes.c_uint64()
    _check(lib().pps_server_submit(srv, state_addr, job_addr,
                                   ctypes.byref(t)))
    return t.value


def pps_server_wait(srv, ticket, timeout_us=-1, mask=None):
    r = pps_server_result()
    _check(lib().pps_server_wait(srv, ticket, timeout_us, ctypes.byref(r),
                                 None if mask is None else mask.ctypes.data))
    return r


def pps_server_replay(srv, frames, jobs, n_matches, frames_per_match, hz,
                      results=None):
    """frames: structured array of pps_state (match-major); jobs: ctypes
    array of n_matches pps_job; results: structured array or None."""
    st = pps_server_stats()
    _check(lib().pps_server_replay(
        srv, frames.ctypes.data, ctypes.addressof(jobs), n_matches,
        frames_per_match, hz,
        None if results is None else results.ctypes.data, ctypes.byref(st)))
    return st


def pps_server_get_stats(srv):
    st = pps_server_stats()
    _check(lib().pps_server_get_stats(srv, ctypes.byref(st)))
    return st


RESULT_DTYPE = np.dtype([("best", BEST_DTYPE), ("ticket", "<u8"),
                         ("latency_ns", "<i8"), ("queue_ns", "<i8"),
                         ("batch_size", "<i4"), ("status", "<i4")])


def pps_net_create(device=0, stream=None, max_batch=256):
    net = c_void_p()
    _check(lib().pps_net_create(device, stream, max_batch, ctypes.byref(net)))
    return net


def pps_net_destroy(net) -> None:
    lib().pps_net_destroy(net)


def pps_net_set_features(net, speeds, params=None) -> int:
    sp = np.ascontiguousarray(np.asarray(speeds, np.float32))
    prm = params if params is None or isinstance(params, pps_params) else \
        params_from_dict(params)
    return _check(lib().pps_net_set_features(
        net, sp.ctypes.data, len(sp),
        ctypes.byref(prm) if prm is not None else None))


def pps_net_sync(net) -> int:
    return _check(lib().pps_net_sync(net))


def pps_net_selftest_timeout(net, states, n) -> int:
    """Status of the bounded-wait self-test (PPS_ETIMEOUT expected)."""
    return lib().pps_net_selftest_timeout(net, states, n)


def pps_net_set_loss(net, top_band=float("inf"), low_weight=1.0,
                     under_weight=1.0) -> int:
    return _check(lib().pps_net_set_loss(net, top_band, low_weight,
                                         under_weight))


def pps_net_set_weights(net, w) -> int:
    w = np.ascontiguousarray(np.asarray(w, np.float32))
    assert w.size == PPS_NET_PARAMS
    return _check(lib().pps_net_set_weights(net, w.ctypes.data))


def pps_net_get_weights(net) -> np.ndarray:
    w = np.zeros(PPS_NET_PARAMS, np.float32)
    _check(lib().pps_net_get_weights(net, w.ctypes.data))
    return w


def pps_net_raster(net, states, n, out) -> int:
    return _check(lib().pps_net_raster(net, states, n, out))


def pps_net_forward(net, states, n, out) -> int:
    return _check(lib().pps_net_forward(net, states, n, out))


def pps_net_forward_layers(net, states, n, out) -> int:
    return _check(lib().pps_net_forward_layers(net, states, n, out))


def pps_net_forward_map(net, maps, n, layers, out) -> int:
    """Device addresses: maps (n x 46 x 61 x 8 bf16 bits), out."""
    return _check(lib().pps_net_forward_map(net, maps, n, int(layers), out))


def pps_net_grad(net, states, labels, n):
    g = np.zeros(PPS_NET_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().pps_net_grad(net, states, labels, n, g.ctypes.data,
                              ctypes.byref(loss)))
    return loss.value, g


def pps_net_grad_map(net, maps, labels, n):
    g = np.zeros(PPS_NET_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().pps_net_grad_map(net, maps, labels, n, g.ctypes.data,
                                  ctypes.byref(loss)))
    return loss.value, g


PPS_NET_TRAIN_TCGEN05 = 0
PPS_NET_TRAIN_MMA_SYNC = 1


def pps_net_set_train_kernels(net, kind) -> int:
    return _check(lib().pps_net_set_train_kernels(net, int(kind)))


def pps_net_train_step(net, states, labels, n, lr, want_loss=True):
    loss = ctypes.c_float()
    _check(lib().pps_net_train_step(net, states, labels, n, lr,
                                    ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def pps_net_labels(net, point_best, n, floor_value, labels) -> int:
    return _check(lib().pps_net_labels(net, point_best, n, floor_value,
                                       labels))


def pps_net_labels_grid(net, point_best, n, fine_grid, floor_value,
                        labels) -> int:
    return _check(lib().pps_net_labels_grid(net, point_best, n,
                                            ctypes.byref(fine_grid),
                                            floor_value, labels))


def pps_propose_jobs(ctx, net, states, jobs, n, spacing, max_speeds, params,
                     topk, flags, out_best, out_cells=None) -> int:
    """Device addresses for states, jobs, out_best, out_cells."""
    return _check(lib().pps_propose_jobs(
        ctx, net, states, jobs, n, spacing, max_speeds,
        ctypes.byref(params) if params is not None else None, topk, flags,
        out_best, out_cells), ctx)


def pps_propose(ctx, net, states, n, fine_grid, speeds, params, topk, flags,
                out_best, out_cells=None) -> int:
    """Device addresses for states, out_best, out_cells; speeds host."""
    sp = np.ascontiguousarray(np.asarray(speeds, np.float32))
    return _check(lib().pps_propose(
        ctx, net, states, n, ctypes.byref(fine_grid), sp.ctypes.data, len(sp),
        ctypes.byref(params) if params is not None else None, topk, flags,
        out_best, out_cells), ctx)


def pps_dpps_default_params() -> pps_dparams:
    p = pps_dparams()
    _check(lib().pps_dpps_default_params(ctypes.byref(p)))
    return p


def pps_dpps_mask_words(params: pps_dparams) -> int:
    return int(lib().pps_dpps_mask_words(ctypes.byref(params)))


def pps_dpps_search(ctx, states, n_states, params, out_best, out_mask=None,
                    out_dbg=None):
    """Device addresses for states, out_best, out_mask and out_dbg."""
    return _check(lib().pps_dpps_search(
        ctx, states, n_states,
        ctypes.byref(params) if params is not None else None, out_best,
        out_mask, out_dbg), ctx)


def pps_pass_powers(ctx, states, n_states, queries, n_queries, buffer,
                    params, out):
    """Device addresses for states, queries and out."""
    return _check(lib().pps_pass_powers(
        ctx, states, n_states, queries, n_queries, buffer,
        ctypes.byref(params) if params is not None else None, out), ctx)


def pps_shoot(ctx, states, n_states, queries, n_queries, v_shot, theta_min,
              params, out):
    """Device addresses for states, queries and out."""
    return _check(lib().pps_shoot(
        ctx, states, n_states, queries, n_queries, v_shot, theta_min,
        ctypes.byref(params) if params is not None else None, out), ctx)


def pps_run_default_params() -> pps_rparams:
    p = pps_rparams()
    _check(lib().pps_run_default_params(ctypes.byref(p)))
    return p


def pps_run_grid(field_len, field_wid, spacing):
    """(nx, ny) of the running-point grid of a field."""
    nx, ny = ctypes.c_int(), ctypes.c_int()
    _check(lib().pps_run_grid(field_len, field_wid, spacing,
                              ctypes.byref(nx), ctypes.byref(ny)))
    return nx.value, ny.value


def pps_run_points(ctx, states, n_states, params, out, pass_best=None,
                   out_scores=None, score_stride=0):
    """Device addresses for states, pass_best, out and out_scores."""
    return _check(lib().pps_run_points(
        ctx, states, n_states,
        ctypes.byref(params) if params is not None else None, pass_best, out,
        out_scores, score_stride), ctx)


def rparams_from_dict(d: dict | None) -> pps_rparams:
    p = pps_run_default_params()
    for k, v in (d or {}).items():
        setattr(p, k, int(v) if k == "n_run" else float(v))
    return p


def dparams_from_dict(d: dict | None) -> pps_dparams:
    p = pps_dpps_default_params()
    for k, v in (d or {}).items():
        setattr(p, k, int(v) if k in ("n_dir", "n_pow") else float(v))
    return p


def pack_dstates(batch: dict) -> np.ndarray:
    """A batch with teammates (team_pos, team_vel) -> pps_dstate records."""
    S = batch["ball"].shape[0]
    out = np.zeros(S, DSTATE_DTYPE)
    out["ball"] = batch["ball"]
    nt, no = batch["team_pos"].shape[1], batch["opp_pos"].shape[1]
    if nt > PPS_MAX_TEAM or no > PPS_MAX_OPP:
        raise ValueError("more robots than PPS_MAX_TEAM / PPS_MAX_OPP")
    out["n_team"] = batch.get("n_team", np.full(S, nt))
    out["n_opp"] = batch["n_opp"]
    out["team_pos"][:, :nt] = batch["team_pos"]
    out["team_vel"][:, :nt] = batch["team_vel"]
    out["opp_pos"][:, :no] = batch["opp_pos"]
    out["opp_vel"][:, :no] = batch["opp_vel"]
    for k in ("ball_decel", "vmax", "amax", "field_len", "field_wid",
              "goal_width", "K"):
        out[k] = batch[k]
    return out


def pps_sync(ctx) -> int:
    return _check(lib().pps_sync(ctx), ctx)


def pps_reset(ctx) -> int:
    return _check(lib().pps_reset(ctx), ctx)


def pps_launch_info(ctx):
    n, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().pps_launch_info(ctx, ctypes.byref(n), ctypes.byref(c)), ctx)
    return n.value, c.value


# ------------------------------------------------------------- marshalling
def params_from_dict(d: dict | None) -> pps_params:
    p = pps_default_params()
    for k, v in (d or {}).items():
        setattr(p, k, float(v))
    return p


def pack_states(batch: dict) -> np.ndarray:
    """A synth batch -> structured array of pps_state records."""
    S = batch["ball"].shape[0]
    out = np.zeros(S, STATE_DTYPE)
    out["ball"] = batch["ball"]
    out["n_opp"] = batch["n_opp"]
    J = batch["opp_pos"].shape[1]
    if J > PPS_MAX_OPP:
        raise ValueError("more opponent slots than PPS_MAX_OPP")
    out["opp_pos"][:, :J] = batch["opp_pos"]
    out["opp_vel"][:, :J] = batch["opp_vel"]
    for k in ("ball_decel", "vmax", "amax", "field_len", "field_wid",
              "goal_width", "K"):
        out[k] = batch[k]
    return out


def unpack_best(raw: np.ndarray) -> np.ndarray:
    """uint8 bytes of pps_best records -> structured array."""
    return np.frombuffer(np.ascontiguousarray(raw).tobytes(), BEST_DTYPE)


class Searcher:
    """A libpps context plus torch buffers.

    ``search`` takes device tensors (uint8 view of pps_state records, see
    ``states_to_device``) and returns device tensors; ``search_host`` takes
    and returns host numpy/pinned buffers through the library's own staging.
    """

    def __init__(self, max_states, max_opp=8, device=0, stream=None,
                 mem_budget_bytes=0, max_K=0, max_points=0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else \
            torch.cuda.current_stream(self.device)
        desc = pps_ctx_desc(max_states=max_states, device=device,
                            stream=self.stream.cuda_stream,
                            mem_budget_bytes=mem_budget_bytes,
                            max_opp=max_opp, max_K=max_K,
                            max_points=max_points)
        self.ctx = pps_create(desc)

    def close(self):
        if self.ctx is not None:
            pps_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def states_to_device(self, batch: dict):
        rec = pack_states(batch)
        t = self.torch.from_numpy(rec.view(np.uint8).reshape(-1).copy())
        return t.to(self.device)

    def alloc_outputs(self, n_states, grid, n_speeds, mask=True, debug=False,
                      T_stride=0):
        torch = self.torch
        out = {"best": torch.empty(n_states * 32, dtype=torch.uint8,
                                   device=self.device)}
        if mask:
            out["mask"] = torch.empty(
                n_states * pps_mask_words(grid, n_speeds), dtype=torch.int32,
                device=self.device)
        if debug:
            P = grid.nx * grid.ny
            out["margin"] = torch.empty((n_states, n_speeds, P),
                                        dtype=torch.float32, device=self.device)
            out["score"] = torch.empty_like(out["margin"])
            if T_stride:
                out["T"] = torch.empty((n_states, P, T_stride),
                                       dtype=torch.float32, device=self.device)
        return out

    def search(self, states_dev, n_states, grid, speeds, params=None,
               out=None, mask=True, debug=False, T_stride=0,
               point_best=None):
        """Enqueue the search on the context's stream (device buffers).
        ``point_best``: optional float32 device tensor of n_states x P that
        receives every point's best score over the speeds."""
        sp = np.ascontiguousarray(np.asarray(speeds, np.float32))
        if out is None:
            out = self.alloc_outputs(n_states, grid, len(sp), mask, debug,
                                     T_stride)
        dbg = None
        if "margin" in out or "T" in out or point_best is not None:
            dbg = pps_debug_out(
                out["margin"].data_ptr() if "margin" in out else None,
                out["score"].data_ptr() if "score" in out else None,
                out["T"].data_ptr() if "T" in out else None,
                out["T"].shape[2] if "T" in out else 0,
                point_best.data_ptr() if point_best is not None else None)
        prm = params if isinstance(params, pps_params) else \
            params_from_dict(params)
        pps_search(self.ctx, states_dev.data_ptr(), n_states, grid,
                   sp.ctypes.data, len(sp), prm, out["best"].data_ptr(),
                   out["mask"].data_ptr() if "mask" in out else None, dbg,
                   PPS_DEVICE_PTRS)
        return out

    def search_host(self, states_np, grid, speeds, params, best_np,
                    mask_np=None):
        """Host buffers (numpy; pinned for async copies): enqueue only."""
        sp = np.ascontiguousarray(np.asarray(speeds, np.float32))
        prm = params if isinstance(params, pps_params) else \
            params_from_dict(params)
        pps_search(self.ctx, states_np.ctypes.data, states_np.shape[0], grid,
                   sp.ctypes.data, len(sp), prm, best_np.ctypes.data,
                   None if mask_np is None else mask_np.ctypes.data, None, 0)

    def sync(self):
        pps_sync(self.ctx)

    @staticmethod
    def best_numpy(best_dev) -> np.ndarray:
        return unpack_best(best_dev.cpu().numpy())


def jobs_from_batch(batch: dict):
    """pps_job records of a batch with per-state shapes (see
    synth.uneven_batch): the grid of each state's field at its spacing."""
    S = batch["ball"].shape[0]
    jobs = (pps_job * S)()
    for i in range(S):
        g = pps_grid_from_field(float(batch["field_len"][i]),
                                float(batch["field_wid"][i]),
                                float(batch["spacing"][i]))
        jobs[i].grid = g
        n = int(batch["n_speeds"][i])
        jobs[i].n_speeds = n
        for v in range(n):
            jobs[i].speeds[v] = float(batch["speeds"][i][v])
        jobs[i].max_opp = int(batch["n_opp"][i])
    return jobs


def jobs_to_bytes(jobs) -> np.ndarray:
    """The raw bytes of a ctypes array of pps_job (for a device copy)."""
    return np.frombuffer(bytes(jobs), np.uint8).copy()


def field_jobs(batch: dict, spacing: float, speeds) -> "ctypes.Array":
    """One pps_job per state of a batch: its own field's grid at `spacing`
    (pps_grid_from_field) and the shared kick speeds."""
    S = batch["ball"].shape[0]
    jobs = (pps_job * S)()
    for i in range(S):
        jobs[i].grid = pps_grid_from_field(float(batch["field_len"][i]),
                                           float(batch["field_wid"][i]),
                                           spacing)
        jobs[i].n_speeds = len(speeds)
        for v, x in enumerate(speeds):
            jobs[i].speeds[v] = float(x)
        jobs[i].max_opp = int(batch["n_opp"][i])
    return jobs


class Plan:
    """A batched plan on a Searcher's context, with device output buffers."""

    def __init__(self, searcher, jobs, n_states, params=None,
                 autotune=True, graph=True):
        self.s = searcher
        self.n = n_states
        self.jobs = jobs
        flags = (PPS_PLAN_AUTOTUNE if autotune else 0) | \
            (PPS_PLAN_GRAPH if graph else 0)
        prm = params if isinstance(params, pps_params) else \
            params_from_dict(params)
        self.plan = pps_plan_create(searcher.ctx, jobs, n_states, prm, flags)
        self.offsets = pps_plan_mask_offsets(self.plan, n_states, searcher.ctx)
        torch = searcher.torch
        self.best = torch.empty(n_states * 32, dtype=torch.uint8,
                                device=searcher.device)
        self.mask = torch.empty(max(1, int(self.offsets[-1])),
                                dtype=torch.int32, device=searcher.device)

    def run(self, states_dev, mask=True):
        pps_plan_run(self.plan, states_dev.data_ptr(), self.best.data_ptr(),
                     self.mask.data_ptr() if mask else None, self.s.ctx)

    def groups(self):
        return pps_plan_groups(self.plan, self.s.ctx)

    def close(self):
        if self.plan is not None:
            pps_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match_jobs(batch: dict):
    """One pps_job per match of a synth.serving_matches batch."""
    M, F = batch["n_matches"], batch["n_frames"]
    first = {k: v[::F] for k, v in batch.items()
             if isinstance(v, np.ndarray)}
    return jobs_from_batch(first)


class Net:
    """The proposal network (weights on the device) with torch buffers."""

    def __init__(self, device=0, stream=None, max_batch=256, weights=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        st = stream if stream is not None else torch.cuda.current_stream(
            self.device)
        self.max_batch = max_batch
        self.net = pps_net_create(device, st.cuda_stream, max_batch)
        if weights is not None:
            pps_net_set_weights(self.net, weights)

    def forward(self, states_dev, n):
        out = self.torch.empty((n, PPS_NET_H, PPS_NET_W),
                               dtype=self.torch.float32, device=self.device)
        pps_net_forward(self.net, states_dev.data_ptr(), n, out.data_ptr())
        return out

    def close(self):
        if self.net is not None:
            pps_net_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fine_grid_12x9():
    """The 0.025 m grid of the 12 x 9 m field the proposal refines on."""
    return pps_grid_from_field(12.0, 9.0, 0.025)


def init_weights(seed: int, zero_output: bool = False) -> np.ndarray:
    """He-style random weights in the flat layout (biases zero).  With
    zero_output the last layer starts at zero, so that the network starts
    as its input's coarse score and training learns the correction."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in [(8, 32), (32, 32), (32, 32), (32, 1)]:
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), 9 * co * ci)
        out.append(w * 0.0 if zero_output and co == 1 else w)
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


# ------------------------------------------------------- proposal weights
WEIGHTS_DIR = os.path.join(PKG, "weights")
# Weights trained by paper_1909_07717_gb300.train_proposal on exact labels
# of 12 x 9 m, 8-opponent states (kick speeds 2, 3.5, 5, 6.5 m/s, K = 64).
PROPOSAL_WEIGHTS = os.path.join(WEIGHTS_DIR, "proposal_12x9_v4_K64_J8.bin")
# the serving workload's network: 12 x 9 and 9 x 6 m fields at 0.05 m
SERVING_WEIGHTS = os.path.join(WEIGHTS_DIR, "proposal_serving_g0.05_K32.bin")
_WMAGIC = b"PPSNET\x00\x01"


def save_net_weights(path: str, w) -> None:
    """Flat float32 weights -> file: 8-byte magic, uint32 count, uint32
    CRC-32 of the data, then the little-endian float32 values."""
    import zlib
    w = np.ascontiguousarray(np.asarray(w, "<f4"))
    if w.size != PPS_NET_PARAMS or not np.all(np.isfinite(w)):
        raise ValueError("weights must be PPS_NET_PARAMS finite values")
    data = w.tobytes()
    hdr = _WMAGIC + np.array([w.size, zlib.crc32(data)], "<u4").tobytes()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(hdr + data)
    os.replace(tmp, path)


def load_net_weights(path: str = PROPOSAL_WEIGHTS) -> np.ndarray:
    """Inverse of save_net_weights; raises on a bad magic, size or CRC."""
    import zlib
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != _WMAGIC or len(raw) < 16:
        raise ValueError(f"{path}: not a proposal weight file")
    n, crc = np.frombuffer(raw[8:16], "<u4")
    data = raw[16:]
    if n != PPS_NET_PARAMS or len(data) != 4 * n:
        raise ValueError(f"{path}: expected {PPS_NET_PARAMS} weights")
    if zlib.crc32(data) != crc:
        raise ValueError(f"{path}: checksum mismatch")
    return np.frombuffer(data, "<f4").astype(np.float32)
