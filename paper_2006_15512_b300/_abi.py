"""ctypes declarations of the C ABI in include/wmc.h (argument marshalling
only).  Importing this module loads the in-tree CUDA library and fails
loudly if it has not been built: there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwmc_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_2006_15512_b300/build.py)")

lib = ctypes.CDLL(LIB_PATH)

WMC_OK = 0
WMC_PENDING = 1
WMC_EINVAL = -1
WMC_ENOMEM = -2
WMC_EPLAN_TOO_BIG = -3
WMC_ECUDA = -4
WMC_ETIMEOUT = -5
WMC_EUNKNOWN_TICKET = -6
WMC_ESHUTDOWN = -7

WMC_FP64 = 0
WMC_SCALED_FP32 = 1

WMC_ORDER_BEST = 0
WMC_ORDER_MINFILL = 1
WMC_ORDER_MINDEGREE = 2
WMC_ORDER_SWEEP = 3
WMC_ORDER_GIVEN = 4

WMC_FLAG_EXACT_INT = 0x1
WMC_FLAG_FP32_FLUSH = 0x2
WMC_FLAG_NO_BOUND = 0x4
WMC_FLAG_DEVICE_TIMEOUT = 0x8
WMC_FLAG_FELL_BACK_FP64 = 0x10

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_u32 = ctypes.c_uint32
c_u64 = ctypes.c_uint64
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p
c_size = ctypes.c_size_t
P = ctypes.POINTER


class wmc_result(ctypes.Structure):
    _fields_ = [("mant", c_dbl), ("exp2", c_i64), ("log10", c_dbl), ("flags", c_u32),
                ("reserved", c_u32), ("rel_err_bound", c_dbl)]


class wmc_network_info_t(ctypes.Structure):
    _fields_ = [("n_vars", c_i64), ("n_clauses_kept", c_i64), ("n_tensors_strict", c_i64),
                ("n_indices_strict", c_i64), ("max_clause_rank", c_i64),
                ("has_empty_clause", c_i32), ("reserved", c_i32)]


class wmc_plan_opts(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("ordering", c_i32), ("max_rank_cap", c_i32),
                ("slice_to_rank", c_i32), ("mem_budget_bytes", c_i64), ("order", P(c_i32)),
                ("factor_clauses_above", c_i32), ("block_fp", c_i32)]


class wmc_plan_info_t(ctypes.Structure):
    _fields_ = [("max_rank", c_i32), ("max_node_rank", c_i32), ("n_leaves", c_i64),
                ("n_nodes", c_i64), ("workspace_bytes", c_i64), ("peak_tensor_bytes", c_i64),
                ("algorithmic_bytes", c_dbl), ("flops", c_dbl), ("precision", c_i32),
                ("ordering_used", c_i32), ("max_path_roundings", c_i32), ("launches_per_walk", c_i32),
                ("n_slice_vars", c_i32), ("slice_vars", c_i32 * 24), ("n_aux_vars", c_i32),
                ("reserved", c_i32)]


class wmc_server_opts(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("max_batch", c_i32), ("max_waves", c_i32),
                ("partial_overlap", c_i32), ("arena_bytes", c_i64), ("max_wave_wait_us", c_i64)]


class wmc_batch_info_t(ctypes.Structure):
    _fields_ = [("n_formulas", c_i64), ("n_nodes", c_i64), ("n_tasks", c_i64),
                ("workspace_bytes", c_i64), ("algorithmic_bytes", c_dbl), ("max_rank", c_i32),
                ("grid", c_i32)]


class wmc_tune_report(ctypes.Structure):
    _fields_ = [("n_candidates", c_i32), ("chosen", c_i32), ("fuse", c_i32 * 8), ("small_phase", c_i32 * 8),
                ("chain_runs", c_i32 * 8), ("launches", c_i32 * 8), ("ms", ctypes.c_float * 8)]


class wmc_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("completed", c_i64), ("waves", c_i64),
                ("failed_waves", c_i64), ("mean_wave_q", c_dbl), ("max_in_flight", c_i64)]


def _decl(name, restype, argtypes):
    f = getattr(lib, name)
    f.restype = restype
    f.argtypes = argtypes
    globals()[name] = f
    return f


EXPORTS = {
    "wmc_network_create": (c_i32, [c_i32, c_i64, P(c_i32), P(c_i64), P(c_dbl), P(c_dbl), P(c_vp)]),
    "wmc_network_destroy": (None, [c_vp]),
    "wmc_network_info": (c_i32, [c_vp, P(wmc_network_info_t)]),
    "wmc_plan": (c_i32, [c_vp, P(wmc_plan_opts), P(c_vp)]),
    "wmc_plan_destroy": (None, [c_vp]),
    "wmc_plan_info": (c_i32, [c_vp, c_i32, P(wmc_plan_info_t)]),
    "wmc_plan_node": (c_i32, [c_vp, c_i64, P(c_i64), P(c_i64), P(c_i32), P(c_i32)]),
    "wmc_plan_leaf": (c_i32, [c_vp, c_i64, P(c_i32), P(c_i32), P(c_i32), P(c_u64)]),
    "wmc_execute": (c_i32, [c_vp, c_i32, P(c_dbl), P(c_dbl), c_vp, P(wmc_result)]),
    "wmc_execute_slices": (c_i32, [c_vp, c_i32, P(c_dbl), P(c_dbl), c_i64, c_i64, c_vp, P(wmc_result)]),
    "wmc_combine_results": (c_i32, [P(wmc_result), c_i64, P(wmc_result)]),
    "wmc_execute_device": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_size, c_vp, c_vp, c_vp, c_vp]),
    "wmc_execute_device_noalloc": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "wmc_contract_pair": (c_i32, [c_i32, c_i32, P(c_i32), c_vp, c_i32, P(c_i32), c_vp, c_i32,
                                  P(c_i32), c_vp, c_vp, c_vp, c_vp, c_vp]),
    "wmc_to_scaled_fp32": (c_i32, [c_vp, c_i64, c_vp, c_vp, c_vp]),
    "wmc_set_autotune": (None, [c_i32]),
    "wmc_autotune_plan": (c_i32, [c_vp, c_i32, c_vp, P(wmc_tune_report)]),
    "wmc_pair_variants": (c_i32, [c_i32, c_i32, P(c_i32), c_i32, P(c_i32), c_i32, P(c_i32), c_i32, c_i32,
                                  P(c_i32), P(c_i64), P(c_i32), P(c_i32)]),
    "wmc_debug_force_pair_variant": (None, [c_i32, c_i64]),
    "wmc_batch_create": (c_i32, [P(c_vp), c_i32, c_i64, P(c_vp), P(c_i32)]),
    "wmc_batch_info": (c_i32, [c_vp, P(wmc_batch_info_t)]),
    "wmc_batch_execute": (c_i32, [c_vp, c_vp, P(wmc_result)]),
    "wmc_batch_formula_info": (c_i32, [c_vp, c_i32, P(c_i64), P(c_i32), P(c_i64)]),
    "wmc_batch_destroy": (None, [c_vp]),
    "wmc_server_create": (c_i32, [c_vp, P(wmc_server_opts), P(c_vp)]),
    "wmc_submit": (c_i32, [c_vp, P(c_dbl), P(c_dbl), P(c_u64)]),
    "wmc_submit_many": (c_i32, [c_vp, c_i64, P(c_dbl), P(c_dbl), P(c_u64)]),
    "wmc_poll": (c_i32, [c_vp, c_u64, P(wmc_result)]),
    "wmc_wait": (c_i32, [c_vp, c_u64, c_i64, P(wmc_result)]),
    "wmc_poll_ex": (c_i32, [c_vp, c_u64, P(wmc_result), P(c_i64)]),
    "wmc_profile_walk": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_size, c_vp, c_vp, c_vp, c_vp,
                                 c_i64, P(ctypes.c_float), P(c_i32), P(c_dbl), P(c_i64)]),
    "wmc_server_stats": (c_i32, [c_vp, P(wmc_server_stats_t)]),
    "wmc_server_destroy": (None, [c_vp]),
    "wmc_last_error": (ctypes.c_char_p, []),
    "wmc_kernel_launch_count": (c_i64, []),
    "wmc_debug_fail_next_allocs": (None, [c_i32]),
    "wmc_debug_stall_copies": (None, [c_i32]),
    "wmc_debug_check_bounds": (c_i32, [c_vp, c_i32, P(c_i64)]),
    "wmc_set_fusion": (None, [c_i32]),
    "wmc_set_small_phase": (None, [c_i32]),
    "wmc_set_dependent_launch": (None, [c_i32]),
    "wmc_set_tensor_cores": (None, [c_i32]),
    "wmc_set_outer_products": (None, [c_i32]),
    "wmc_set_batched_pairs": (None, [c_i32]),
    "wmc_set_fp64_fallback": (None, [c_i32]),
    "wmc_set_chain_runs": (None, [c_i32]),
    "wmc_set_cta_walk": (None, [c_i32]),
    "wmc_set_batch_schedule": (None, [c_i32, c_i32]),
    "wmc_set_batch_fusion": (None, [c_i32]),
    "wmc_set_batch_subtrees": (None, [c_i32]),
}

for _name, (_res, _args) in EXPORTS.items():
    _decl(_name, _res, _args)


class WmcError(RuntimeError):
    def __init__(self, status, where):
        msg = lib.wmc_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def check(status, where):
    if status < 0:
        raise WmcError(status, where)
    return status
