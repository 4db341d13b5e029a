"""B300 execution stage for tensor-network weighted model counting
(Dudek & Vardi, "Parallel Weighted Model Counting with Tensor Networks").

A thin Python binding of the C ABI in include/wmc.h: every function below
only marshals arguments (numpy arrays, torch tensors' device pointers,
integer stream handles) into one C call.  All work runs in the CUDA library
libwmc_b300.so; importing this package fails if that library is missing.

Raw ABI functions keep their C names (``wmc_network_create``, ``wmc_plan``,
``wmc_execute``, ``wmc_execute_device``, ``wmc_contract_pair``,
``wmc_submit``, ``wmc_poll`` ...); the classes are small owners of the
opaque handles.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import _abi
from ._abi import *  # noqa: F401,F403  (the C names)
from ._abi import check, lib

__all__ = ["Network", "Plan", "Server", "Batch", "Result", "contract_pair", "to_scaled_fp32",
           "launch_count", "slice_range", "combine_results", "pair_variants", "PAIR_KINDS"] + list(_abi.EXPORTS)

P = ctypes.POINTER


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(P(ct))


@dataclass(frozen=True)
class Result:
    """value = mant * 2**exp2 (Def. 2.1's W(phi))."""
    mant: float
    exp2: int
    log10: float
    flags: int
    rel_err_bound: float

    @staticmethod
    def from_c(r: _abi.wmc_result) -> "Result":
        return Result(r.mant, int(r.exp2), r.log10, int(r.flags), r.rel_err_bound)

    def to_float(self) -> float:
        return math.ldexp(self.mant, self.exp2) if self.mant != 0 else 0.0


def launch_count() -> int:
    return int(lib.wmc_kernel_launch_count())


def slice_range(n_slices: int, rank: int, world: int):
    """Index slicing across processes (Alg. 3 with one share of the slices
    per process): the contiguous range [lo, hi) of slice assignments that
    process `rank` of `world` runs; the ranges cover [0, n_slices) once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return n_slices * rank // world, n_slices * (rank + 1) // world


def combine_results(parts: Sequence[Result]) -> Result:
    """wmc_combine_results: the sum of partial results mant * 2**exp2 (e.g.
    the slice shares of several processes, Thm 4.2), computed in the C
    library."""
    parts = list(parts)
    arr = (_abi.wmc_result * max(len(parts), 1))()
    for i, r in enumerate(parts):
        arr[i].mant, arr[i].exp2, arr[i].log10 = r.mant, r.exp2, r.log10
        arr[i].flags, arr[i].rel_err_bound = r.flags, r.rel_err_bound
    out = _abi.wmc_result()
    check(lib.wmc_combine_results(arr, len(parts), ctypes.byref(out)), "wmc_combine_results")
    return Result.from_c(out)


class Network:
    """Reduction of Thm 3.2: owns a wmc_network_t."""

    def __init__(self, n_vars: int, lits: np.ndarray, clause_off: np.ndarray,
                 w_pos: Optional[np.ndarray] = None, w_neg: Optional[np.ndarray] = None):
        lits = np.ascontiguousarray(lits, dtype=np.int32)
        off = np.ascontiguousarray(clause_off, dtype=np.int64)
        n_clauses = int(off.size) - 1
        if lits.size == 0:
            lits = np.zeros(1, dtype=np.int32)
        wp = wn = None
        if w_pos is not None:
            wp = np.ascontiguousarray(w_pos, dtype=np.float64)
            wn = np.ascontiguousarray(w_neg, dtype=np.float64)
        h = ctypes.c_void_p()
        check(lib.wmc_network_create(int(n_vars), n_clauses, _ptr(lits, ctypes.c_int32),
                                     _ptr(off, ctypes.c_int64),
                                     _ptr(wp, ctypes.c_double) if wp is not None else None,
                                     _ptr(wn, ctypes.c_double) if wn is not None else None,
                                     ctypes.byref(h)), "wmc_network_create")
        self.handle = h
        self.n_vars = int(n_vars)

    @classmethod
    def from_cnf(cls, cnf, w_pos=None, w_neg=None) -> "Network":
        lits, off = cnf.flat()
        return cls(cnf.n_vars, lits, off, w_pos, w_neg)

    def info(self) -> _abi.wmc_network_info_t:
        out = _abi.wmc_network_info_t()
        check(lib.wmc_network_info(self.handle, ctypes.byref(out)), "wmc_network_info")
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            lib.wmc_network_destroy(self.handle)
            self.handle = None


class Plan:
    """Planning stage (Sec. 3.3): owns a wmc_plan_t."""

    def __init__(self, net: Network, precision: int = _abi.WMC_SCALED_FP32,
                 ordering: int = _abi.WMC_ORDER_BEST, max_rank_cap: int = 0,
                 mem_budget_bytes: int = 0, order: Optional[Sequence[int]] = None,
                 slice_to_rank: int = 0, factor_clauses_above: int = 0, block_fp: int = 0):
        o = _abi.wmc_plan_opts()
        o.block_fp = block_fp
        o.precision = precision
        o.ordering = ordering
        o.max_rank_cap = max_rank_cap
        o.slice_to_rank = slice_to_rank
        o.factor_clauses_above = factor_clauses_above
        o.mem_budget_bytes = mem_budget_bytes
        self._order = None
        if order is not None:
            self._order = np.ascontiguousarray(order, dtype=np.int32)
            o.order = _ptr(self._order, ctypes.c_int32)
            o.ordering = _abi.WMC_ORDER_GIVEN
        h = ctypes.c_void_p()
        check(lib.wmc_plan(net.handle, ctypes.byref(o), ctypes.byref(h)), "wmc_plan")
        self.handle = h
        self.net = net
        self.n_vars = net.n_vars
        self.precision = precision

    def info(self, Q: int = 1) -> _abi.wmc_plan_info_t:
        out = _abi.wmc_plan_info_t()
        check(lib.wmc_plan_info(self.handle, int(Q), ctypes.byref(out)), "wmc_plan_info")
        return out

    def nodes(self):
        """[(left, right, labels)] in post-order (tensor ids: leaves first)."""
        n = self.info(1).n_nodes
        res = []
        lab = (ctypes.c_int32 * 64)()
        for i in range(n):
            l = ctypes.c_int64(); r = ctypes.c_int64(); k = ctypes.c_int32()
            check(lib.wmc_plan_node(self.handle, i, ctypes.byref(l), ctypes.byref(r), ctypes.byref(k), lab),
                  "wmc_plan_node")
            res.append((l.value, r.value, [lab[j] for j in range(k.value)]))
        return res

    def leaves(self):
        """[(kind, labels, fals)] for every leaf id."""
        n = self.info(1).n_leaves
        res = []
        lab = (ctypes.c_int32 * 64)()
        for i in range(n):
            kind = ctypes.c_int32(); k = ctypes.c_int32(); f = ctypes.c_uint64()
            check(lib.wmc_plan_leaf(self.handle, i, ctypes.byref(kind), ctypes.byref(k), lab,
                                    ctypes.byref(f)), "wmc_plan_leaf")
            res.append((kind.value, [lab[j] for j in range(k.value)], f.value))
        return res

    def execute(self, w_pos_q: Optional[np.ndarray] = None, w_neg_q: Optional[np.ndarray] = None,
                Q: Optional[int] = None, stream: int = 0) -> List[Result]:
        """wmc_execute with host buffers ([Q][n_vars] float64 each, or None
        for the network's default weights)."""
        if w_pos_q is not None:
            wp = np.ascontiguousarray(w_pos_q, dtype=np.float64).reshape(-1, max(self.n_vars, 1) if self.n_vars else 1)
            wn = np.ascontiguousarray(w_neg_q, dtype=np.float64).reshape(wp.shape)
            Q = wp.shape[0] if self.n_vars else (Q or 1)
            pw, nw = _ptr(wp, ctypes.c_double), _ptr(wn, ctypes.c_double)
        else:
            Q = Q or 1
            pw = nw = None
        out = (_abi.wmc_result * Q)()
        check(lib.wmc_execute(self.handle, int(Q), pw, nw, ctypes.c_void_p(stream), out), "wmc_execute")
        return [Result.from_c(out[i]) for i in range(Q)]

    @property
    def slice_vars(self) -> List[int]:
        i = self.info(1)
        return [int(i.slice_vars[k]) for k in range(i.n_slice_vars)]

    def execute_slices(self, slice_lo: int, slice_hi: int, w_pos_q: Optional[np.ndarray] = None,
                       w_neg_q: Optional[np.ndarray] = None, Q: Optional[int] = None,
                       stream: int = 0) -> List[Result]:
        """wmc_execute_slices: the partial sum over slice assignments
        [slice_lo, slice_hi) of a sliced plan."""
        if w_pos_q is not None:
            wp = np.ascontiguousarray(w_pos_q, dtype=np.float64).reshape(-1, max(self.n_vars, 1))
            wn = np.ascontiguousarray(w_neg_q, dtype=np.float64).reshape(wp.shape)
            Q = wp.shape[0]
            pw, nw = _ptr(wp, ctypes.c_double), _ptr(wn, ctypes.c_double)
        else:
            Q = Q or 1
            pw = nw = None
        out = (_abi.wmc_result * Q)()
        check(lib.wmc_execute_slices(self.handle, int(Q), pw, nw, ctypes.c_int64(slice_lo),
                                     ctypes.c_int64(slice_hi), ctypes.c_void_p(stream), out),
              "wmc_execute_slices")
        return [Result.from_c(out[i]) for i in range(Q)]

    def autotune(self, Q: int, stream: int = 0) -> dict:
        """wmc_autotune_plan: time the walk's layouts for batch size Q and
        install the fastest; returns the report as a dict."""
        rep = _abi.wmc_tune_report()
        check(lib.wmc_autotune_plan(self.handle, int(Q), ctypes.c_void_p(stream), ctypes.byref(rep)),
              "wmc_autotune_plan")
        n = rep.n_candidates
        return {"chosen": rep.chosen,
                "layouts": [{"fuse": rep.fuse[i], "small_phase": rep.small_phase[i],
                             "chain_runs": rep.chain_runs[i], "launches": rep.launches[i],
                             "ms": rep.ms[i]} for i in range(n)]}

    def execute_device(self, Q: int, d_w_pos, d_w_neg, workspace, d_mant, d_exp2, d_flags,
                       stream: int = 0) -> None:
        """wmc_execute_device on torch tensors (or raw integer pointers)."""
        ws_ptr, ws_bytes = _dptr(workspace), _nbytes(workspace)
        check(lib.wmc_execute_device(self.handle, int(Q), _dptr(d_w_pos), _dptr(d_w_neg),
                                     ws_ptr, ws_bytes, _dptr(d_mant), _dptr(d_exp2),
                                     _dptr(d_flags), ctypes.c_void_p(stream)),
              "wmc_execute_device")

    def __del__(self):
        if getattr(self, "handle", None):
            lib.wmc_plan_destroy(self.handle)
            self.handle = None


def _dptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _nbytes(t):
    return int(t.numel() * t.element_size())


def contract_pair(precision: int, labels_a, a, labels_b, b, labels_c, c,
                  exp_a=None, exp_b=None, exp_c=None, stream: int = 0) -> None:
    """wmc_contract_pair on device tensors (see include/wmc.h)."""
    la = np.ascontiguousarray(labels_a, dtype=np.int32)
    lb = np.ascontiguousarray(labels_b, dtype=np.int32)
    lc = np.ascontiguousarray(labels_c, dtype=np.int32)
    pad = lambda x: x if x.size else np.zeros(1, dtype=np.int32)
    la_, lb_, lc_ = pad(la), pad(lb), pad(lc)
    check(lib.wmc_contract_pair(int(precision), la.size, _ptr(la_, ctypes.c_int32), _dptr(a),
                                lb.size, _ptr(lb_, ctypes.c_int32), _dptr(b),
                                lc.size, _ptr(lc_, ctypes.c_int32), _dptr(c),
                                _dptr(exp_a), _dptr(exp_b), _dptr(exp_c),
                                ctypes.c_void_p(stream)), "wmc_contract_pair")


PAIR_KINDS = {0: "k1_generic", 1: "k2_stream", 2: "k2_tma", 3: "k4_dense", 4: "k4_outer", 5: "k4_tc",
              6: "k4_dense split", 7: "k2_stream_s16q"}


def pair_variants(precision: int, labels_a, labels_b, labels_c, c_aligned16: bool = True):
    """wmc_pair_variants: ([(kind, blocks)], index of the current choice)."""
    la = np.ascontiguousarray(labels_a, dtype=np.int32)
    lb = np.ascontiguousarray(labels_b, dtype=np.int32)
    lc = np.ascontiguousarray(labels_c, dtype=np.int32)
    pad = lambda x: x if x.size else np.zeros(1, dtype=np.int32)
    la_, lb_, lc_ = pad(la), pad(lb), pad(lc)
    kinds = (ctypes.c_int32 * 32)()
    blocks = (ctypes.c_int64 * 32)()
    n = ctypes.c_int32(); chosen = ctypes.c_int32()
    check(lib.wmc_pair_variants(int(precision), la.size, _ptr(la_, ctypes.c_int32), lb.size,
                                _ptr(lb_, ctypes.c_int32), lc.size, _ptr(lc_, ctypes.c_int32),
                                int(bool(c_aligned16)), 32, kinds, blocks, ctypes.byref(n),
                                ctypes.byref(chosen)), "wmc_pair_variants")
    return [(int(kinds[i]), int(blocks[i])) for i in range(min(n.value, 32))], int(chosen.value)


def to_scaled_fp32(x, out, exp_out, stream: int = 0) -> None:
    check(lib.wmc_to_scaled_fp32(_dptr(x), int(x.numel()), _dptr(out), _dptr(exp_out),
                                 ctypes.c_void_p(stream)), "wmc_to_scaled_fp32")


class Batch:
    """Uneven batch of formulas in one persistent launch (wmc_batch_*)."""

    def __init__(self, plans, mem_budget_bytes: int = 0):
        arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
        h = ctypes.c_void_p()
        n = ctypes.c_int32()
        check(lib.wmc_batch_create(arr, len(plans), int(mem_budget_bytes), ctypes.byref(h),
                                   ctypes.byref(n)), "wmc_batch_create")
        self.handle = h
        self.plans = list(plans)[: n.value]
        self.n_admitted = n.value

    def info(self) -> _abi.wmc_batch_info_t:
        out = _abi.wmc_batch_info_t()
        check(lib.wmc_batch_info(self.handle, ctypes.byref(out)), "wmc_batch_info")
        return out

    def formula_info(self, i: int):
        """(workspace byte offset, max rank, node count) of admitted formula i."""
        off = ctypes.c_int64(); r = ctypes.c_int32(); n = ctypes.c_int64()
        check(lib.wmc_batch_formula_info(self.handle, int(i), ctypes.byref(off), ctypes.byref(r),
                                         ctypes.byref(n)), "wmc_batch_formula_info")
        return int(off.value), int(r.value), int(n.value)

    def execute(self, stream: int = 0) -> List[Result]:
        out = (_abi.wmc_result * self.n_admitted)()
        check(lib.wmc_batch_execute(self.handle, ctypes.c_void_p(stream), out), "wmc_batch_execute")
        return [Result.from_c(out[i]) for i in range(self.n_admitted)]

    def __del__(self):
        if getattr(self, "handle", None):
            lib.wmc_batch_destroy(self.handle)
            self.handle = None


class Server:
    """Continuous-batching server (wmc_server_create / wmc_submit /
    wmc_poll / wmc_wait)."""

    def __init__(self, plan: Plan, max_batch: int = 256, max_waves: int = 2,
                 arena_bytes: int = 0, max_wave_wait_us: int = 0, partial_overlap: int = 0):
        o = _abi.wmc_server_opts()
        o.precision = plan.precision
        o.max_batch = max_batch
        o.max_waves = max_waves
        o.partial_overlap = partial_overlap
        o.arena_bytes = arena_bytes
        o.max_wave_wait_us = max_wave_wait_us
        h = ctypes.c_void_p()
        check(lib.wmc_server_create(plan.handle, ctypes.byref(o), ctypes.byref(h)), "wmc_server_create")
        self.handle = h
        self.plan = plan
        self.n_vars = plan.n_vars

    def submit(self, w_pos, w_neg) -> int:
        wp = np.ascontiguousarray(w_pos, dtype=np.float64)
        wn = np.ascontiguousarray(w_neg, dtype=np.float64)
        if wp.size == 0:
            wp = np.zeros(1); wn = np.zeros(1)
        t = ctypes.c_uint64()
        check(lib.wmc_submit(self.handle, _ptr(wp, ctypes.c_double), _ptr(wn, ctypes.c_double),
                             ctypes.byref(t)), "wmc_submit")
        return int(t.value)

    def submit_many(self, w_pos, w_neg):
        """Queries as rows of [n][n_vars] arrays; returns their tickets."""
        wp = np.ascontiguousarray(w_pos, dtype=np.float64)
        wn = np.ascontiguousarray(w_neg, dtype=np.float64)
        n = int(wp.shape[0])
        if wp.shape != wn.shape or (self.n_vars and wp.shape[1] != self.n_vars):
            raise ValueError("w_pos, w_neg must both be [n][n_vars]")
        t = np.zeros(n, dtype=np.uint64)
        check(lib.wmc_submit_many(self.handle, ctypes.c_int64(n), _ptr(wp, ctypes.c_double),
                                  _ptr(wn, ctypes.c_double), _ptr(t, ctypes.c_uint64)), "wmc_submit_many")
        return [int(x) for x in t]

    def poll(self, ticket: int) -> Optional[Result]:
        r = _abi.wmc_result()
        rc = check(lib.wmc_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r)), "wmc_poll")
        return None if rc == _abi.WMC_PENDING else Result.from_c(r)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> Result:
        r = _abi.wmc_result()
        check(lib.wmc_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_s * 1e6), ctypes.byref(r)),
              "wmc_wait")
        return Result.from_c(r)

    def poll_ex(self, ticket: int):
        """(Result or None, completion time in CLOCK_MONOTONIC ns)."""
        r = _abi.wmc_result()
        t = ctypes.c_int64()
        rc = check(lib.wmc_poll_ex(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r),
                                   ctypes.byref(t)), "wmc_poll_ex")
        return (None, 0) if rc == _abi.WMC_PENDING else (Result.from_c(r), int(t.value))

    def collect_done_ns(self, tickets, timeout_s: float = 60.0):
        """Waits for every ticket; returns their server-stamped completion
        times (ns)."""
        import time as _t
        out = [None] * len(tickets)
        left = set(range(len(tickets)))
        deadline = _t.monotonic() + timeout_s
        while left:
            for j in list(left):
                res, ns = self.poll_ex(tickets[j])
                if res is not None:
                    out[j] = ns
                    left.discard(j)
            if left:
                if _t.monotonic() > deadline:
                    raise TimeoutError(f"{len(left)} tickets still pending")
                _t.sleep(0.001)
        return out

    def stats(self) -> _abi.wmc_server_stats_t:
        s = _abi.wmc_server_stats_t()
        check(lib.wmc_server_stats(self.handle, ctypes.byref(s)), "wmc_server_stats")
        return s

    def close(self):
        if getattr(self, "handle", None):
            lib.wmc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
