"""CPU oracle for literal-weighted model counting (Def. 2.1) and for one
pairwise tensor contraction (Eq. (1) on a two-tensor network).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  It shares no code
with the CUDA path and never imports it.

Functions
---------
brute_force(cnf, w_pos, w_neg)      Def. 2.1 by enumeration (n <= 30).
bucket_elim(cnf, w_pos, w_neg, ...) variable elimination in long double.
count_exact(cnf, ...)               exact unweighted count (unsigned __int128).
contract_pair(...)                  entries of C = A . B by direct summation.
min_degree_order(cnf)               the oracle's own elimination order.
min_fill_order(cnf)                 a second order (min-fill), for formulas
                                    whose min-degree order is too wide.
induced_width(cnf, order)           the largest bucket an order creates.

Values are returned as ``Big(mant, exp2)`` meaning ``mant * 2**exp2`` so
counts far below the float64 range (grid formulas reach 1e-956) survive.

Parity pins: every function here is pinned by ``tests/test_oracle.py``
against closed forms, the paper's worked example (Fig. 1) and brute force.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from fractions import Fraction
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-std=gnu11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_brute_force.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i64p,
                                           _f64p, _f64p, _f64p, _i64p, _u64p]
        lib.oracle_bucket_elim.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i64p,
                                           _f64p, _f64p, _i32p, ctypes.c_int32,
                                           _f64p, _i64p, _i32p]
        lib.oracle_bucket_exact.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i64p,
                                            _i32p, ctypes.c_int32, _u64p, _u64p, _i32p]
        lib.oracle_min_degree_order.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p,
                                                _i64p, _i32p]
        lib.oracle_contract_pair.argtypes = [ctypes.c_int32, _i32p, _f64p,
                                             ctypes.c_int32, _i32p, _f64p,
                                             ctypes.c_int32, _i32p, ctypes.c_int64,
                                             _i64p, _f64p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


@dataclass(frozen=True)
class Big:
    """mant * 2**exp2 (mant in [0.5, 1) or 0)."""
    mant: float
    exp2: int

    def to_float(self) -> float:
        return math.ldexp(self.mant, self.exp2) if self.mant != 0 else 0.0

    def log10(self) -> float:
        if self.mant == 0:
            return float("-inf")
        return math.log10(abs(self.mant)) + self.exp2 * math.log10(2.0)

    def to_fraction(self) -> Fraction:
        f = Fraction(self.mant)
        return f * (Fraction(2) ** self.exp2)

    def rel_diff(self, other: "Big") -> float:
        """|self - other| / |other|, computed without leaving the exponent
        range (0 when both are 0)."""
        if other.mant == 0:
            return 0.0 if self.mant == 0 else float("inf")
        a = math.ldexp(self.mant, self.exp2 - other.exp2)
        return abs(a - other.mant) / abs(other.mant)


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _cnf_arrays(cnf):
    lits, off = cnf.flat()
    lits = np.ascontiguousarray(lits, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    if lits.size == 0:
        lits = np.zeros(1, dtype=np.int32)
    return lits, off


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def brute_force(cnf, w_pos, w_neg):
    """(W(phi) as Big, number of satisfying assignments) by enumerating all
    2^n assignments (Def. 2.1)."""
    lib = _load()
    lits, off = _cnf_arrays(cnf)
    wp = np.ascontiguousarray(w_pos, dtype=np.float64)
    wn = np.ascontiguousarray(w_neg, dtype=np.float64)
    if wp.size == 0:
        wp = np.zeros(1); wn = np.zeros(1)
    mant = ctypes.c_double(); e = ctypes.c_int64(); cnt = ctypes.c_uint64()
    rc = lib.oracle_brute_force(cnf.n_vars, cnf.n_clauses, _ptr(lits, _i32p), _ptr(off, _i64p),
                                _ptr(wp, _f64p), _ptr(wn, _f64p), ctypes.byref(mant),
                                ctypes.byref(e), ctypes.byref(cnt))
    _check(rc, "oracle_brute_force")
    return Big(mant.value, e.value), int(cnt.value)


def bucket_elim(cnf, w_pos, w_neg, order: Optional[Sequence[int]] = None,
                max_width: int = 30, return_width: bool = False):
    """W(phi) by variable elimination in long double.  `order` is a list of
    1-based variable ids (default: the oracle's min-degree order)."""
    lib = _load()
    lits, off = _cnf_arrays(cnf)
    wp = np.ascontiguousarray(w_pos, dtype=np.float64)
    wn = np.ascontiguousarray(w_neg, dtype=np.float64)
    if wp.size == 0:
        wp = np.zeros(1); wn = np.zeros(1)
    ordp = None
    if order is not None:
        ordarr = np.ascontiguousarray(order, dtype=np.int32)
        if ordarr.size != cnf.n_vars:
            raise ValueError("order must list every variable once")
        ordp = _ptr(ordarr, _i32p)
    mant = ctypes.c_double(); e = ctypes.c_int64(); w = ctypes.c_int32()
    rc = lib.oracle_bucket_elim(cnf.n_vars, cnf.n_clauses, _ptr(lits, _i32p), _ptr(off, _i64p),
                                _ptr(wp, _f64p), _ptr(wn, _f64p), ordp, max_width,
                                ctypes.byref(mant), ctypes.byref(e), ctypes.byref(w))
    _check(rc, "oracle_bucket_elim")
    r = Big(mant.value, e.value)
    return (r, int(w.value)) if return_width else r


def count_exact(cnf, order: Optional[Sequence[int]] = None, max_width: int = 24) -> int:
    """Exact unweighted model count (all weights 1) by variable elimination
    over unsigned 128-bit integers."""
    lib = _load()
    lits, off = _cnf_arrays(cnf)
    ordp = None
    if order is not None:
        ordarr = np.ascontiguousarray(order, dtype=np.int32)
        ordp = _ptr(ordarr, _i32p)
    lo = ctypes.c_uint64(); hi = ctypes.c_uint64(); w = ctypes.c_int32()
    rc = lib.oracle_bucket_exact(cnf.n_vars, cnf.n_clauses, _ptr(lits, _i32p), _ptr(off, _i64p),
                                 ordp, max_width, ctypes.byref(lo), ctypes.byref(hi),
                                 ctypes.byref(w))
    _check(rc, "oracle_bucket_exact")
    return int(lo.value) | (int(hi.value) << 64)


def min_degree_order(cnf):
    lib = _load()
    lits, off = _cnf_arrays(cnf)
    out = np.zeros(max(cnf.n_vars, 1), dtype=np.int32)
    rc = lib.oracle_min_degree_order(cnf.n_vars, cnf.n_clauses, _ptr(lits, _i32p),
                                     _ptr(off, _i64p), _ptr(out, _i32p))
    _check(rc, "oracle_min_degree_order")
    return [int(v) for v in out[:cnf.n_vars]]


def _primal_graph(cnf):
    adj = [set() for _ in range(cnf.n_vars)]
    for cl in cnf.clauses:
        vs = sorted({abs(l) - 1 for l in cl})
        for a in vs:
            adj[a].update(v for v in vs if v != a)
    return adj


def min_fill_order(cnf):
    """An elimination order (1-based ids) chosen greedily by the fewest
    fill edges, ties by degree then lowest id.  Any order gives the same
    W (Thm 3.1); this one only keeps buckets narrow where min-degree does
    not.  Pure Python, O(n^3): for formulas of up to a few hundred
    variables."""
    adj = _primal_graph(cnf)
    alive = set(range(cnf.n_vars))
    order = []
    while alive:
        best, best_key = -1, None
        for v in sorted(alive):
            nb = sorted(adj[v])
            fill = sum(1 for i, a in enumerate(nb) for b in nb[i + 1:] if b not in adj[a])
            key = (fill, len(nb), v)
            if best_key is None or key < best_key:
                best, best_key = v, key
        nb = list(adj[best])
        for a in nb:
            adj[a].update(b for b in nb if b != a)
            adj[a].discard(best)
        alive.discard(best)
        order.append(best + 1)
    return order


def induced_width(cnf, order) -> int:
    """The largest number of variables multiplied together in one bucket
    when eliminating along `order` (the width bucket_elim reports)."""
    adj = _primal_graph(cnf)
    width = 0
    for x in order:
        v = x - 1
        nb = list(adj[v])
        width = max(width, len(nb) + 1)
        for a in nb:
            adj[a].update(b for b in nb if b != a)
            adj[a].discard(v)
        adj[v] = set()
    return width


def contract_pair(labels_a, a, labels_b, b, labels_c, out_offsets=None):
    """Entries of C = A . B (Eq. (1) on the network {A, B}).  Bit j of each
    tensor's linear offset is the index labels[j]; summed indices are those
    absent from labels_c.  Returns all 2^len(labels_c) entries, or the
    entries at `out_offsets`."""
    lib = _load()
    la = np.ascontiguousarray(labels_a, dtype=np.int32)
    lb = np.ascontiguousarray(labels_b, dtype=np.int32)
    lc = np.ascontiguousarray(labels_c, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if out_offsets is None:
        n_out = 1 << len(lc)
        offp = None
    else:
        offs = np.ascontiguousarray(out_offsets, dtype=np.int64)
        n_out = offs.size
        offp = _ptr(offs, _i64p)
    out = np.zeros(max(n_out, 1), dtype=np.float64)
    pad = lambda x: x if x.size else np.zeros(1, dtype=x.dtype)
    rc = lib.oracle_contract_pair(len(la), _ptr(pad(la), _i32p), _ptr(a, _f64p),
                                  len(lb), _ptr(pad(lb), _i32p), _ptr(b, _f64p),
                                  len(lc), _ptr(pad(lc), _i32p), n_out, offp,
                                  _ptr(out, _f64p))
    _check(rc, "oracle_contract_pair")
    return out[:n_out]
