"""Seeded synthetic input generators shared by the oracle tests, the GPU
parity tests and the benchmark.

This module produces *inputs only*: CNF formulas (DIMACS-style signed
literals), literal-weight vectors, query streams and dense Boolean tensors
with index labels.  It contains none of the weighted-model-counting
arithmetic (no reduction, no contraction, no summation), so the CPU oracle
and the CUDA path can both draw from it without sharing any of the method.

Every generator takes an integer ``seed`` and draws from
``numpy.random.Generator(PCG64(seed))``.

Formats
-------
A CNF is returned as ``Cnf(n_vars, clauses)`` where ``clauses`` is a list of
lists of nonzero ints; literal ``+v`` is variable ``v`` (1-based) and ``-v``
its negation.  ``Cnf.flat()`` gives the flattened ``(lits int32[],
clause_off int64[n_clauses+1])`` pair used by the C ABI.

Weights are ``(w_pos, w_neg)`` float64 arrays of length ``n_vars``:
``w_pos[v-1] = W(x_v, 1)`` and ``w_neg[v-1] = W(x_v, 0)`` (Def. 2.1).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class Cnf:
    n_vars: int
    clauses: List[List[int]]

    @property
    def n_clauses(self) -> int:
        return len(self.clauses)

    def flat(self) -> Tuple[np.ndarray, np.ndarray]:
        off = np.zeros(len(self.clauses) + 1, dtype=np.int64)
        for i, c in enumerate(self.clauses):
            off[i + 1] = off[i] + len(c)
        lits = np.zeros(int(off[-1]), dtype=np.int32)
        for i, c in enumerate(self.clauses):
            lits[off[i]:off[i + 1]] = np.asarray(c, dtype=np.int32)
        return lits, off

    def to_dimacs(self) -> str:
        out = [f"p cnf {self.n_vars} {len(self.clauses)}"]
        out += [" ".join(str(l) for l in c) + " 0" for c in self.clauses]
        return "\n".join(out) + "\n"


def parse_dimacs(text: str) -> Cnf:
    n = 0
    clauses: List[List[int]] = []
    cur: List[int] = []
    for line in text.splitlines():
        line = line.strip()
        if not line or line.startswith("c"):
            continue
        if line.startswith("p"):
            n = int(line.split()[2])
            continue
        for tok in line.split():
            v = int(tok)
            if v == 0:
                clauses.append(cur)
                cur = []
            else:
                cur.append(v)
    if cur:
        clauses.append(cur)
    return Cnf(n, clauses)


# ---------------------------------------------------------------- formulas

def random_kcnf(n_vars: int, n_clauses: int, seed: int, k: int = 3) -> Cnf:
    """Random k-CNF: each clause draws k distinct variables uniformly and
    each sign with probability 1/2; clauses are independent (duplicates
    allowed)."""
    rng = rng_for(seed)
    clauses = []
    for _ in range(n_clauses):
        vs = rng.choice(n_vars, size=k, replace=False) + 1
        sg = rng.integers(0, 2, size=k)
        clauses.append([int(v) if s else -int(v) for v, s in zip(vs, sg)])
    return Cnf(n_vars, clauses)


def grid_cnf(height: int, width: int, seed: int) -> Cnf:
    """Grid CNF on a height x width lattice (variable id = i*width + j + 1).

    For every cell (i, j) with i < height-1 and j < width-1: one 3-literal
    clause over the cell, its right neighbour and its down neighbour, and
    one 2-literal clause over the cell and its down-right diagonal
    neighbour.  Every sign is drawn with probability 1/2."""
    rng = rng_for(seed)
    vid = lambda i, j: i * width + j + 1
    clauses = []
    for i in range(height - 1):
        for j in range(width - 1):
            tri = [vid(i, j), vid(i, j + 1), vid(i + 1, j)]
            sg = rng.integers(0, 2, size=3)
            clauses.append([v if s else -v for v, s in zip(tri, sg)])
            diag = [vid(i, j), vid(i + 1, j + 1)]
            sg = rng.integers(0, 2, size=2)
            clauses.append([v if s else -v for v, s in zip(diag, sg)])
    return Cnf(height * width, clauses)


def fig1_example() -> Tuple[Cnf, List[str]]:
    """The worked example of Fig. 1: (w | x | ~y) & (w | y | z) & (~x | ~y)
    & (~y | ~z) with variables w=1, x=2, y=3, z=4."""
    return Cnf(4, [[1, 2, -3], [1, 3, 4], [-2, -3], [-3, -4]]), ["w", "x", "y", "z"]


def psi_family(n: int) -> Cnf:
    """psi = (x_1 | ... | x_n) & (~x_1 | ... | ~x_n), the example of
    Sec. 3.3 whose incidence treewidth is 2 and primal treewidth n-1."""
    return Cnf(n, [list(range(1, n + 1)), [-v for v in range(1, n + 1)]])


def chain_or(n: int) -> Cnf:
    """(x_1 | x_2) & (x_2 | x_3) & ... & (x_{n-1} | x_n)."""
    return Cnf(n, [[i, i + 1] for i in range(1, n)])


def chain_implication(n: int) -> Cnf:
    """x_1 -> x_2 -> ... -> x_n, i.e. clauses (~x_i | x_{i+1})."""
    return Cnf(n, [[-i, i + 1] for i in range(1, n)])


def independent_clauses(n_clauses: int, width: int, seed: int) -> Cnf:
    """n_clauses clauses over pairwise disjoint variable sets of size
    `width`, random signs."""
    rng = rng_for(seed)
    clauses = []
    for c in range(n_clauses):
        vs = np.arange(c * width, (c + 1) * width) + 1
        sg = rng.integers(0, 2, size=width)
        clauses.append([int(v) if s else -int(v) for v, s in zip(vs, sg)])
    return Cnf(n_clauses * width, clauses)


def uneven_candidates(seed: int, n3: Tuple[int, int] = (40, 120), ratio=(2.0, 3.5),
                      grid_w=(6, 20), grid_h=(20, 150)):
    """Endless stream of uneven-batch candidates: random 3-CNF (n in n3,
    clause ratio in `ratio`) and grid CNFs (width in grid_w, height in
    grid_h), alternating, each with complementary weights U(0.05, 0.95).
    Yields (kind, cnf, w_pos, w_neg, sub_seed) with kind "3cnf" or
    "grid<H>x<W>".  Candidates whose plans are too wide are skipped by the
    caller (rejection sampling)."""
    rng = rng_for(seed)
    i = 0
    while True:
        sub = int(rng.integers(0, 2 ** 31 - 1))
        if i % 2 == 0:
            n = int(rng.integers(n3[0], n3[1] + 1))
            m = int(round(n * rng.uniform(*ratio)))
            cnf = random_kcnf(n, m, sub)
            kind = "3cnf"
        else:
            w = int(rng.integers(grid_w[0], grid_w[1] + 1))
            h = int(rng.integers(grid_h[0], grid_h[1] + 1))
            cnf = grid_cnf(h, w, sub)
            kind = f"grid{h}x{w}"
        wp, wn = weights_complementary(cnf.n_vars, sub, 0.05, 0.95)
        yield kind, cnf, wp, wn, sub
        i += 1


# ----------------------------------------------------------------- weights

def grid_column_order(height: int, width: int) -> List[int]:
    """Column-by-column variable order of grid_cnf (an input for the
    oracle's elimination; it carries no arithmetic)."""
    return [i * width + j + 1 for j in range(width) for i in range(height)]


def weights_complementary(n_vars: int, seed: int, lo: float, hi: float):
    """w(x) ~ U(lo, hi), w(~x) = 1 - w(x)."""
    rng = rng_for(seed)
    wp = rng.uniform(lo, hi, size=n_vars)
    return wp.astype(np.float64), (1.0 - wp).astype(np.float64)


def weights_independent(n_vars: int, seed: int, lo: float, hi: float):
    """w(x), w(~x) drawn independently from U(lo, hi)."""
    rng = rng_for(seed)
    return (rng.uniform(lo, hi, size=n_vars).astype(np.float64),
            rng.uniform(lo, hi, size=n_vars).astype(np.float64))


def weights_unit(n_vars: int):
    return np.ones(n_vars, dtype=np.float64), np.ones(n_vars, dtype=np.float64)


def query_weights(n_vars: int, n_queries: int, seed: int, lo: float, hi: float):
    """A batch of weight-vector queries, query-major: arrays of shape
    (n_queries, n_vars); w(~x) = 1 - w(x)."""
    rng = rng_for(seed)
    wp = rng.uniform(lo, hi, size=(n_queries, n_vars))
    return np.ascontiguousarray(wp), np.ascontiguousarray(1.0 - wp)


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds, starting near 0) of a Poisson stream."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


# ------------------------------------------------------ pairwise tensors

@dataclass
class PairCase:
    """Two dense Boolean tensors for one pairwise contraction.  Bit j of a
    tensor's linear offset is the index labels[j] (extent 2 per index)."""
    labels_a: List[int]
    labels_b: List[int]
    labels_c: List[int]
    a: np.ndarray
    b: np.ndarray


def pair_case(rank_a: int, rank_b: int, n_batch: int, n_summed: int, seed: int,
              shuffle: bool = True, with_data: bool = True,
              dtype=np.float64) -> PairCase:
    """A pairwise contraction C = A . B whose shared indices are split into
    n_batch batch indices (kept in C) and n_summed summed indices; the rest
    of each operand's indices are free.  Entries are U(0, 1).  With
    shuffle=True each tensor's index order is a random permutation."""
    f_a = rank_a - n_batch - n_summed
    f_b = rank_b - n_batch - n_summed
    if f_a < 0 or f_b < 0:
        raise ValueError("rank too small for the shared indices")
    rng = rng_for(seed)
    lab = 0
    batch = list(range(lab, lab + n_batch)); lab += n_batch
    summed = list(range(lab, lab + n_summed)); lab += n_summed
    fa = list(range(lab, lab + f_a)); lab += f_a
    fb = list(range(lab, lab + f_b)); lab += f_b
    la = fa + batch + summed
    lb = summed + batch + fb
    lc = fa + batch + fb
    if shuffle:
        la = [la[i] for i in rng.permutation(len(la))]
        lb = [lb[i] for i in rng.permutation(len(lb))]
        lc = [lc[i] for i in rng.permutation(len(lc))]
    a = b = None
    if with_data:
        a = rng.random(1 << rank_a, dtype=np.float64).astype(dtype)
        b = rng.random(1 << rank_b, dtype=np.float64).astype(dtype)
    return PairCase(la, lb, lc, a, b)
