"""Pins for the CPU oracle: closed forms, the worked example of Fig. 1,
theorems used as invariants, and library routines for the pairwise
contraction.  None of these compute the oracle's own formula a second time;
each checks it against something the paper or the mathematics fixes."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import wmcgen
from oracle import Big

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def big_of_fraction(fr: Fraction) -> Big:
    if fr == 0:
        return Big(0.0, 0)
    m, e = math.frexp(float(fr))
    return Big(m, e)


def rel(a: Big, b: Big) -> float:
    return a.rel_diff(b)


# ------------------------------------------------------------ Fig. 1

def _fig1():
    with open(os.path.join(GOLDEN, "fig1.json")) as f:
        g = json.load(f)
    return g, wmcgen.parse_dimacs(g["cnf_dimacs"])


def test_fig1_unweighted_count():
    """Fig. 1 formula has exactly 7 models."""
    g, cnf = _fig1()
    ones = wmcgen.weights_unit(cnf.n_vars)
    val, cnt = oracle.brute_force(cnf, *ones)
    assert cnt == g["unweighted_count"] == 7
    assert val.to_float() == 7.0
    assert oracle.count_exact(cnf) == 7
    assert oracle.bucket_elim(cnf, *ones).to_float() == 7.0


def test_fig1_weighted_closed_form():
    """Weighted count of Fig. 1 against its hand derivation (Def. 2.1),
    evaluated in exact rationals."""
    g, cnf = _fig1()
    wp = g["weighted_example"]["w_pos"]
    wn = g["weighted_example"]["w_neg"]
    F = lambda v: Fraction(v)
    w1, x1, y1, z1 = (F(v) for v in wp)
    w0, x0, y0, z0 = (F(v) for v in wn)
    exact = w1 * x0 * y1 * z0 + y0 * (x0 + x1) * ((w0 + w1) * (z0 + z1) - w0 * z0)
    want = big_of_fraction(exact)
    bf, _ = oracle.brute_force(cnf, np.array(wp), np.array(wn))
    be = oracle.bucket_elim(cnf, np.array(wp), np.array(wn))
    assert rel(bf, want) < 1e-15
    assert rel(be, want) < 1e-15
    # swapping the roles of W(x,0) and W(x,1) must change the value
    bs, _ = oracle.brute_force(cnf, np.array(wn), np.array(wp))
    assert rel(bs, want) > 1e-3


def _strict_network(cnf, w_pos, w_neg):
    """The network of Thm 3.2 exactly as constructed there: one index (x, C)
    per variable occurrence, one COPY-like tensor A_x per variable over its
    indices, one clause tensor B_C per clause."""
    idx = {}
    for c, cl in enumerate(cnf.clauses):
        for v in sorted(set(abs(l) for l in cl)):
            idx[(v, c)] = len(idx)
    tensors = []
    for v in range(1, cnf.n_vars + 1):
        mine = [i for (x, c), i in idx.items() if x == v]
        t = np.zeros((2,) * len(mine))
        if mine:
            t[(0,) * len(mine)] = w_neg[v - 1]
            t[(1,) * len(mine)] = w_pos[v - 1]
        else:
            t = np.array(w_neg[v - 1] + w_pos[v - 1])  # reading: a variable in no clause
        tensors.append((t, mine))
    for c, cl in enumerate(cnf.clauses):
        vs = sorted(set(abs(l) for l in cl))
        mine = [idx[(v, c)] for v in vs]
        t = np.zeros((2,) * len(vs))
        for assign in itertools.product((0, 1), repeat=len(vs)):
            val = dict(zip(vs, assign))
            t[assign] = float(any((l > 0 and val[l]) or (l < 0 and not val[-l]) for l in cl))
        tensors.append((t, mine))
    return tensors, len(idx)


def _contract_strict(tensors):
    args = []
    for t, lab in tensors:
        args += [t, lab]
    return float(np.einsum(*args, [], optimize="greedy"))


def test_fig1_reduction_structure():
    """Thm 3.2 on Fig. 1: 8 tensors and 10 indices, and the contraction of
    that network equals the oracle's count."""
    g, cnf = _fig1()
    wp = np.array(g["weighted_example"]["w_pos"])
    wn = np.array(g["weighted_example"]["w_neg"])
    tensors, n_idx = _strict_network(cnf, wp, wn)
    assert len(tensors) == g["n_tensors"] == 8
    assert n_idx == g["n_indices"] == 10
    val = _contract_strict(tensors)
    assert abs(val - oracle.brute_force(cnf, wp, wn)[0].to_float()) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_strict_form_equals_oracle(seed):
    """Reading: the hyperedge form (COPY tensors contracted into variables)
    equals the strict form of Thm 3.2 on random small formulas."""
    cnf = wmcgen.random_kcnf(7, 8, seed=100 + seed)
    wp, wn = wmcgen.weights_independent(7, seed, 0.1, 2.0)
    tensors, _ = _strict_network(cnf, wp, wn)
    val = _contract_strict(tensors)
    bf = oracle.brute_force(cnf, wp, wn)[0].to_float()
    be = oracle.bucket_elim(cnf, wp, wn).to_float()
    assert abs(val - bf) <= 1e-12 * abs(bf)
    assert abs(be - bf) <= 1e-15 * abs(bf) + 1e-300


# ------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_psi_family(n):
    """psi = (x1|..|xn) & (~x1|..|~xn): W = prod(W0+W1) - prod W1 - prod W0;
    unweighted 2^n - 2 (Sec. 3.3 example)."""
    cnf = wmcgen.psi_family(n)
    wp, wn = wmcgen.weights_independent(n, 7 + n, 0.05, 1.5)
    exact = math.prod(Fraction(a) + Fraction(b) for a, b in zip(wp, wn)) \
        - math.prod(Fraction(a) for a in wp) - math.prod(Fraction(b) for b in wn)
    want = big_of_fraction(exact)
    assert rel(oracle.brute_force(cnf, wp, wn)[0], want) < 1e-14
    assert rel(oracle.bucket_elim(cnf, wp, wn), want) < 1e-14
    assert oracle.count_exact(cnf) == 2 ** n - 2
    assert oracle.brute_force(cnf, *wmcgen.weights_unit(n))[1] == 2 ** n - 2


@pytest.mark.parametrize("n", [0, 1, 9, 20])
def test_no_clauses(n):
    """Empty CNF: prod_x (W0+W1); all weights 1 gives 2^n."""
    cnf = wmcgen.Cnf(n, [])
    wp, wn = wmcgen.weights_independent(max(n, 1), 3, 0.1, 3.0)
    wp, wn = wp[:n], wn[:n]
    exact = math.prod((Fraction(a) + Fraction(b) for a, b in zip(wp, wn)), start=Fraction(1))
    assert rel(oracle.bucket_elim(cnf, wp, wn), big_of_fraction(exact)) < 1e-15
    assert oracle.count_exact(cnf) == 2 ** n
    if n <= 20:
        assert rel(oracle.brute_force(cnf, wp, wn)[0], big_of_fraction(exact)) < 1e-15


def test_large_unit_and_complementary():
    """4800 free variables: 2^4800 unweighted (beyond float64); with
    w + w' = 1 every variable contributes exactly 1."""
    n = 4800
    cnf = wmcgen.Cnf(n, [])
    one = oracle.bucket_elim(cnf, *wmcgen.weights_unit(n))
    assert one.mant == 0.5 and one.exp2 == n + 1
    wp = np.full(n, 0.25); wn = np.full(n, 0.75)
    v = oracle.bucket_elim(cnf, wp, wn)
    assert v.to_float() == 1.0


def test_empty_clause_and_tautology():
    """An empty clause makes W = 0; a tautology x | ~x changes nothing."""
    wp, wn = wmcgen.weights_independent(3, 5, 0.1, 1.0)
    base = wmcgen.Cnf(3, [[1, -2], [2, 3]])
    with_empty = wmcgen.Cnf(3, [[1, -2], [], [2, 3]])
    with_taut = wmcgen.Cnf(3, [[1, -2], [3, -3], [2, 3]])
    with_dup = wmcgen.Cnf(3, [[1, 1, -2], [2, 3, 3]])
    b = oracle.brute_force(base, wp, wn)[0]
    assert oracle.brute_force(with_empty, wp, wn)[0].to_float() == 0.0
    assert oracle.bucket_elim(with_empty, wp, wn).to_float() == 0.0
    assert rel(oracle.bucket_elim(with_taut, wp, wn), b) < 1e-15
    assert rel(oracle.bucket_elim(with_dup, wp, wn), b) < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_independent_clauses(seed):
    """Disjoint clauses: W = prod_C (prod_{x in C}(W0+W1) - prod_{l in C}
    W(falsifying value of l))."""
    cnf = wmcgen.independent_clauses(5, 3, seed)
    wp, wn = wmcgen.weights_independent(cnf.n_vars, seed + 11, 0.1, 2.0)
    exact = Fraction(1)
    for cl in cnf.clauses:
        full = math.prod(Fraction(wp[abs(l) - 1]) + Fraction(wn[abs(l) - 1]) for l in cl)
        fals = math.prod(Fraction(wn[l - 1]) if l > 0 else Fraction(wp[-l - 1]) for l in cl)
        exact *= full - fals
    want = big_of_fraction(exact)
    assert rel(oracle.brute_force(cnf, wp, wn)[0], want) < 1e-14
    assert rel(oracle.bucket_elim(cnf, wp, wn), want) < 1e-14
    assert oracle.count_exact(cnf) == 7 ** 5


def _fib(k):
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


@pytest.mark.parametrize("n", [2, 3, 10, 22])
def test_or_chain_fibonacci(n):
    """(x1|x2)&(x2|x3)&...: unweighted count F(n+2)."""
    cnf = wmcgen.chain_or(n)
    assert oracle.count_exact(cnf) == _fib(n + 2)
    if n <= 22:
        assert oracle.brute_force(cnf, *wmcgen.weights_unit(n))[1] == _fib(n + 2)


@pytest.mark.parametrize("n", [3, 15, 4800])
def test_or_chain_transfer_matrix(n):
    """Weighted or-chain by a 2x2 transfer-matrix recursion (an independent
    algorithm): exact rationals for short chains, 60-digit decimals for a
    4800-variable chain whose value is far below the float64 range."""
    import decimal
    cnf = wmcgen.chain_or(n)
    wp, wn = wmcgen.weights_complementary(n, 40 + n, 0.05, 0.95)
    num = Fraction if n <= 15 else (lambda x: decimal.Decimal(float(x)))
    ctx = decimal.localcontext()
    ctx.__enter__()
    decimal.getcontext().prec = 60
    decimal.getcontext().Emin = -999999
    # v[b] = total weight of the prefix ending with x_i = b
    v0, v1 = num(wn[0]), num(wp[0])
    for i in range(1, n):
        a0, a1 = num(wn[i]), num(wp[i])
        v0, v1 = v1 * a0, (v0 + v1) * a1      # x_i = 0 needs x_{i-1} = 1
    exact = v0 + v1
    ctx.__exit__(None, None, None)
    be = oracle.bucket_elim(cnf, wp, wn, order=list(range(1, n + 1)))
    if n <= 15:
        want = big_of_fraction(exact)
        assert rel(oracle.brute_force(cnf, wp, wn)[0], want) < 1e-14
        assert rel(be, want) < 1e-14
    else:
        got = decimal.Decimal(be.mant) * (decimal.Decimal(2) ** be.exp2)
        assert abs(got / exact - 1) < decimal.Decimal("1e-12")
        assert be.log10() < -400


@pytest.mark.parametrize("n", [1, 2, 8, 60])
def test_implication_chain(n):
    """x1 -> x2 -> ... -> xn has exactly n+1 models."""
    cnf = wmcgen.chain_implication(n)
    assert oracle.count_exact(cnf) == n + 1
    if n <= 20:
        assert oracle.brute_force(cnf, *wmcgen.weights_unit(n))[1] == n + 1


@pytest.mark.parametrize("n", [64, 65, 100, 127])
def test_exact_count_beyond_64_bits_free_variables(n):
    """Unweighted count of n free variables is 2^n (Def. 2.1 with unit
    weights): counts at and beyond 2^64 exercise the upper half of the
    128-bit result."""
    assert oracle.count_exact(wmcgen.Cnf(n, [])) == 2 ** n


@pytest.mark.parametrize("n", [92, 100, 180])
def test_exact_count_beyond_64_bits_or_chain(n):
    """(x1|x2)&...&(x_{n-1}|x_n) has F(n+2) models; F(94) > 2^64, F(182)
    is just below 2^125."""
    assert _fib(n + 2) >= 2 ** 64
    assert oracle.count_exact(wmcgen.chain_or(n)) == _fib(n + 2)


def test_exact_count_beyond_64_bits_independent_clauses():
    """40 disjoint 3-literal clauses: 7^40 (about 2^112) models."""
    assert oracle.count_exact(wmcgen.independent_clauses(40, 3, seed=2)) == 7 ** 40


# ------------------------------------------ theorems used as invariants

@pytest.mark.parametrize("seed", range(8))
def test_bucket_matches_brute_force(seed):
    """O1b against O1a on random 3-CNF (n <= 20): exact counts identical,
    weighted values within 1e-15 relative."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 21))
    m = int(rng.integers(n, 4 * n))
    cnf = wmcgen.random_kcnf(n, m, seed=seed)
    wp, wn = wmcgen.weights_complementary(n, seed, 0.1, 0.9)
    bf, cnt = oracle.brute_force(cnf, wp, wn)
    assert oracle.count_exact(cnf) == cnt
    assert rel(oracle.bucket_elim(cnf, wp, wn), bf) < 1e-15


@pytest.mark.parametrize("seed", range(4))
def test_order_independence(seed):
    """Thm 3.1: any valid plan gives the same value.  Random elimination
    orders agree bit-exactly on integer counts and to 1e-15 otherwise."""
    cnf = wmcgen.random_kcnf(16, 40, seed=50 + seed)
    wp, wn = wmcgen.weights_complementary(16, seed, 0.1, 0.9)
    ref = oracle.bucket_elim(cnf, wp, wn)
    cref = oracle.count_exact(cnf)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        order = list(rng.permutation(16) + 1)
        assert rel(oracle.bucket_elim(cnf, wp, wn, order=order), ref) < 1e-15
        assert oracle.count_exact(cnf, order=order) == cref


def test_min_fill_order_and_induced_width():
    """The second elimination order is a permutation and gives brute
    force's value (Thm 3.1); induced_width equals the bucket size the
    elimination reports, and known widths: an or-chain eliminated in
    order has buckets of 2 variables, one clause over k variables a bucket
    of k, an H x W grid eliminated column by column buckets of H + 2."""
    for seed in range(4):
        cnf = wmcgen.random_kcnf(18, 60, seed=90 + seed)
        wp, wn = wmcgen.weights_complementary(18, seed, 0.1, 0.9)
        o = oracle.min_fill_order(cnf)
        assert sorted(o) == list(range(1, 19))
        v, wd = oracle.bucket_elim(cnf, wp, wn, order=o, return_width=True)
        assert rel(v, oracle.brute_force(cnf, wp, wn)[0]) < 1e-15
        assert oracle.induced_width(cnf, o) == wd
    assert oracle.induced_width(wmcgen.chain_or(30), list(range(1, 31))) == 2
    assert oracle.induced_width(wmcgen.Cnf(9, [list(range(1, 10))]), list(range(1, 10))) == 9
    assert oracle.induced_width(wmcgen.grid_cnf(6, 10, 1), wmcgen.grid_column_order(6, 10)) == 8
    assert oracle.bucket_elim(wmcgen.grid_cnf(6, 10, 1), *wmcgen.weights_unit(60),
                              order=wmcgen.grid_column_order(6, 10), return_width=True)[1] == 8


@pytest.mark.parametrize("seed", range(3))
def test_conditioning_identity(seed):
    """Thm 4.2 with one sliced variable: W(phi) = W(phi|x=0) + W(phi|x=1),
    where conditioning zeroes the other literal weight of x."""
    cnf = wmcgen.random_kcnf(14, 40, seed=70 + seed)
    wp, wn = wmcgen.weights_complementary(14, seed, 0.1, 0.9)
    full = oracle.bucket_elim(cnf, wp, wn).to_fraction()
    x = 3
    wp0, wn1 = wp.copy(), wn.copy()
    wp0[x] = 0.0
    wn1[x] = 0.0
    part = oracle.bucket_elim(cnf, wp0, wn).to_fraction() + oracle.bucket_elim(cnf, wp, wn1).to_fraction()
    assert abs(part - full) <= Fraction(1, 10 ** 15) * full


def test_grid_orders_agree():
    """16x100 grid: two unrelated elimination orders (column sweep and
    reversed column sweep) give the same count to 1e-13; the value is below
    the float64 range, which long double holds."""
    H, W = 16, 100
    cnf = wmcgen.grid_cnf(H, W, seed=1)
    wp, wn = wmcgen.weights_complementary(H * W, 1, 0.05, 0.95)
    col = [i * W + j + 1 for j in range(W) for i in range(H)]
    a, wa = oracle.bucket_elim(cnf, wp, wn, order=col, return_width=True)
    b = oracle.bucket_elim(cnf, wp, wn, order=col[::-1])
    assert wa <= 19
    assert rel(a, b) < 1e-13
    assert a.log10() < -150


# --------------------------------------------- pairwise contraction pins

@pytest.mark.parametrize("ra,rb,nb,nk,seed", [
    (6, 5, 0, 1, 0), (8, 7, 2, 3, 1), (9, 9, 4, 4, 2), (10, 6, 1, 1, 3), (7, 7, 0, 7, 4),
])
def test_contract_pair_vs_einsum(ra, rb, nb, nk, seed):
    """Direct summation against torch.einsum in float64 (a library routine)
    with random index orders."""
    torch = pytest.importorskip("torch")
    case = wmcgen.pair_case(ra, rb, nb, nk, seed=seed)
    got = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c)
    letters = {}
    def sub(labels):
        # bit j of the offset is labels[j]: numpy/torch C-order puts bit 0 last
        return "".join(letters.setdefault(l, chr(ord("a") + len(letters))) for l in reversed(labels))
    ea, eb, ec = sub(case.labels_a), sub(case.labels_b), sub(case.labels_c)
    A = torch.from_numpy(case.a).reshape((2,) * ra)
    B = torch.from_numpy(case.b).reshape((2,) * rb)
    C = torch.einsum(f"{ea},{eb}->{ec}", A, B).reshape(-1).numpy()
    np.testing.assert_allclose(got, C, rtol=1e-14, atol=0)


def test_contract_pair_matmul_and_samples():
    """A plain matrix product (labels laid out as [k | i] and [j | k]) equals
    numpy's matmul; sampled offsets equal the full evaluation."""
    rng = np.random.default_rng(5)
    i_bits, j_bits, k_bits = 3, 4, 5
    Am = rng.random((2 ** i_bits, 2 ** k_bits))   # A[i, k]
    Bm = rng.random((2 ** k_bits, 2 ** j_bits))   # B[k, j]
    ki = list(range(0, k_bits)); ii = list(range(10, 10 + i_bits)); jj = list(range(20, 20 + j_bits))
    # row-major A[i, k]: offset = i * 2^k + k, so the low bits are k
    la, lb, lc = ki + ii, jj + ki, jj + ii
    got = oracle.contract_pair(la, Am.reshape(-1), lb, Bm.reshape(-1), lc)
    want = (Am @ Bm).reshape(-1)  # C[i, j]: offset = i * 2^j + j
    np.testing.assert_allclose(got, want, rtol=1e-14)
    offs = rng.integers(0, 2 ** (i_bits + j_bits), size=17)
    np.testing.assert_array_equal(oracle.contract_pair(la, Am.reshape(-1), lb, Bm.reshape(-1), lc, offs), got[offs])
