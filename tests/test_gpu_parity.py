"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Tolerances (all weights nonnegative, so relative bounds apply):
  * unweighted counts below 2^53: bit-exact;
  * FP64 path: relative 1e-10 (the a-priori bound d * 2^-53 is far below);
  * scaled-FP32 path: relative 1e-4, and never above the bound the library
    states per result (gamma_d with u = 2^-24).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import wmcgen
from oracle import Big

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FP64, FP32 = 0, 1
TOL = {FP64: 1e-10, FP32: 1e-4}


@pytest.fixture(scope="module")
def w():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2006_15512_b300 as lib
    return lib


def rel(res, big: Big) -> float:
    return Big(res.mant, res.exp2).rel_diff(big)


def plan_for(w, cnf, wp, wn, precision, **kw):
    return w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=precision, **kw)


# ------------------------------------------------------ random 3-CNF

@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("seed", range(6))
def test_random_3cnf_n20(w, precision, seed):
    """Random 3-CNF, n=20, m=60, w(x)~U(0.1,0.9), w(~x)=1-w(x), vs brute
    force over 2^20 assignments."""
    cnf = wmcgen.random_kcnf(20, 60, seed=seed)
    wp, wn = wmcgen.weights_complementary(20, seed, 0.1, 0.9)
    want, _ = oracle.brute_force(cnf, wp, wn)
    res = plan_for(w, cnf, wp, wn, precision).execute()[0]
    r = rel(res, want)
    assert r <= TOL[precision], r
    assert r <= res.rel_err_bound + 1e-16


@pytest.mark.parametrize("seed", range(4))
def test_unweighted_bit_exact(w, seed):
    """All weights 1: the FP64 path returns the exact model count."""
    cnf = wmcgen.random_kcnf(20, 50, seed=10 + seed)
    _, cnt = oracle.brute_force(cnf, *wmcgen.weights_unit(20))
    for precision in (FP64, FP32):
        res = plan_for(w, cnf, None, None, precision).execute()[0]
        assert res.to_float() == float(cnt)
        if precision == FP64:
            assert res.flags & w.WMC_FLAG_EXACT_INT


def test_closed_forms(w):
    cases = []
    cnf, _ = wmcgen.fig1_example()
    cases.append((cnf, 7))
    cases.append((wmcgen.psi_family(20), 2 ** 20 - 2))
    cases.append((wmcgen.Cnf(60, []), 2 ** 60))
    cases.append((wmcgen.chain_implication(1000), 1001))
    cases.append((wmcgen.Cnf(3, [[1, 2], [], [3]]), 0))
    cases.append((wmcgen.Cnf(0, []), 1))
    a, b = 0, 1
    for _ in range(302):
        a, b = b, a + b
    cases.append((wmcgen.chain_or(300), a))   # Fibonacci F(302) ~ 1.6e62
    for cnf, want in cases:
        for precision in (FP64, FP32):
            res = plan_for(w, cnf, None, None, precision).execute()[0]
            if want == 0:
                assert res.mant == 0.0
                continue
            got = Big(res.mant, res.exp2)
            m, e = math.frexp(float(want))
            r = got.rel_diff(Big(m, e))
            if want < 2 ** 53 and precision == FP64:
                assert r == 0.0, (cnf.n_vars, want, got)
            else:
                assert r <= TOL[precision], (cnf.n_vars, r)


def test_psi_weighted(w):
    n = 18
    cnf = wmcgen.psi_family(n)
    wp, wn = wmcgen.weights_independent(n, 3, 0.1, 0.9)
    want = oracle.bucket_elim(cnf, wp, wn)
    for precision in (FP64, FP32):
        assert rel(plan_for(w, cnf, wp, wn, precision).execute()[0], want) <= TOL[precision]


# ------------------------------------------------------ query batching

@pytest.mark.parametrize("precision", [FP64, FP32])
def test_query_batch_matches_oracle_and_is_batch_invariant(w, precision):
    cnf = wmcgen.random_kcnf(22, 70, seed=7)
    plan = plan_for(w, cnf, None, None, precision)
    wq, wnq = wmcgen.query_weights(22, 64, seed=8, lo=0.05, hi=0.95)
    alone = [plan.execute(wq[i:i + 1], wnq[i:i + 1])[0] for i in range(64)]
    for Q in (3, 8, 64):
        batch = plan.execute(wq[:Q], wnq[:Q])
        for i in range(Q):
            assert (batch[i].mant, batch[i].exp2) == (alone[i].mant, alone[i].exp2)
    for i in range(0, 64, 9):
        want = oracle.bucket_elim(cnf, wq[i], wnq[i])
        assert rel(alone[i], want) <= TOL[precision]


def _fuzz_cases():
    """Seeded mix of formula families, widths and batch sizes: random
    k-CNF (k = 2..5, clause ratios around each k's hard region), small
    grids and the psi family, with odd query counts (padded lanes)."""
    rng = np.random.default_rng(2006)
    cases = []
    for i in range(16):
        fam = ("kcnf", "kcnf", "kcnf", "grid", "psi")[i % 5]
        if fam == "kcnf":
            k = int(rng.integers(2, 6))
            n = int(rng.integers(10, 33))
            ratio = {2: 1.0, 3: 3.2, 4: 7.0, 5: 14.0}[k] * float(rng.uniform(0.6, 1.1))
            cnf = wmcgen.random_kcnf(n, max(1, int(ratio * n)), seed=100 + i, k=k)
        elif fam == "grid":
            cnf = wmcgen.grid_cnf(int(rng.integers(3, 9)), int(rng.integers(4, 30)), seed=100 + i)
        else:
            cnf = wmcgen.psi_family(int(rng.integers(4, 18)))
        cases.append((i, cnf, int((1, 5, 33)[i % 3])))
    # taller grids: frontiers past the small-node phase, so the walk runs
    # streaming passes and chains of frontier eliminations
    # (the oracle eliminates these column by column)
    for j, (h, wd, Q) in enumerate(((12, 24, 1), (14, 30, 3), (16, 22, 17), (18, 20, 2))):
        cases.append((16 + j, wmcgen.grid_cnf(h, wd, seed=300 + j), Q, wmcgen.grid_column_order(h, wd)))
    return [c if len(c) == 4 else c + (None,) for c in cases]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("case", range(20))
def test_walk_fuzz_against_the_oracle(w, precision, case):
    """Default walk layout on a seeded mix of families and batch sizes:
    every sampled query within the tolerance of the oracle's bucket
    elimination and within the result's stated bound, each query's bits
    the same alone as in its batch, and the same bits with one pass per
    contraction and with runs of six frontier eliminations."""
    i, cnf, Q, order = _fuzz_cases()[case]
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=200 + i, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, precision)
    got = plan.execute(wq, wnq)
    try:
        for fuse in (0, 6):
            w.wmc_set_fusion(fuse)
            other = plan_for(w, cnf, None, None, precision).execute(wq, wnq)
            for q in range(Q):
                assert (other[q].mant, other[q].exp2) == (got[q].mant, got[q].exp2), (fuse, q)
    finally:
        w.wmc_set_fusion(-1)
    for q in sorted({0, Q // 2, Q - 1}):
        want = oracle.bucket_elim(cnf, wq[q], wnq[q], order=order)
        r = rel(got[q], want)
        assert r <= TOL[precision], (q, r)
        assert r <= got[q].rel_err_bound + 1e-16, (q, r)
        alone = plan.execute(wq[q:q + 1], wnq[q:q + 1])[0]
        assert (alone.mant, alone.exp2) == (got[q].mant, got[q].exp2), q


def test_evidence_zero_weight(w):
    """Evidence as a zero weight equals conditioning (Thm 4.2)."""
    cnf = wmcgen.random_kcnf(16, 40, seed=3)
    wp, wn = wmcgen.weights_complementary(16, 3, 0.1, 0.9)
    wp0 = wp.copy(); wp0[5] = 0.0
    want = oracle.bucket_elim(cnf, wp0, wn)
    for precision in (FP64, FP32):
        assert rel(plan_for(w, cnf, wp0, wn, precision).execute()[0], want) <= TOL[precision]


def test_fp32_flush_is_flagged(w):
    """A weight ratio beyond float32's range underflows a mantissa: without
    the fallback the result carries WMC_FLAG_FP32_FLUSH; FP64 stays
    exact-to-tolerance."""
    cnf = wmcgen.random_kcnf(12, 30, seed=4)
    wp, wn = wmcgen.weights_complementary(12, 4, 0.2, 0.8)
    wn[2] = 1e-60
    want = oracle.bucket_elim(cnf, wp, wn)
    try:
        w.wmc_set_fp64_fallback(0)
        r32 = plan_for(w, cnf, wp, wn, FP32).execute()[0]
    finally:
        w.wmc_set_fp64_fallback(1)
    assert r32.flags & w.WMC_FLAG_FP32_FLUSH
    assert not r32.flags & w.WMC_FLAG_FELL_BACK_FP64
    r64 = plan_for(w, cnf, wp, wn, FP64).execute()[0]
    assert rel(r64, want) <= TOL[FP64]


def test_fp32_flush_falls_back_to_fp64(w):
    """With the fallback (default), the flushed queries of a scaled-FP32
    batch run again in FP64 on the same tree: they carry
    WMC_FLAG_FELL_BACK_FP64 and FP64's accuracy; the other queries keep
    their FP32 values, bit for bit."""
    n = 14
    cnf = wmcgen.random_kcnf(n, 36, seed=6)
    cnf = wmcgen.Cnf(n, cnf.clauses + [[3]])  # x_3 forced true: a tiny w(x_3) survives
    Q = 8
    wq, wnq = wmcgen.query_weights(n, Q, seed=9, lo=0.1, hi=0.9)
    for q in (1, 4, 5):
        wq[q, 2] = 1e-41  # below float32's smallest normal
    plan = plan_for(w, cnf, None, None, FP32)
    res = plan.execute(wq, wnq)
    try:
        w.wmc_set_fp64_fallback(0)
        raw = plan.execute(wq, wnq)
    finally:
        w.wmc_set_fp64_fallback(1)
    for q in range(Q):
        want = oracle.bucket_elim(cnf, wq[q], wnq[q])
        if q in (1, 4, 5):
            assert raw[q].flags & w.WMC_FLAG_FP32_FLUSH
            assert res[q].flags & w.WMC_FLAG_FELL_BACK_FP64 and not res[q].flags & w.WMC_FLAG_FP32_FLUSH
            assert rel(res[q], want) <= TOL[FP64]
        else:
            assert not res[q].flags & (w.WMC_FLAG_FELL_BACK_FP64 | w.WMC_FLAG_FP32_FLUSH)
            assert (res[q].mant, res[q].exp2) == (raw[q].mant, raw[q].exp2)
            assert rel(res[q], want) <= TOL[FP32]


# ------------------------------------------- block floating point (f4)

@pytest.mark.parametrize("block_fp", [1, 3, 6])
@pytest.mark.parametrize("Q", [1, 8])
def test_block_fp_random_3cnf(w, block_fp, Q):
    """Block-floating-point float32 (one exponent per block of 2^(block_fp-1)
    index assignments and lane) against brute force on random 3-CNF."""
    cnf = wmcgen.random_kcnf(20, 60, seed=block_fp)
    wq, wnq = wmcgen.query_weights(20, Q, seed=40 + Q, lo=0.1, hi=0.9)
    plan = plan_for(w, cnf, None, None, FP32, block_fp=block_fp)
    res = plan.execute(wq, wnq)
    for q in range(Q):
        want = oracle.brute_force(cnf, wq[q], wnq[q])[0]
        r = rel(res[q], want)
        assert r <= TOL[FP32] and r <= res[q].rel_err_bound + 1e-16, (q, r)
        assert not res[q].flags & (w.WMC_FLAG_FP32_FLUSH | w.WMC_FLAG_FELL_BACK_FP64)


def test_block_fp_grid(w):
    """The 16x100 grid (the serving network, values near 1e-300) in
    block-floating-point form, 8 queries, against the oracle."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, 8, seed=3, lo=0.05, hi=0.95)
    col = [i * 100 + j + 1 for j in range(100) for i in range(16)]
    plan = plan_for(w, cnf, None, None, FP32, block_fp=4)
    res = plan.execute(wq, wnq)
    for q in (0, 7):
        assert rel(res[q], oracle.bucket_elim(cnf, wq[q], wnq[q], order=col)) <= TOL[FP32]


@pytest.mark.parametrize("block_fp", [1, 2])
def test_block_fp_keeps_weights_beyond_float_range(w, block_fp):
    """Weight ratios far beyond float32's range inside one tensor (1e-41,
    1e-300 against ~1): the scaled-FP32 walk flushes them (and, with the
    fallback off, only flags the query), while block floating point keeps
    every query within 1e-4 of the oracle in float32 storage, with no flush
    flag and no FP64 re-execution."""
    n = 14
    cnf = wmcgen.random_kcnf(n, 36, seed=6)
    cnf = wmcgen.Cnf(n, cnf.clauses + [[3]])  # x_3 forced true: its tiny weight survives
    Q = 8
    wq, wnq = wmcgen.query_weights(n, Q, seed=9, lo=0.1, hi=0.9)
    for q, tiny in ((1, 1e-41), (4, 1e-41), (5, 1e-300), (6, 3e-200)):
        wq[q, 2] = tiny
    try:
        w.wmc_set_fp64_fallback(0)
        raw = plan_for(w, cnf, None, None, FP32).execute(wq, wnq)
        res = plan_for(w, cnf, None, None, FP32, block_fp=block_fp).execute(wq, wnq)
    finally:
        w.wmc_set_fp64_fallback(1)
    assert all(raw[q].flags & w.WMC_FLAG_FP32_FLUSH for q in (1, 4, 5, 6))
    for q in range(Q):
        want = oracle.bucket_elim(cnf, wq[q], wnq[q])
        assert not res[q].flags & (w.WMC_FLAG_FP32_FLUSH | w.WMC_FLAG_FELL_BACK_FP64), q
        assert rel(res[q], want) <= TOL[FP32], (q, rel(res[q], want))


# ------------------------------------------------------------ grids

@pytest.mark.parametrize("precision", [FP64, FP32])
def test_grid_16x100(w, precision):
    """16x100 grid (the serving network), value ~1e-300, below the float64
    range for some seeds: per-tensor exponents keep it."""
    H, W_ = 16, 100
    cnf = wmcgen.grid_cnf(H, W_, 1)
    wp, wn = wmcgen.weights_complementary(H * W_, 1, 0.05, 0.95)
    col = [i * W_ + j + 1 for j in range(W_) for i in range(H)]
    want = oracle.bucket_elim(cnf, wp, wn, order=col)
    res = plan_for(w, cnf, wp, wn, precision).execute()[0]
    assert rel(res, want) <= TOL[precision]


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_grid_24x200_full_size(w, precision):
    """24x200 grid at full size (max-rank 25, 2^25-entry tensors) against
    the stored oracle value."""
    with open(os.path.join(GOLDEN, "grid_24x200.json")) as f:
        g = json.load(f)
    for v in g["values"][:1]:
        seed = v["seed"]
        cnf = wmcgen.grid_cnf(24, 200, seed)
        wp, wn = wmcgen.weights_complementary(24 * 200, seed, 0.05, 0.95)
        res = plan_for(w, cnf, wp, wn, precision).execute()[0]
        assert rel(res, Big(v["mant"], v["exp2"])) <= TOL[precision]
        assert res.log10 < -300


# ------------------------------------------------ pairwise contraction

def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype=dtype)


def _pair_tol(k, precision):
    if precision == FP64:
        return 1e-12
    d = (2 ** min(k, 8)) + (2 ** max(k - 8, 0)) + 4
    return d * 2.0 ** -24 * 1.01


SWEEP_SMALL = [(ra, rb, b, k) for (b, k) in [(0, 1), (2, 1), (4, 1), (0, 4), (2, 4), (4, 4),
                                              (0, 8), (2, 8), (4, 8), (0, 16)]
               for (ra, rb) in [(b + k + 3, b + k + 2), (b + k + 9, b + k + 1)]]
# dense batched products (at least 2^6 free values on each side): the tiled kernel
SWEEP_SMALL += [(13, 14, 2, 5), (15, 14, 0, 8), (16, 16, 4, 6), (14, 14, 0, 8)]
# streaming products with four summed and/or four S-free indices (one lane per thread)
SWEEP_SMALL += [(10, 8, 0, 4), (12, 10, 2, 4), (9, 7, 0, 3), (13, 9, 2, 4), (14, 8, 4, 4)]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("ra,rb,b,k", SWEEP_SMALL)
@pytest.mark.parametrize("shuffle", [False, True])
def test_pair_small(w, precision, ra, rb, b, k, shuffle):
    """Every output of C = A . B against direct long-double summation."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=ra * 1000 + rb * 10 + b + k, shuffle=shuffle)
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c)
    got = _run_pair(w, case, precision)
    err = np.abs(got - want) / np.abs(want)
    assert err.max() <= _pair_tol(k, precision), err.max()


def _run_pair(w, case, precision, out_offsets=None):
    rc = len(case.labels_c)
    A64, B64 = _dev(case.a, torch.float64), _dev(case.b, torch.float64)
    if precision == FP64:
        C = torch.empty(1 << rc, dtype=torch.float64, device="cuda")
        w.contract_pair(FP64, case.labels_a, A64, case.labels_b, B64, case.labels_c, C)
        torch.cuda.synchronize()
        out = C
        scale = 1.0
    else:
        A = torch.empty(A64.numel(), dtype=torch.float32, device="cuda")
        B = torch.empty(B64.numel(), dtype=torch.float32, device="cuda")
        e = torch.zeros(3, dtype=torch.int64, device="cuda")
        w.to_scaled_fp32(A64, A, e[0:1])
        w.to_scaled_fp32(B64, B, e[1:2])
        del A64, B64
        C = torch.empty(1 << rc, dtype=torch.float32, device="cuda")
        w.contract_pair(FP32, case.labels_a, A, case.labels_b, B, case.labels_c, C, e[0:1], e[1:2], e[2:3])
        torch.cuda.synchronize()
        assert int(e[2]) == int(e[0]) + int(e[1])
        out = C.double()
        scale = 2.0 ** int(e[2])
    if out_offsets is not None:
        idx = torch.from_numpy(np.asarray(out_offsets)).to("cuda")
        return out[idx].cpu().numpy() * scale
    return out.cpu().numpy() * scale


# (rank A, rank B, batch, summed); outputs of rank 30, 28, 30, 30, 12
SWEEP_FULL = [(29, 5, 2, 1), (28, 12, 4, 4), (17, 17, 2, 1), (24, 22, 0, 8), (22, 22, 0, 16)]


@pytest.fixture(autouse=True)
def _free_device_memory():
    import gc
    yield
    gc.collect()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("ra,rb,b,k", SWEEP_FULL)
def test_pair_full_size_sampled(w, precision, ra, rb, b, k):
    """Full-size sweep cases (outputs up to 2^30): sampled outputs against
    the oracle, which evaluates those entries one by one."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=7 + ra + rb + k, shuffle=False)
    rc = len(case.labels_c)
    offs = np.random.default_rng(0).integers(0, 1 << rc, size=48)
    offs[0], offs[-1] = 0, (1 << rc) - 1
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c, offs)
    got = _run_pair(w, case, precision, offs)
    err = np.abs(got - want) / np.abs(want)
    assert err.max() <= _pair_tol(k, precision), err.max()
    torch.cuda.empty_cache()


# nodes summing more than 2^16 terms (Eq. (1) with 17..20 summed indices):
# (rank A, rank B, batch, summed); the last one would be a dense batched
# product (2^6 x 2^6 free values) if its summed range were short
SWEEP_LONG_SUM = [(24, 22, 0, 18), (22, 21, 2, 17), (21, 21, 1, 20), (23, 23, 0, 17)]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("ra,rb,b,k", SWEEP_LONG_SUM)
def test_pair_long_summed_range_accumulates_in_fp64(w, precision, ra, rb, b, k):
    """A node whose summed extent exceeds 2^16 accumulates in float64 even
    on the scaled-FP32 path.  The float32 result then differs from the
    exact sum only by the rounding of the float32 inputs (2 u per product)
    and of the output (u), u = 2^-24: a tolerance of 4 u.  Summing 2^17 or
    more terms in float32 (even in 256-term blocks) drifts well past it."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=300 + ra + rb + k, shuffle=True)
    rc = len(case.labels_c)
    offs = np.random.default_rng(k).integers(0, 1 << rc, size=min(48, 1 << rc))
    offs[0], offs[-1] = 0, (1 << rc) - 1
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c, offs)
    got = _run_pair(w, case, precision, offs)
    err = np.abs(got - want) / np.abs(want)
    tol = 1e-12 if precision == FP64 else 4 * 2.0 ** -24
    assert err.max() <= tol, err.max()


# shapes with several same-order variants: streaming (and TMA-staged),
# dense tiled / outer product, and the generic kernel
SWEEP_VARIANTS = [(20, 3, 2, 1), (18, 6, 0, 2), (15, 14, 1, 2), (13, 14, 2, 5), (12, 10, 2, 4), (16, 8, 4, 4)]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("ra,rb,b,k", SWEEP_VARIANTS)
def test_pair_variants_give_the_same_bits(w, precision, ra, rb, b, k):
    """Every variant the autotuner may pick for a node (wmc_pair_variants)
    adds the summed terms in the canonical order: forced one by one, each
    returns the fixed rule's bits (and exponent), which match the oracle."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=500 + ra + rb + k, shuffle=False)
    variants, chosen = w.pair_variants(precision, case.labels_a, case.labels_b, case.labels_c)
    assert chosen == 0 and len(variants) >= 2
    ref = None
    try:
        for kind, blocks in variants:
            w.wmc_debug_force_pair_variant(kind, blocks)
            got = _run_pair_raw(w, case, precision)
            if ref is None:
                ref = got
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1], (w.PAIR_KINDS[kind], blocks)
    finally:
        w.wmc_debug_force_pair_variant(-1, 0)
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c)
    err = np.abs(ref[0].astype(np.float64) * 2.0 ** ref[1] - want) / np.abs(want)
    assert err.max() <= _pair_tol(k, precision)


def _run_pair_raw(w, case, precision):
    """(C as stored, C's exponent) of one wmc_contract_pair call."""
    rc = len(case.labels_c)
    A64, B64 = _dev(case.a, torch.float64), _dev(case.b, torch.float64)
    if precision == FP64:
        C = torch.empty(1 << rc, dtype=torch.float64, device="cuda")
        w.contract_pair(FP64, case.labels_a, A64, case.labels_b, B64, case.labels_c, C)
        torch.cuda.synchronize()
        return C.cpu().numpy(), 0
    A = torch.empty(A64.numel(), dtype=torch.float32, device="cuda")
    B = torch.empty(B64.numel(), dtype=torch.float32, device="cuda")
    e = torch.zeros(3, dtype=torch.int64, device="cuda")
    w.to_scaled_fp32(A64, A, e[0:1])
    w.to_scaled_fp32(B64, B, e[1:2])
    C = torch.empty(1 << rc, dtype=torch.float32, device="cuda")
    w.contract_pair(FP32, case.labels_a, A, case.labels_b, B, case.labels_c, C, e[0:1], e[1:2], e[2:3])
    torch.cuda.synchronize()
    return C.cpu().numpy(), int(e[2])


def test_pair_autotune_keeps_the_bits(w):
    """With autotuning on, the first call of a shape times its variants and
    later calls use the fastest: the results stay the fixed rule's bits."""
    cases = [wmcgen.pair_case(ra, rb, b, k, seed=600 + ra + k, shuffle=False) for (ra, rb, b, k) in SWEEP_VARIANTS]
    fixed = [_run_pair_raw(w, c, FP32) for c in cases]
    try:
        w.wmc_set_autotune(1)
        for c, ref in zip(cases, fixed):
            for _ in range(2):  # the tuning call, then a tuned call
                got = _run_pair_raw(w, c, FP32)
                assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
            variants, chosen = w.pair_variants(FP32, c.labels_a, c.labels_b, c.labels_c)
            assert 0 <= chosen < len(variants)
    finally:
        w.wmc_set_autotune(0)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_plan_autotune_keeps_the_bits(w, precision):
    """wmc_autotune_plan times the walk's layouts and installs the fastest:
    no layout is rejected (all return the same bits), and the tuned plan's
    results equal the untuned plan's bit for bit."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    Q = 16
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=23, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, precision)
    before = plan.execute(wq, wnq)
    rep = plan.autotune(Q)
    ms = [l["ms"] for l in rep["layouts"]]
    assert len(ms) >= 5 and min(ms) >= 0
    assert ms[rep["chosen"]] == min(ms)
    assert plan.info(Q).launches_per_walk == rep["layouts"][rep["chosen"]]["launches"]
    after = plan.execute(wq, wnq)
    for q in range(Q):
        assert (after[q].mant, after[q].exp2, after[q].flags) == (before[q].mant, before[q].exp2, before[q].flags)


def test_pair_edge_cases(w):
    """Rank-0 output (full inner product), no summed index (outer product),
    a summed index present in one operand only."""
    rng = np.random.default_rng(1)
    for la, lb, lc in [([0, 1, 2], [2, 1, 0], []), ([0, 1], [2, 3], [3, 0, 2, 1]),
                       ([0, 1, 5], [1, 2], [2, 0]), ([4], [], [4])]:
        a = rng.random(1 << len(la)); b = rng.random(1 << len(lb))
        case = wmcgen.PairCase(la, lb, lc, a, b)
        want = oracle.contract_pair(la, a, lb, b, lc)
        for precision in (FP64, FP32):
            got = _run_pair(w, case, precision)
            assert np.max(np.abs(got - want) / np.abs(want)) <= _pair_tol(3, precision)


def test_pair_rejects_bad_labels(w):
    A = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(w._abi.WmcError):
        w.contract_pair(FP64, [0, 1], A, [1, 2], A, [0, 7], A)
    with pytest.raises(w._abi.WmcError):
        w.contract_pair(FP64, [0, 0], A, [1, 2], A, [0], A)


# ------------------------------------------------- device path, server

@pytest.mark.parametrize("precision", [FP64, FP32])
def test_execute_device_matches_host(w, precision):
    cnf = wmcgen.grid_cnf(8, 40, 2)
    plan = plan_for(w, cnf, None, None, precision)
    Q = 16
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=5, lo=0.05, hi=0.95)
    host = plan.execute(wq, wnq)
    info = plan.info(Q)
    ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device="cuda")
    dwp, dwn = _dev(wq, torch.float64), _dev(wnq, torch.float64)
    mant = torch.empty(Q, dtype=torch.float64, device="cuda")
    ex = torch.empty(Q, dtype=torch.int64, device="cuda")
    fl = torch.empty(Q, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        plan.execute_device(Q, dwp, dwn, ws, mant, ex, fl, stream=s)
        torch.cuda.synchronize()
        for q in range(Q):
            m, e = math.frexp(float(mant[q]))
            assert (m, e + int(ex[q])) == (host[q].mant, host[q].exp2)
    with pytest.raises(w._abi.WmcError) as err:
        plan.execute_device(Q, dwp, dwn, ws[: info.workspace_bytes // 2], mant, ex, fl, stream=s)
    assert err.value.status == w.WMC_EINVAL


def test_server_continuous_batching(w):
    """Queries submitted in bursts while earlier waves run: each result is
    identical to the same query run alone."""
    import time
    cnf = wmcgen.grid_cnf(10, 60, 3)
    plan = plan_for(w, cnf, None, None, FP32)
    n = 96
    wq, wnq = wmcgen.query_weights(cnf.n_vars, n, seed=6, lo=0.05, hi=0.95)
    alone = [plan.execute(wq[i:i + 1], wnq[i:i + 1])[0] for i in range(n)]
    srv = w.Server(plan, max_batch=32, max_waves=3)
    tickets = []
    for i in range(n):
        tickets.append(srv.submit(wq[i], wnq[i]))
        if i % 7 == 0:
            time.sleep(0.002)
    for i, t in enumerate(tickets):
        r = srv.wait(t, timeout_s=60)
        assert (r.mant, r.exp2) == (alone[i].mant, alone[i].exp2)
    st = srv.stats()
    assert st.completed == n and st.failed_waves == 0
    assert st.waves >= 2
    with pytest.raises(w._abi.WmcError) as e:
        srv.poll(tickets[0])  # already consumed
    assert e.value.status == w.WMC_EUNKNOWN_TICKET
    srv.close()


@pytest.mark.parametrize("partial_overlap", [0, 1])
def test_server_waves_overlap_under_load(w, partial_overlap):
    """A burst of four full waves: full waves run in both slots at once
    (their work overlaps on the device) under either wave-start policy, and
    every result equals the query run alone; trickling queries afterwards
    are admitted into later waves."""
    import time
    cnf = wmcgen.grid_cnf(10, 60, 3)
    plan = plan_for(w, cnf, None, None, FP32)
    n = 4 * 32 + 24
    wq, wnq = wmcgen.query_weights(cnf.n_vars, n, seed=16, lo=0.05, hi=0.95)
    alone = plan.execute(wq, wnq)
    srv = w.Server(plan, max_batch=32, max_waves=2, partial_overlap=partial_overlap)
    tickets = srv.submit_many(wq[:128], wnq[:128])
    for i in range(128, n):
        tickets.append(srv.submit(wq[i], wnq[i]))
        time.sleep(0.0005)
    for i, t in enumerate(tickets):
        r = srv.wait(t, timeout_s=60)
        assert (r.mant, r.exp2) == (alone[i].mant, alone[i].exp2), i
    st = srv.stats()
    assert st.completed == n and st.failed_waves == 0
    assert st.max_in_flight == 2
    srv.close()


def test_server_submit_many_matches_single_submits(w):
    """A block of queries submitted in one call gets consecutive tickets and
    the same results as the queries submitted one by one (and run alone)."""
    cnf = wmcgen.grid_cnf(10, 60, 3)
    plan = plan_for(w, cnf, None, None, FP32)
    n = 80
    wq, wnq = wmcgen.query_weights(cnf.n_vars, n, seed=8, lo=0.05, hi=0.95)
    alone = plan.execute(wq, wnq)
    srv = w.Server(plan, max_batch=32, max_waves=2)
    t_single = [srv.submit(wq[i], wnq[i]) for i in range(0, 20)]
    t_block = srv.submit_many(wq[20:], wnq[20:])
    assert t_block == list(range(t_block[0], t_block[0] + n - 20))
    assert t_block[0] > t_single[-1]
    for i, t in enumerate(t_single + t_block):
        r = srv.wait(t, timeout_s=60)
        assert (r.mant, r.exp2) == (alone[i].mant, alone[i].exp2), i
    assert srv.submit_many(wq[:0], wnq[:0]) == []
    srv.close()


def test_alloc_failure_is_reported(w):
    cnf = wmcgen.random_kcnf(14, 40, seed=9)
    plan = plan_for(w, cnf, None, None, FP32)
    w.wmc_debug_fail_next_allocs(1)
    with pytest.raises(w._abi.WmcError) as e:
        plan.execute()
    assert e.value.status == w.WMC_ENOMEM
    w.wmc_debug_fail_next_allocs(0)
    plan2 = plan_for(w, cnf, None, None, FP32)
    assert plan2.execute()[0].mant != 0.0


def test_bounded_wait_times_out_cleanly(w):
    """Failure detection without a GPU fault: the test hook keeps the TMA
    kernel's first copy from being issued, its bounded mbarrier wait runs
    out, the call returns WMC_ETIMEOUT, and the context stays usable."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    w.wmc_debug_stall_copies(1)
    try:
        plan = plan_for(w, cnf, None, None, FP32)
        wq, wnq = wmcgen.query_weights(cnf.n_vars, 64, seed=2, lo=0.05, hi=0.95)
        with pytest.raises(w._abi.WmcError) as e:
            plan.execute(wq, wnq)
        assert e.value.status == w.WMC_ETIMEOUT
    finally:
        w.wmc_debug_stall_copies(0)
    plan2 = plan_for(w, cnf, None, None, FP32)
    res = plan2.execute(wq[:4], wnq[:4])
    col = [i * 100 + j + 1 for j in range(100) for i in range(16)]
    want = oracle.bucket_elim(cnf, wq[0], wnq[0], order=col)
    assert rel(res[0], want) <= TOL[FP32]


# ---------------------------------------------------------- uneven batch

def _uneven(w, count, precision, **kw):
    plans, cnfs, rejected = [], [], 0
    for kind, cnf, wp, wn, sub in wmcgen.uneven_candidates(**kw):
        try:
            plans.append(w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=precision, max_rank_cap=20))
            cnfs.append((cnf, wp, wn))
        except w._abi.WmcError:
            rejected += 1
        if len(plans) == count:
            return plans, cnfs, rejected


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_uneven_batch_persistent(w, precision):
    """Mixed random 3-CNF and grid formulas in one persistent launch: each
    result equals the oracle and the formula's own graph walk."""
    plans, cnfs, _ = _uneven(w, 24, precision, seed=5, n3=(14, 40), grid_w=(3, 8), grid_h=(4, 30))
    batch = w.Batch(plans)
    assert batch.n_admitted == 24
    for rep in range(2):
        res = batch.execute()
        for i, (p, (cnf, wp, wn)) in enumerate(zip(plans, cnfs)):
            alone = p.execute()[0]
            assert Big(res[i].mant, res[i].exp2).rel_diff(Big(alone.mant, alone.exp2)) <= TOL[precision]
            if i % 3 == 0:
                want = oracle.bucket_elim(cnf, wp, wn, max_width=26)
                assert rel(res[i], want) <= TOL[precision], (i, rep)


def test_uneven_batch_with_chain_sized_formulas(w):
    """Formulas large enough that their own single-query walks fuse frontier
    chains: the persistent batch (one pass per node, its own layout) still
    gives each formula's result."""
    cnfs = [wmcgen.grid_cnf(h, wd, seed) for h, wd, seed in ((48, 16, 2), (64, 16, 5), (30, 12, 3))]
    plans = []
    for cnf in cnfs:
        wp, wn = wmcgen.weights_complementary(cnf.n_vars, 4, 0.05, 0.95)
        plans.append(plan_for(w, cnf, wp, wn, FP32))
    try:
        w.wmc_set_fusion(0)  # (a plan is laid out at its first info/execute)
        unfused = [plan_for(w, c, *wmcgen.weights_complementary(c.n_vars, 4, 0.05, 0.95), FP32) for c in cnfs]
        n_unfused = [p.info(1).launches_per_walk for p in unfused]
    finally:
        w.wmc_set_fusion(-1)
    assert any(p.info(1).launches_per_walk < n for p, n in zip(plans, n_unfused))  # chains formed
    batch = w.Batch(plans)
    assert batch.n_admitted == len(plans)
    res = batch.execute()
    for i, p in enumerate(plans):
        alone = p.execute()[0]
        assert Big(res[i].mant, res[i].exp2).rel_diff(Big(alone.mant, alone.exp2)) <= TOL[FP32], i


def _narrow_order(cnf):
    """The narrowest of the oracle's elimination orders for this formula:
    min-degree, variable-id order (row by row on the generator's grids) and,
    for formulas of up to 200 variables, min-fill."""
    orders = [oracle.min_degree_order(cnf), list(range(1, cnf.n_vars + 1))]
    if cnf.n_vars <= 200:
        orders.append(oracle.min_fill_order(cnf))
    return min(orders, key=lambda o: oracle.induced_width(cnf, o))


def test_uneven_batch_schedules_give_the_same_bits(w):
    """Task size and order change only how a node's outputs are split and
    when they run: the results are the same bits (round-robin over 2^15-
    output tasks, list scheduling over 2^13 and over 2^9), in both
    precisions, and each equals the formula's own walk and the oracle."""
    for precision in (FP32, FP64):
        plans, cnfs, _ = _uneven(w, 16, precision, seed=9, n3=(20, 44), grid_w=(4, 12), grid_h=(10, 60))
        got = []
        try:
            for chunk, order in ((15, 1), (13, 0), (9, 0)):
                w.wmc_set_batch_schedule(chunk, order)
                b = w.Batch(plans)
                got.append([(r.mant, r.exp2, r.flags) for r in b.execute()])
                del b
        finally:
            w.wmc_set_batch_schedule(0, 0)
        assert got[0] == got[1] == got[2]
        for i, (p, (cnf, wp, wn)) in enumerate(zip(plans, cnfs)):
            alone = p.execute()[0]
            assert Big(got[0][i][0], got[0][i][1]).rel_diff(Big(alone.mant, alone.exp2)) <= TOL[precision]
            if i % 4 == 0:
                want = oracle.bucket_elim(cnf, wp, wn, order=_narrow_order(cnf), max_width=30)
                r = Big(got[1][i][0], got[1][i][1]).rel_diff(want)
                assert r <= TOL[precision], (i, r)


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_uneven_batch_chains_and_subtrees_keep_the_bits(w, precision):
    """Runs of frontier eliminations in one pass (chains of up to 2 and 4
    steps) and small subtrees as one task each (output ranks <= 6 and <=
    12), against one pass per contraction, every node a task: the same bits
    for every formula (a chain's inner tensors are not rescaled, and the
    scales are powers of two), fewer algorithmic bytes, and the oracle's
    value."""
    plans, cnfs, _ = _uneven(w, 16, precision, seed=11, n3=(20, 40), grid_w=(4, 8), grid_h=(6, 30))
    got, infos = [], []
    try:
        for fz, sub in ((0, 0), (2, 0), (4, 0), (0, 6), (4, 6), (4, 12)):
            w.wmc_set_batch_fusion(fz)
            w.wmc_set_batch_subtrees(sub)
            b = w.Batch(plans)
            infos.append(b.info())
            got.append([(r.mant, r.exp2, r.flags) for r in b.execute()])
            del b
    finally:
        w.wmc_set_batch_fusion(4)
        w.wmc_set_batch_subtrees(12)
    assert all(g == got[0] for g in got)
    assert infos[2].algorithmic_bytes < infos[1].algorithmic_bytes < infos[0].algorithmic_bytes
    assert infos[2].n_nodes < infos[1].n_nodes < infos[0].n_nodes
    assert infos[3].algorithmic_bytes == infos[0].algorithmic_bytes and infos[3].n_nodes < infos[0].n_nodes
    for i in range(0, len(plans), 3):
        cnf, wp, wn = cnfs[i]
        want = oracle.bucket_elim(cnf, wp, wn, order=_narrow_order(cnf))
        assert Big(got[2][i][0], got[2][i][1]).rel_diff(want) <= TOL[precision], i


def test_uneven_batch_admission(w):
    """Admission by workspace bytes: only the prefix that fits is taken."""
    plans, _, _ = _uneven(w, 10, FP32, seed=6, n3=(14, 30), grid_w=(3, 6), grid_h=(4, 20))
    # formula i's workspace starts where the first i formulas' end (each
    # rounded up to 256 bytes)
    whole = w.Batch(plans)
    budget = whole.formula_info(4)[0]
    del whole
    batch = w.Batch(plans, mem_budget_bytes=budget)
    assert batch.n_admitted == 4
    assert len(batch.execute()) == 4
    assert w.Batch(plans, mem_budget_bytes=budget - 1).n_admitted == 3


_C5_CACHE = {}


def _c5_formulas(w, precision):
    """The uneven-batch configuration at full scale: the first 512 candidates
    (random 3-CNF n in [40, 120], clause ratio [2.0, 3.5]; grids of width
    6..20 and height 20..150; seed 3) whose plans have max-rank <= 26,
    planned on host threads (the planner releases the GIL)."""
    if precision in _C5_CACHE:
        return _C5_CACHE[precision]
    from concurrent.futures import ThreadPoolExecutor
    cands = []
    gen = wmcgen.uneven_candidates(3)
    plans = []
    with ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        while len(plans) < 512:
            chunk = [next(gen) for _ in range(64)]

            def one(c):
                kind, cnf, wp, wn, sub = c
                try:
                    return w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=precision, max_rank_cap=26)
                except w._abi.WmcError:
                    return None
            for c, p in zip(chunk, ex.map(one, chunk)):
                if p is not None and len(plans) < 512:
                    plans.append(p)
                    cands.append(c)
    _C5_CACHE[precision] = (plans, cands)
    return plans, cands


_C5_ORACLE = {}


def _c5_want(i, cand):
    if i not in _C5_ORACLE:
        kind, cnf, wp, wn, sub = cand
        if kind.startswith("grid"):  # row by row or column by column
            h_, w_ = (int(v) for v in kind[4:].split("x"))
            orders = (list(range(1, cnf.n_vars + 1)), wmcgen.grid_column_order(h_, w_))
        else:  # the oracle's two greedy orders
            orders = (oracle.min_degree_order(cnf), oracle.min_fill_order(cnf))
        order = min(orders, key=lambda o: oracle.induced_width(cnf, o))
        _C5_ORACLE[i] = oracle.bucket_elim(cnf, wp, wn, order=order, max_width=30)
    return _C5_ORACLE[i]


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_uneven_batch_full_scale(w, precision):
    """The uneven-batch configuration as benchmarked: 512 formulas in one
    persistent launch, a workspace of many GiB.  Compared with the oracle
    (bucket elimination, long double): every formula of max-rank 26, and
    formulas laid out past byte 2^32 of the batch workspace, one of each
    kind per GiB beyond it."""
    plans, cands = _c5_formulas(w, precision)
    batch = w.Batch(plans)
    assert batch.n_admitted == 512
    assert batch.info().workspace_bytes > 2 ** 32
    layout = [batch.formula_info(i) for i in range(512)]
    sample = [i for i, (off, r, n) in enumerate(layout) if r == 26]
    assert len(sample) >= 8
    seen = set()
    for i, (off, r, n) in enumerate(layout):
        key = (off >> 30, cands[i][0][:4])
        if off >= 2 ** 32 and r <= 17 and key not in seen:
            seen.add(key)
            sample.append(i)
    assert any(layout[i][0] >= 2 ** 32 and layout[i][1] == 26 for i in sample)
    assert layout[-1][0] >= 2 ** 32
    sample.append(511)
    for rep in range(2):
        res = batch.execute()
        for i in sorted(set(sample)):
            r = rel(res[i], _c5_want(i, cands[i]))
            assert r <= TOL[precision], (i, cands[i][0], layout[i], r)
            assert r <= res[i].rel_err_bound + 1e-16, (i, r, res[i].rel_err_bound)
    del batch


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_fused_chains_match_unfused(w, precision):
    """Consecutive frontier eliminations contracted in one pass (k2_chain,
    chains of up to 2, 3, 4; k2_chain_direct, runs of 5 and 6 in float32)
    give the same values as one pass per elimination (the intermediates'
    pow2 scales only move into the exponent), and match the oracle; longer
    chains move fewer bytes."""
    H, W_ = 16, 100
    cnf = wmcgen.grid_cnf(H, W_, 1)
    Q = 64
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=12, lo=0.05, hi=0.95)
    res, nbytes = {}, {}
    try:
        for level in (0, 1, 2, 3, 4, 5, 6):
            w.wmc_set_fusion(level)
            plan = plan_for(w, cnf, None, None, precision)
            res[level] = plan.execute(wq, wnq)
            nbytes[level] = plan.info(Q).algorithmic_bytes
    finally:
        w.wmc_set_fusion(-1)
    assert nbytes[4] < 0.7 * nbytes[0]
    assert nbytes[4] < nbytes[2] <= nbytes[0]
    if precision == FP32:
        # (a 16-step grid column: growth 4 + 6 + shrink 6 at six; still four
        # passes at five, 4 + 5 + 5 + 2)
        assert nbytes[6] < 0.8 * nbytes[4] and nbytes[5] <= nbytes[4]
    a = res[0]
    for level in (1, 2, 3, 4, 5, 6):
        b = res[level]
        for q in range(Q):
            assert (a[q].mant, a[q].exp2) == (b[q].mant, b[q].exp2), (level, q)
    col = wmcgen.grid_column_order(H, W_)
    for q in (0, 33):
        assert rel(res[4][q], oracle.bucket_elim(cnf, wq[q], wnq[q], order=col)) <= TOL[precision]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("case", ["random3cnf", "grid", "psi"])
def test_small_phase_matches_per_node_launches(w, precision, case):
    """The small-node phase (every node with at most 2^16 outputs and 2^8
    summed terms, run as tasks of one persistent launch in post-order)
    gives bit-identical values and flags to one launch per node, and the
    oracle's values; it replaces most launches of the walk."""
    if case == "random3cnf":
        cnf, Q, order = wmcgen.random_kcnf(24, 80, seed=21), 256, None
    elif case == "grid":
        cnf, Q, order = wmcgen.grid_cnf(16, 100, 1), 64, wmcgen.grid_column_order(16, 100)
    else:
        cnf, Q, order = wmcgen.psi_family(12), 3, None
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=14, lo=0.05, hi=0.95)
    try:
        w.wmc_set_small_phase(0)
        plain = plan_for(w, cnf, None, None, precision)
        a = plain.execute(wq, wnq)
        n_plain = plain.info(Q).launches_per_walk
    finally:
        w.wmc_set_small_phase(1)
    small = plan_for(w, cnf, None, None, precision)
    b = small.execute(wq, wnq)
    assert small.info(Q).launches_per_walk < n_plain
    for q in range(Q):
        assert (a[q].mant, a[q].exp2, a[q].flags) == (b[q].mant, b[q].exp2, b[q].flags), q
    for q in (0, Q - 1):
        want = oracle.bucket_elim(cnf, wq[q], wnq[q], order=order)
        assert rel(b[q], want) <= TOL[precision]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("Q,seed", [(1, 1), (1, 5), (2, 2), (1, 6)])
def test_cta_walk_matches_small_phase(w, precision, Q, seed):
    """A small formula's whole walk in one block (leaves and intermediates in
    shared memory, the nodes level by level between block barriers) gives
    the bits of the small-node phase and the oracle's value, in a handful
    of launches."""
    cnf = wmcgen.random_kcnf(20, 60, seed=seed)
    wq, wnq = wmcgen.query_weights(20, Q, seed=30 + seed, lo=0.1, hi=0.9)
    ref_plan = plan_for(w, cnf, None, None, precision)
    ref = ref_plan.execute(wq, wnq)
    try:
        w.wmc_set_cta_walk(1)
        plan = plan_for(w, cnf, None, None, precision)
        got = plan.execute(wq, wnq)
    finally:
        w.wmc_set_cta_walk(0)
    assert plan.info(Q).launches_per_walk == 2 < ref_plan.info(Q).launches_per_walk  # the walk, the finaliser
    for q in range(Q):
        assert (got[q].mant, got[q].exp2, got[q].flags) == (ref[q].mant, ref[q].exp2, ref[q].flags), q
        assert rel(got[q], oracle.brute_force(cnf, wq[q], wnq[q])[0]) <= TOL[precision]


# ------------------------------------------------------ index slicing (Alg. 3)

@pytest.mark.parametrize("precision", [FP64, FP32])
def test_sliced_walk_matches_unsliced(w, precision):
    """Index slicing: the walk runs once per slice assignment with the sliced
    variables fixed (clauses their literals satisfy become ones, their
    weights multiply the root) and the results are summed (Thm 4.2); the sum
    equals the unsliced walk and the oracle for several queries."""
    cnf = wmcgen.random_kcnf(20, 60, seed=2)
    Q = 3
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=13, lo=0.1, hi=0.9)
    full = plan_for(w, cnf, None, None, precision).execute(wq, wnq)
    r0 = plan_for(w, cnf, None, None, precision).info(1).max_rank
    sliced = plan_for(w, cnf, None, None, precision, slice_to_rank=r0 - 4)
    assert sliced.info(1).n_slice_vars >= 2
    got = sliced.execute(wq, wnq)
    for q in range(Q):
        want = oracle.brute_force(cnf, wq[q], wnq[q])[0]
        assert rel(got[q], want) <= TOL[precision], q
        assert Big(got[q].mant, got[q].exp2).rel_diff(Big(full[q].mant, full[q].exp2)) <= 2 * TOL[precision]
        assert rel(got[q], want) <= got[q].rel_err_bound  # the stated bound holds


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_batched_pairs_match_generic(w, precision):
    """Joins of two large operands with few free and summed indices on the
    batched small-contraction kernel (operands' batch indices in any order,
    query lanes one operand lacks broadcast, many free indices on one side
    as broadcast batch indices): the same bits as the generic kernel, and the
    oracle's value, for several queries."""
    cnf = wmcgen.random_kcnf(34, 110, seed=0)  # (max rank 21)
    Q = 5
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=21, lo=0.1, hi=0.9)
    out = {}
    try:
        for on in (1, 0):
            w.wmc_set_batched_pairs(on)
            plan = plan_for(w, cnf, None, None, precision)
            kinds = _launch_kinds(w, plan, Q, wq, wnq)
            out[on] = ([(r.mant, r.exp2, r.flags) for r in plan.execute(wq, wnq)], kinds)
    finally:
        w.wmc_set_batched_pairs(1)
    assert 11 in out[1][1] and 11 not in out[0][1]
    assert out[1][0] == out[0][0]
    order = _narrow_order(cnf)
    for q in (0, Q - 1):
        want = oracle.bucket_elim(cnf, wq[q], wnq[q], order=order)
        assert Big(out[1][0][q][0], out[1][0][q][1]).rel_diff(want) <= TOL[precision], q


def test_sliced_unweighted_count_is_exact(w):
    """Unit weights in FP64: the sliced count is the exact model count."""
    cnf = wmcgen.random_kcnf(20, 60, seed=5)
    exact = oracle.count_exact(cnf)
    r0 = w.Plan(w.Network.from_cnf(cnf), precision=FP64).info(1).max_rank
    plan = w.Plan(w.Network.from_cnf(cnf), precision=FP64, slice_to_rank=r0 - 3)
    assert plan.info(1).n_slice_vars >= 2
    r = plan.execute()[0]
    assert r.to_float() == float(exact)
    assert r.flags & w.WMC_FLAG_EXACT_INT


def test_slice_ranges_sum_to_the_whole(w):
    """Partial sums over disjoint slice ranges (one per process in a sharded
    run) combine to the full result; an empty range is zero."""
    cnf = wmcgen.random_kcnf(30, 90, seed=1)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, 2, seed=3, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, FP32, slice_to_rank=16)
    n = 1 << plan.info(1).n_slice_vars
    assert n >= 4
    whole = plan.execute(wq, wnq)
    cuts = [0, 1, n // 2, n]
    parts = [plan.execute_slices(cuts[i], cuts[i + 1], wq, wnq) for i in range(3)]
    assert plan.execute_slices(2, 2, wq, wnq)[0].mant == 0.0
    for q in range(2):
        tot = w.combine_results([p[q] for p in parts])
        assert Big(tot.mant, tot.exp2).rel_diff(Big(whole[q].mant, whole[q].exp2)) <= 1e-12
    with pytest.raises(w._abi.WmcError) as e:
        plan.execute_slices(0, n + 1, wq, wnq)
    assert e.value.status == w.WMC_EINVAL


def test_sliced_psi_beyond_the_rank_cap(w):
    """psi(34) has no plan within rank 30; sliced to 28 it runs and gives
    the closed form prod(w0 + w1) - prod(w1) - prod(w0)."""
    n = 34
    cnf = wmcgen.psi_family(n)
    wp, wn = wmcgen.weights_complementary(n, 7, 0.2, 0.8)
    plan = plan_for(w, cnf, wp, wn, FP64, slice_to_rank=28)
    r = plan.execute()[0]
    assert Big(r.mant, r.exp2).rel_diff(_psi_closed_form(wp, wn)) <= TOL[FP64]


def test_sliced_device_path_and_server(w):
    """The device entry and the server run every slice too."""
    cnf = wmcgen.random_kcnf(30, 90, seed=1)
    Q = 4
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=5, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, FP32, slice_to_rank=16)
    host = plan.execute(wq, wnq)
    info = plan.info(Q)
    dwp = torch.from_numpy(wq).cuda(); dwn = torch.from_numpy(wnq).cuda()
    ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device="cuda")
    m = torch.empty(Q, dtype=torch.float64, device="cuda"); e = torch.empty(Q, dtype=torch.int64, device="cuda")
    f = torch.empty(Q, dtype=torch.int32, device="cuda")
    plan.execute_device(Q, dwp, dwn, ws, m, e, f, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for q in range(Q):
        assert Big(*_norm_pair(float(m[q]), int(e[q]))).rel_diff(Big(host[q].mant, host[q].exp2)) == 0.0
    srv = w.Server(plan, max_batch=4, max_waves=2)
    ts = srv.submit_many(wq, wnq)
    for q, t in enumerate(ts):
        r = srv.wait(t, timeout_s=60)
        assert (r.mant, r.exp2) == (host[q].mant, host[q].exp2)
    srv.close()


def _norm_pair(mant, e):
    import math
    fm, fe = math.frexp(mant)
    return fm, (e + fe) if mant != 0.0 else 0


# dense float32 products with 2^7 x 2^7 output tiles: the tcgen05 kernel
# (rank A, rank B, batch, summed): 128- and 256-column accumulators, one
# 16-term chunk, a ring of stages that wraps within a tile (16 chunks), and
# more tiles than blocks (both accumulators reused, 512 tiles)
SWEEP_TC = [(13, 13, 1, 5), (16, 15, 0, 8), (17, 17, 2, 6), (15, 16, 1, 7), (12, 13, 0, 4), (18, 17, 1, 5)]


@pytest.mark.parametrize("ra,rb,b,k", SWEEP_TC)
@pytest.mark.parametrize("shuffle", [False, True])
def test_pair_tensor_cores(w, ra, rb, b, k, shuffle):
    """Dense float32 products on the tensor cores (tcgen05, 3xTF32): every
    output against direct long-double summation, and against the scalar
    tiled kernel, within float32 rounding of the two summation orders."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=ra * 100 + rb + 31 * k, shuffle=shuffle)
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c)
    got = _run_pair(w, case, FP32)
    try:
        w.wmc_set_tensor_cores(0)
        scalar = _run_pair(w, case, FP32)
    finally:
        w.wmc_set_tensor_cores(1)
    # 3 MMAs per 8-term step into a float32 accumulator, 2^-21 per product
    tol = (3 * (2 ** k) / 8 + 8) * 2.0 ** -24 + 2.0 ** -21
    assert (np.abs(got - want) / np.abs(want)).max() <= tol
    assert (np.abs(got - scalar) / np.abs(scalar)).max() <= tol + _pair_tol(k, FP32)


# dense products with one or two summed bits and 2^24 or more outputs: the
# streaming outer-product kernel; (rank A, rank B, batch, summed, swap): with
# swap the operands are passed as (B, A), so C's low bits are the second
# operand's free indices
SWEEP_OUTER = [(13, 13, 0, 1, False), (15, 14, 1, 2, False), (15, 14, 1, 2, True), (14, 15, 2, 1, True)]


@pytest.mark.parametrize("ra,rb,b,k,swap", SWEEP_OUTER)
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_pair_outer_products(w, ra, rb, b, k, swap, precision):
    """Short summed ranges with a large output: every output against the
    oracle, and the same bits as the tiled kernel (same summation order)."""
    case = wmcgen.pair_case(ra, rb, b, k, seed=ra * 7 + rb + 13 * k, shuffle=False)
    if swap:
        case = wmcgen.PairCase(case.labels_b, case.labels_a, case.labels_c, case.b, case.a)
    assert len(case.labels_c) >= 24
    want = oracle.contract_pair(case.labels_a, case.a, case.labels_b, case.b, case.labels_c)
    got = _run_pair(w, case, precision)
    try:
        w.wmc_set_outer_products(0)
        tiled = _run_pair(w, case, precision)
    finally:
        w.wmc_set_outer_products(1)
    assert np.array_equal(got, tiled)
    assert (np.abs(got - want) / np.abs(want)).max() <= _pair_tol(k, precision)


def test_pair_outer_products_full_size(w):
    """The sweep's (17, 17, b2, k1) row, 2^30 outputs: the same bits as the
    tiled kernel on sampled outputs, and those outputs against the oracle's
    sum over the two summed values."""
    case = wmcgen.pair_case(17, 17, 2, 1, seed=7 + 17 + 17 + 1, shuffle=False)
    rng = np.random.default_rng(3)
    offs = np.concatenate([np.arange(4096), rng.integers(0, 1 << 30, 60000), (1 << 30) - 1 - np.arange(64)])
    got = _run_pair(w, case, FP32, out_offsets=offs)
    try:
        w.wmc_set_outer_products(0)
        tiled = _run_pair(w, case, FP32, out_offsets=offs)
    finally:
        w.wmc_set_outer_products(1)
    assert np.array_equal(got, tiled)
    # C = [fa (14 bits), batch (2), fb (14)]; A = [fa, batch, s]; B = [s, batch, fb]
    i = offs & ((1 << 14) - 1); bb = (offs >> 14) & 3; j = offs >> 16
    want = sum(case.a[i + (bb << 14) + (s << 16)] * case.b[s + (bb << 1) + (j << 3)] for s in (0, 1))
    assert (np.abs(got - want) / np.abs(want)).max() <= _pair_tol(1, FP32)


# ------------------------------------------------------ clause factoring

def _psi_closed_form(wp, wn):
    """W(psi_n) = prod(w0 + w1) - prod(w1) - prod(w0), exactly (Sec. 3.3's
    example: every assignment but all-true and all-false satisfies psi)."""
    import math
    from fractions import Fraction
    pa, p1, p0 = Fraction(1), Fraction(1), Fraction(1)
    for a, b in zip(wp, wn):
        fa, fb = Fraction(float(a)), Fraction(float(b))
        pa *= fa + fb
        p1 *= fa
        p0 *= fb
    want = pa - p1 - p0
    e = want.numerator.bit_length() - want.denominator.bit_length()
    mant = float(want / Fraction(2) ** e) if e >= 0 else float(want * Fraction(2) ** (-e))
    m, fe = math.frexp(mant)
    return Big(m, e + fe)


def _long_clause_cnf(n, n_short, n_long, k_long, seed):
    short = wmcgen.random_kcnf(n, n_short, seed=seed)
    long_ = wmcgen.random_kcnf(n, n_long, seed=seed + 1000, k=k_long)
    return wmcgen.Cnf(n, short.clauses + long_.clauses)


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("seed", range(3))
def test_factored_long_clauses_match_oracle(w, precision, seed):
    """Clause factoring (Def. 3.4, Thm 3.3): formulas with 12-literal
    clauses, factored into rank-3 gate clauses, against brute force and
    against the unfactored plan."""
    n = 22
    cnf = _long_clause_cnf(n, 40, 4, 12, seed)
    wp, wn = wmcgen.weights_complementary(n, seed, 0.05, 0.95)
    want = oracle.brute_force(cnf, wp, wn)[0]
    fac = plan_for(w, cnf, wp, wn, precision, factor_clauses_above=3)
    assert fac.info(1).n_aux_vars == 4 * 10
    got = fac.execute()[0]
    assert rel(got, want) <= TOL[precision]
    assert rel(plan_for(w, cnf, wp, wn, precision).execute()[0], want) <= TOL[precision]


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("n", [64, 1000])
def test_factored_psi_closed_form(w, precision, n):
    """psi_n with rank-n clauses (no plan within rank 30 unfactored; n = 1000
    is beyond the network's 62-literal clause masks) against its closed
    form; unit weights give 2^n - 2."""
    cnf = wmcgen.psi_family(n)
    wp, wn = wmcgen.weights_independent(n, 11, 0.3, 1.2)
    r = plan_for(w, cnf, wp, wn, precision, factor_clauses_above=3).execute()[0]
    assert Big(r.mant, r.exp2).rel_diff(_psi_closed_form(wp, wn)) <= TOL[precision]
    u = plan_for(w, cnf, None, None, precision, factor_clauses_above=3).execute()[0]
    assert Big(u.mant, u.exp2).rel_diff(_psi_closed_form([1.0] * n, [1.0] * n)) <= TOL[precision]


def test_factored_query_batch_and_slicing(w):
    """A factored plan batches queries (each against the oracle) and slices
    (the sliced factored walk equals the unsliced one)."""
    n = 26
    cnf = _long_clause_cnf(n, 60, 5, 10, 5)
    Q = 16
    wq, wnq = wmcgen.query_weights(n, Q, seed=6, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, FP32, factor_clauses_above=3)
    got = plan.execute(wq, wnq)
    for i in range(Q):
        assert rel(got[i], oracle.bucket_elim(cnf, wq[i], wnq[i])) <= TOL[FP32]
    r0 = plan.info(1).max_rank
    sliced = plan_for(w, cnf, None, None, FP64, factor_clauses_above=3, slice_to_rank=r0 - 2)
    assert sliced.info(1).n_slice_vars > 0
    s = sliced.execute(wq, wnq)
    for i in range(Q):
        assert rel(s[i], oracle.bucket_elim(cnf, wq[i], wnq[i])) <= TOL[FP64]


# ------------------------------------------------------ runs of chains

def _launch_kinds(w, plan, Q, wq, wnq):
    """Kinds of the walk's launches (wmc_profile_walk: 8 chain, 9 run of chains)."""
    import ctypes
    info = plan.info(Q)
    dev = torch.device("cuda", 0)
    d_wp = torch.from_numpy(np.ascontiguousarray(wq[:Q])).to(dev)
    d_wn = torch.from_numpy(np.ascontiguousarray(wnq[:Q])).to(dev)
    ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device=dev)
    mant = torch.empty(Q, dtype=torch.float64, device=dev)
    ex = torch.empty(Q, dtype=torch.int64, device=dev)
    fl = torch.empty(Q, dtype=torch.int32, device=dev)
    nmax = 8192
    node_ms = (ctypes.c_float * nmax)()
    kinds = (ctypes.c_int32 * nmax)()
    nbytes = (ctypes.c_double * nmax)()
    nl = ctypes.c_int64()
    w.check(w.wmc_profile_walk(plan.handle, Q, ctypes.c_void_p(d_wp.data_ptr()), ctypes.c_void_p(d_wn.data_ptr()),
                               ctypes.c_void_p(ws.data_ptr()), info.workspace_bytes, ctypes.c_void_p(mant.data_ptr()),
                               ctypes.c_void_p(ex.data_ptr()), ctypes.c_void_p(fl.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), nmax, node_ms, kinds, nbytes,
                               ctypes.byref(nl)), "wmc_profile_walk")
    return [kinds[i] for i in range(min(nl.value, nmax))]


@pytest.mark.parametrize("Q", [4, 16, 64])
def test_chain_runs_match_single_launches(w, Q):
    """Runs of consecutive chains in one launch (k2_chain_seq: tiles handed
    out in chain order, each block waiting for the previous chain's
    completion count) give the bits of one launch per chain, and the
    oracle's values."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=12, lo=0.05, hi=0.95)
    try:
        w.wmc_set_fusion(4)  # (runs join chains of four steps)
        single = plan_for(w, cnf, None, None, FP32)
        n1 = single.info(Q).launches_per_walk
        r1 = single.execute(wq, wnq)
        w.wmc_set_chain_runs(512)
        runs = plan_for(w, cnf, None, None, FP32)
        n2 = runs.info(Q).launches_per_walk
        assert 9 in _launch_kinds(w, runs, Q, wq, wnq)
        r2 = runs.execute(wq, wnq)
    finally:
        w.wmc_set_chain_runs(0)
        w.wmc_set_fusion(-1)
    assert n2 * 4 < n1
    for q in range(Q):
        assert (r1[q].mant, r1[q].exp2, r1[q].flags) == (r2[q].mant, r2[q].exp2, r2[q].flags)
    col = [i * 100 + j + 1 for j in range(100) for i in range(16)]
    for q in (0, Q - 1):
        assert rel(r2[q], oracle.bucket_elim(cnf, wq[q], wnq[q], order=col)) <= TOL[FP32]


def test_chain_runs_on_two_streams(w):
    """Two walks whose runs of chains execute at the same time on two
    streams (no block waits on work that a non-running block holds) give
    the results of the walks one at a time."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    Q = 8
    wq, wnq = wmcgen.query_weights(cnf.n_vars, 2 * Q, seed=13, lo=0.05, hi=0.95)
    try:
        w.wmc_set_fusion(4)  # (runs join chains of four steps)
        w.wmc_set_chain_runs(512)
        plan = plan_for(w, cnf, None, None, FP32)
        info = plan.info(Q)
    finally:
        w.wmc_set_chain_runs(0)
        w.wmc_set_fusion(-1)
    ref = [plan.execute(wq[k * Q:(k + 1) * Q], wnq[k * Q:(k + 1) * Q]) for k in range(2)]
    dev = torch.device("cuda", 0)
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    bufs = []
    for k in range(2):
        d_wp = torch.from_numpy(np.ascontiguousarray(wq[k * Q:(k + 1) * Q])).to(dev)
        d_wn = torch.from_numpy(np.ascontiguousarray(wnq[k * Q:(k + 1) * Q])).to(dev)
        ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device=dev)
        bufs.append((d_wp, d_wn, ws, torch.empty(Q, dtype=torch.float64, device=dev),
                     torch.empty(Q, dtype=torch.int64, device=dev), torch.empty(Q, dtype=torch.int32, device=dev)))
    torch.cuda.synchronize()
    for rep in range(6):
        for k in range(2):
            d_wp, d_wn, ws, m, e, f = bufs[k]
            plan.execute_device(Q, d_wp, d_wn, ws, m, e, f, stream=streams[k].cuda_stream)
    torch.cuda.synchronize()
    for k in range(2):
        m, e = bufs[k][3].cpu().numpy(), bufs[k][4].cpu().numpy()
        for q in range(Q):
            r = ref[k][q]
            got = Big(float(m[q]), int(e[q]))
            assert got.rel_diff(Big(r.mant, r.exp2)) <= 1e-15


def test_chain_run_bounded_wait_times_out_cleanly(w):
    """Failure detection inside a run of chains without a GPU fault: the
    test hook keeps the first tile of the run's first chain from being
    copied; the block's bounded wait runs out, the others' waits for that
    chain see the error word, the call returns WMC_ETIMEOUT and the context
    stays usable."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    Q = 8
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=14, lo=0.05, hi=0.95)
    w.wmc_set_fusion(4)  # (runs join chains of four steps)
    w.wmc_set_chain_runs(512)
    try:
        probe = plan_for(w, cnf, None, None, FP32)
        assert 9 in _launch_kinds(w, probe, Q, wq, wnq)  # the walk has runs of chains
        w.wmc_debug_stall_copies(2)
        plan = plan_for(w, cnf, None, None, FP32)
        with pytest.raises(w._abi.WmcError) as e:
            plan.execute(wq, wnq)
        assert e.value.status == w.WMC_ETIMEOUT
    finally:
        w.wmc_debug_stall_copies(0)
        w.wmc_set_chain_runs(0)
        w.wmc_set_fusion(-1)
    plan2 = plan_for(w, cnf, None, None, FP32)
    res = plan2.execute(wq, wnq)
    col = [i * 100 + j + 1 for j in range(100) for i in range(16)]
    assert rel(res[0], oracle.bucket_elim(cnf, wq[0], wnq[0], order=col)) <= TOL[FP32]


def test_serving_config_as_benchmarked(w):
    """The timed configuration itself: the 16x100 grid network, waves of
    Q = 256 queries from the pool w ~ U(0.05, 0.95) (seed 1), two waves in
    flight on two streams with their own workspaces (graph replays); sampled
    queries of each wave against the oracle, one by one."""
    H, W_, Q = 16, 100, 256
    cnf = wmcgen.grid_cnf(H, W_, 1)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, 4096, seed=1, lo=0.05, hi=0.95)  # the pool
    plan = plan_for(w, cnf, None, None, FP32)
    info = plan.info(Q)
    dev = torch.device("cuda", 0)
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    slots = []
    for k in range(2):
        slots.append((torch.from_numpy(np.ascontiguousarray(wq[k * Q:(k + 1) * Q])).to(dev),
                      torch.from_numpy(np.ascontiguousarray(wnq[k * Q:(k + 1) * Q])).to(dev),
                      torch.empty(info.workspace_bytes, dtype=torch.uint8, device=dev),
                      torch.empty(Q, dtype=torch.float64, device=dev), torch.empty(Q, dtype=torch.int64, device=dev),
                      torch.empty(Q, dtype=torch.int32, device=dev)))
    torch.cuda.synchronize()
    for rep in range(3):
        for k in range(2):
            d_wp, d_wn, ws, m, e, f = slots[k]
            plan.execute_device(Q, d_wp, d_wn, ws, m, e, f, stream=streams[k].cuda_stream)
    torch.cuda.synchronize()
    col = [i * W_ + j + 1 for j in range(W_) for i in range(H)]
    for k in range(2):
        m, e, f = (slots[k][3].cpu().numpy(), slots[k][4].cpu().numpy(), slots[k][5].cpu().numpy())
        for q in (0, 37, 128, Q - 1):
            assert int(f[q]) & 0x8 == 0
            want = oracle.bucket_elim(cnf, wq[k * Q + q], wnq[k * Q + q], order=col)
            assert Big(float(m[q]), int(e[q])).rel_diff(want) <= TOL[FP32]


def test_large_batch_chains_are_batch_invariant(w):
    """Waves of 512 queries (bucket tensors of 2^13 entries with the query
    bits: one work unit per thread beside the staged S_i) still run as
    chains, and give each query the bits it gets alone."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    Q = 512
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=15, lo=0.05, hi=0.95)
    plan = plan_for(w, cnf, None, None, FP32)
    assert plan.info(Q).launches_per_walk < 500
    res = plan.execute(wq, wnq)
    for q in (0, 300, Q - 1):
        alone = plan.execute(wq[q:q + 1], wnq[q:q + 1])[0]
        assert (res[q].mant, res[q].exp2) == (alone.mant, alone.exp2)
    col = [i * 100 + j + 1 for j in range(100) for i in range(16)]
    assert rel(res[300], oracle.bucket_elim(cnf, wq[300], wnq[300], order=col)) <= TOL[FP32]


def test_single_lane_chains_match_unfused(w):
    """One query on the 24x200 grid (max rank 25: one lane per thread, the
    chains' FAST variant whose bucket tensors hold one value for all lanes)
    gives the bits of one pass per elimination."""
    cnf = wmcgen.grid_cnf(24, 200, 1)
    wp, wn = wmcgen.weights_complementary(4800, 1, 0.05, 0.95)
    out = {}
    try:
        for fuse in (4, 6, 0):
            w.wmc_set_fusion(fuse)
            plan = plan_for(w, cnf, wp, wn, FP32)
            r = plan.execute()[0]
            out[fuse] = (r.mant, r.exp2, plan.info(1).launches_per_walk)
    finally:
        w.wmc_set_fusion(-1)
    assert out[4][2] * 2 < out[0][2] and out[6][2] < out[4][2]
    assert out[4][:2] == out[0][:2] == out[6][:2]
