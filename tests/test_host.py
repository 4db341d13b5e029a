"""Host-side tests of the C ABI library (no GPU needed): every declared
symbol is exported, the reduction matches Thm 3.2's structure, the planner's
contraction tree is a valid tree whose evaluation (done here in numpy, from
the tree the library reports) equals the oracle, and malformed input is
rejected with the documented status codes."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import wmcgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2006_15512_b300 as w
    return w


def test_every_declared_symbol_is_exported():
    w = _lib()
    hdr = open(os.path.join(ROOT, "include", "wmc.h")).read()
    declared = set(re.findall(r"\b(wmc_[a-z0-9_]+)\s*\(", hdr))
    declared = {d for d in declared if not d.endswith("_t")}
    out = subprocess.check_output(["nm", "-D", "--defined-only", w._abi.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (wmc_[a-z0-9_]+)$", out, flags=re.M))
    assert declared, "no declarations parsed"
    assert declared <= exported, f"missing: {sorted(declared - exported)}"
    assert declared <= set(w._abi.EXPORTS), f"binding lacks: {sorted(declared - set(w._abi.EXPORTS))}"


def test_fig1_network_structure():
    """Thm 3.2 on Fig. 1: 8 tensors, 10 indices."""
    w = _lib()
    cnf, _ = wmcgen.fig1_example()
    info = w.Network.from_cnf(cnf).info()
    assert info.n_tensors_strict == 8
    assert info.n_indices_strict == 10
    assert info.max_clause_rank == 3


def _leaf_tensor(kind, labels, fals, wp, wn):
    r = len(labels)
    if kind == 0:
        t = np.ones(1 << r)
        t[fals] = 0.0
    elif kind == 1:
        x = labels[0]
        t = np.array([wn[x], wp[x]])
    else:
        t = np.ones(1)
    return t


def _einsum_labels(labels, letters):
    return "".join(letters.setdefault(l, chr(ord("a") + len(letters)) if len(letters) < 26
                                      else chr(ord("A") + len(letters) - 26))
                   for l in reversed(labels))


def evaluate_plan_numpy(plan, wp, wn):
    """Walk the library's contraction tree bottom-up with numpy (test-side
    evaluation of Algorithm 2)."""
    leaves = plan.leaves()
    nodes = plan.nodes()
    tens = []
    labs = []
    for kind, labels, fals in leaves:
        tens.append(_leaf_tensor(kind, labels, fals, wp, wn))
        labs.append(labels)
    for a, b, lc in nodes:
        letters = {}
        ea, eb = _einsum_labels(labs[a], letters), _einsum_labels(labs[b], letters)
        ec = _einsum_labels(lc, letters)
        A = tens[a].reshape((2,) * len(labs[a]))
        B = tens[b].reshape((2,) * len(labs[b]))
        C = np.einsum(f"{ea},{eb}->{ec}", A, B)
        tens.append(np.asarray(C).reshape(-1))
        labs.append(lc)
    assert len(labs[-1]) == 0
    return float(tens[-1][0])


def _check_tree_shape(plan):
    """Every tensor id is consumed exactly once except the root; children
    precede their parent (post-order)."""
    n_leaves = plan.info(1).n_leaves
    nodes = plan.nodes()
    used = {}
    for i, (a, b, _) in enumerate(nodes):
        cid = n_leaves + i
        assert a < cid and b < cid and a != b
        used[a] = used.get(a, 0) + 1
        used[b] = used.get(b, 0) + 1
    total = n_leaves + len(nodes)
    for t in range(total - 1):
        assert used.get(t, 0) == 1, f"tensor {t} used {used.get(t, 0)} times"
    assert used.get(total - 1, 0) == 0


@pytest.mark.parametrize("ordering", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", range(5))
def test_plan_tree_evaluates_to_oracle(ordering, seed):
    """Thm 3.1: any valid plan gives W(phi); checked for every ordering."""
    w = _lib()
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 15))
    cnf = wmcgen.random_kcnf(n, int(rng.integers(n, 3 * n)), seed=seed)
    wp, wn = wmcgen.weights_independent(n, seed, 0.1, 1.0)
    net = w.Network.from_cnf(cnf, wp, wn)
    plan = w.Plan(net, precision=0, ordering=ordering)
    _check_tree_shape(plan)
    got = evaluate_plan_numpy(plan, wp, wn)
    want = oracle.brute_force(cnf, wp, wn)[0].to_float()
    assert abs(got - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("cnf", [
    wmcgen.Cnf(0, []), wmcgen.Cnf(3, []), wmcgen.Cnf(2, [[]]), wmcgen.Cnf(3, [[1, -1], [2]]),
    wmcgen.Cnf(4, [[1, 1, 2], [-2, 3]]), wmcgen.psi_family(6), wmcgen.Cnf(5, [[2, 3]]),
], ids=["n0", "free3", "empty-clause", "tautology", "dup-literal", "psi6", "isolated-vars"])
def test_plan_edge_cases(cnf):
    w = _lib()
    wp, wn = wmcgen.weights_independent(max(cnf.n_vars, 1), 9, 0.2, 1.3)
    wp, wn = wp[:cnf.n_vars], wn[:cnf.n_vars]
    net = w.Network.from_cnf(cnf, wp, wn)
    plan = w.Plan(net, precision=0)
    _check_tree_shape(plan)
    got = evaluate_plan_numpy(plan, wp, wn)
    want = oracle.brute_force(cnf, wp, wn)[0].to_float()
    assert abs(got - want) <= 1e-13 * max(abs(want), 1e-300)


def test_grid_plan_width():
    """The order portfolio finds the sweep on the configs' grids: max-rank
    25 on 24x200 and 17 on 16x100 (min-fill alone reaches 32+)."""
    w = _lib()
    for (H, W_, cap) in [(24, 200, 26), (16, 100, 18)]:
        net = w.Network.from_cnf(wmcgen.grid_cnf(H, W_, 0))
        info = w.Plan(net).info(1)
        assert info.max_rank <= cap, (H, W_, info.max_rank)
        with pytest.raises(w._abi.WmcError) as e:   # min-fill alone is far wider
            w.Plan(net, ordering=1, max_rank_cap=cap + 2)
        assert e.value.status == w.WMC_EPLAN_TOO_BIG


def test_layouts_keep_big_operand_order():
    """Layout rule: in each node the kept indices of the larger operand
    keep their relative order in the output."""
    w = _lib()
    plan = w.Plan(w.Network.from_cnf(wmcgen.grid_cnf(6, 30, 1)))
    labs = [l for _, l, _ in plan.leaves()]
    for a, b, lc in plan.nodes():
        P = labs[a] if len(labs[a]) >= len(labs[b]) else labs[b]
        kept = [l for l in P if l in lc]
        assert [l for l in lc if l in P] == kept
        labs.append(lc)


def test_invalid_inputs():
    w = _lib()
    with pytest.raises(w._abi.WmcError) as e:
        w.Network(3, np.array([1, 4], dtype=np.int32), np.array([0, 2]))
    assert e.value.status == w.WMC_EINVAL
    with pytest.raises(w._abi.WmcError) as e:
        w.Network(3, np.array([1, 0], dtype=np.int32), np.array([0, 2]))
    assert e.value.status == w.WMC_EINVAL
    with pytest.raises(w._abi.WmcError) as e:
        w.Network(3, np.array([1, 2], dtype=np.int32), np.array([0, 2, 1]))
    assert e.value.status == w.WMC_EINVAL
    net = w.Network.from_cnf(wmcgen.grid_cnf(16, 100, 0))
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net, max_rank_cap=10)
    assert e.value.status == w.WMC_EPLAN_TOO_BIG
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net, mem_budget_bytes=1 << 20)
    assert e.value.status == w.WMC_EPLAN_TOO_BIG
    plan = w.Plan(net)
    with pytest.raises(w._abi.WmcError) as e:
        plan.info(0)
    assert e.value.status == w.WMC_EINVAL
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net, order=[1] * net.n_vars)
    assert e.value.status == w.WMC_EINVAL


def test_workspace_grows_with_q():
    w = _lib()
    plan = w.Plan(w.Network.from_cnf(wmcgen.grid_cnf(16, 100, 0)))
    a, b = plan.info(1), plan.info(256)
    # a lone float32 query on this small network runs as two lanes
    assert plan.info(2).workspace_bytes == a.workspace_bytes
    assert b.workspace_bytes > 50 * a.workspace_bytes
    # (chains of eliminations differ between the two layouts: not exactly 128x)
    assert b.algorithmic_bytes > 50 * a.algorithmic_bytes
    # FP64 keeps one lane
    p64 = w.Plan(w.Network.from_cnf(wmcgen.grid_cnf(16, 100, 0)), precision=w.WMC_FP64)
    assert p64.info(1).workspace_bytes < p64.info(2).workspace_bytes


@pytest.mark.parametrize("Q", [1, 3, 256])
def test_bounds_check_of_every_launch(Q):
    """CPU replay of every contraction launch's index arithmetic (bulk
    copies of every tile, extreme and sampled per-thread offsets): every
    access stays inside its tensor."""
    import ctypes
    w = _lib()
    for cnf in (wmcgen.grid_cnf(16, 100, 1), wmcgen.random_kcnf(30, 90, 2), wmcgen.psi_family(16),
                wmcgen.grid_cnf(8, 40, 2)):
        for precision in (0, 1):
            plan = w.Plan(w.Network.from_cnf(cnf), precision=precision)
            n = ctypes.c_int64()
            rc = w.wmc_debug_check_bounds(plan.handle, Q, ctypes.byref(n))
            assert rc == 0, w.wmc_last_error()
            assert n.value > 0


@pytest.mark.parametrize("Q", [1, 2, 4])
def test_bounds_check_of_one_block_walks(Q):
    """The one-block walk's level layout on the CPU: levels partition the
    node list, each level's lookup tables and outputs sit back to back in
    their shared-memory region, and every node's operands and output stay
    inside their arena tensors (children are freed only after their whole
    level)."""
    import ctypes
    w = _lib()
    try:
        w.wmc_set_cta_walk(1)
        for seed in range(6):
            for precision in (0, 1):
                plan = w.Plan(w.Network.from_cnf(wmcgen.random_kcnf(20, 60, seed)), precision=precision)
                n = ctypes.c_int64()
                assert w.wmc_debug_check_bounds(plan.handle, Q, ctypes.byref(n)) == 0, w.wmc_last_error()
                assert n.value > 0
    finally:
        w.wmc_set_cta_walk(0)


def test_slicing_plan_meets_its_target():
    """Index slicing (Alg. 3): the planner fixes variables until the largest
    tensor fits the target; the sliced variables are distinct, appear in no
    leaf, and every launch of the sliced walk stays in bounds."""
    w = _lib()
    cnf = wmcgen.random_kcnf(20, 60, seed=0)
    base = w.Plan(w.Network.from_cnf(cnf), precision=w.WMC_FP64)
    r0 = base.info(1).max_rank
    assert base.info(1).n_slice_vars == 0
    same = w.Plan(w.Network.from_cnf(cnf), precision=w.WMC_FP64, slice_to_rank=r0)
    assert same.info(1).n_slice_vars == 0  # already within the target
    for target in (r0 - 2, r0 - 5):
        p = w.Plan(w.Network.from_cnf(cnf), precision=w.WMC_FP64, slice_to_rank=target)
        info = p.info(1)
        sv = p.slice_vars
        assert info.max_rank <= target and 0 < len(sv) == info.n_slice_vars
        assert len(set(sv)) == len(sv) and all(0 <= v < 20 for v in sv)
        for kind, labels, _ in p.leaves():
            assert not set(labels) & set(sv)
        for Q in (1, 4):
            n = ctypes.c_int64()
            assert w.wmc_debug_check_bounds(p.handle, Q, ctypes.byref(n)) == w.WMC_OK, w.wmc_last_error()


def test_slicing_makes_a_too_wide_formula_plannable():
    """psi with 34 literals per clause has rank-34 clause tensors: no plan
    within rank 30; slicing to 28 fixes 6 variables (64 slices)."""
    w = _lib()
    net = w.Network.from_cnf(wmcgen.psi_family(34))
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net)
    assert e.value.status == w.WMC_EPLAN_TOO_BIG
    p = w.Plan(net, slice_to_rank=28)
    assert p.info(1).max_rank <= 28 and p.info(1).n_slice_vars == 6


def test_slice_ranges_and_combination():
    """slice_range splits [0, n) into contiguous per-process ranges that
    cover it once; combine_results sums exponent-aligned values."""
    w = _lib()
    for n in (1, 2, 7, 64):
        for world in (1, 2, 3, 8):
            rs = [w.slice_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    R = w.Result
    parts = [R(0.75, 10, 0, 0, 0.0), R(0.5, -3, 0, 2, 1e-9), R(0.0, 0, 0, 0, 0.0), R(0.625, 12, 0, 0, 0.0)]
    tot = w.combine_results(parts)
    want = 0.75 * 2 ** 10 + 0.5 * 2 ** -3 + 0.625 * 2 ** 12
    assert math.isclose(tot.to_float(), want, rel_tol=1e-15)
    assert tot.flags == 2 and tot.rel_err_bound >= 1e-9
    tiny = w.combine_results([R(0.5, -5000, 0, 0, 0.0), R(0.5, -5001, 0, 0, 0.0)])
    assert (tiny.mant, tiny.exp2) == (0.75, -5000)
    assert w.combine_results([]).mant == 0.0
    # exact integer shares stay flagged exact while the total is below 2^53
    E = w.WMC_FLAG_EXACT_INT
    ex = w.combine_results([R(0.5, 52, 0, E, 0.0), R(0.75, 2, 0, E, 0.0)])
    assert ex.to_float() == 2.0 ** 51 + 3 and ex.flags == E
    big = w.combine_results([R(0.5, 53, 0, E, 0.0), R(0.5, 53, 0, E, 0.0)])
    assert big.to_float() == 2.0 ** 53 and not big.flags & E
    assert not w.combine_results([R(0.5, 2, 0, E, 0.0), R(0.5, 2, 0, 0, 0.0)]).flags & E
    # exponents far apart: the small part is below the sum's last bit
    far = w.combine_results([R(0.5, 5000, 0, 0, 0.0), R(0.5, -5000, 0, 0, 0.0)])
    assert (far.mant, far.exp2) == (0.5, 5000)
    # unnormalised mantissas are accepted (value = mant * 2^exp2)
    un = w.combine_results([R(3.0, 4, 0, 0, 0.0), R(-1.0, 4, 0, 0, 0.0)])
    assert un.to_float() == 32.0
    assert math.isclose(un.log10, math.log10(32.0), rel_tol=1e-15)
    # error bound: the largest part bound plus one rounding per addition
    b3 = w.combine_results([R(0.5, 1, 0, 0, 1e-7), R(0.5, 1, 0, 0, 3e-7), R(0.5, 1, 0, 0, 0.0)])
    assert b3.rel_err_bound == 3e-7 + 2 * 2.0 ** -53
    out = w._abi.wmc_result()
    assert w.wmc_combine_results(None, -1, ctypes.byref(out)) == w.WMC_EINVAL
    nan = (w._abi.wmc_result * 1)()
    nan[0].mant = float("nan")
    assert w.wmc_combine_results(nan, 1, ctypes.byref(out)) == w.WMC_EINVAL


def test_pair_variants_listing():
    """wmc_pair_variants lists the fixed rule's kernel first and, for
    shapes in the canonical summation order, the other same-order kernels
    the autotuner may pick; shapes whose rule picks another order (the
    tensor-core product, the split summed range) list only that one."""
    w = _lib()
    K = {v: k for k, v in w.PAIR_KINDS.items()}
    def kinds(ra, rb, b, k, prec):
        pc = wmcgen.pair_case(ra, rb, b, k, seed=1, shuffle=False, with_data=False)
        v, ch = w.pair_variants(prec, pc.labels_a, pc.labels_b, pc.labels_c)
        assert ch == 0
        return [x[0] for x in v]
    assert kinds(29, 5, 2, 1, 1)[0] == K["k2_tma"] and K["k2_stream"] in kinds(29, 5, 2, 1, 1)
    assert kinds(17, 17, 2, 1, 1)[:2] == [K["k4_outer"], K["k4_dense"]]
    assert kinds(24, 22, 0, 8, 1) == [K["k4_tc"]]
    assert kinds(24, 22, 0, 8, 0)[0] == K["k4_dense"]
    assert kinds(22, 22, 0, 16, 1) == [K["k4_dense split"]]
    for sh in [(29, 5, 2, 1), (17, 17, 2, 1), (13, 14, 2, 5), (12, 10, 2, 4)]:
        assert kinds(*sh, 1)[-1] == K["k1_generic"]


def test_block_fp_options():
    """Block floating point: at most 9, scaled-FP32 plans only, not with
    index slicing, blocks of at most 2^11 outputs with the query bits; its
    walks pass the host bounds replay, exponent arrays included."""
    w = _lib()
    import ctypes
    cnf = wmcgen.random_kcnf(20, 60, seed=3)
    net = w.Network.from_cnf(cnf)
    for bad in (dict(block_fp=10), dict(block_fp=-1), dict(block_fp=2, precision=w.WMC_FP64),
                dict(block_fp=2, slice_to_rank=10)):
        kw = dict(precision=w.WMC_SCALED_FP32)
        kw.update(bad)
        with pytest.raises(w._abi.WmcError) as e:
            w.Plan(net, **kw)
        assert e.value.status == w.WMC_EINVAL
    p = w.Plan(net, precision=w.WMC_SCALED_FP32, block_fp=5)  # blocks of 16 assignments
    with pytest.raises(w._abi.WmcError):
        p.info(1024)  # 10 query bits + 4 block bits > 11
    for Q in (1, 4, 64):
        n = ctypes.c_int64()
        assert w.wmc_debug_check_bounds(p.handle, Q, ctypes.byref(n)) == w.WMC_OK
        assert n.value >= p.info(Q).n_nodes  # every node (and the weight table)
    plans = [w.Plan(net, precision=w.WMC_SCALED_FP32, block_fp=1)]
    with pytest.raises(w._abi.WmcError):
        w.Batch(plans)


def test_batch_chain_tables():
    """Host side of the uneven batch's chains and small-subtree tasks:
    longer chains leave fewer nodes and tasks and fewer algorithmic bytes;
    subtree tasks leave the bytes and cut the scheduled units; the layout
    replay (every operand live when read, no output over a live tensor)
    passes for every setting; chains need 2 steps at least."""
    w = _lib()
    plans = []
    for h, wd, seed in ((30, 8, 1), (24, 7, 2), (16, 9, 3)):
        plans.append(w.Plan(w.Network.from_cnf(wmcgen.grid_cnf(h, wd, seed)), precision=w.WMC_SCALED_FP32))
    plans.append(w.Plan(w.Network.from_cnf(wmcgen.random_kcnf(40, 100, seed=4)), precision=w.WMC_FP64))
    infos = {}
    try:
        for sub in (0, 6):
            w.wmc_set_batch_subtrees(sub)
            for fz in (0, 1, 2, 3, 4, 9):
                w.wmc_set_batch_fusion(fz)
                for prec_plans in (plans[:3], plans[3:]):
                    b = w.Batch(prec_plans)
                    assert b.n_admitted == len(prec_plans)
                    infos.setdefault((sub, fz), []).append(b.info())
    finally:
        w.wmc_set_batch_fusion(4)
        w.wmc_set_batch_subtrees(12)
    g = {fz: v[0] for (sub, fz), v in infos.items() if sub == 0}  # the grids, every node a task
    assert g[0].n_nodes == g[1].n_nodes and g[0].algorithmic_bytes == g[1].algorithmic_bytes
    assert g[4].n_nodes == g[9].n_nodes  # (at most 4 steps)
    assert g[4].n_nodes < g[3].n_nodes < g[2].n_nodes < g[0].n_nodes
    assert g[4].algorithmic_bytes < g[3].algorithmic_bytes < g[2].algorithmic_bytes < g[0].algorithmic_bytes
    assert g[4].n_tasks < g[0].n_tasks
    # small subtrees (output rank <= 6) as one task each: the same
    # contractions (bytes), far fewer scheduled units, in both precisions
    for i in range(2):
        assert infos[(6, 0)][i].algorithmic_bytes == infos[(0, 0)][i].algorithmic_bytes
        assert infos[(6, 0)][i].n_nodes < infos[(0, 0)][i].n_nodes / 2
        assert infos[(6, 4)][i].n_nodes <= infos[(6, 0)][i].n_nodes


# ------------------------------------------------------ clause factoring

def _long_clause_cnf(n, n_short, n_long, k_long, seed):
    """Random 3-CNF clauses plus a few long clauses (k_long literals)."""
    short = wmcgen.random_kcnf(n, n_short, seed=seed)
    long_ = wmcgen.random_kcnf(n, n_long, seed=seed + 1000, k=k_long)
    return wmcgen.Cnf(n, short.clauses + long_.clauses)


def _leaves_as_cnf(plan, n_vars):
    """The plan's clause leaves read back as a CNF over the formula's and the
    auxiliary variables (bit j of fals = the falsifying value of labels[j])."""
    n_aux = plan.info(1).n_aux_vars
    clauses = []
    for kind, labels, fals in plan.leaves():
        if kind == 0:
            clauses.append([-(v + 1) if (fals >> j) & 1 else v + 1 for j, v in enumerate(labels)])
    return wmcgen.Cnf(n_vars + n_aux, clauses), n_aux


@pytest.mark.parametrize("seed", range(4))
def test_factored_network_keeps_the_count(seed):
    """Clause factoring (Def. 3.4, Thm 3.3): every factored clause leaf has
    rank <= 3, and the factored network, read back through the ABI, has the
    oracle's weighted count of the original formula when the auxiliary
    variables weigh 1 for both values; the factored tree evaluated with
    numpy gives the same value."""
    w = _lib()
    n = 14
    cnf = _long_clause_cnf(n, 18, 3, 9, seed)
    wp, wn = wmcgen.weights_independent(n, seed, 0.1, 1.0)
    plan = w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=w.WMC_FP64, factor_clauses_above=3)
    fcnf, n_aux = _leaves_as_cnf(plan, n)
    assert n_aux == 3 * (9 - 2)
    assert max(len(c) for c in fcnf.clauses) <= 3
    want = oracle.brute_force(cnf, wp, wn)[0]
    got = oracle.bucket_elim(fcnf, np.concatenate([wp, np.ones(n_aux)]), np.concatenate([wn, np.ones(n_aux)]))
    assert want.rel_diff(got) <= 1e-15
    assert abs(evaluate_plan_numpy(plan, wp, wn) - want.to_float()) <= 1e-13 * want.to_float()
    # clauses at or below the threshold are kept as they are
    same = w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=w.WMC_FP64, factor_clauses_above=9)
    assert same.info(1).n_aux_vars == 0


def test_factoring_makes_psi_plannable():
    """psi(300): two rank-300 clause tensors, no plan within rank 30;
    factored, 2 x 298 auxiliary indices, every leaf of rank <= 3 and a
    small largest tensor; every launch of the walk stays in bounds."""
    w = _lib()
    net = w.Network.from_cnf(wmcgen.psi_family(300))
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net, precision=w.WMC_FP64)
    assert e.value.status == w.WMC_EPLAN_TOO_BIG
    p = w.Plan(net, precision=w.WMC_FP64, factor_clauses_above=3)
    info = p.info(1)
    assert info.n_aux_vars == 2 * 298
    assert info.max_rank <= 6
    assert all(len(labels) <= 3 for _, labels, _ in p.leaves())
    for Q in (1, 4):
        n = ctypes.c_int64()
        assert w.wmc_debug_check_bounds(p.handle, Q, ctypes.byref(n)) == w.WMC_OK, w.wmc_last_error()


def test_factoring_option_errors():
    w = _lib()
    net = w.Network.from_cnf(wmcgen.psi_family(8))
    for bad in (1, 2, -1):
        with pytest.raises(w._abi.WmcError) as e:
            w.Plan(net, factor_clauses_above=bad)
        assert e.value.status == w.WMC_EINVAL
    with pytest.raises(w._abi.WmcError) as e:
        w.Plan(net, factor_clauses_above=3, order=list(range(1, 9)))
    assert e.value.status == w.WMC_EINVAL
