"""The allocation-free entry point, wmc_execute_device_noalloc, called
through the C ABI.

It exists for callers that cannot allocate device memory when they run a
count: a library embedded in a process whose device memory belongs to
another allocator, or code that must not call cudaMalloc/cudaFree once it
is running (both can synchronise the device).  It runs the same walk and
kernels as wmc_execute_device on a static scratch array, so it must return
the same bits, on two calls in a row (the second call finds the first
call's contents still in the shared scratch), for plans with several slice
assignments, with runs of chains and with the one-block walk, and after
another plan has used the scratch in between.  It must reject plans that do not fit its fixed
scratch.

This file is collected last so that a run stopping at its first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import wmcgen
from oracle import Big

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-4}


@pytest.fixture(scope="module")
def w():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required")
    import paper_2006_15512_b300 as lib
    return lib


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _norm(m, e):
    import math
    fm, fe = math.frexp(m)
    return fm, (e + fe) if m != 0.0 else 0


def _device_inputs(cnf, Q, seed):
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=seed, lo=0.05, hi=0.95)
    return wq, wnq, torch.from_numpy(wq).cuda(), torch.from_numpy(wnq).cuda()


def _execute_device(plan, Q, dwp, dwn):
    """The allocating device entry (caller-owned workspace)."""
    info = plan.info(Q)
    ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device="cuda")
    m = torch.empty(Q, dtype=torch.float64, device="cuda")
    e = torch.empty(Q, dtype=torch.int64, device="cuda")
    f = torch.empty(Q, dtype=torch.int32, device="cuda")
    plan.execute_device(Q, dwp, dwn, ws, m, e, f, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return m, e, f


def _execute_noalloc(w, plan, Q, dwp, dwn):
    # outputs pre-filled with garbage: the call must overwrite every entry
    m = torch.full((Q,), -1.0, dtype=torch.float64, device="cuda")
    e = torch.full((Q,), 12345, dtype=torch.int64, device="cuda")
    f = torch.full((Q,), 7, dtype=torch.int32, device="cuda")
    rc = w.wmc_execute_device_noalloc(plan.handle, Q, _vp(dwp), _vp(dwn), _vp(m), _vp(e), _vp(f),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == w.WMC_OK, w.wmc_last_error()
    torch.cuda.synchronize()
    return m, e, f


def _assert_same_bits(got, want):
    for g, x in zip(got, want):
        assert torch.equal(g, x), (g, x)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["random3cnf", "grid"])
def test_noalloc_matches_execute_device(w, precision, kind):
    """Same bits as wmc_execute_device on two calls in a row; the random
    3-CNF (n = 20, m = 60) also against the oracle's brute-force count."""
    if kind == "random3cnf":
        cnf = wmcgen.random_kcnf(20, 60, seed=3)
        Q = 2
    else:
        cnf = wmcgen.grid_cnf(16, 100, 1)
        Q = 4
    plan = w.Plan(w.Network.from_cnf(cnf), precision=precision)
    wq, wnq, dwp, dwn = _device_inputs(cnf, Q, 11)
    want = _execute_device(plan, Q, dwp, dwn)
    for call in range(2):
        got = _execute_noalloc(w, plan, Q, dwp, dwn)
        _assert_same_bits(got, want)
    if kind == "random3cnf":
        for q in range(Q):
            exact = oracle.brute_force(cnf, wq[q], wnq[q])[0]
            assert Big(*_norm(float(got[0][q]), int(got[1][q]))).rel_diff(exact) <= TOL[precision]


def test_noalloc_after_another_plan_used_the_scratch(w):
    """Two plans alternating on the one scratch: each call finds the other
    plan's tables and workspace there and still returns its own bits."""
    a = wmcgen.random_kcnf(20, 60, seed=5)
    b = wmcgen.grid_cnf(10, 40, 2)
    pa = w.Plan(w.Network.from_cnf(a), precision=1)
    pb = w.Plan(w.Network.from_cnf(b), precision=1)
    _, _, awp, awn = _device_inputs(a, 1, 21)
    _, _, bwp, bwn = _device_inputs(b, 8, 22)
    want_a = _execute_device(pa, 1, awp, awn)
    want_b = _execute_device(pb, 8, bwp, bwn)
    for _ in range(2):
        _assert_same_bits(_execute_noalloc(w, pa, 1, awp, awn), want_a)
        _assert_same_bits(_execute_noalloc(w, pb, 8, bwp, bwn), want_b)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_sliced_plan(w, precision):
    """A plan with index slicing (Alg. 3): one walk per slice assignment,
    the later ones adding into the outputs; same bits as the device entry,
    which runs every slice too, and the oracle's value."""
    cnf = wmcgen.random_kcnf(24, 70, seed=8)
    Q = 2
    plan = w.Plan(w.Network.from_cnf(cnf), precision=precision, slice_to_rank=12)
    assert plan.info(Q).n_slice_vars >= 2
    wq, wnq, dwp, dwn = _device_inputs(cnf, Q, 31)
    want = _execute_device(plan, Q, dwp, dwn)
    for _ in range(2):
        got = _execute_noalloc(w, plan, Q, dwp, dwn)
        _assert_same_bits(got, want)
    for q in range(Q):
        exact = oracle.bucket_elim(cnf, wq[q], wnq[q])
        assert Big(*_norm(float(got[0][q]), int(got[1][q]))).rel_diff(exact) <= TOL[precision]


def test_noalloc_with_runs_of_chains(w):
    """Runs of chains in one launch (their parameter table sits in the
    scratch and their pointers are rebased against it): same bits as the
    device entry."""
    cnf = wmcgen.grid_cnf(16, 100, 1)
    Q = 4
    try:
        w.wmc_set_fusion(4)  # (runs join chains of four steps)
        w.wmc_set_chain_runs(512)
        plan = w.Plan(w.Network.from_cnf(cnf), precision=1)
        assert plan.info(Q).launches_per_walk < 100  # chains were grouped into runs
    finally:
        w.wmc_set_chain_runs(0)
        w.wmc_set_fusion(-1)
    _, _, dwp, dwn = _device_inputs(cnf, Q, 41)
    want = _execute_device(plan, Q, dwp, dwn)
    for _ in range(2):
        _assert_same_bits(_execute_noalloc(w, plan, Q, dwp, dwn), want)


def test_noalloc_with_one_block_walk(w):
    """The one-block walk (its node program and leaf descriptors sit in the
    scratch): same bits as the device entry."""
    cnf = wmcgen.random_kcnf(20, 60, seed=2)
    Q = 1
    try:
        w.wmc_set_cta_walk(1)
        plan = w.Plan(w.Network.from_cnf(cnf), precision=0)
        assert plan.info(Q).launches_per_walk == 2  # the walk and the finaliser
    finally:
        w.wmc_set_cta_walk(0)
    _, _, dwp, dwn = _device_inputs(cnf, Q, 51)
    want = _execute_device(plan, Q, dwp, dwn)
    for _ in range(2):
        _assert_same_bits(_execute_noalloc(w, plan, Q, dwp, dwn), want)


def test_noalloc_rejects_plans_beyond_its_scratch(w):
    cnf = wmcgen.grid_cnf(16, 100, 1)
    plan = w.Plan(w.Network.from_cnf(cnf), precision=1)
    Q = 256  # workspace of several hundred MiB
    dummy = torch.zeros(Q * cnf.n_vars, dtype=torch.float64, device="cuda")
    out = torch.zeros(Q, dtype=torch.float64, device="cuda")
    rc = w.wmc_execute_device_noalloc(plan.handle, Q, _vp(dummy), _vp(dummy), _vp(out), _vp(out),
                                      _vp(out), ctypes.c_void_p(0))
    assert rc == w.WMC_EINVAL
    assert b"static scratch holds" in w.wmc_last_error()
