"""The allocation-free entry point, wmc_execute_device_noalloc, called
through the C ABI.

It exists for callers that cannot allocate device memory (work enqueued
during stream capture, latency-bound serving loops, hosts whose memory
belongs to another allocator).  It must return what wmc_execute_device
returns for the same plan and inputs, on two calls in a row (the second
call finds the first call's contents still in the shared scratch), and
reject plans that do not fit its fixed scratch.

This file is collected last so that a run stopping at its first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def _results(mant, ex):
    return [Big(*_norm(float(mant[i]), int(ex[i]))) for i in range(mant.numel())]


def _norm(m, e):
    import math
    fm, fe = math.frexp(m)
    return fm, (e + fe) if m != 0.0 else 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["random3cnf", "grid"])
def test_noalloc_matches_execute_device(w, precision, kind):
    if kind == "random3cnf":
        cnf = wmcgen.random_kcnf(20, 60, seed=3)
        Q = 1
    else:
        cnf = wmcgen.grid_cnf(16, 100, 1)
        Q = 4
    plan = w.Plan(w.Network.from_cnf(cnf), precision=precision)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, Q, seed=11, lo=0.05, hi=0.95)
    dwp = torch.from_numpy(wq).cuda()
    dwn = torch.from_numpy(wnq).cuda()
    info = plan.info(Q)
    ws = torch.empty(info.workspace_bytes, dtype=torch.uint8, device="cuda")
    m0 = torch.empty(Q, dtype=torch.float64, device="cuda")
    e0 = torch.empty(Q, dtype=torch.int64, device="cuda")
    f0 = torch.empty(Q, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    plan.execute_device(Q, dwp, dwn, ws, m0, e0, f0, stream=s)
    torch.cuda.synchronize()
    want = _results(m0, e0)
    for call in range(2):
        m1 = torch.full((Q,), -1.0, dtype=torch.float64, device="cuda")
        e1 = torch.zeros(Q, dtype=torch.int64, device="cuda")
        f1 = torch.full((Q,), 7, dtype=torch.int32, device="cuda")
        rc = w.wmc_execute_device_noalloc(plan.handle, Q, _vp(dwp), _vp(dwn), _vp(m1), _vp(e1),
                                          _vp(f1), ctypes.c_void_p(s))
        assert rc == w.WMC_OK, w.wmc_last_error()
        torch.cuda.synchronize()
        got = _results(m1, e1)
        for q in range(Q):
            assert got[q].rel_diff(want[q]) <= TOL[precision], (call, q)
        assert torch.equal(f1, f0)


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
