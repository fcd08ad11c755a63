"""amrfd_dt_noalloc against amrfd_dt, through the C ABI.

Some callers cannot allocate device memory (they run inside someone else's
memory pool or a fixed device budget, or must not take the allocator's locks
on a hot path); amrfd_dt_noalloc serves them from a fixed scratch array inside
the library. Its time steps must equal those of the handle-based amrfd_dt,
bit for bit, on consecutive calls (the scratch keeps the previous call's
contents and must not leak into the next). This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_2052_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _via_c_abi(A, w, U, active=None, dt_scope=0, t=0.0, t_end=float("inf")):
    L = A.load()
    cfg = A.Config(w.physics, w.ndim, w.integrator, dt_scope, w.gamma, w.cfl, w.glm_cr)
    doms = A.domains_c(w.domains)
    out = torch.full((len(w.domains),), -1.0, dtype=torch.float64, device="cuda")
    act = ctypes.c_void_p(active.data_ptr()) if active is not None else None
    rc = L.amrfd_dt_noalloc(ctypes.byref(cfg), doms, len(w.domains), act, ctypes.c_void_p(U.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), t, t_end,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == A.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_dt_matches_handle_dt_on_consecutive_calls():
    from paper_1407_2052_gb300 import amrfd as A
    cases = [W.batched(nblocks=300), W.blast3d(16, 8)]
    cases[1].active = np.array([1, 0, 1, 1, 0, 1, 1, 0], np.uint8)
    for w in cases:  # two calls in a row, the second with fewer domains than the first
        s = A.Solver.from_workload(w)
        U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
        want = s.dt(U, t=0.0, t_end=10.0).cpu().numpy()
        act = torch.from_numpy(w.active).cuda()
        got = _via_c_abi(A, w, U, active=act, t=0.0, t_end=10.0)
        assert np.array_equal(got, want)
        s.close()
    # global scope, all blocks active, again right after the calls above
    w = W.batched(nblocks=50)
    s = A.Solver.from_workload(w, dt_scope=A.DT_GLOBAL)
    s.set_active(torch.ones(len(w.domains), dtype=torch.uint8, device="cuda"))
    U = torch.from_numpy(w.U).cuda()
    want = s.dt(U).cpu().numpy()
    got = _via_c_abi(A, w, U, active=None, dt_scope=A.DT_GLOBAL)
    assert np.array_equal(got, want)


def test_noalloc_rejects_too_many_domains():
    from paper_1407_2052_gb300 import amrfd as A
    w = W.batched(nblocks=1025, sizes=(8,))
    U = torch.from_numpy(w.U).cuda()
    L = A.load()
    cfg = A.Config(w.physics, w.ndim, w.integrator, 0, w.gamma, w.cfl, w.glm_cr)
    out = torch.empty(len(w.domains), dtype=torch.float64, device="cuda")
    rc = L.amrfd_dt_noalloc(ctypes.byref(cfg), A.domains_c(w.domains), len(w.domains), None,
                            ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()), 0.0, 1.0, None)
    assert rc == A.ERR_INVALID_ARG
