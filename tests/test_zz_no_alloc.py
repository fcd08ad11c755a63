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


def _dt_both(A, w, U, dt_scope=0, t=0.0, t_end=float("inf")):
    """(handle amrfd_dt, amrfd_dt_noalloc) on the same inputs and the workload's active
    flags, as numpy arrays, and the handle's error latch."""
    s = A.Solver.from_workload(w, dt_scope=dt_scope)
    active = torch.from_numpy(w.active).cuda() if w.active is not None else None
    want = s.dt(U, t=t, t_end=t_end).cpu().numpy()
    err = s.error()
    s.close()
    got = _via_c_abi(A, w, U, active=active, dt_scope=dt_scope, t=t, t_end=t_end)
    return want, got, err


def test_noalloc_more_shapes_bitwise():
    """The 3- and 4-variable Euler kernels, the t_end clamp deciding the step, and domains
    whose cell counts are not multiples of the 4096-cell work chunk beside smaller ones
    (the chunk-to-domain search), with the global scope."""
    from paper_1407_2052_gb300 import amrfd as A
    w = W.sod(512)
    U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
    want, got, _ = _dt_both(A, w, U, t=0.1, t_end=0.1 + 1e-7)
    assert np.array_equal(got, want) and got[0] <= 1.0000001e-7
    want, got, _ = _dt_both(A, w, U, t=0.0, t_end=0.2)
    assert np.array_equal(got, want) and got[0] > 1e-7
    w = W.sine_advection(96, ndim=2)
    U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
    want, got, _ = _dt_both(A, w, U)
    assert np.array_equal(got, want)
    w = W.batched(nblocks=40, sizes=(8, 24))
    assert {d.n[0] for d in w.domains} == {8, 24}
    U = torch.from_numpy(w.U).cuda()
    for scope in (A.DT_PER_DOMAIN, A.DT_GLOBAL):
        want, got, _ = _dt_both(A, w, U, dt_scope=scope)
        assert np.array_equal(got, want)
    w.active = None  # every block active
    for scope in (A.DT_PER_DOMAIN, A.DT_GLOBAL):
        want, got, _ = _dt_both(A, w, U, dt_scope=scope)
        assert np.array_equal(got, want) and np.all(np.isfinite(got))


def test_noalloc_flags_a_nonphysical_domain_with_nan():
    """A domain with a cell of negative pressure gets dt = NaN (the handle's amrfd_dt leaves
    the cell out and latches AMRFD_ERR_NONPHYSICAL); the other domains keep amrfd_dt's value.
    With the global scope every domain gets NaN."""
    from paper_1407_2052_gb300 import amrfd as A
    w = W.batched(nblocks=12, sizes=(8, 12))
    bad = int(np.flatnonzero(w.active)[2])
    d = w.domains[bad]
    w.U[d.offset + 4 * d.ncell + 17] = -1.0  # total energy below the kinetic + magnetic part
    U = torch.from_numpy(w.U).cuda()
    want, got, err = _dt_both(A, w, U)
    assert err == A.ERR_NONPHYSICAL
    assert np.isnan(got[bad])
    keep = np.arange(len(w.domains)) != bad
    assert np.array_equal(got[keep], want[keep])
    _, got, _ = _dt_both(A, w, U, dt_scope=A.DT_GLOBAL)
    assert np.all(np.isnan(got))
    # the next call on physical data is unaffected by the flags the previous one left
    w2 = W.batched(nblocks=12, sizes=(8, 12))
    U2 = torch.from_numpy(w2.U).cuda()
    want, got, err = _dt_both(A, w2, U2)
    assert err == A.OK and np.array_equal(got, want)


def test_noalloc_call_leaves_device_memory_unchanged():
    """The point of the entry point: after the library is loaded and the first call has
    looked up the scratch, further calls change neither torch's allocator statistics nor
    the device's free memory."""
    from paper_1407_2052_gb300 import amrfd as A
    w = W.batched(nblocks=64)
    U = torch.from_numpy(w.U).cuda()
    act = torch.from_numpy(w.active).cuda()
    out = torch.empty(len(w.domains), dtype=torch.float64, device="cuda")
    A.dt_noalloc(w.physics, w.ndim, w.gamma, w.cfl, w.domains, U, out, active=act)
    first = out.clone()
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        A.dt_noalloc(w.physics, w.ndim, w.gamma, w.cfl, w.domains, U, out, active=act)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert after == before
    assert torch.equal(out, first)
