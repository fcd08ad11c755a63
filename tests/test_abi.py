"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/amrfd.h declares; argument validation runs on the host."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|void|size_t|const char\s*\*)\s*(amrfd_\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1407_2052_gb300 import amrfd, build
    build.build()
    return amrfd.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    from paper_1407_2052_gb300 import amrfd
    assert set(amrfd.EXPORTS) <= set(declared)


def test_strerror(lib):
    assert lib.amrfd_strerror(0) == b"ok"
    assert b"invalid" in lib.amrfd_strerror(1)
    assert b"non-physical" in lib.amrfd_strerror(4)


@pytest.mark.parametrize("bad", ["physics", "ndim", "gamma", "periodic_small", "overlap", "nb", "unpaired_bc",
                                 "bc_kind", "mirror_small", "mirror_mask", "recon", "limo3_r", "no_domains",
                                 "zero_cells", "dx_nan", "dx_negative", "cfl", "integrator", "dt_scope",
                                 "negative_offset", "block_edge", "huge_domain"])
def test_create_rejects_bad_arguments_on_host(lib, bad):
    """Validation happens before any CUDA call, so this needs no GPU."""
    from paper_1407_2052_gb300 import amrfd as A
    from paper_1407_2052_gb300 import workloads as W
    cfg = A.Config(A.MHD_GLM, 3, A.SSPRK3, 0, 5 / 3, 0.3, 0.18)
    doms = [W.Domain((8, 8, 8), (0.1,) * 3), W.Domain((8, 8, 8), (0.1,) * 3, offset=9 * 512)]
    if bad == "physics":
        cfg.physics = 7
    elif bad == "ndim":
        cfg.ndim = 4
    elif bad == "gamma":
        cfg.gamma = 1.0
    elif bad == "periodic_small":
        doms[0] = W.Domain((2, 8, 8), (0.1,) * 3)
    elif bad == "overlap":
        doms[1] = W.Domain((8, 8, 8), (0.1,) * 3, offset=100)
    elif bad == "nb":
        doms[0] = W.Domain((8, 8, 8), (0.1,) * 3, nb=(3, 1, 1))
    elif bad == "unpaired_bc":
        doms[0] = W.Domain((8, 8, 8), (0.1,) * 3, bc=((A.PERIODIC, A.OUTFLOW),) * 3)
    elif bad == "bc_kind":
        doms[0] = W.Domain((8, 8, 8), (0.1,) * 3, bc=((A.OUTFLOW, 3),) * 3)
    elif bad == "mirror_small":
        doms[0] = W.Domain((8, 2, 8), (0.1,) * 3, bc=((0, 0), (A.SYMMETRIC, A.OUTFLOW), (0, 0)))
    elif bad == "mirror_mask":  # MHD has 9 variables: bit 9 does not exist
        doms[0] = W.Domain((8, 8, 8), (0.1,) * 3, bc=((A.SYMMETRIC, A.SYMMETRIC), (0, 0), (0, 0)),
                           asym=((1 << 9, 0), (0, 0), (0, 0)))
    elif bad == "recon":
        cfg.recon = 2
    elif bad == "limo3_r":
        cfg.recon, cfg.limo3_r = A.LIMO3, 0.0
    elif bad == "zero_cells":
        doms[0] = W.Domain((0, 8, 8), (0.1,) * 3)
    elif bad == "dx_nan":
        doms[0] = W.Domain((8, 8, 8), (float("nan"), 0.1, 0.1))
    elif bad == "dx_negative":
        doms[0] = W.Domain((8, 8, 8), (0.1, -0.1, 0.1))
    elif bad == "cfl":
        cfg.cfl = 0.0
    elif bad == "integrator":
        cfg.integrator = 9
    elif bad == "dt_scope":
        cfg.dt_scope = 5
    elif bad == "negative_offset":
        doms[0] = W.Domain((8, 8, 8), (0.1,) * 3, offset=-9)
    elif bad == "block_edge":  # a block edge beyond 32767 cells
        doms[0] = W.Domain((40000, 8, 8), (0.1,) * 3)
        doms[1] = W.Domain((8, 8, 8), (0.1,) * 3, offset=9 * 40000 * 64)
    elif bad == "huge_domain":  # more than 2^31 - 1 cells in one domain
        doms[0] = W.Domain((2048, 2048, 1024), (0.1,) * 3, nb=(128, 128, 64))
        doms[1] = W.Domain((8, 8, 8), (0.1,) * 3, offset=9 * 2048 * 2048 * 1024)
    h = ctypes.c_void_p()
    nd = 0 if bad == "no_domains" else len(doms)
    rc = lib.amrfd_create(ctypes.byref(h), ctypes.byref(cfg), A.domains_c(doms), nd, None, None)
    assert rc == A.ERR_INVALID_ARG
    assert not h.value


def test_dt_noalloc_binding_rejects_bad_tensors_before_the_call():
    """The kernels of amrfd_dt_noalloc trust the sizes they are given, so the binding checks
    the flags, the output and the state first (no library call, no GPU needed)."""
    torch = pytest.importorskip("torch")
    from paper_1407_2052_gb300 import amrfd as A
    from paper_1407_2052_gb300 import workloads as W
    doms = [W.Domain((8, 8, 8), (0.1,) * 3), W.Domain((8, 8, 8), (0.1,) * 3, offset=9 * 512)]
    U = torch.zeros(2 * 9 * 512, dtype=torch.float64)
    out = torch.zeros(2, dtype=torch.float64)

    def call(**kw):
        args = dict(U=U, out=out, active=None)
        args.update(kw)
        A.dt_noalloc(A.MHD_GLM, 3, 5 / 3, 0.3, doms, args["U"], args["out"], active=args["active"])

    with pytest.raises(TypeError):
        call(active=torch.ones(2, dtype=torch.bool))
    with pytest.raises(TypeError):
        call(active=torch.ones(2, dtype=torch.int64))
    with pytest.raises(ValueError):
        call(active=torch.ones(1, dtype=torch.uint8))
    with pytest.raises(TypeError):
        call(active=torch.ones(4, dtype=torch.uint8)[::2])
    with pytest.raises(TypeError):  # right size and type, but host memory
        call(active=torch.ones(2, dtype=torch.uint8))
    with pytest.raises(ValueError):
        call(out=torch.zeros(1, dtype=torch.float64))
    with pytest.raises(TypeError):
        call(out=torch.zeros(2, dtype=torch.float32))
    with pytest.raises(ValueError):
        call(U=torch.zeros(9 * 512, dtype=torch.float64))
