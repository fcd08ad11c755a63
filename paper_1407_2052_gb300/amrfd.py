"""Python binding of libamrfd.so (argument marshalling only).

Every step of the update runs in the CUDA kernels behind include/amrfd.h; this
module converts torch CUDA tensors to device pointers and the current torch
stream to a cudaStream_t. There is no CPU fallback: if the library is missing
or no GPU is present, calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamrfd.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libamrfd_checked.so")

EULER, MHD_GLM = 0, 1
SSPRK3, SSPRK54, SSPRK43 = 0, 1, 2
PERIODIC, OUTFLOW, SYMMETRIC = 0, 1, 2
MP5, LIMO3 = 0, 1
DT_PER_DOMAIN, DT_GLOBAL = 0, 1
OK, ERR_INVALID_ARG, ERR_CUDA, ERR_UNSUPPORTED, ERR_NONPHYSICAL, ERR_CHECK = 0, 1, 2, 3, 4, 5

EXPORTS = ("amrfd_create", "amrfd_set_active", "amrfd_dt", "amrfd_step", "amrfd_step_batched",
           "amrfd_adjoint", "amrfd_autotune", "amrfd_set_tile", "amrfd_get_tile", "amrfd_get_alpha",
           "amrfd_get_error", "amrfd_destroy", "amrfd_strerror", "amrfd_timing_begin", "amrfd_timing_end",
           "amrfd_dt_noalloc", "amrfd_flag_steady", "amrfd_activate", "amrfd_get_active",
           "amrfd_step_cfl", "amrfd_fp64_peak", "amrfd_set_adjoint_tile", "amrfd_record_bytes",
           "amrfd_step_record", "amrfd_adjoint_recorded")


class Config(ctypes.Structure):
    _fields_ = [("physics", ctypes.c_int), ("ndim", ctypes.c_int), ("integrator", ctypes.c_int),
                ("dt_scope", ctypes.c_int), ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("glm_cr", ctypes.c_double), ("recon", ctypes.c_int), ("reserved_", ctypes.c_int),
                ("limo3_r", ctypes.c_double)]


class DomainC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nb", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", (ctypes.c_int * 2) * 3), ("asym", (ctypes.c_uint32 * 2) * 3), ("offset", ctypes.c_int64)]


class AmrfdError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (code %d)" % (what, _strerror(code), code))


_libs = {}


def load(checked=False):
    """Load libamrfd.so (checked: libamrfd_checked.so, the build with kernel index
    checks), built by paper_1407_2052_gb300.build; raise if absent."""
    if checked in _libs:
        return _libs[checked]
    path = LIB_CHECKED_PATH if checked else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run `python -c 'import __graft_entry__ as g; g.build()'`"
                           % os.path.basename(path))
    L = ctypes.CDLL(path)
    vp, dp, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    L.amrfd_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Config), ctypes.POINTER(DomainC), i, vp, vp]
    L.amrfd_set_active.argtypes = [vp, vp, vp]
    L.amrfd_flag_steady.argtypes = [vp, vp, vp, dp, vp, vp]
    L.amrfd_activate.argtypes = [vp, vp, i, vp]
    L.amrfd_get_active.argtypes = [vp, vp, vp]
    L.amrfd_dt.argtypes = [vp, vp, vp, dp, dp, vp]
    L.amrfd_step.argtypes = [vp, vp, vp, vp]
    L.amrfd_step_batched.argtypes = [vp, vp, vp, vp]
    L.amrfd_step_cfl.argtypes = [vp, vp, vp, dp, dp, vp]
    L.amrfd_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
    L.amrfd_autotune.argtypes = [vp, vp, vp, vp]
    L.amrfd_set_tile.argtypes = [vp, i, i, i]
    L.amrfd_set_adjoint_tile.argtypes = [vp, i, i, i]
    L.amrfd_record_bytes.argtypes = [vp]
    L.amrfd_step_record.argtypes = [vp, vp, vp, vp, vp]
    L.amrfd_adjoint_recorded.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.amrfd_get_tile.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.amrfd_get_alpha.argtypes = [vp, vp, i, vp]
    L.amrfd_get_error.argtypes = [vp, vp]
    L.amrfd_timing_begin.argtypes = [vp, i]
    L.amrfd_timing_end.argtypes = [vp, vp, vp, vp]
    L.amrfd_dt_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(DomainC), i, vp, vp, vp, dp, dp, vp]
    L.amrfd_fp64_peak.argtypes = [dp, vp, vp]
    L.amrfd_destroy.argtypes = [vp]
    L.amrfd_destroy.restype = None
    L.amrfd_strerror.argtypes = [i]
    L.amrfd_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("amrfd_destroy", "amrfd_strerror", "amrfd_record_bytes"):
            getattr(L, name).restype = i
    L.amrfd_record_bytes.restype = ctypes.c_size_t
    _libs[checked] = L
    return L


def _strerror(code):
    try:
        return load().amrfd_strerror(code).decode()
    except Exception:  # pragma: no cover - library missing
        return "error"


def _check(rc, what):
    if rc != OK:
        raise AmrfdError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def domains_c(domains):
    arr = (DomainC * len(domains))()
    for i, d in enumerate(domains):
        for k in range(3):
            arr[i].n[k] = int(d.n[k])
            arr[i].nb[k] = int(d.nb[k])
            arr[i].dx[k] = float(d.dx[k])
            arr[i].bc[k][0] = int(d.bc[k][0])
            arr[i].bc[k][1] = int(d.bc[k][1])
            asym = getattr(d, "asym", None)
            if asym is not None:
                arr[i].asym[k][0] = int(asym[k][0])
                arr[i].asym[k][1] = int(asym[k][1])
        arr[i].offset = int(d.offset)
    return arr


def dt_noalloc(physics, ndim, gamma, cfl, domains, U, out, active=None, t=0.0, t_end=float("inf"),
               dt_scope=DT_PER_DOMAIN, stream=None):
    """amrfd_dt_noalloc: the CFL time step without a handle or any device allocation
    (for callers that cannot allocate; `out` is a caller-owned float64 CUDA tensor).
    The tensors are checked here, before the call, because the kernels trust their sizes:
    `active` a contiguous CUDA uint8 tensor with one flag per block, `out` a float64 CUDA
    tensor of at least len(domains) values, `U` large enough for every domain."""
    import torch
    nv = 2 + ndim if physics == EULER else 9
    nblocks = sum(int(d.nb[0]) * int(d.nb[1]) * int(d.nb[2]) for d in domains)
    need = max((int(d.offset) + nv * int(d.n[0]) * int(d.n[1]) * int(d.n[2]) for d in domains), default=0)
    if active is not None:
        if not isinstance(active, torch.Tensor) or active.dtype != torch.uint8 or not active.is_contiguous():
            raise TypeError("active: expected a contiguous uint8 tensor")
        if active.numel() != nblocks:
            raise ValueError("active: %d flags for %d blocks" % (active.numel(), nblocks))
        if not active.is_cuda:
            raise TypeError("active: expected a CUDA tensor")
    if not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or not out.is_contiguous():
        raise TypeError("out: expected a contiguous float64 tensor")
    if out.numel() < len(domains):
        raise ValueError("out: %d values for %d domains" % (out.numel(), len(domains)))
    if not isinstance(U, torch.Tensor) or U.numel() < need:
        raise ValueError("U: the domains need %d elements" % need)
    cfg = Config(physics, ndim, SSPRK3, dt_scope, gamma, cfl, 0.0)
    doms = domains_c(domains)
    act = ctypes.c_void_p(active.data_ptr()) if active is not None else None
    _check(load().amrfd_dt_noalloc(ctypes.byref(cfg), doms, len(domains), act, _ptr(U), _ptr(out), float(t),
                                   float(t_end), _stream(stream)), "amrfd_dt_noalloc")
    return out


def fp64_peak(seconds=2.0, stream=None):
    """amrfd_fp64_peak: measured FP64 throughput of the current GPU,
    {"burst_tflops", "sustained_tflops", "launch_ms", "fma_per_launch"}."""
    out = np.zeros(4)
    _check(load().amrfd_fp64_peak(float(seconds), out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "amrfd_fp64_peak")
    return {"burst_tflops": float(out[0]), "sustained_tflops": float(out[1]), "launch_ms": float(out[2]),
            "fma_per_launch": float(out[3])}


class Solver:
    """One amrfd handle: a set of domains advanced together on the current GPU."""

    def __init__(self, physics, ndim, integrator, gamma, cfl, domains, active=None, glm_cr=0.18,
                 dt_scope=DT_PER_DOMAIN, stream=None, recon=MP5, limo3_r=1.0, checked=False):
        L = self._L = load(checked)
        self.cfg = Config(physics, ndim, integrator, dt_scope, gamma, cfl, glm_cr, recon, 0, limo3_r)
        self.domains = list(domains)
        self.ndom = len(self.domains)
        self.nv = 2 + ndim if physics == EULER else 9
        self.nstages = {SSPRK3: 3, SSPRK54: 5, SSPRK43: 4}[integrator]
        self.nblocks = sum(int(d.nb[0]) * int(d.nb[1]) * int(d.nb[2]) for d in self.domains)
        self.nelem = max(int(d.offset) + self.nv * int(d.n[0]) * int(d.n[1]) * int(d.n[2]) for d in self.domains)
        doms = domains_c(self.domains)
        act = None
        if active is not None:
            a = np.ascontiguousarray(active, dtype=np.uint8).ravel()
            if a.size != self.nblocks:
                raise ValueError("one active flag per block")
            self._active_host = a
            act = a.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        _check(L.amrfd_create(ctypes.byref(h), ctypes.byref(self.cfg), doms, self.ndom, act, _stream(stream)),
               "amrfd_create")
        self._h = h

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.physics, w.ndim, w.integrator, w.gamma, w.cfl, w.domains, active=w.active,
                   glm_cr=w.glm_cr, recon=w.recon, limo3_r=w.limo3_r, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._L.amrfd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_active(self, active_dev, stream=None):
        import torch
        if active_dev.dtype != torch.uint8 or not active_dev.is_cuda or active_dev.numel() != self.nblocks:
            raise TypeError("expected a CUDA uint8 tensor with one flag per block")
        _check(self._L.amrfd_set_active(self._h, ctypes.c_void_p(active_dev.data_ptr()), _stream(stream)),
               "amrfd_set_active")

    def _flags(self, t):
        import torch
        if t.dtype != torch.uint8 or not t.is_cuda or t.numel() != self.nblocks or not t.is_contiguous():
            raise TypeError("expected a contiguous CUDA uint8 tensor with one flag per block")
        return ctypes.c_void_p(t.data_ptr())

    def flag_steady(self, U, U_ref, tol, out=None, stream=None):
        """amrfd_flag_steady: 1 per block whose cells all lie within tol of U_ref."""
        import torch
        if out is None:
            out = torch.empty(self.nblocks, dtype=torch.uint8, device=U.device)
        _check(self._L.amrfd_flag_steady(self._h, _ptr(U), _ptr(U_ref), float(tol), self._flags(out),
                                        _stream(stream)), "amrfd_flag_steady")
        return out

    def activate(self, flag, belt=1, stream=None):
        """amrfd_activate: passive candidates `flag`, `belt` safety layers, device work lists rebuilt."""
        _check(self._L.amrfd_activate(self._h, self._flags(flag), int(belt), _stream(stream)), "amrfd_activate")

    def active(self, stream=None):
        """Current per-block active flags (CUDA uint8 tensor)."""
        import torch
        out = torch.empty(self.nblocks, dtype=torch.uint8, device="cuda")
        _check(self._L.amrfd_get_active(self._h, self._flags(out), _stream(stream)), "amrfd_get_active")
        return out

    def dt(self, U, t=0.0, t_end=float("inf"), out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.ndom, dtype=torch.float64, device=U.device)
        _check(self._L.amrfd_dt(self._h, _ptr(U), _ptr(out), float(t), float(t_end), _stream(stream)), "amrfd_dt")
        return out

    def step(self, U, dt, stream=None):
        _check(self._L.amrfd_step(self._h, _ptr(U), _ptr(dt), _stream(stream)), "amrfd_step")
        return U

    def step_batched(self, U, dt, stream=None):
        _check(self._L.amrfd_step_batched(self._h, _ptr(U), _ptr(dt), _stream(stream)), "amrfd_step_batched")
        return U

    def step_cfl(self, U, t=0.0, t_end=float("inf"), out=None, stream=None):
        """amrfd_step_cfl: CFL dt of U (returned, also in `out`) and one step with it."""
        import torch
        if out is None:
            out = torch.empty(self.ndom, dtype=torch.float64, device=U.device)
        _check(self._L.amrfd_step_cfl(self._h, _ptr(U), _ptr(out), float(t), float(t_end), _stream(stream)),
               "amrfd_step_cfl")
        return out

    def adjoint(self, U_n, dt, gU_np1, gU_n, stream=None):
        _check(self._L.amrfd_adjoint(self._h, _ptr(U_n), _ptr(dt), _ptr(gU_np1), _ptr(gU_n), _stream(stream)),
               "amrfd_adjoint")
        return gU_n

    def record_bytes(self):
        """amrfd_record_bytes: bytes of one step record of this handle."""
        return int(self._L.amrfd_record_bytes(self._h))

    def new_record(self):
        """A device buffer for one step record (uint8 CUDA tensor)."""
        import torch
        return torch.empty(self.record_bytes(), dtype=torch.uint8, device="cuda")

    def _record(self, rec):
        import torch
        if (not isinstance(rec, torch.Tensor) or not rec.is_cuda or rec.dtype != torch.uint8 or not rec.is_contiguous()
                or rec.numel() < self.record_bytes() or rec.data_ptr() % 16):
            raise TypeError("expected a contiguous 16-byte aligned CUDA uint8 tensor of record_bytes() bytes")
        return ctypes.c_void_p(rec.data_ptr())

    def step_record(self, U, dt, record, stream=None):
        """amrfd_step_record: one step of U in place that also fills `record` for its adjoint."""
        _check(self._L.amrfd_step_record(self._h, _ptr(U), _ptr(dt), self._record(record), _stream(stream)),
               "amrfd_step_record")
        return U

    def adjoint_recorded(self, U_n, dt, record, gU_np1, gU_n, stream=None):
        """amrfd_adjoint_recorded: the adjoint of the recorded step (U_n: the state before it)."""
        _check(self._L.amrfd_adjoint_recorded(self._h, _ptr(U_n), _ptr(dt), self._record(record), _ptr(gU_np1),
                                             _ptr(gU_n), _stream(stream)), "amrfd_adjoint_recorded")
        return gU_n

    def tile_key(self):
        """Key of the autotuner cache: physics, dimensions, reconstruction, the multiset of
        (cells, blocks) shapes and the device's SM count."""
        import hashlib
        import torch
        shapes = sorted((tuple(int(x) for x in d.n), tuple(int(x) for x in d.nb)) for d in self.domains)
        h = hashlib.sha1(repr(shapes).encode()).hexdigest()[:16]
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        return "p%d-d%d-r%d-%s-sm%d" % (self.cfg.physics, self.cfg.ndim, self.cfg.recon, h, sms)

    def autotune(self, U, dt, stream=None, cache=None):
        """amrfd_autotune; with `cache` (a JSON file path) a tile chosen before for the same
        key (tile_key) is reused instead of timing the candidates again."""
        import json
        key = self.tile_key() if cache else None
        if cache and os.path.exists(cache):
            try:
                known = json.load(open(cache)).get(key)
            except (OSError, ValueError):
                known = None
            if known:
                # a tile the library no longer accepts (another version's limits) is tuned again
                if self._L.amrfd_set_tile(self._h, *(int(x) for x in known)) == OK:
                    return self.get_tile()
        _check(self._L.amrfd_autotune(self._h, _ptr(U), _ptr(dt), _stream(stream)), "amrfd_autotune")
        tile = self.get_tile()
        if cache:
            data = {}
            if os.path.exists(cache):
                try:
                    data = json.load(open(cache))
                except (OSError, ValueError):
                    data = {}
            data[key] = list(tile)
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return tile

    def set_tile(self, seg, lines, threads):
        _check(self._L.amrfd_set_tile(self._h, seg, lines, threads), "amrfd_set_tile")

    def set_adjoint_tile(self, seg, lines, threads):
        """amrfd_set_adjoint_tile: the tile of the adjoint's transposed flux pass."""
        _check(self._L.amrfd_set_adjoint_tile(self._h, seg, lines, threads), "amrfd_set_adjoint_tile")

    def get_tile(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._L.amrfd_get_tile(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "amrfd_get_tile")
        return a.value, b.value, c.value

    def alpha(self, nstage=None, stream=None):
        """Raw per-stage splitting speeds of the last step, shape (nstage, ndom, 3)."""
        nstage = self.nstages if nstage is None else nstage
        out = np.zeros((nstage, self.ndom, 3))
        _check(self._L.amrfd_get_alpha(self._h, out.ctypes.data_as(ctypes.c_void_p), nstage, _stream(stream)),
               "amrfd_get_alpha")
        return out

    KINDS = ("speeds", "flux", "combine", "dt")

    def timing_begin(self, capacity):
        _check(self._L.amrfd_timing_begin(self._h, int(capacity)), "amrfd_timing_begin")

    def timing_end(self, stream=None):
        """{kind: (total_ms, launches)} for the launches since timing_begin."""
        ms = np.zeros(4)
        cnt = np.zeros(4, dtype=np.int32)
        _check(self._L.amrfd_timing_end(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                       cnt.ctypes.data_as(ctypes.c_void_p), _stream(stream)), "amrfd_timing_end")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KINDS)}

    def error(self, stream=None):
        return self._L.amrfd_get_error(self._h, _stream(stream))
