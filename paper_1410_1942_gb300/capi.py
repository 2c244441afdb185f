"""Thin ctypes binding to ``libpoisson.so`` (the C ABI of ``include/poisson.h``).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.  Arrays
may be numpy float64 arrays (host memory) or CUDA torch tensors (device memory, passed by
``data_ptr()``); the library tells the two apart.  The library must have been built
(``paper_1410_1942_gb300.build.build()``); loading raises if it is missing -- there is no other
implementation behind these names.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, PENDING = 0, 1
EINVAL, ENOMEM, ENOTCONV, EBREAKDOWN, ETIMEOUT, ENOTREADY, ECUDA, ENOMEM_BUDGET, ENOTICKET = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9
ETOOLARGE = -10
FP64, FP32, FP32_BF16COEF = 0, 1, 2
JACOBI, RBSSOR, MG = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1

PRECISION = {"fp64": FP64, "fp32": FP32, "bf16": FP32_BF16COEF}
PRECOND = {"jacobi": JACOBI, "rbssor": RBSSOR, "ssor": RBSSOR, "mg": MG}

# every symbol include/poisson.h declares
EXPORTS = ["poisson_default_opts", "poisson_create", "poisson_destroy", "poisson_set_density",
           "poisson_solve", "poisson_apply", "poisson_precond_apply", "poisson_get_operator",
           "poisson_batch_submit", "poisson_poll", "poisson_kernel_launches", "poisson_profile",
           "poisson_profile_read", "poisson_describe", "poisson_residual_noalloc",
           "poisson_divergence", "poisson_project", "poisson_set_apertures", "poisson_strerror",
           "poisson_version", "poisson_test_unreachable_barrier", "poisson_hydrostatic_force",
           "poisson_required_bytes", "poisson_handle_bytes", "poisson_test_fail_alloc",
           "poisson_test_live_allocations"]
K_CG_A, K_CG_B, K_RESIDUAL, K_OTHER, K_PCG = 0, 1, 2, 3, 4
K_NAMES = ["cg_phase_a", "cg_phase_b", "residual64", "other", "pcg_persistent"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("omega", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("inner_tol", ctypes.c_double), ("tile", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("dirichlet_walls", ctypes.c_int),
                ("periodic_x", ctypes.c_int)]


# poisson_opts.dirichlet_walls bits: side/bottom walls with p = 0 on the wall face
WALL_XM, WALL_XP, WALL_YM, WALL_YP, WALL_ZM = 1, 2, 4, 8, 16


class Stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 5), ("ms", ctypes.c_double * 5)]

    def as_dict(self):
        return {K_NAMES[q]: {"launches": int(self.launches[q]), "ms": float(self.ms[q])}
                for q in range(5)}


class PoissonError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s: %s (%d)" % (what, strerror(status), status))
        self.status = status


_lib = None


def load(path=None):
    """Load the library (built in-tree); raises OSError if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError("libpoisson.so not built (%s); run paper_1410_1942_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.poisson_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.poisson_default_opts.restype = None
    lib.poisson_create.argtypes = [i, i, i, d, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    lib.poisson_destroy.argtypes = [vp]
    lib.poisson_set_density.argtypes = [vp, vp, d, d, i]
    lib.poisson_solve.argtypes = [vp, vp, vp, d, ctypes.POINTER(Stats)]
    lib.poisson_apply.argtypes = [vp, vp, vp, i]
    lib.poisson_precond_apply.argtypes = [vp, vp, vp, i, i]
    lib.poisson_get_operator.argtypes = [vp, vp, vp, vp, vp]
    lib.poisson_batch_submit.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(d), i, ctypes.POINTER(ctypes.c_uint64)]
    lib.poisson_poll.argtypes = [ctypes.c_uint64, ctypes.POINTER(Stats)]
    lib.poisson_strerror.argtypes = [i]
    lib.poisson_strerror.restype = ctypes.c_char_p
    lib.poisson_version.argtypes = []
    lib.poisson_version.restype = ctypes.c_char_p
    lib.poisson_kernel_launches.argtypes = []
    lib.poisson_kernel_launches.restype = ctypes.c_uint64
    lib.poisson_profile.argtypes = [vp, i]
    lib.poisson_profile_read.argtypes = [vp, ctypes.POINTER(KernelTimes)]
    lib.poisson_describe.argtypes = [vp, ctypes.c_char_p, i]
    lib.poisson_residual_noalloc.argtypes = [i, i, i, d, vp, d, d, vp, vp, vp, vp]
    lib.poisson_residual_noalloc.restype = i
    lib.poisson_divergence.argtypes = [vp, vp, vp, vp, d, vp]
    lib.poisson_divergence.restype = i
    lib.poisson_project.argtypes = [vp, vp, vp, vp, vp, d]
    lib.poisson_project.restype = i
    lib.poisson_set_apertures.argtypes = [vp, vp, vp, vp, vp, i]
    lib.poisson_set_apertures.restype = i
    lib.poisson_required_bytes.argtypes = [i, i, i, ctypes.POINTER(Opts), ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint64)]
    lib.poisson_required_bytes.restype = i
    lib.poisson_handle_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.poisson_handle_bytes.restype = i
    lib.poisson_hydrostatic_force.argtypes = [vp, vp, d, d, d, d, d, vp, vp, vp]
    lib.poisson_hydrostatic_force.restype = i
    lib.poisson_test_unreachable_barrier.argtypes = [vp, i]
    lib.poisson_test_unreachable_barrier.restype = i
    lib.poisson_test_fail_alloc.argtypes = [i]
    lib.poisson_test_fail_alloc.restype = i
    lib.poisson_test_live_allocations.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    lib.poisson_test_live_allocations.restype = i
    for name in EXPORTS[1:10] + ["poisson_profile", "poisson_profile_read", "poisson_describe"]:
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def strerror(status):
    try:
        return load().poisson_strerror(int(status)).decode()
    except OSError:
        return "status %d" % status


def _addr(a):
    """Address of a float64 array: numpy (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def _check(rc, what, ok=(OK,)):
    if rc not in ok:
        raise PoissonError(rc, what)
    return rc


def default_opts():
    o = Opts()
    load().poisson_default_opts(ctypes.byref(o))
    return o


def make_opts(precision="fp32", precond="jacobi", omega=1.0, max_iters=20000, inner_tol=1e-4,
              tile=0, stream=None, dirichlet_walls=0, periodic_x=False):
    o = default_opts()
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
    o.omega, o.max_iters, o.inner_tol, o.tile = omega, max_iters, inner_tol, tile
    o.stream = stream if (stream is None or isinstance(stream, int)) else stream.cuda_stream
    o.dirichlet_walls = dirichlet_walls
    o.periodic_x = 1 if periodic_x else 0
    return o


def required_bytes(nx, ny, nz, budget=0, **opts):
    """(status, bytes): the device bytes a handle of this grid and options would hold, and
    ENOMEM_BUDGET when they exceed ``budget`` (> 0); OK otherwise."""
    b = ctypes.c_uint64(0)
    rc = load().poisson_required_bytes(nx, ny, nz, ctypes.byref(make_opts(**opts)),
                                       ctypes.c_uint64(int(budget)), ctypes.byref(b))
    _check(rc, "poisson_required_bytes", ok=(OK, ENOMEM_BUDGET))
    return rc, int(b.value)


class Poisson:
    """One grid: ``poisson_create`` ... ``poisson_destroy``."""

    def __init__(self, nx, ny, nz, h, precision="fp32", precond="jacobi", omega=1.0,
                 max_iters=20000, inner_tol=1e-4, tile=0, stream=None, dirichlet_walls=0,
                 periodic_x=False):
        lib = load()
        o = make_opts(precision, precond, omega, max_iters, inner_tol, tile, stream,
                      dirichlet_walls, periodic_x)
        self.shape = (nz, ny, nx)
        self.h = h
        self.opts = o
        hnd = ctypes.c_void_p()
        _check(lib.poisson_create(nx, ny, nz, h, ctypes.byref(o), ctypes.byref(hnd)), "poisson_create")
        self._h = hnd

    @property
    def handle(self):
        return self._h

    def close(self):
        """Destroys the handle; refused (PoissonError EINVAL, handle kept) while a batch job
        that poll() has not reported uses it."""
        if self._h:
            _check(load().poisson_destroy(self._h), "poisson_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_density(self, F, rho_air=1.0, rho_water=1000.0):
        mem = MEM_HOST if isinstance(F, np.ndarray) or not getattr(F, "is_cuda", False) else MEM_DEVICE
        _check(load().poisson_set_density(self._h, _addr(F), rho_air, rho_water, mem),
               "poisson_set_density")

    def solve(self, rhs, p, tol, allow=(OK,)):
        """Solves in place into ``p``; returns (status, stats dict)."""
        st = Stats()
        rc = load().poisson_solve(self._h, _addr(rhs), _addr(p), tol, ctypes.byref(st))
        _check(rc, "poisson_solve", ok=allow)
        return rc, st.as_dict()

    def apply(self, x, y, precision="fp64"):
        _check(load().poisson_apply(self._h, _addr(x), _addr(y), PRECISION[precision]), "poisson_apply")

    def precond_apply(self, r, z, kind="jacobi", precision="fp64"):
        _check(load().poisson_precond_apply(self._h, _addr(r), _addr(z), PRECOND[kind],
                                            PRECISION[precision]), "poisson_precond_apply")

    def profile(self, enable=True):
        _check(load().poisson_profile(self._h, 1 if enable else 0), "poisson_profile")

    def profile_read(self):
        t = KernelTimes()
        _check(load().poisson_profile_read(self._h, ctypes.byref(t)), "poisson_profile_read")
        return t.as_dict()

    def test_unreachable_barrier(self, extra):
        """Testing aid: the next persistent launches wait at their grid barriers for ``extra``
        CTAs more than they launch (0 restores), so a solve ends with ETIMEOUT."""
        _check(load().poisson_test_unreachable_barrier(self._h, int(extra)),
               "poisson_test_unreachable_barrier")

    def device_bytes(self):
        """Device bytes the handle holds (poisson_handle_bytes)."""
        b = ctypes.c_uint64(0)
        _check(load().poisson_handle_bytes(self._h, ctypes.byref(b)), "poisson_handle_bytes")
        return int(b.value)

    def describe(self):
        buf = ctypes.create_string_buffer(256)
        _check(load().poisson_describe(self._h, buf, 256), "poisson_describe")
        return buf.value.decode()

    def set_apertures(self, ax=None, ay=None, az=None, vol=None):
        """Free-slip cut cells: open fractions of the MAC faces and fluid fractions of the cells
        (numpy or CUDA float64); call set_density afterwards.  No arguments: the plain operator."""
        if ax is None:
            _check(load().poisson_set_apertures(self._h, None, None, None, None, MEM_HOST),
                   "poisson_set_apertures")
            return
        mem = MEM_HOST if isinstance(ax, np.ndarray) or not getattr(ax, "is_cuda", False) else MEM_DEVICE
        _check(load().poisson_set_apertures(self._h, _addr(ax), _addr(ay), _addr(az), _addr(vol),
                                            mem), "poisson_set_apertures")

    def divergence(self, u, v, w, dt, s):
        """``s = div_h(u) / dt`` from face velocities ``u`` ``(nz, ny, nx+1)``, ``v``
        ``(nz, ny+1, nx)``, ``w`` ``(nz+1, ny, nx)`` (numpy or CUDA float64) into ``s``."""
        _check(load().poisson_divergence(self._h, _addr(u), _addr(v), _addr(w), dt, _addr(s)),
               "poisson_divergence")

    def project(self, u, v, w, p, dt):
        """In place: ``u -= dt beta_f grad_h p`` on every face (walls unchanged)."""
        _check(load().poisson_project(self._h, _addr(u), _addr(v), _addr(w), _addr(p), dt),
               "poisson_project")

    def hydrostatic_force(self, F, u, v, w, g, z_o, dt, rho_air=1.0, rho_water=1000.0):
        """Adds dt times the reduced-pressure force to the face velocities in place."""
        _check(load().poisson_hydrostatic_force(self._h, _addr(F), rho_air, rho_water, g, z_o, dt,
                                                _addr(u), _addr(v), _addr(w)),
               "poisson_hydrostatic_force")

    def projection_step(self, u, v, w, dt, p, tol, s=None):
        """One pressure projection of a provisional face velocity, in place: ``s =
        div(u)/dt``, ``p`` solves the pressure equation (``p`` is the warm start on entry), then
        ``u -= dt beta grad p``.  ``s``: optional scratch of the cell shape (same kind of array
        as ``p``).  Returns the solve's (status, stats)."""
        if s is None:
            s = np.empty(self.shape) if isinstance(p, np.ndarray) else p.new_empty(self.shape)
        self.divergence(u, v, w, dt, s)
        rc, st = self.solve(s, p, tol)
        self.project(u, v, w, p, dt)
        return rc, st

    def get_operator(self, bx=None, by=None, bz=None, diag=None):
        _check(load().poisson_get_operator(self._h, _addr(bx), _addr(by), _addr(bz), _addr(diag)),
               "poisson_get_operator")


def residual_noalloc(nx, ny, nz, h, F, rho_air, rho_water, rhs, p, out=None, stream=None):
    """FP64 relative residual of ``p`` through ``poisson_residual_noalloc`` (no device allocation
    in the library during the call; for callers that cannot allocate).  ``F``, ``rhs``, ``p`` are
    CUDA float64 tensors; with ``out`` (a one-element CUDA float64 tensor) the result is written
    there on the stream and None is returned, else the value is returned."""
    st = stream if (stream is None or isinstance(stream, int)) else stream.cuda_stream
    if out is not None:
        rc = load().poisson_residual_noalloc(nx, ny, nz, h, _addr(F), rho_air, rho_water,
                                             _addr(rhs), _addr(p), _addr(out), st)
        _check(rc, "poisson_residual_noalloc")
        return None
    v = ctypes.c_double(0.0)
    rc = load().poisson_residual_noalloc(nx, ny, nz, h, _addr(F), rho_air, rho_water, _addr(rhs),
                                         _addr(p), ctypes.addressof(v), st)
    _check(rc, "poisson_residual_noalloc")
    return v.value


def kernel_launches():
    """CUDA kernels launched by the library since it was loaded."""
    return int(load().poisson_kernel_launches())


def test_fail_alloc(n):
    """Testing aid: the n-th device or pinned-host allocation of the library from now on fails
    as if memory were exhausted (0: none)."""
    _check(load().poisson_test_fail_alloc(int(n)), "poisson_test_fail_alloc")


def live_allocations():
    """The library's device and pinned-host allocations not yet released."""
    v = ctypes.c_longlong()
    _check(load().poisson_test_live_allocations(ctypes.byref(v)), "poisson_test_live_allocations")
    return int(v.value)


def batch_submit(solvers, rhs, p, tol):
    n = len(solvers)
    H = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    R = (ctypes.c_void_p * n)(*[_addr(a) for a in rhs])
    P = (ctypes.c_void_p * n)(*[_addr(a) for a in p])
    T = (ctypes.c_double * n)(*([tol] * n if np.isscalar(tol) else list(tol)))
    tickets = (ctypes.c_uint64 * n)()
    _check(load().poisson_batch_submit(H, R, P, T, n, tickets), "poisson_batch_submit")
    return list(tickets)


def poll(ticket):
    """Returns (status, stats dict or None); status PENDING while running."""
    st = Stats()
    rc = load().poisson_poll(ctypes.c_uint64(ticket), ctypes.byref(st))
    return rc, (st.as_dict() if rc != PENDING else None)
