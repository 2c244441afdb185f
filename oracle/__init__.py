"""FP64 CPU oracle for the variable-coefficient pressure Poisson solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the GPU library never does, and the two share no code.

The arithmetic lives in ``poisson_oracle.c`` (plain C loops, FP64, optional OpenMP), compiled on
first use into ``oracle/_build/liboracle.so``; this module is the numpy-facing wrapper.  Every
array is float64, shape ``(nz, ny, nx)``, C order (x fastest).

What it computes (Formulation, eqs. (density) and (pois); Introduction on the preconditioned
conjugate-gradient solve of the second-order, variable-coefficient Poisson equation):
``rho = rho_air + F (rho_water - rho_air)``; face coefficients are the harmonic means
``2 / (rho_c + rho_n)`` of ``1/rho``; Neumann walls on x, y and the bottom; Dirichlet ``p = 0`` on
the top face.  ``A = -h^2 div_h(beta grad_h)`` is SPD and ``A p = -h^2 s`` is solved by PCG with a
Jacobi or red-black SSOR preconditioner.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py`` against closed forms,
library dense solves, series-resistance layered solutions and second-order convergence.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "poisson_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OK, EINVAL, ENOMEM, ENOTCONV, EBREAKDOWN = 0, -1, -2, -3, -4
JACOBI, SSOR = 0, 1
MEAN_HARMONIC, MEAN_ARITHMETIC = 0, 1
_PRECOND = {"jacobi": JACOBI, "ssor": SSOR, "rbssor": SSOR}

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile ``poisson_oracle.c`` with gcc (OpenMP if available, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_faces.argtypes = [i, i, i, P, d, d, i, P, P, P, P]
        lib.oracle_faces.restype = i
        lib.oracle_faces_bc.argtypes = [i, i, i, P, d, d, i, i, P, P, P, P]
        lib.oracle_faces_bc.restype = i
        lib.oracle_faces_cut.argtypes = [i, i, i, P, d, d, i, i, P, P, P, P, P, P, P, P]
        lib.oracle_faces_cut.restype = i
        lib.oracle_divergence_cut.argtypes = [i, i, i, d, d, P, P, P, P, P, P, P, P]
        lib.oracle_divergence_cut.restype = None
        lib.oracle_project_cut.argtypes = [i, i, i, d, d, P, d, d, i, P, P, P, P, P, P, P, P, P,
                                           P, P]
        lib.oracle_project_cut.restype = None
        lib.oracle_apply.argtypes = [i, i, i, P, P, P, P, P, P]
        lib.oracle_apply.restype = None
        lib.oracle_precond.argtypes = [i, i, i, P, P, P, P, i, d, P, P]
        lib.oracle_precond.restype = None
        lib.oracle_residual.argtypes = [i, i, i, P, P, P, P, P, P, P]
        lib.oracle_residual.restype = d
        lib.oracle_pcg.argtypes = [i, i, i, P, P, P, P, P, P, d, i, d, i,
                                   ctypes.POINTER(ctypes.c_int), P, P]
        lib.oracle_pcg.restype = i
        lib.oracle_divergence.argtypes = [i, i, i, d, d, P, P, P, P]
        lib.oracle_divergence.restype = None
        lib.oracle_project.argtypes = [i, i, i, d, d, P, d, d, P, P, P, P, P, P, P]
        lib.oracle_project.restype = None
        lib.oracle_project_bc.argtypes = [i, i, i, d, d, P, d, d, i, P, P, P, P, P, P, P]
        lib.oracle_project_bc.restype = None
        lib.oracle_hydrostatic_force.argtypes = [i, i, i, d, P, d, d, d, d, i, d, P, P, P]
        lib.oracle_hydrostatic_force.restype = None
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = i
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_set_threads.restype = None
        _lib = lib
        return lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads():
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def set_threads(n):
    _load().oracle_set_threads(int(n))


@dataclasses.dataclass
class Operator:
    """The FP64 operator ``A = -h^2 div_h(beta grad_h)``: low-side face arrays and diagonal."""
    nx: int
    ny: int
    nz: int
    bx: np.ndarray
    by: np.ndarray
    bz: np.ndarray
    diag: np.ndarray
    walls: int = 0
    apertures: tuple | None = None  # (ax, ay, az, vol) of a cut-cell operator

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def args(self):
        return (self.nx, self.ny, self.nz, _ptr(self.bx), _ptr(self.by), _ptr(self.bz),
                _ptr(self.diag))


WALL_XM, WALL_XP, WALL_YM, WALL_YP, WALL_ZM = 1, 2, 4, 8, 16
PERIODIC_X = 32  # in ``walls``: x periodic (no x walls)


def operator(F, rho_air=1.0, rho_water=1000.0, mean="harmonic", walls=0, apertures=None):
    """Assemble the operator from the water fraction ``F`` (shape ``(nz, ny, nx)``).  ``walls``:
    bitmask of side/bottom walls with p = 0 on the wall face (WALL_XM | ...); the others, as in
    the paper's configuration, have a zero normal gradient; the top face always has p = 0.
    ``PERIODIC_X`` in ``walls`` makes x periodic (the strut run of the Results), with no x
    walls; red-black SSOR then needs an even nx.  ``apertures = (ax, ay, az, vol)``: open
    fractions of the MAC faces (shapes of u, v, w) and fluid fractions of the cells for free-slip
    cut cells (Enforcement of Body Boundary Conditions): every face coefficient is scaled by its
    open fraction, a face of a cell with vol = 0 is closed, and such a cell is inactive
    (diagonal 1, no coupling)."""
    if walls & PERIODIC_X and walls & (WALL_XM | WALL_XP):
        raise ValueError("periodic x has no x walls")
    F = _f64(F)
    nz, ny, nx = F.shape
    bx, by, bz, dg = (np.empty_like(F) for _ in range(4))
    m = MEAN_HARMONIC if mean == "harmonic" else MEAN_ARITHMETIC
    if apertures is None:
        rc = _load().oracle_faces_bc(nx, ny, nz, _ptr(F), float(rho_air), float(rho_water), m,
                                     int(walls), _ptr(bx), _ptr(by), _ptr(bz), _ptr(dg))
    else:
        ap = tuple(_f64(a) for a in apertures)
        assert tuple(a.shape for a in ap[:3]) == _faces_shapes(nx, ny, nz) and ap[3].shape == F.shape
        rc = _load().oracle_faces_cut(nx, ny, nz, _ptr(F), float(rho_air), float(rho_water), m,
                                      int(walls), *(_ptr(a) for a in ap), _ptr(bx), _ptr(by),
                                      _ptr(bz), _ptr(dg))
        apertures = ap
    if rc != OK:
        raise RuntimeError("oracle_faces failed: %d" % rc)
    return Operator(nx, ny, nz, bx, by, bz, dg, int(walls), apertures)


def apply(op: Operator, x):
    """``y = A x``."""
    x = _f64(x).reshape(op.shape)
    y = np.empty_like(x)
    _load().oracle_apply(*op.args, _ptr(x), _ptr(y))
    return y


def precond(op: Operator, r, kind="jacobi", omega=1.0):
    """``z = M^{-1} r`` for the Jacobi or red-black SSOR(omega) preconditioner."""
    r = _f64(r).reshape(op.shape)
    z = np.empty_like(r)
    _load().oracle_precond(*op.args, _PRECOND[kind], float(omega), _ptr(r), _ptr(z))
    return z


def residual(op: Operator, b, x):
    """``(r, ||r||_2)`` with ``r = b - A x``."""
    b = _f64(b).reshape(op.shape)
    x = _f64(x).reshape(op.shape)
    r = np.empty_like(b)
    nrm = _load().oracle_residual(*op.args, _ptr(b), _ptr(x), _ptr(r))
    return r, float(nrm)


def rel_residual(op: Operator, b, x):
    """``||b - A x||_2 / ||b||_2`` in FP64."""
    b = _f64(b)
    _, nrm = residual(op, b, x)
    bn = float(np.linalg.norm(b.ravel()))
    return 0.0 if bn == 0.0 else nrm / bn


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    rel_residual: float
    status: int
    history: np.ndarray | None = None


def pcg(op: Operator, b, x0=None, tol=1e-12, precond="jacobi", omega=1.0, max_iters=100000,
        history=False):
    """Preconditioned conjugate gradients on ``A x = b``.  ``tol <= 0`` runs exactly
    ``max_iters`` iterations."""
    b = _f64(b).reshape(op.shape)
    x = np.zeros_like(b) if x0 is None else _f64(x0).reshape(op.shape).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.zeros(max(max_iters, 1)) if history else None
    st = _load().oracle_pcg(*op.args, _ptr(b), _ptr(x), float(tol), _PRECOND[precond],
                            float(omega), int(max_iters), ctypes.byref(it), ctypes.byref(rr),
                            _ptr(hist) if history else None)
    return PCGResult(x, it.value, rr.value, st, hist[:it.value] if history else None)


def _faces_shapes(nx, ny, nz):
    return (nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)


def divergence(u, v, w, h, dt, apertures=None):
    """``s = div_h(u) / dt`` at cell centres from MAC face velocities ``u`` ``(nz, ny, nx+1)``,
    ``v`` ``(nz, ny+1, nx)``, ``w`` ``(nz+1, ny, nx)`` (w's last plane is the top boundary):
    the flux difference of each cell divided by ``h dt`` (Numerical Time Integration: the
    pressure equation's source).  With ``apertures = (ax, ay, az, vol)`` the fluxes are
    ``a u`` and the difference is divided by ``vol`` as well (0 in inactive cells)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    nz, ny, nx1 = u.shape
    nx = nx1 - 1
    assert (v.shape, w.shape) == _faces_shapes(nx, ny, nz)[1:]
    s = np.empty((nz, ny, nx))
    if apertures is None:
        _load().oracle_divergence(nx, ny, nz, float(h), float(dt), _ptr(u), _ptr(v), _ptr(w),
                                  _ptr(s))
    else:
        ap = tuple(_f64(a) for a in apertures)
        _load().oracle_divergence_cut(nx, ny, nz, float(h), float(dt), _ptr(u), _ptr(v), _ptr(w),
                                      *(_ptr(a) for a in ap), _ptr(s))
    return s


def project(op: Operator, F, u, v, w, p, h, dt, rho_air=1.0, rho_water=1000.0):
    """The velocity correction ``u - dt beta_f grad_h p`` on every face (new arrays): interior
    faces use the operator's face coefficients and ``(p_n - p_c)/h``; the top face and the
    operator's Dirichlet walls, where ``p = 0``, use ``1/rho_c`` and the difference to 0 over
    ``h/2``; zero-gradient wall faces are unchanged.  Then
    ``divergence(u_new) = (A p - b)/h^2`` for ``b = rhs(divergence(u), h)``."""
    u, v, w = _f64(u).copy(), _f64(v).copy(), _f64(w).copy()
    p, F = _f64(p).reshape(op.shape), _f64(F).reshape(op.shape)
    assert (u.shape, v.shape, w.shape) == _faces_shapes(op.nx, op.ny, op.nz)
    if op.apertures is None:
        _load().oracle_project_bc(op.nx, op.ny, op.nz, float(h), float(dt), _ptr(F),
                                  float(rho_air), float(rho_water), op.walls, _ptr(op.bx),
                                  _ptr(op.by), _ptr(op.bz), _ptr(p), _ptr(u), _ptr(v), _ptr(w))
    else:
        _load().oracle_project_cut(op.nx, op.ny, op.nz, float(h), float(dt), _ptr(F),
                                   float(rho_air), float(rho_water), op.walls,
                                   *(_ptr(a) for a in op.apertures), _ptr(op.bx), _ptr(op.by),
                                   _ptr(op.bz), _ptr(p), _ptr(u), _ptr(v), _ptr(w))
    return u, v, w


def hydrostatic_force(F, u, v, w, h, g, z_o, dt=1.0, rho_air=1.0, rho_water=1000.0, walls=0):
    """The face velocities plus ``dt`` times the force of the reduced-pressure formulation (new
    arrays; Entrance and Exit Boundary Conditions, hydrostatic-pressure method).  The solve is
    then for ``P_r = P - rho g (z - z_o)``; the force on the face between cells c and n (n on the
    +axis side) is ``-(z_f - z_o) g beta_f (rho_n - rho_c) / h`` with the operator's face
    coefficient ``beta_f = 2/(rho_c + rho_n)`` and ``z_f`` the face's height; boundary faces get
    none; ``walls`` matters only through ``PERIODIC_X`` (the wrap face)."""
    F = _f64(F)
    nz, ny, nx = F.shape
    u, v, w = _f64(u).copy(), _f64(v).copy(), _f64(w).copy()
    assert (u.shape, v.shape, w.shape) == _faces_shapes(nx, ny, nz)
    _load().oracle_hydrostatic_force(nx, ny, nz, float(h), _ptr(F), float(rho_air),
                                     float(rho_water), float(g), float(z_o), int(walls), float(dt),
                                     _ptr(u), _ptr(v), _ptr(w))
    return u, v, w


def rhs(s, h, vol=None):
    """``b = -h^2 s``: the right side of ``A p = b`` for ``div((1/rho) grad p) = s``; with cut
    cells ``b = -h^2 (vol s)`` (the cell's fluid fraction times its source)."""
    if vol is None:
        return -(h * h) * _f64(s)
    return -(h * h) * (_f64(vol) * _f64(s))


def solve(F, s, h, tol=1e-12, precond="jacobi", omega=1.0, x0=None, rho_air=1.0,
          rho_water=1000.0, max_iters=100000):
    """Solve ``div((1/rho(F)) grad p) = s`` to relative residual ``tol``; returns
    ``(PCGResult, Operator)``."""
    op = operator(F, rho_air, rho_water)
    res = pcg(op, rhs(s, h), x0=x0, tol=tol, precond=precond, omega=omega, max_iters=max_iters)
    return res, op
