"""Seeded synthetic inputs for the pressure Poisson solve of a Cartesian-grid ship-wave run.

This module produces the two fields a two-phase ship-wave code hands to its pressure projection
(Formulation section, eqs. (density) and (pois); Numerical Time Integration): the water volume
fraction ``F`` of every cell (0 = air, 1 = water) and the Poisson source ``s = div_h(u*) / dt``
built from a face-centred provisional velocity ``u*``.  It is shared by the CPU oracle tests and
the GPU library's tests and benchmark, and it deliberately holds none of the solver's arithmetic:
no density, no face coefficients, no operator, no preconditioner.

Conventions (shared by every consumer):

* grid ``nx x ny x nz`` cells of spacing ``h``; domain ``[0, nx h] x [0, ny h] x [0, nz h]``;
  cell ``(i, j, k)`` has its centre at ``((i+1/2)h, (j+1/2)h, (k+1/2)h)``;
* arrays are numpy float64, shape ``(nz, ny, nx)``, C order (x fastest, linear index
  ``i + nx*(j + ny*k)``);
* walls ``x = 0, x = Lx, y = 0, y = Ly, z = 0`` are impermeable (wall-normal face velocity 0);
  the top face ``z = Lz`` keeps its velocity (it is the open, Dirichlet-pressure boundary).

The free surface is ``z = z0 + eta(x, y)`` with ``z0 = 1/2`` of the domain height.  The fraction is
a mollified step of the signed vertical distance to it (the paper smooths the density jump with a
mollified step, Formulation, eq. (density)); a hull given by a signed distance ``psi`` (positive
outside, Enforcement of Body Boundary Conditions) is filled with water-density fluid.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RHO_AIR = 1.0
RHO_WATER = 1000.0
DT = 1.0e-3
N_MODES = 8
MODE_AMPLITUDE = 0.1


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    h: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def lengths(self):
        return (self.nx * self.h, self.ny * self.h, self.nz * self.h)

    def centres(self, axis):
        n = (self.nx, self.ny, self.nz)[axis]
        return (np.arange(n, dtype=np.float64) + 0.5) * self.h


@dataclasses.dataclass
class Case:
    """One synthetic solve: the grid, the water fraction, the source and the target tolerance."""
    name: str
    grid: Grid
    F: np.ndarray
    s: np.ndarray
    tol: float
    meta: dict


def smoothed_step(d, eps):
    """Mollified Heaviside of half-width ``eps``: 0 below ``-eps``, 1 above ``eps``, and the
    sinusoidal ramp ``(1 + d/eps + sin(pi d/eps)/pi) / 2`` in between."""
    d = np.asarray(d, dtype=np.float64)
    out = np.where(d > eps, 1.0, 0.0)
    ramp = np.abs(d) <= eps
    if np.any(ramp):
        dr = d[ramp] / eps
        out[ramp] = 0.5 * (1.0 + dr + np.sin(math.pi * dr) / math.pi)
    return out


# ----------------------------------------------------------------------------------- velocity
@dataclasses.dataclass(frozen=True)
class Mode:
    a: tuple      # unit amplitude direction (3,)
    k: tuple      # integer wave numbers per axis, each in {1, 2, 3}
    phase: float  # in [0, 2 pi)


def fourier_modes(rng: np.random.Generator, n=N_MODES):
    """``n`` random smooth Fourier modes ``a sin(2 pi k . (x / L) + phase)`` of ``u*``."""
    modes = []
    for _ in range(n):
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        k = rng.integers(1, 4, size=3)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        modes.append(Mode(tuple(float(v) for v in a), tuple(int(v) for v in k), float(ph)))
    return modes


def advect_modes(modes, grid: Grid, dt, c=(-1.0, 0.0, 0.0)):
    """Translate every mode by ``c dt`` (the free stream of the entrance/exit conditions)."""
    L = grid.lengths
    out = []
    for m in modes:
        shift = sum(2.0 * math.pi * m.k[d] * c[d] * dt / L[d] for d in range(3))
        out.append(Mode(m.a, m.k, (m.phase - shift) % (2.0 * math.pi)))
    return out


def _face_mask(n, open_top):
    m = np.ones(n + 1)
    m[0] = 0.0
    if not open_top:
        m[n] = 0.0
    return m


def face_velocity(grid: Grid, modes, amp=MODE_AMPLITUDE):
    """Face-centred ``u*`` from the modes: ``(u, v, w)`` with shapes ``(nz, ny, nx+1)``,
    ``(nz, ny+1, nx)``, ``(nz+1, ny, nx)``; wall-normal faces are zero, the top face is kept."""
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    L = grid.lengths
    xc, yc, zc = grid.centres(0), grid.centres(1), grid.centres(2)
    xf, yf, zf = (np.arange(nx + 1) * h, np.arange(ny + 1) * h, np.arange(nz + 1) * h)
    u = np.zeros((nz, ny, nx + 1))
    v = np.zeros((nz, ny + 1, nx))
    w = np.zeros((nz + 1, ny, nx))
    for m in modes:
        tx = lambda x: 2 * math.pi * m.k[0] * x / L[0]
        ty = lambda y: 2 * math.pi * m.k[1] * y / L[1]
        tz = lambda z: 2 * math.pi * m.k[2] * z / L[2]
        u += amp * m.a[0] * np.sin(tz(zc)[:, None, None] + ty(yc)[None, :, None]
                                   + tx(xf)[None, None, :] + m.phase)
        v += amp * m.a[1] * np.sin(tz(zc)[:, None, None] + ty(yf)[None, :, None]
                                   + tx(xc)[None, None, :] + m.phase)
        w += amp * m.a[2] * np.sin(tz(zf)[:, None, None] + ty(yc)[None, :, None]
                                   + tx(xc)[None, None, :] + m.phase)
    u *= _face_mask(nx, False)[None, None, :]
    v *= _face_mask(ny, False)[None, :, None]
    w *= _face_mask(nz, True)[:, None, None]
    return u, v, w


def divergence_source(grid: Grid, modes, dt=DT, amp=MODE_AMPLITUDE, zchunk=32):
    """``s = div_h(u*) / dt`` at cell centres, the discrete flux difference of the face velocity of
    :func:`face_velocity` divided by ``h dt``.

    Each mode is separable, ``sin(tx + ty + tz + phase) = Im(e^{i phase} e^{i tx} e^{i ty}
    e^{i tz})``, so the flux difference of one velocity component is an outer product of 1-D
    factors; the sum is built plane-block by plane-block to bound host memory on large grids.
    """
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    L = grid.lengths
    s = np.empty(grid.shape)
    fac = []
    for m in modes:
        ex_c = np.exp(1j * 2 * math.pi * m.k[0] * grid.centres(0) / L[0])
        ey_c = np.exp(1j * 2 * math.pi * m.k[1] * grid.centres(1) / L[1])
        ez_c = np.exp(1j * 2 * math.pi * m.k[2] * grid.centres(2) / L[2])
        ex_f = np.exp(1j * 2 * math.pi * m.k[0] * np.arange(nx + 1) * h / L[0]) * _face_mask(nx, False)
        ey_f = np.exp(1j * 2 * math.pi * m.k[1] * np.arange(ny + 1) * h / L[1]) * _face_mask(ny, False)
        ez_f = np.exp(1j * 2 * math.pi * m.k[2] * np.arange(nz + 1) * h / L[2]) * _face_mask(nz, True)
        dx, dy, dz = np.diff(ex_f), np.diff(ey_f), np.diff(ez_f)
        c = amp * np.exp(1j * m.phase)
        # (z, y) factors multiplying the x-difference and the x-centre values
        P = c * m.a[0] * (ez_c[:, None] * ey_c[None, :])
        Q = c * (m.a[1] * ez_c[:, None] * dy[None, :] + m.a[2] * dz[:, None] * ey_c[None, :])
        fac.append((P, Q, dx, ex_c))
    for k0 in range(0, nz, zchunk):
        k1 = min(nz, k0 + zchunk)
        acc = np.zeros((k1 - k0, ny, nx))
        for P, Q, dx, ex_c in fac:
            acc += (P[k0:k1, :, None] * dx[None, None, :]
                    + Q[k0:k1, :, None] * ex_c[None, None, :]).imag
        s[k0:k1] = acc / (h * dt)
    return s


# ----------------------------------------------------------------------------------- geometry
def ellipse_sdf(x, y, xc, yc, a, b):
    """Approximate signed distance of a vertical elliptic strut (semi-axes ``a`` in x, ``b`` in
    y), negative inside; exact on the minor axis, good to within a cell near the surface."""
    r = np.sqrt(((x - xc) / a) ** 2 + ((y - yc) / b) ** 2)
    return (r - 1.0) * b


def wedge_sdf(x, y, xa, yc, half_angle):
    """Signed distance to a wedge of half-angle ``half_angle`` whose bow (apex) sits at
    ``(xa, yc)`` and which opens towards +x to the end of the domain: the larger of the signed
    distances to its two side planes (negative inside)."""
    sn, cs = math.sin(half_angle), math.cos(half_angle)
    xp, yp = x - xa, y - yc
    return np.maximum(yp * cs - xp * sn, -yp * cs - xp * sn)


def cut_apertures(grid: Grid, psi_fn, sub=4):
    """Open fractions of the MAC faces and fluid fractions of the cells for a body given by a
    signed distance ``psi(x, y, z)`` (positive outside, in the fluid): the share of ``sub x sub``
    sample points on each face (``sub^3`` in each cell) where ``psi > 0``.  Returns
    ``(ax, ay, az, vol)`` with the shapes of ``u, v, w`` and of the cells.  Geometry input for
    free-slip cut cells; no part of the solve."""
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    o = (np.arange(sub) + 0.5) / sub  # sample offsets inside a cell / face, in cells

    def frac(x, y, z):
        return (psi_fn(x, y, z) > 0).mean(axis=-1)

    def grid3(a, b, c):
        return np.meshgrid(a, b, c, indexing="ij")

    xf, yf, zf = np.arange(nx + 1) * h, np.arange(ny + 1) * h, np.arange(nz + 1) * h
    xs = ((np.arange(nx)[:, None] + o[None, :]) * h)  # (nx, sub) sample x inside each cell
    ys = ((np.arange(ny)[:, None] + o[None, :]) * h)
    zs = ((np.arange(nz)[:, None] + o[None, :]) * h)
    ax = np.empty((nz, ny, nx + 1))
    ay = np.empty((nz, ny + 1, nx))
    az = np.empty((nz + 1, ny, nx))
    vol = np.empty((nz, ny, nx))
    for k in range(nz):
        Z = zs[k]
        # x faces: samples over (y, z) of each face
        Y, Zg = np.meshgrid(ys.ravel(), Z, indexing="ij")  # (ny*sub, sub)
        for i in range(nx + 1):
            v = (psi_fn(np.full_like(Y, xf[i]), Y, Zg) > 0).reshape(ny, sub * sub)
            ax[k, :, i] = v.mean(axis=1)
        X, Zg = np.meshgrid(xs.ravel(), Z, indexing="ij")  # (nx*sub, sub)
        for j in range(ny + 1):
            v = (psi_fn(X, np.full_like(X, yf[j]), Zg) > 0).reshape(nx, sub * sub)
            ay[k, j, :] = v.mean(axis=1)
        X, Y, Zg = grid3(xs.ravel(), ys.ravel(), Z)  # (nx*sub, ny*sub, sub)
        v = (psi_fn(X, Y, Zg) > 0).reshape(nx, sub, ny, sub, sub)
        vol[k] = v.mean(axis=(1, 3, 4)).T
    for k in range(nz + 1):
        X, Y = np.meshgrid(xs.ravel(), ys.ravel(), indexing="ij")
        v = (psi_fn(X, Y, np.full_like(X, zf[k])) > 0).reshape(nx, sub, ny, sub)
        az[k] = v.mean(axis=(1, 3)).T
    return ax, ay, az, vol


def water_fraction(grid: Grid, eta_fn, psi_fn=None, z0=None, eps_cells=1.5, breaking=None,
                   zchunk=32):
    """Water fraction ``F = H_eps(z0 + eta(x, y) - z)`` at cell centres, with ``eps = 1.5 h``;
    a body ``psi(x, y) < 0`` is filled with water (``F = max(F, H_eps(-psi))``).  ``breaking``
    is ``(rng, prob)``: each near-surface cell (``|d| <= 2h``) is, with probability ``prob``,
    replaced by a random sharp 0 or 1 (overturned, breaking-like patches)."""
    h = grid.h
    eps = eps_cells * h
    if z0 is None:
        z0 = 0.5 * grid.lengths[2]
    x, y, z = grid.centres(0), grid.centres(1), grid.centres(2)
    surf = z0 + eta_fn(x[None, :], y[:, None])           # (ny, nx)
    body = None
    if psi_fn is not None:
        body = smoothed_step(-psi_fn(x[None, :], y[:, None]), eps)   # (ny, nx), full depth
    F = np.empty(grid.shape)
    for k0 in range(0, grid.nz, zchunk):
        k1 = min(grid.nz, k0 + zchunk)
        d = surf[None, :, :] - z[k0:k1, None, None]
        Fk = smoothed_step(d, eps)
        if body is not None:
            Fk = np.maximum(Fk, body[None, :, :])
        if breaking is not None:
            rng, prob = breaking
            near = np.abs(d) <= 2.0 * h
            flip = near & (rng.random(d.shape) < prob)
            vals = (rng.random(d.shape) < 0.5).astype(np.float64)
            Fk = np.where(flip, vals, Fk)
            if body is not None:
                Fk = np.maximum(Fk, body[None, :, :])
        F[k0:k1] = Fk
    return F


# ----------------------------------------------------------------------------------- the cases
def flat_case(nx=32, ny=32, nz=32, seed=0, tol=1e-10, h=None):
    """Flat free surface ``z = 1/2 + 0.02 sin(2 pi x) cos(2 pi y)`` (no body); source from 8
    random modes of amplitude 0.1 with ``dt = 1e-3``."""
    grid = Grid(nx, ny, nz, h if h is not None else 1.0 / nz)
    rng = np.random.default_rng(seed)
    eta = lambda x, y: 0.02 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y)
    F = water_fraction(grid, eta)
    modes = fourier_modes(rng)
    s = divergence_source(grid, modes)
    return Case("flat", grid, F, s, tol, {"seed": seed, "modes": modes})


def strut_case(nx=256, ny=128, nz=128, seed=0, tol=1e-9):
    """Surface-piercing elliptic strut (semi-axes 0.1 x 0.02, full depth, water density) at the
    domain centre, Kelvin-like surface ``eta = 0.01 sin(k (x - xc)) exp(-|y - yc| / 0.2)`` with a
    seeded ``k`` in [8, 16]; source as in :func:`flat_case`."""
    grid = Grid(nx, ny, nz, 1.0 / nz)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = grid.lengths
    xc, yc = 0.5 * Lx, 0.5 * Ly
    kw = rng.uniform(8.0, 16.0)
    eta = lambda x, y: 0.01 * np.sin(kw * (x - xc)) * np.exp(-np.abs(y - yc) / 0.2)
    psi = lambda x, y: ellipse_sdf(x, y, xc, yc, 0.1, 0.02)
    F = water_fraction(grid, eta, psi)
    modes = fourier_modes(rng)
    s = divergence_source(grid, modes)
    return Case("strut", grid, F, s, tol, {"seed": seed, "k": kw, "modes": modes})


def wedge_case(nx=1024, ny=512, nz=256, seed=0, tol=1e-9):
    """Wedge-like hull (half-angle seeded in [10, 30] degrees, bow at ``x = Lx/4``), Kelvin-like
    surface as in :func:`strut_case` measured from the bow, and breaking-like patches: 5 % of the
    near-surface cells set to a random sharp 0 or 1."""
    grid = Grid(nx, ny, nz, 1.0 / nz)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = grid.lengths
    xa, yc = 0.25 * Lx, 0.5 * Ly
    theta = math.radians(rng.uniform(10.0, 30.0))
    kw = rng.uniform(8.0, 16.0)
    eta = lambda x, y: 0.01 * np.sin(kw * (x - xa)) * np.exp(-np.abs(y - yc) / 0.2)
    psi = lambda x, y: wedge_sdf(x, y, xa, yc, theta)
    F = water_fraction(grid, eta, psi, breaking=(rng, 0.05))
    modes = fourier_modes(rng)
    s = divergence_source(grid, modes)
    return Case("wedge", grid, F, s, tol,
                {"seed": seed, "theta_deg": math.degrees(theta), "k": kw, "modes": modes})


def draw_shape(rng, lo=(32, 32, 32), hi=(128, 64, 64), mult=16, max_aspect=4.0):
    """A grid shape with every dimension a multiple of ``mult`` in ``[lo, hi]``, drawn uniformly
    and redrawn while the aspect ratio exceeds ``max_aspect``."""
    while True:
        dims = [int(rng.integers(lo[d] // mult, hi[d] // mult + 1)) * mult for d in range(3)]
        if max(dims) / min(dims) <= max_aspect:
            return tuple(dims)


def mixed_case(shape, seed, tol=1e-9):
    """One solve of a batch or request mix: its own seeded surface phases, a strut at a seeded
    position and a source of 8 modes (the flat case's recipe plus a body)."""
    nx, ny, nz = shape
    grid = Grid(nx, ny, nz, 1.0 / nz)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = grid.lengths
    px, py = rng.uniform(0.0, 2 * math.pi, size=2)
    eta = lambda x, y: 0.02 * np.sin(2 * math.pi * x / Lx + px) * np.cos(2 * math.pi * y / Ly + py)
    xc = rng.uniform(0.3, 0.7) * Lx
    yc = rng.uniform(0.3, 0.7) * Ly
    psi = lambda x, y: ellipse_sdf(x, y, xc, yc, 0.1, 0.02)
    F = water_fraction(grid, eta, psi)
    modes = fourier_modes(rng)
    s = divergence_source(grid, modes)
    return Case("mixed", grid, F, s, tol, {"seed": seed, "modes": modes, "strut": (xc, yc)})


def batch_cases(n=64, seed=0, lo=(32, 32, 32), hi=(128, 64, 64), tol=1e-9):
    """``n`` independent solves of uneven size (the batched workload)."""
    rng = np.random.default_rng(seed)
    shapes = [draw_shape(rng, lo, hi) for _ in range(n)]
    return [mixed_case(sh, seed * 100003 + 17 * i + 1, tol) for i, sh in enumerate(shapes)]


# ----------------------------------------------------------------------------- torch twins
# The same fields computed with torch (float64) on any device, for workloads that generate
# inputs inside a running loop (the served request stream).  Same formulas as the numpy
# versions above; tests check the two agree.
def _torch():
    import torch
    return torch


def smoothed_step_t(d, eps):
    torch = _torch()
    dr = d / eps
    ramp = 0.5 * (1.0 + dr + torch.sin(math.pi * dr) / math.pi)
    return torch.where(d > eps, torch.ones_like(d), torch.where(d < -eps, torch.zeros_like(d), ramp))


def water_fraction_t(grid: Grid, eta_fn, psi_fn=None, z0=None, eps_cells=1.5, device="cpu"):
    """:func:`water_fraction` (without breaking patches) in torch, shape (nz, ny, nx)."""
    torch = _torch()
    h = grid.h
    eps = eps_cells * h
    if z0 is None:
        z0 = 0.5 * grid.lengths[2]
    f64 = torch.float64
    x = (torch.arange(grid.nx, dtype=f64, device=device) + 0.5) * h
    y = (torch.arange(grid.ny, dtype=f64, device=device) + 0.5) * h
    z = (torch.arange(grid.nz, dtype=f64, device=device) + 0.5) * h
    surf = z0 + eta_fn(x[None, :], y[:, None])
    F = smoothed_step_t(surf[None, :, :] - z[:, None, None], eps)
    if psi_fn is not None:
        F = torch.maximum(F, smoothed_step_t(-psi_fn(x[None, :], y[:, None]), eps)[None, :, :])
    return F


def divergence_source_t(grid: Grid, modes, dt=DT, amp=MODE_AMPLITUDE, device="cpu"):
    """:func:`divergence_source` in torch (complex128 outer products), shape (nz, ny, nx)."""
    torch = _torch()
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    L = grid.lengths
    c128, f64 = torch.complex128, torch.float64
    acc = torch.zeros(grid.shape, dtype=f64, device=device)

    def e(kk, pos, Ld):
        return torch.exp(1j * (2 * math.pi * kk / Ld) * pos.to(c128))

    def mask(n, open_top):
        m = torch.ones(n + 1, dtype=c128, device=device)
        m[0] = 0
        if not open_top:
            m[n] = 0
        return m

    cx = (torch.arange(nx, dtype=f64, device=device) + 0.5) * h
    cy = (torch.arange(ny, dtype=f64, device=device) + 0.5) * h
    cz = (torch.arange(nz, dtype=f64, device=device) + 0.5) * h
    fx = torch.arange(nx + 1, dtype=f64, device=device) * h
    fy = torch.arange(ny + 1, dtype=f64, device=device) * h
    fz = torch.arange(nz + 1, dtype=f64, device=device) * h
    for m in modes:
        ex_c, ey_c, ez_c = e(m.k[0], cx, L[0]), e(m.k[1], cy, L[1]), e(m.k[2], cz, L[2])
        dx = torch.diff(e(m.k[0], fx, L[0]) * mask(nx, False))
        dy = torch.diff(e(m.k[1], fy, L[1]) * mask(ny, False))
        dz = torch.diff(e(m.k[2], fz, L[2]) * mask(nz, True))
        c = amp * complex(math.cos(m.phase), math.sin(m.phase))
        P = c * m.a[0] * (ez_c[:, None] * ey_c[None, :])
        Q = c * (m.a[1] * ez_c[:, None] * dy[None, :] + m.a[2] * dz[:, None] * ey_c[None, :])
        acc += (P[:, :, None] * dx[None, None, :] + Q[:, :, None] * ex_c[None, None, :]).imag
    return acc / (h * dt)


def mixed_fields_t(shape, seed, device="cpu"):
    """The density field and first source of :func:`mixed_case` computed with torch, plus the
    modes (for drifting the source step by step).  Returns (grid, F, s, modes)."""
    nx, ny, nz = shape
    grid = Grid(nx, ny, nz, 1.0 / nz)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = grid.lengths
    px, py = rng.uniform(0.0, 2 * math.pi, size=2)
    torch = _torch()
    eta = lambda x, y: 0.02 * torch.sin(2 * math.pi * x / Lx + px) * torch.cos(2 * math.pi * y / Ly + py)
    xc = rng.uniform(0.3, 0.7) * Lx
    yc = rng.uniform(0.3, 0.7) * Ly

    def psi(x, y):
        r = torch.sqrt(((x - xc) / 0.1) ** 2 + ((y - yc) / 0.02) ** 2)
        return (r - 1.0) * 0.02

    F = water_fraction_t(grid, eta, psi, device=device)
    modes = fourier_modes(rng)
    s = divergence_source_t(grid, modes, device=device)
    return grid, F, s, modes


def wedge_fields_t(shape=(1024, 512, 256), seed=0, device="cpu"):
    """The wedge workload of :func:`wedge_case` computed with torch on ``device``: same hull,
    surface and source; the breaking patches come from their own numpy generator (seed + 12345,
    one float32 pair per cell, z-chunk by z-chunk), so every device gets the same patches (they
    differ from the numpy version's).  Returns (grid, F, s, meta)."""
    torch = _torch()
    nx, ny, nz = shape
    grid = Grid(nx, ny, nz, 1.0 / nz)
    rng = np.random.default_rng(seed)
    Lx, Ly, _ = grid.lengths
    xa, yc = 0.25 * Lx, 0.5 * Ly
    theta = math.radians(rng.uniform(10.0, 30.0))
    kw = rng.uniform(8.0, 16.0)
    sn, cs = math.sin(theta), math.cos(theta)
    eta = lambda x, y: 0.01 * torch.sin(kw * (x - xa)) * torch.exp(-torch.abs(y - yc) / 0.2)
    psi = lambda x, y: torch.maximum((y - yc) * cs - (x - xa) * sn, -(y - yc) * cs - (x - xa) * sn)
    F = water_fraction_t(grid, eta, psi, device=device)
    # breaking-like patches: 5 % of the cells within 2h of the surface set to a sharp 0 or 1
    h = grid.h
    f64 = torch.float64
    x = (torch.arange(nx, dtype=f64, device=device) + 0.5) * h
    y = (torch.arange(ny, dtype=f64, device=device) + 0.5) * h
    z = (torch.arange(nz, dtype=f64, device=device) + 0.5) * h
    surf = 0.5 * grid.lengths[2] + eta(x[None, :], y[:, None])
    body = smoothed_step_t(-psi(x[None, :], y[:, None]), 1.5 * h)
    gen = np.random.default_rng(int(seed) + 12345)
    for k0 in range(0, nz, 32):
        k1 = min(nz, k0 + 32)
        d = surf[None, :, :] - z[k0:k1, None, None]
        near = torch.abs(d) <= 2.0 * h
        u = torch.from_numpy(gen.random((2,) + tuple(d.shape), dtype=np.float32)).to(device)
        flip = near & (u[0] < 0.05)
        vals = (u[1] < 0.5).to(f64)
        F[k0:k1] = torch.maximum(torch.where(flip, vals, F[k0:k1]), body[None, :, :])
    modes = fourier_modes(rng)
    s = divergence_source_t(grid, modes, device=device)
    return grid, F, s, {"seed": seed, "theta_deg": math.degrees(theta), "k": kw}
