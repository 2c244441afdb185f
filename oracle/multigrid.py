"""FP64 CPU oracle of the multigrid V-cycle preconditioner (beyond the paper: its PCG
preconditioner is not specified, and a V-cycle is the standard stronger choice for the
variable-coefficient pressure Poisson equation of Formulation, eq. (pois)).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the GPU library never does, and the two share no code.

What it computes, step by step (plain numpy on whole arrays; the stencil applications go through
the oracle's own C ``apply``):

* Hierarchy.  Level 0 is the operator ``A``.  Level l+1 aggregates cells of level l in blocks
  of ``fx x fy x fz`` (2 along every axis with more than one cell; along a periodic x axis only
  while nx is even and at least 4, else 1; the last block of an odd axis has one cell).  With
  ``P`` the 0/1 matrix that maps an aggregate to its cells, the coarse operator is the Galerkin
  product ``A_{l+1} = P^T A_l P``: again a symmetric 7-point stencil whose face coupling is the
  sum of the fine couplings across the coarse face and whose diagonal is the sum of the fine
  diagonals of the block minus twice its internal couplings.  Level 0 is always coarsened
  once; coarsening stops at ``COARSE_MAX`` cells or when no axis can be coarsened.
* V-cycle ``y = V_l(r)``: ``x = omega D^-1 r`` (one damped Jacobi sweep from zero);
  ``e = V_{l+1}(P^T (r - A x))``; ``x += alpha P e``; ``y = x + omega D^-1 (r - A x)``.  On the
  coarsest level ``COARSE_SWEEPS`` damped Jacobi sweeps from zero.  As a matrix,
  ``V_l = 2B - BAB + alpha (I - BA) P V_{l+1} P^T (I - AB)`` with ``B = omega D^-1``: symmetric,
  and positive definite for 0 < omega < 1 (``lambda(D^-1 A) < 2`` for these diagonally dominant
  operators), so it is a valid PCG preconditioner for any alpha > 0.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import Operator, PERIODIC_X, apply

OMEGA = 0.9          # damping of the Jacobi smoother
ALPHA = 1.5          # scaling of the coarse-grid correction
COARSE_MAX = 512     # coarsest level: at most this many cells
COARSE_SWEEPS = 16   # damped Jacobi sweeps on the coarsest level


@dataclasses.dataclass
class Level:
    op: Operator
    f: tuple  # (fx, fy, fz): aggregation factors to the next level (None on the coarsest)


def factors(nx, ny, nz, periodic):
    """Aggregation factors of one coarsening step (1 = that axis is not coarsened)."""
    if periodic:
        fx = 2 if (nx % 2 == 0 and nx >= 4) else 1
    else:
        fx = 2 if nx > 1 else 1
    return fx, 2 if ny > 1 else 1, 2 if nz > 1 else 1


def _block_sum(a, f, nc):
    """Sum of ``a`` (shape (nz, ny, nx)) over aggregates of size f = (fx, fy, fz); nc = coarse
    shape (nzc, nyc, nxc).  Missing cells of a partial block count as zero."""
    fx, fy, fz = f
    nzc, nyc, nxc = nc
    pad = np.zeros((nzc * fz, nyc * fy, nxc * fx))
    pad[:a.shape[0], :a.shape[1], :a.shape[2]] = a
    return pad.reshape(nzc, fz, nyc, fy, nxc, fx).sum(axis=(1, 3, 5))


def galerkin(op: Operator, f):
    """``P^T A P`` for the aggregation with factors f, as an Operator of the coarse shape."""
    fx, fy, fz = f
    nz, ny, nx = op.shape
    nc = (-(-nz // fz), -(-ny // fy), -(-nx // fx))
    nzc, nyc, nxc = nc
    # couplings across the coarse low faces: the fine low faces of each block's first layer
    bx_low = np.zeros((nz, ny, nxc))
    bx_low[:, :, :] = op.bx[:, :, 0::fx][:, :, :nxc]
    by_low = np.zeros((nz, nyc, nx))
    by_low[:, :, :] = op.by[:, 0::fy, :][:, :nyc, :]
    bz_low = np.zeros((nzc, ny, nx))
    bz_low[:, :, :] = op.bz[0::fz, :, :][:nzc]
    BX = _block_sum(bx_low, (1, fy, fz), nc)
    BY = _block_sum(by_low, (fx, 1, fz), nc)
    BZ = _block_sum(bz_low, (fx, fy, 1), nc)
    # couplings inside a block: the low faces of its second layer (when the axis is coarsened)
    inner = np.zeros(op.shape)
    if fx == 2:
        m = np.zeros(nx, bool)
        m[1::2] = True
        inner += np.where(m[None, None, :], op.bx, 0.0)
    if fy == 2:
        m = np.zeros(ny, bool)
        m[1::2] = True
        inner += np.where(m[None, :, None], op.by, 0.0)
    if fz == 2:
        m = np.zeros(nz, bool)
        m[1::2] = True
        inner += np.where(m[:, None, None], op.bz, 0.0)
    D = _block_sum(op.diag, f, nc) - 2.0 * _block_sum(inner, f, nc)
    walls = op.walls & PERIODIC_X
    return Operator(nxc, nyc, nzc, BX, BY, BZ, D, walls)


def hierarchy(op: Operator, coarse_max=COARSE_MAX):
    """The levels of the V-cycle, finest first."""
    levels = []
    cur = op
    while True:
        nz, ny, nx = cur.shape
        f = factors(nx, ny, nz, bool(cur.walls & PERIODIC_X))
        if (levels and nx * ny * nz <= coarse_max) or f == (1, 1, 1):
            levels.append(Level(cur, None))
            return levels
        levels.append(Level(cur, f))
        cur = galerkin(cur, f)


def restrict(r, f, nc):
    """``P^T r``: the sum over each aggregate."""
    return _block_sum(r, f, nc)


def prolong(e, f, shape):
    """``P e``: every cell takes its aggregate's value."""
    fx, fy, fz = f
    up = np.repeat(np.repeat(np.repeat(e, fz, axis=0), fy, axis=1), fx, axis=2)
    return up[:shape[0], :shape[1], :shape[2]]


def vcycle(levels, r, l=0, omega=OMEGA, alpha=ALPHA, coarse_sweeps=COARSE_SWEEPS):
    """``y = V_l(r)`` (see the module docstring)."""
    lev = levels[l]
    op = lev.op
    D = op.diag
    x = omega * r / D
    if lev.f is None:
        for _ in range(coarse_sweeps - 1):
            x = x + omega * (r - apply(op, x)) / D
        return x
    nxt = levels[l + 1].op
    rc = restrict(r - apply(op, x), lev.f, nxt.shape)
    e = vcycle(levels, rc, l + 1, omega, alpha, coarse_sweeps)
    x = x + alpha * prolong(e, lev.f, op.shape)
    return x + omega * (r - apply(op, x)) / D


def pcg_mg(op: Operator, b, x0=None, tol=1e-12, max_iters=10000, levels=None, **kw):
    """PCG with the V-cycle preconditioner (the oracle's PCG steps, Jacobi replaced by
    ``z = V_0(r)``); stops when ``|b - A x| <= tol |b|`` on the recurrence residual.  Returns a
    PCGResult with the true relative residual."""
    from . import PCGResult, OK, ENOTCONV
    levels = levels or hierarchy(op)
    b = np.asarray(b, dtype=np.float64).reshape(op.shape)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(op.shape)
    r = b - apply(op, x)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return PCGResult(np.zeros_like(b), 0, 0.0, OK)
    z = vcycle(levels, r, **kw)
    p = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    while np.linalg.norm(r) > tol * bn and it < max_iters:
        q = apply(op, p)
        a = rz / float(np.sum(p * q))
        x = x + a * p
        r = r - a * q
        it += 1
        if np.linalg.norm(r) <= tol * bn:
            break
        z = vcycle(levels, r, **kw)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    rel = float(np.linalg.norm(b - apply(op, x))) / bn
    return PCGResult(x, it, rel, OK if rel <= 10 * tol else ENOTCONV)
