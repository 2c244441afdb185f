"""CPU cross-check of the rearranged CG that the one-sweep kernels run.

The paper solves the pressure equation by preconditioned conjugate gradients (Introduction); the
oracle holds that textbook PCG.  The library's one-sweep kernels run the Chronopoulos-Gear
rearrangement of Jacobi PCG (both inner products of an iteration from one reduction).  This file
restates those recurrences in numpy, in the kernels' variables, and checks that they are a
rearrangement and nothing else: the same iterates as the oracle's textbook Jacobi PCG at every k,
and the dense direct solution at convergence.  It is test code, not part of the oracle, and no
GPU test compares against it: the GPU tests take the oracle's textbook PCG as the reference.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle

RHO_A, RHO_W = 1.0, 1000.0


def cg_single_reduction(op, b, tol=1e-12, max_iters=100000):
    """Jacobi PCG (M = D) as the Chronopoulos-Gear recurrences, zero start:

        u = M^-1 r,  s^ = M^-1 A p,  w^ = M^-1 A u
        p = u + beta p;  s^ = w^ + beta s^;  x += alpha p;  u = u - alpha s^;  w^ = M^-1 A u
        gamma = (D u, u);  delta = (A u, u);  |r|^2 = |D u|^2
        beta = gamma / gamma_old;  alpha = gamma / (delta - beta gamma / alpha_old)

    Stops when |r| <= tol |r_0| (tol <= 0: exactly max_iters iterations).  Returns (x, iters)."""
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(op.shape)
    D = op.diag
    x = np.zeros_like(b)
    u = b / D
    Au = oracle.apply(op, u)
    w = Au / D
    gamma = float(np.sum(D * u * u))
    delta = float(np.sum(Au * u))
    rr0 = float(np.sum((D * u) ** 2))
    stop2 = (tol * tol) * rr0 if tol > 0 else -1.0
    if rr0 == 0.0:
        return x, 0
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    alpha, beta = gamma / delta, 0.0
    it = 0
    while it < max_iters:
        p = u + beta * p
        s = w + beta * s
        x = x + alpha * p
        u = u - alpha * s
        Au = oracle.apply(op, u)
        w = Au / D
        g_new = float(np.sum(D * u * u))
        delta = float(np.sum(Au * u))
        rr = float(np.sum((D * u) ** 2))
        it += 1
        if rr <= stop2:
            break
        beta = g_new / gamma
        alpha = g_new / (delta - beta * g_new / alpha)
        gamma = g_new
    return x, it


def _rand_F(shape, seed, sharp=False):
    rng = np.random.default_rng(seed)
    if sharp:
        return (rng.random(shape) < 0.5).astype(np.float64)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


def _dense(op):
    n = op.nx * op.ny * op.nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = oracle.apply(op, e).ravel()
        e[j] = 0.0
    return A


@pytest.mark.parametrize("shape,sharp", [((4, 4, 4), False), ((5, 5, 5), True), ((3, 5, 4), True)])
def test_single_reduction_cg_matches_dense_lu(shape, sharp):
    op = oracle.operator(_rand_F(shape, 13, sharp), RHO_A, RHO_W)
    b = np.random.default_rng(14).standard_normal(shape)
    ref = scipy.linalg.solve(_dense(op), b.ravel(), assume_a="sym").reshape(shape)
    x, _ = cg_single_reduction(op, b, tol=1e-13)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-10


def test_single_reduction_cg_has_the_iterates_of_the_oracle_pcg():
    """The same x_k as the oracle's textbook Jacobi PCG at every k (to rounding)."""
    shape = (6, 5, 7)
    op = oracle.operator(_rand_F(shape, 63), RHO_A, RHO_W)
    b = np.random.default_rng(64).standard_normal(shape)
    for it in range(1, 25):
        a1, n1 = cg_single_reduction(op, b, tol=0.0, max_iters=it)
        a2 = oracle.pcg(op, b, tol=0.0, precond="jacobi", max_iters=it).x
        assert n1 == it
        assert np.linalg.norm(a1 - a2) <= 1e-9 * np.linalg.norm(a2), it
