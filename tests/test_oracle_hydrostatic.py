"""Pins of the oracle's reduced-pressure force (Entrance and Exit Boundary Conditions,
hydrostatic-pressure method) against what the formulation fixes, not against its own formula.

* Substituting P = P_r + rho g (z - z_o) into the face-centred pressure gradient plus gravity,
  beta_f grad_h P - g e_z, must leave exactly beta_f grad_h P_r minus the force: on every interior
  face the force equals -beta_f (Psi_n - Psi_c)/h + g [z face], Psi = rho g (z - z_o).  The
  identity holds only with the harmonic-mean face coefficient and the face heights of the
  reading, so it fixes both, and the sign.
* Boundary faces carry no force; the periodic wrap face carries the same force on faces 0 and nx.
* Hydrostatic rest: for a layered density F(z) and no flow, adding the force, solving for P_r and
  projecting must leave no velocity, and P_r must be the column that jumps by
  (z_f - z_o) g (rho_above - rho_below) across every face (the paper's jump condition), with
  P_r = 0 in the top layer (p = 0 on the top face, no force there).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle

RHO_A, RHO_W = 1.0, 1000.0
G = -9.81      # the coefficient as the paper writes it
Z_O = 0.43


def _rand_F(shape, seed):
    rng = np.random.default_rng(seed)
    F = rng.random(shape)
    F[rng.random(shape) < 0.3] = 0.0
    F[rng.random(shape) < 0.3] = 1.0
    return F


def _zeros_faces(nz, ny, nx):
    return np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))


def _force(F, h, walls=0, g=G, z_o=Z_O):
    nz, ny, nx = F.shape
    return oracle.hydrostatic_force(F, *_zeros_faces(nz, ny, nx), h, g, z_o, dt=1.0,
                                    walls=walls)


@pytest.mark.parametrize("shape,walls", [((5, 6, 7), 0), ((9, 3, 4), 0), ((6, 5, 8), oracle.PERIODIC_X)])
def test_force_is_the_reduced_form_of_face_gravity(shape, walls):
    nz, ny, nx = shape
    h = 1.0 / nz
    F = _rand_F(shape, 3 + nx)
    op = oracle.operator(F, RHO_A, RHO_W, walls=walls)   # beta_f: the operator's own faces
    fu, fv, fw = _force(F, h, walls)
    rho = RHO_A + F * (RHO_W - RHO_A)
    zc = (np.arange(nz) + 0.5) * h
    psi = rho * G * (zc[:, None, None] - Z_O)
    atol = 1e-12 * np.abs(psi).max() / h
    # x faces i >= 1 (the low face of cell i), and the wrap face when periodic
    ex = -op.bx[:, :, 1:] * (psi[:, :, 1:] - psi[:, :, :-1]) / h
    assert np.allclose(fu[:, :, 1:nx], ex, rtol=0, atol=atol)
    if walls & oracle.PERIODIC_X:
        ew = -op.bx[:, :, 0] * (psi[:, :, 0] - psi[:, :, -1]) / h
        assert np.allclose(fu[:, :, 0], ew, rtol=0, atol=atol)
        assert np.array_equal(fu[:, :, 0], fu[:, :, nx])
        assert np.abs(fu[:, :, 0]).max() > 0
    ey = -op.by[:, 1:, :] * (psi[:, 1:, :] - psi[:, :-1, :]) / h
    assert np.allclose(fv[:, 1:ny, :], ey, rtol=0, atol=atol)
    ez = -op.bz[1:] * (psi[1:] - psi[:-1]) / h + G
    assert np.allclose(fw[1:nz], ez, rtol=0, atol=atol)
    assert np.abs(fw[1:nz]).max() > 1.0  # the case does exercise the force


@pytest.mark.parametrize("walls", [0, 31])
def test_boundary_faces_carry_no_force(walls):
    shape = (6, 5, 7)
    F = _rand_F(shape, 11)
    fu, fv, fw = _force(F, 1.0 / 6, walls)
    for a in (fu[:, :, 0], fu[:, :, -1], fv[:, 0, :], fv[:, -1, :], fw[0], fw[-1]):
        assert not a.any()


def test_no_force_without_gravity_or_a_density_change():
    shape = (4, 5, 6)
    u0 = [np.random.default_rng(s).standard_normal(a.shape) for s, a in
          enumerate(_zeros_faces(*shape))]
    F = _rand_F(shape, 2)
    for FF, g in ((F, 0.0), (np.full(shape, 0.7), G)):
        out = oracle.hydrostatic_force(FF, *u0, 0.25, g, Z_O, dt=0.1)
        for a, b in zip(out, u0):
            assert np.array_equal(a, b)


def _dense(op):
    n = op.nx * op.ny * op.nz
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = oracle.apply(op, e).ravel()
        e[j] = 0.0
    return A


@pytest.mark.parametrize("z_s", [0.43, 0.6])
def test_hydrostatic_rest_of_a_layered_column(z_s):
    """Surface at z_s (at the static level z_o or above it), mollified over 1.5 cells."""
    nx, ny, nz = 4, 3, 24
    h = 1.0 / nz
    zc = (np.arange(nz) + 0.5) * h
    eps = 1.5 * h
    d = z_s - zc
    Fz = np.where(d > eps, 1.0, np.where(d < -eps, 0.0,
                                         0.5 * (1 + d / eps + np.sin(np.pi * d / eps) / np.pi)))
    F = np.broadcast_to(Fz[:, None, None], (nz, ny, nx)).copy()
    dt = 1e-3
    u1, v1, w1 = oracle.hydrostatic_force(F, *_zeros_faces(nz, ny, nx), h, G, Z_O, dt=dt)
    s = oracle.divergence(u1, v1, w1, h, dt)
    op = oracle.operator(F, RHO_A, RHO_W)
    b = oracle.rhs(s, h)
    x = scipy.linalg.solve(_dense(op), b.ravel(), assume_a="sym").reshape(F.shape)
    # the closed-form column: P_r = 0 in the top layer, jumps across every face
    rho = RHO_A + Fz * (RHO_W - RHO_A)
    col = np.zeros(nz)
    for k in range(nz - 1, 0, -1):
        col[k - 1] = col[k] + (k * h - Z_O) * G * (rho[k] - rho[k - 1])
    assert np.abs(col).max() > 1e-3
    assert np.abs(x - col[:, None, None]).max() <= 1e-9 * np.abs(col).max()
    u2, v2, w2 = oracle.project(op, F, u1, v1, w1, x, h, dt, RHO_A, RHO_W)
    ref = np.abs(w1).max()
    assert ref > 0
    for a in (u2, v2, w2):
        assert np.abs(a).max() <= 1e-9 * ref
