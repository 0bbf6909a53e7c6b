"""Pins of the oracle's extended particles (solid spheres with moving link
bounce-back, Sec. 4.1-4.2).

- Eq. (EOMUsol) and the U~ equation: for m dU/dt = -zeta U + F with a
  symmetric matrix zeta the update equals expm(-zeta h / m) U +
  zeta^-1 (1 - expm(-zeta h / m)) F (scipy's matrix exponential), and
  m (U(t+h) - U(t)) = F - zeta U~, the momentum balance that makes the
  coupling conservative.
- Sec. 4.1: the combined momentum of fluid and spheres is conserved by the
  moving bounce-back, also while moving spheres cover and uncover nodes.
- Eq. (MBB): a sphere whose surface moves with the velocity of a uniform
  fluid at equilibrium leaves that state unchanged (the returned population
  is exactly the equilibrium one): Galilean invariance of the rule.
- With rotation (Eq. NodeVel, u_b = U + Omega x (r_b - R)): the 6 x 6
  update equals the matrix exponential of M^-1 Z (scipy), linear momentum
  is still conserved while rotating spheres move, a spinning sphere at a
  lattice-symmetric position exerts no net force, and the steady torque on a
  sphere held spinning is within a few per cent of Stokes' 8 pi eta a^3
  Omega (0.954 for a = 4; the staircase surface of the discrete sphere is a
  little smaller than the sphere of radius a).
- Sec. 4.1: the drag of a periodic array of fixed spheres agrees with the
  Hasimoto / Sangani-Acrivos series for a simple cubic array within a few
  per cent (the paper reports ~1 % for larger spheres with kinetic
  eigenvalues tied to the viscosity); here with the two-rate relation
  (tau_e - 1/2)(tau_o - 1/2) = 3/16.
"""
import numpy as np
import pytest

from paper_0803_2826_gb300 import inputs


def test_velocity_update_is_the_matrix_exponential(ora):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(0)
    for m in (0.5, 2.0, 50.0):
        A = rng.normal(size=(3, 3))
        Z = A @ A.T + 0.3 * np.eye(3)
        U, F = rng.normal(size=3), rng.normal(size=3)
        un, ut = ora.sphere_velocity(Z, m, U, F)
        E = scipy_linalg.expm(-Z / m)
        want = E @ U + np.linalg.solve(Z, (np.eye(3) - E) @ F)
        assert np.allclose(un, want, rtol=1e-12, atol=1e-14)
        assert np.allclose(m * (un - U), F - Z @ ut, rtol=1e-12, atol=1e-13)
    # a direction without links: free motion U + F/m, U~ = U + F/(2m)
    Z = np.diag([2.0, 0.0, 1.0])
    un, ut = ora.sphere_velocity(Z, 4.0, np.ones(3), np.array([0.0, 8.0, 0.0]))
    assert np.isclose(un[1], 3.0) and np.isclose(ut[1], 2.0)


def test_moving_spheres_conserve_momentum(ora):
    shape = (16, 16, 16)
    p = ora.make_params(shape, kT=1e-4, seed=3, gamma_shear=0.1)
    c, a, e, w, opp = ora.tables()
    pops = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.01))
    R = np.array([[4.3, 5.1, 6.2], [11.2, 10.7, 9.9]])
    U = np.array([[0.05, -0.03, 0.02], [-0.04, 0.02, 0.06]])
    mass = np.array([40.0, 60.0])
    rad = 2.6
    owner = ora.sphere_owner(p, R, rad)

    def total(pops, owner, U):
        fl = owner.reshape(-1) < 0
        return (pops.reshape(19, -1)[:, fl] - a[:, None]).sum(1) @ c + (mass[:, None] * U).sum(0)

    P0 = total(pops, owner, U)
    changed = 0
    for s in range(12):
        o0 = owner
        pops, owner, R, U, _, ut, st = ora.step_spheres(p, pops, owner, R, U, rad, mass, step=s)
        assert st == 0
        changed += int((o0 != owner).sum())
    assert changed > 5  # nodes were covered and uncovered
    assert np.allclose(total(pops, owner, U), P0, rtol=0, atol=1e-12)


def test_bounce_back_is_galilean(ora):
    """Fixed sphere (mass <= 0) whose surface moves with the fluid's uniform
    velocity: the equilibrium state is stationary."""
    shape = (12, 12, 12)
    p = ora.make_params(shape)
    u0 = np.array([0.03, -0.02, 0.01])
    uu = np.zeros((3,) + shape[::-1])
    for d in range(3):
        uu[d] = u0[d]
    pops = ora.equilibrium(p, None, uu)
    R = np.array([[6.2, 5.9, 6.4]])
    owner = ora.sphere_owner(p, R, 3.1)
    fl = owner < 0
    out = pops
    for s in range(5):
        out, owner, R2, U2, _, ut, st = ora.step_spheres(p, out, owner, R, u0[None], 3.1, [0.0], step=s)
    assert np.abs(out[:, fl] - pops[:, fl]).max() < 1e-15


def _hasimoto_K(c):
    """Sangani-Acrivos series for the drag of a simple cubic array of spheres
    (volume fraction c): F = 6 pi eta a U / K(c)."""
    return 1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2 + 3.9799 * c ** (8 / 3) - 3.0734 * c ** (10 / 3)


def test_fixed_sphere_array_drag(ora):
    L, rad, g = 16, 3.5, 1e-6
    te = 1.0
    go = 1.0 - 1.0 / (0.5 + (3.0 / 16.0) / (te - 0.5))
    p = ora.make_params((L, L, L), body_force=(g, 0, 0), gamma_odd=go)
    R = np.array([[L / 2 + 0.1, L / 2 + 0.2, L / 2 + 0.3]])
    owner = ora.sphere_owner(p, R, rad)
    pops = ora.equilibrium(p)
    U = np.zeros((1, 3))
    for s in range(3000):
        pops, owner, R, U, _, ut, st = ora.step_spheres(p, pops, owner, R, U, rad, [0.0], step=s)
    rho, j, _ = ora.moments(p, pops)
    fl = owner < 0
    Us = j[0][fl].sum() / L ** 3             # superficial velocity
    F = g * fl.sum()                         # steady state: drag = force on the fluid
    ratio = F / (6 * np.pi * (1 / 6) * rad * Us) * _hasimoto_K(4 / 3 * np.pi * rad ** 3 / L ** 3)
    assert abs(ratio - 1) < 0.05, ratio


def test_rotation_update_is_the_matrix_exponential(ora):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    for m, inertia in ((3.0, 0.7), (50.0, 200.0)):
        A = rng.normal(size=(6, 6))
        Z = A @ A.T + 0.2 * np.eye(6)
        V, F = rng.normal(size=6), rng.normal(size=6)
        vn, vt = ora.sphere_velocity6(Z, m, inertia, V, F)
        M = np.diag([m, m, m, inertia, inertia, inertia])
        E = scipy_linalg.expm(-np.linalg.solve(M, Z))
        want = E @ V + np.linalg.solve(Z, M @ (np.eye(6) - E) @ np.linalg.solve(M, F))
        assert np.allclose(vn, want, rtol=1e-11, atol=1e-13)
        assert np.allclose(M @ (vn - V), F - Z @ vt, rtol=1e-11, atol=1e-13)


def test_rotating_spheres_conserve_momentum(ora):
    shape = (16, 16, 16)
    p = ora.make_params(shape, gamma_shear=0.1)
    c, a, e, w, opp = ora.tables()
    pops = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.01))
    R = np.array([[4.3, 5.1, 6.2], [11.2, 10.7, 9.9]])
    U = np.array([[0.05, -0.03, 0.02], [-0.04, 0.02, 0.06]])
    Om = np.array([[0.01, -0.02, 0.015], [0.0, 0.02, -0.01]])
    mass = np.array([40.0, 60.0])
    owner = ora.sphere_owner(p, R, 2.6)

    def total(pops, owner, U):
        fl = owner.reshape(-1) < 0
        return (pops.reshape(19, -1)[:, fl] - a[:, None]).sum(1) @ c + (mass[:, None] * U).sum(0)

    P0 = total(pops, owner, U)
    Om0 = Om.copy()
    for s in range(12):
        pops, owner, R, U, Om, ut, st = ora.step_spheres(p, pops, owner, R, U, 2.6, mass, omega=Om, step=s)
        assert st == 0
    assert np.allclose(total(pops, owner, U), P0, rtol=0, atol=1e-12)
    assert np.abs(Om - Om0).max() > 1e-4  # the spheres exchanged angular momentum with the fluid


def test_spinning_sphere_torque(ora):
    go = 1.0 - 1.0 / (0.5 + (3.0 / 16.0) / 0.5)
    ratios = []
    for L, rad in ((24, 4.0),):
        p = ora.make_params((L, L, L), gamma_odd=go)
        R = np.array([[L / 2, L / 2, L / 2]])
        owner = ora.sphere_owner(p, R, rad)
        pops = ora.equilibrium(p)
        Om = np.array([[0.0, 0.0, 1e-3]])
        FT = np.zeros((1, 6))
        U = np.zeros((1, 3))
        for s in range(1200):
            pops, owner, R, U, _, ut, st = ora.step_spheres(p, pops, owner, R, U, rad, [0.0], omega=Om, step=s,
                                                          forces=FT)
        assert np.abs(FT[0, :3]).max() < 1e-14          # no net force by symmetry
        ratios.append(-FT[0, 5] / (8 * np.pi * (1 / 6) * rad ** 3 * 1e-3))
    assert all(0.9 < r < 1.05 for r in ratios), ratios
