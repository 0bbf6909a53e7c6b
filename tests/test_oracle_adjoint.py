"""Pin of the oracle's reverse pass (kT = 0) against central finite
differences of the oracle's own forward run (FP64).

The loss is the fluid kinetic energy L = 1/2 sum |j|^2 / rho over a sub-box
after T steps (j = sum n c + f/2, Sec. 3.7); the parameters are the force
field f.  L is smooth in f, so central differences with eps = 1e-3 relative
to the field scale are accurate to O(eps^2).
"""
import numpy as np
import pytest

from paper_0803_2826_gb300 import inputs


@pytest.mark.parametrize("walls", [False, True])
def test_adjoint_matches_finite_differences(ora, walls):
    shape = (6, 5, 7)
    p = ora.make_params(shape, gamma_shear=0.2, gamma_bulk=-0.3, gamma_odd=0.4, gamma_even=-0.1,
                        body_force=(2e-4, -1e-4, 0.0 if walls else 1e-4), walls=walls)
    u = inputs.shear_wave(shape, 0.02) + inputs.gaussian_field(shape, 3, 5e-3, seed=1)
    rho = 1.0 + inputs.gaussian_field(shape, 1, 1e-2, seed=2)[0]
    if walls:
        u[:, 0] = u[:, -1] = 0
    pops0 = ora.equilibrium(p, rho, u)
    f = inputs.gaussian_field(shape, 3, 1e-3, seed=3)
    if walls:
        f[:, 0] = f[:, -1] = 0
    lo, hi, T = (1, 1, 2), (5, 4, 6), 6
    L, g = ora.kinetic_energy_and_grad(p, pops0, f, T, lo, hi)
    assert np.isclose(L, ora.kinetic_energy(p, pops0, f, T, lo, hi), rtol=1e-13)
    rng = np.random.default_rng(4)
    zr = range(1, shape[2] - 1) if walls else range(shape[2])
    for _ in range(16):
        c, z, y, x = rng.integers(0, 3), rng.choice(list(zr)), rng.integers(0, shape[1]), rng.integers(0, shape[0])
        eps = 1e-3 * 1e-3
        fp = f.copy()
        fp[c, z, y, x] += eps
        fm = f.copy()
        fm[c, z, y, x] -= eps
        fd = (ora.kinetic_energy(p, pops0, fp, T, lo, hi) - ora.kinetic_energy(p, pops0, fm, T, lo, hi)) / (2 * eps)
        assert np.isclose(g[c, z, y, x], fd, rtol=1e-6, atol=1e-12 * abs(L) / 1e-3), (g[c, z, y, x], fd)


def test_adjoint_linear_in_lambda_and_transposes_step(ora):
    """<lam, J v> = <J^T lam, v> for the one-step map (directional derivative
    by central differences in the state direction v)."""
    shape = (5, 4, 6)
    p = ora.make_params(shape, gamma_shear=0.3, gamma_odd=-0.2, body_force=(1e-3, 0, 0))
    u = inputs.gaussian_field(shape, 3, 1e-2, seed=5)
    s0 = ora.equilibrium(p, None, u)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(s0.shape) * 1e-3
    lam = rng.standard_normal(s0.shape)
    f = inputs.gaussian_field(shape, 3, 1e-3, seed=7)
    h = 1e-4
    jv = (ora.step(p, s0 + h * v, f) - ora.step(p, s0 - h * v, f)) / (2 * h)
    jt, _ = ora.adjoint_step(p, s0, lam, f)
    assert np.isclose(np.sum(lam * jv), np.sum(jt * v), rtol=1e-8)


def test_checkpointed_reverse_pass_is_identical(ora):
    shape = (5, 6, 4)
    p = ora.make_params(shape, gamma_shear=0.1)
    f = inputs.gaussian_field(shape, 3, 1e-3, seed=9)
    s0 = ora.equilibrium(p, None, inputs.gaussian_field(shape, 3, 1e-2, seed=8))
    L1, g1 = ora.kinetic_energy_and_grad(p, s0, f, 7, (0, 0, 0), (5, 6, 4))
    L2, g2 = ora.kinetic_energy_and_grad(p, s0, f, 7, (0, 0, 0), (5, 6, 4), checkpoint_every=3)
    assert L1 == L2 and np.array_equal(g1, g2)


def _coupled_case(ora, walls):
    from paper_0803_2826_gb300 import inputs
    shape = (8, 7, 8)
    p = ora.make_params(shape, kT=0.0, walls=walls)
    rng = np.random.default_rng(11)
    force = rng.normal(0.0, 1e-4, size=(3, 8, 7, 8))
    u = inputs.shear_wave(shape, 0.02) + inputs.gaussian_field(shape, 3, 2e-3, seed=12)
    if walls:
        u[:, 0] = 0
        u[:, -1] = 0
        force[:, 0] = 0
        force[:, -1] = 0
    pops0 = ora.equilibrium(p, None, u)
    n = 5
    pos0 = rng.uniform(0.0, 1.0, (n, 3)) * np.array(shape, dtype=float)
    mom0 = rng.normal(0.0, 0.02, (n, 3))
    if walls:  # three particles heading into the walls, so that they reflect
        pos0[:, 2] = rng.uniform(1.2, 5.8, n)
        pos0[0, 2], mom0[0, 2] = 1.02, -0.3
        pos0[1, 2], mom0[1, 2] = 5.97, 0.35
        pos0[2, 2], mom0[2, 2] = 1.05, -0.2
    kw = dict(dt=0.1, n_substeps=5, nsteps=4, lo=(1, 1, 1), hi=(7, 6, 7))
    return p, pops0, force, pos0, mom0, kw


@pytest.mark.parametrize("walls", [False, True])
def test_coupled_reverse_pass_matches_central_differences(ora, walls):
    """Reverse of (couple free particles at kT = 0, then step) x 4 against
    central differences of the forward loss in the force field, the initial
    positions and the initial momenta (Sec. 4.5 with Eqs. Delta, 2point)."""
    p, pops0, force, pos0, mom0, kw = _coupled_case(ora, walls)
    L, g, lpos, lmom = ora.coupled_kinetic_energy_and_grad(p, pops0, force, pos0, mom0, 1.0, 2.0, **kw)
    assert L == pytest.approx(ora.coupled_kinetic_energy(p, pops0, force, pos0, mom0, 1.0, 2.0, **kw), rel=1e-13)

    def fd(fun, x, idx, eps):
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        return (fun(xp) - fun(xm)) / (2 * eps)

    for idx in [(0, 2, 3, 4), (1, 3, 1, 1), (2, 5, 6, 7)]:
        d = fd(lambda F: ora.coupled_kinetic_energy(p, pops0, F, pos0, mom0, 1.0, 2.0, **kw), force, idx, 1e-4)
        assert g[idx] == pytest.approx(d, rel=1e-5, abs=1e-9)
    for idx in [(0, 0), (1, 2), (2, 2), (3, 1)]:
        d = fd(lambda P: ora.coupled_kinetic_energy(p, pops0, force, P, mom0, 1.0, 2.0, **kw), pos0, idx, 1e-6)
        assert lpos[idx] == pytest.approx(d, rel=1e-4, abs=1e-10)
    for idx in [(0, 2), (1, 2), (4, 1)]:
        d = fd(lambda M: ora.coupled_kinetic_energy(p, pops0, force, pos0, M, 1.0, 2.0, **kw), mom0, idx, 1e-5)
        assert lmom[idx] == pytest.approx(d, rel=1e-4, abs=1e-10)


def test_coupled_reverse_without_particles_is_the_lb_reverse(ora):
    """With no particles the coupled reverse pass is the plain one."""
    p, pops0, force, pos0, mom0, kw = _coupled_case(ora, False)
    L, g, _, _ = ora.coupled_kinetic_energy_and_grad(p, pops0, force, pos0[:0], mom0[:0], 1.0, 2.0, **kw)
    L2, g2 = ora.kinetic_energy_and_grad(p, pops0, force, kw["nsteps"], kw["lo"], kw["hi"])
    assert L == pytest.approx(L2, rel=1e-14)
    assert np.allclose(g, g2, rtol=1e-12, atol=1e-18)
