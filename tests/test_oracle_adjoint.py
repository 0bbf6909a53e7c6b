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
