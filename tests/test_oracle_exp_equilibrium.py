"""Pins of the oracle's exponential equilibrium (Sec. 3.6, Eq.
(equildist_lagrange)) and of the collision that uses it.

- Eqs. (constraint_mass), (constraint_mom): sum n^eq = rho and sum n^eq c = j.
- Sec. 3.6: the quadratic equilibrium of Eq. (original_equil_distrib) is its
  expansion to second order in u, so the two differ by O(u^3).
- Eq. (Smax): n^eq maximises the entropy of Eq. (boltzmann_entropy_function)
  (with nu_bar_i = a_i rho) among populations with the same rho and j.
- With the exponential equilibrium in the collision, a uniform state at that
  equilibrium is a fixed point, every step conserves mass and momentum, and
  a small shear wave decays at the rate of the same viscosity (Eq.
  shearviscosity) as with the quadratic equilibrium.
"""
import numpy as np

from paper_0803_2826_gb300 import inputs


def test_constraints(ora):
    c = ora.tables()[0]
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.15, 0.15, 3)
        n = ora.exp_equilibrium(rho, u)
        assert np.all(n > 0)
        assert abs(n.sum() - rho) < 1e-14 * rho
        assert np.allclose(n @ c, rho * u, rtol=0, atol=1e-15)


def test_quadratic_form_is_the_second_order_expansion(ora):
    p = ora.make_params((1, 1, 1))
    direction = np.array([0.7, -0.4, 0.5])
    ratios = []
    for s in (1e-2, 1e-3):
        u = direction * s
        uu = np.zeros((3, 1, 1, 1))
        uu[:, 0, 0, 0] = u
        nq = ora.equilibrium(p, np.full((1, 1, 1), 1.1), uu)[:, 0, 0, 0]
        ne = ora.exp_equilibrium(1.1, u)
        ratios.append(np.abs(ne - nq).max() / s ** 3)
    assert ratios[0] > 1e-3                       # a genuine third-order difference
    assert abs(ratios[0] / ratios[1] - 1) < 0.05  # that scales as u^3


def _entropy(n, nbar):
    return -np.sum(n * np.log(n) - n - n * np.log(nbar) + nbar)


def test_maximum_entropy(ora):
    c, a, e, w, opp = ora.tables()
    rho, u = 1.05, np.array([0.08, -0.05, 0.03])
    n = ora.exp_equilibrium(rho, u)
    nbar = a * rho
    # directions that keep rho and j: the complement of span{1, c_x, c_y, c_z}
    A = np.vstack([np.ones(19), c.T])
    _, _, vt = np.linalg.svd(A)
    null = vt[4:]
    rng = np.random.default_rng(2)
    S0 = _entropy(n, nbar)
    for _ in range(50):
        d = rng.normal(size=null.shape[0]) @ null
        d *= 1e-3 / np.abs(d).max()
        assert _entropy(n + d, nbar) < S0
        assert _entropy(n - d, nbar) < S0


def test_collision_fixed_point_and_conservation(ora):
    c, a, e, w, opp = ora.tables()
    shape = (4, 3, 5)
    u0 = np.array([0.05, -0.03, 0.02])
    p = ora.make_params(shape, gamma_shear=0.3, gamma_bulk=-0.2, gamma_odd=0.4, gamma_even=-0.1, equilibrium=1)
    ne = ora.exp_equilibrium(1.02, u0)
    pops = np.repeat(ne[:, None], np.prod(shape), axis=1).reshape((19,) + shape[::-1])
    out = ora.step(p, pops)
    assert np.abs(out - pops).max() < 1e-15
    # a thermal, forced state: mass and momentum per step
    p = ora.make_params(shape, kT=1e-4, seed=4, gamma_shear=0.1, body_force=(1e-4, 0, -2e-4), equilibrium=1)
    pops = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.03))
    for t in range(3):
        out = ora.step(p, pops, None, t)
        assert abs(out.sum() - pops.sum()) < 1e-13 * pops.sum()
        dj = (out.reshape(19, -1).sum(1) - pops.reshape(19, -1).sum(1)) @ c
        assert np.allclose(dj, np.array([1e-4, 0, -2e-4]) * np.prod(shape), rtol=0, atol=1e-13)
        pops = out


def test_shear_wave_viscosity_unchanged(ora):
    L = 64
    rates = []
    for eq in (0, 1):
        p = ora.make_params((1, 1, L), gamma_shear=0.2, gamma_bulk=0.2, equilibrium=eq)
        pops = ora.equilibrium(p, None, inputs.shear_wave((1, 1, L), 1e-4))
        s = np.sin(2 * np.pi * np.arange(L) / L)

        def amp(pp):
            rho, j, _ = ora.moments(p, pp)
            return 2.0 / L * np.sum(j[0, :, 0, 0] / rho[:, 0, 0] * s)

        pops = ora.run(p, pops, 20)
        a0 = amp(pops)
        pops = ora.run(p, pops, 200, step0=20)
        rates.append(-np.log(amp(pops) / a0) / 200)
    assert abs(rates[1] / rates[0] - 1) < 1e-6
