"""Pins of the oracle's particle side against what the paper fixes.

- Sec. 4.6 Eqs. (DnormDiscrete), (C1), (C2): the stencils of phi_2, phi_3
  and phi_4 sum to one and reproduce the particle position exactly; the
  product form of Eq. (Delta) interpolates any linear velocity field exactly,
  and the coupling interpolates u, not j (Sec. 4.5).  Eq. (C3): sum phi^2 is
  1/2 for phi_3 and 3/8 for phi_4 wherever the particle is; phi_3 has a
  continuous first derivative.
- Sec. 4.5: total particle + fluid momentum is conserved by the coupling plus
  the following LB step (pair forces, uniform Gamma/m).
- Eq. (langevin_momentum_update) is the exact Ornstein-Uhlenbeck solution:
  stationary <p^2>/(3m) = kT and <p/m> = u for a frozen uniform fluid.
- Sec. 4.5: the three-point noise has the Gaussian moments to fourth order.
- Sec. 2.1 Eqs. (ulennardjones), (ufene): forces are minus the gradient of the
  potentials, vanish at the WCA cut-off, and sum to zero (pair forces).
"""
import numpy as np
import pytest

from paper_0803_2826_gb300 import inputs


@pytest.mark.parametrize("kernel", [2, 3, 4])
def test_stencil_moment_conditions(ora, kernel):
    """Eqs. C1, C2 for the 3-d stencil of phi_2, phi_3, phi_4: weights sum to
    1 and their first moments give the position (unwrapped node coordinates)."""
    p = ora.make_params((8, 9, 10))
    rng = np.random.default_rng(0)
    K = kernel
    for _ in range(50):
        r = rng.uniform(0, 1, 3) * np.array([8, 9, 10])
        node, wt = ora.stencil(p, r, kernel)
        assert len(wt) == K ** 3
        assert np.isclose(wt.sum(), 1.0, rtol=0, atol=1e-14)
        assert np.all(wt >= 0)
        b = np.floor(r + 0.5) - 1 if K == 3 else (np.floor(r) - 1 if K == 4 else np.floor(r))
        q = 0
        acc = np.zeros(3)
        for dz in range(K):
            for dy in range(K):
                for dx in range(K):
                    acc += wt[q] * (b + np.array([dx, dy, dz]))
                    q += 1
        assert np.allclose(acc, r, rtol=0, atol=1e-13)


@pytest.mark.parametrize("kernel,C", [(3, 0.5), (4, 0.375)])
def test_phi_moment_conditions(ora, kernel, C):
    """Eqs. C1-C3 in one dimension for phi_3 (Eq. 3point) and phi_4 (Eq.
    4point): sum phi = 1, sum j phi = u and sum phi^2 = C independent of u
    (1/2 and 3/8); phi_2 satisfies C1, C2 but not C3."""
    us = np.linspace(-3.0, 3.0, 611) + 1e-3
    js = np.arange(-8, 9)
    for u in us:
        ph = np.array([ora.phi(kernel, u - j) for j in js])
        assert abs(ph.sum() - 1.0) < 1e-14
        assert abs((js * ph).sum() - u) < 1e-13
        assert abs((ph * ph).sum() - C) < 1e-14
    s2 = [sum(ora.phi(2, u - j) ** 2 for j in js) for u in us]
    assert max(s2) - min(s2) > 0.4  # 1/2 .. 1


def test_phi3_first_derivative_continuous(ora):
    """phi_3 has a continuous first derivative (Sec. 4.6), also at the
    branch points |u| = 1/2 and 3/2; phi_2 has a jump at 0."""
    h = 1e-7
    for b in (-1.5, -0.5, 0.5, 1.5):
        left = (ora.phi(3, b) - ora.phi(3, b - h)) / h
        right = (ora.phi(3, b + h) - ora.phi(3, b)) / h
        assert abs(left - right) < 1e-4, (b, left, right)
    left = (ora.phi(2, 0.0) - ora.phi(2, -h)) / h
    right = (ora.phi(2, h) - ora.phi(2, 0.0)) / h
    assert abs(left - right) > 1.9


def test_interpolates_linear_u_not_j(ora):
    """Nodes carry u(r) = U0 + G r (linear) and a non-uniform rho; in the
    interior the interpolated velocity equals U0 + G r_p exactly."""
    shape = (12, 12, 12)
    p = ora.make_params(shape)
    z, y, x = np.meshgrid(np.arange(12), np.arange(12), np.arange(12), indexing="ij")
    G = np.array([[1e-4, 2e-4, -1e-4], [0, -2e-4, 3e-4], [1e-4, 0, 2e-4]])
    U0 = np.array([0.01, -0.005, 0.002])
    u = np.stack([U0[a] + G[a, 0] * x + G[a, 1] * y + G[a, 2] * z for a in range(3)])
    rho = 1.0 + 0.05 * np.sin(x + 2 * y) * np.cos(z)
    # stored state = post-collision; make the pre-collision (pulled) state the
    # equilibrium by inverting the pull on the equilibrium field
    c, a, e, w, opp = ora.tables()
    neq = ora.equilibrium(p, rho, u)
    pops = np.empty_like(neq)
    for i in range(19):
        pops[i] = np.roll(neq[i], shift=(-c[i][2], -c[i][1], -c[i][0]), axis=(0, 1, 2))
    rr, jj, _ = ora.moments(p, pops)
    assert np.allclose(jj / rr, u, rtol=1e-12, atol=1e-16)
    pos = inputs.uniform_particles(40, (1, 1, 1), seed=1) * 6 + 3  # interior
    for kernel in (2, 3, 4):  # Eq. C2 makes every kernel exact for a linear field
        up = ora.interpolate(p, pops, pos, kernel=kernel)
        want = U0[None, :] + pos @ G.T
        assert np.allclose(up, want, rtol=1e-12, atol=1e-15)
        # interpolating j and dividing by interpolated rho would not be exact
        assert np.abs(up - want).max() < 1e-14


@pytest.mark.parametrize("kernel", [2, 3, 4])
def test_momentum_conservation_coupled(ora, kernel):
    """Sigma p + fluid momentum is unchanged by couple() followed by the LB
    step that applies the spread impulses (FP64 <= 1e-12 relative), for each
    interpolation function (Eq. C1)."""
    shape = (10, 10, 10)
    kT = 1e-4
    p = ora.make_params(shape, kT=kT, seed=1)
    c, a, e, w, opp = ora.tables()
    u = inputs.shear_wave(shape, 0.01)
    pops = ora.equilibrium(p, None, u)
    pos = inputs.random_walk_chains(2, 12, shape, seed=3)
    mom = inputs.maxwell_momenta(pos.shape[0], 1.0, kT, seed=4)
    md = ora.make_md(2, 12, eps=0.01, k_fene=0.3)
    fluid0 = pops.reshape(19, -1).sum(1) @ c
    P0 = mom.sum(0) + fluid0
    pos1, mom1, facc, broken = ora.couple(p, pops, pos, mom, 1.0, 2.0, dt=0.1, n_substeps=10,
                                          seed=9, md=md, kernel=kernel)
    assert broken == 0
    # impulse bookkeeping: particles + accumulator conserved
    assert np.allclose(mom1.sum(0) + facc.reshape(3, -1).sum(1), mom.sum(0), rtol=0, atol=1e-14)
    out = ora.step(p, pops, facc, 0)
    P1 = mom1.sum(0) + out.reshape(19, -1).sum(1) @ c
    assert np.allclose(P1, P0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kernel", [2, 3, 4])
def test_wall_band_keeps_stencil_off_solid_planes(ora, kernel):
    """With walls, positions reflect into z in [K/2, nz-1-K/2] (a project
    reading) so that the K-node stencil of phi_K never reaches a solid plane:
    no impulse lands on z = 0 or nz-1, and the impulses still sum to the
    momentum the particles gave up (Eq. C1)."""
    shape = (8, 8, 10)
    p = ora.make_params(shape, walls=True)
    u = inputs.shear_wave(shape, 0.02)
    pops = ora.equilibrium(p, None, u)
    rng = np.random.default_rng(5)
    n = 60
    pos = np.column_stack([rng.uniform(0, 8, n), rng.uniform(0, 8, n), rng.uniform(1.0, 8.0, n)])
    mom = rng.normal(0, 0.5, (n, 3))
    mom[:, 2] = np.where(pos[:, 2] < 4.5, -1.5, 1.5)  # drive them towards the walls
    pos1, mom1, facc, _ = ora.couple(p, pops, pos, mom, 1.0, 0.5, dt=0.2, n_substeps=4, seed=2,
                                     kernel=kernel)
    b = kernel / 2.0
    assert np.all(pos1[:, 2] >= b) and np.all(pos1[:, 2] <= shape[2] - 1 - b)
    assert np.all(facc[:, 0] == 0.0) and np.all(facc[:, -1] == 0.0)
    assert np.abs(facc).max() > 0
    # reflections flip p_z, so only x and y of the impulse balance are checked
    assert np.allclose(mom1.sum(0)[:2] + facc.reshape(3, -1).sum(1)[:2], mom.sum(0)[:2], rtol=0, atol=1e-13)


def test_ou_update_stationary(ora):
    """Frozen uniform fluid with velocity U, no conservative forces: the exact
    OU momentum update gives <p/m> -> U and <(p - mU)^2>/(3m) -> kT."""
    shape = (4, 4, 4)
    kT, m, G = 1e-4, 2.0, 3.0
    U = np.array([0.01, -0.02, 0.005])
    p = ora.make_params(shape, kT=kT, seed=2)
    uu = np.zeros((3,) + shape[::-1])
    for d in range(3):
        uu[d] = U[d]
    c, a, e, w, opp = ora.tables()
    neq = ora.equilibrium(p, None, uu)
    pos = inputs.uniform_particles(2000, shape, seed=5)
    mom = np.zeros_like(pos)
    pos1, mom1, facc, _ = ora.couple(p, neq, pos, mom, m, G, dt=0.5, n_substeps=40, seed=6)
    v = mom1 / m
    assert np.allclose(v.mean(0), U, atol=4 * np.sqrt(kT / m / 2000))
    T = ((mom1 - m * U) ** 2).mean() / m
    assert abs(T / kT - 1) < 0.05


def test_three_point_noise_moments(ora):
    """P(theta) = 2/3 delta(0) + 1/6 delta(+-sqrt 3): mean 0, <theta^2> = 1,
    <theta^4> = 3, and the same stationary temperature as the Gaussian."""
    shape = (4, 4, 4)
    kT, m, G = 1e-4, 1.0, 2.0
    p = ora.make_params(shape, kT=kT, seed=2)
    pops = ora.equilibrium(p)
    pos = inputs.uniform_particles(3000, shape, seed=8)
    mom = np.zeros_like(pos)
    _, mom1, _, _ = ora.couple(p, pops, pos, mom, m, G, dt=0.2, n_substeps=1, seed=3,
                               noise_kind=1)
    C1 = np.exp(-G * 0.2 / m)
    C3 = np.sqrt(m * kT * (1 - C1 ** 2))
    th = mom1 / C3
    vals = np.unique(np.round(th, 9))
    assert set(vals.tolist()) <= {round(-np.sqrt(3), 9), 0.0, round(np.sqrt(3), 9)}
    assert abs(th.mean()) < 0.03
    assert abs((th ** 2).mean() - 1) < 0.03
    assert abs((th ** 4).mean() - 3) < 0.1
    _, mom2, _, _ = ora.couple(p, pops, pos, mom, m, G, dt=0.2, n_substeps=60, seed=4,
                               noise_kind=1)
    assert abs((mom2 ** 2).mean() / (m * kT) - 1) < 0.06


def _energy(pos, L, eps, sigma, k, r0, chain_len):
    n = pos.shape[0]
    E = 0.0
    rc = 2 ** (1 / 6) * sigma
    for i in range(n):
        for j in range(i + 1, n):
            d = pos[i] - pos[j]
            d -= L * np.round(d / L)
            r = np.sqrt(d @ d)
            if r < rc:
                E += 4 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6 + 0.25)
            if j == i + 1 and i // chain_len == j // chain_len:
                E += -0.5 * k * r0 ** 2 * np.log(1 - (r / r0) ** 2)
    return E


def test_md_forces_are_gradients(ora):
    L = 8.0
    p = ora.make_params((8, 8, 8))
    pos = inputs.random_walk_chains(2, 6, (8, 8, 8), bond=0.97, min_dist=0.9, seed=2)
    md = ora.make_md(2, 6, eps=1.0, sigma=1.0, k_fene=30.0, r0=1.5)
    F, broken = ora.md_forces(p, md, pos)
    assert broken == 0
    assert np.allclose(F.sum(0), 0, atol=1e-10)
    h = 1e-6
    for i in range(pos.shape[0]):
        for a in range(3):
            pp = pos.copy()
            pp[i, a] += h
            em = pos.copy()
            em[i, a] -= h
            g = (_energy(pp, L, 1.0, 1.0, 30.0, 1.5, 6) - _energy(em, L, 1.0, 1.0, 30.0, 1.5, 6)) / (2 * h)
            assert np.isclose(F[i, a], -g, rtol=1e-5, atol=1e-5)


def test_wca_cutoff_and_fene_limits(ora):
    p = ora.make_params((10, 10, 10))
    md = ora.make_md(1, 2, eps=1.0, sigma=1.0, k_fene=30.0, r0=1.5, use_wca=True)
    rc = 2 ** (1 / 6)
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + rc * (1 - 1e-12), 5.0, 5.0]])
    F, _ = ora.md_forces(p, md, pos)
    fene = 30.0 * rc / (1 - rc ** 2 / 2.25)  # attraction only, WCA ~ 0 at r_c
    assert np.isclose(F[0, 0], fene, rtol=1e-6)
    pos = np.array([[5.0, 5.0, 5.0], [6.6, 5.0, 5.0]])  # bond beyond R0
    F, broken = ora.md_forces(p, md, pos)
    assert broken == 2  # counted once from each end


def test_particles_thermalise_with_the_fluid_at_weak_friction(ora):
    """Sec. 4.5: the coupled fluid-particle system satisfies the
    fluctuation-dissipation theorem, so free particles in a thermal fluid
    reach <p^2>/(3m) = kT.  At weak friction (Gamma mu_inf ~ 0.06) the
    discrete scheme (fluid frozen over the LB step, u without the particles'
    own half force) gives kT to a few per cent; the temperature at stronger
    friction is a measured property of the scheme, not a pin."""
    shape, kT, n = (8, 8, 8), 1e-3, 200
    p = ora.make_params(shape, kT=kT, seed=1)
    pops = ora.equilibrium(p)
    pos = inputs.uniform_particles(n, shape, seed=2)
    mom = np.zeros((n, 3))
    T = []
    for t in range(600):
        pos, mom, facc, _ = ora.couple(p, pops, pos, mom, 1.0, 0.2, dt=0.1, n_substeps=10, seed=3, md_step0=10 * t)
        pops = ora.step(p, pops, facc, t)
        if t >= 200:
            T.append((mom ** 2).mean())
    assert abs(np.mean(T) / kT - 1) < 0.06
