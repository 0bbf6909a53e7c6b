"""GPU parity of the point-particle coupling (Sec. 4.5, 4.6) and the
Kremer-Grest forces (Sec. 2.1) against the FP64 oracle, through the C ABI.

Every comparison asserts the field-wide relative L2 error and the worst
element (relative to the field's largest entry); the bars are about three
times the errors measured on a GB300:
  - positions: 1e-6 absolute (FP32 cell offsets: ~3e-7 measured);
  - free particles (no pair forces): momenta, spread impulses and the
    populations after the LB step that applies them at ~2e-7 relative
    (FP32 rounding of the interpolation and the OU update);
  - FENE/WCA chains: momenta ~1e-5, impulses ~3e-6.  The WCA force is steep
    (d ln F / d ln r ~ 14 at r ~ sigma), so the ~2e-7 rounding of the FP32
    offsets over the sub-steps becomes ~3e-6 in a force and ~1e-5 in the
    momentum it accumulates; the impulses to the fluid, which see the forces
    only through (C2 - dt) F^c, stay smaller.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check, check_pos, tid  # noqa: E402

# Bars (relative L2, worst element relative to the field's largest entry);
# see the module docstring.
MOM = (6e-7, 1e-6)          # free particles
FACC = (1.2e-6, 3e-6)
NEXT = (6e-7, 1.2e-6)
CHAIN_MOM = (3e-5, 4e-5)    # FENE/WCA chains
CHAIN_FACC = (1e-5, 1.2e-5)


def _check_run(r, shape, pos_tol, next_bar=NEXT, mom=MOM, facc=FACC):
    t = tid()
    check_pos(t + " positions", r["gpos"], r["opos"], shape, pos_tol)
    check(t + " momenta", r["gmom"], r["omom"], *mom)
    check(t + " impulses", r["gfacc"], r["ofacc"], *facc)
    if "got_next" in r and next_bar is not None:
        c, a, e, w, opp = r["tables"]
        aa = a[:, None, None, None]
        check(t + " next populations", r["got_next"] - aa, r["want_next"] - aa, *next_bar)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x, dt=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dt is not None:
        t = t.to(dt)
    return t.cuda()


def _run(ora, shape, pos, mom, *, kT, walls=False, chains=None, nsub=10, dt=0.1, gamma=2.0, mass=1.0,
         noise_kind=0, u_amp=0.01, lb_after=True, body_force=(0.0, 0.0, 0.0), per_substep=False, kernel=2,
         fext=(0.0, 0.0, 0.0)):
    mom32 = mom.astype(np.float32).astype(np.float64)
    p = ora.make_params(shape, kT=kT, seed=4, walls=walls, body_force=body_force)
    u = inputs.shear_wave(shape, u_amp) + inputs.gaussian_field(shape, 3, 1e-3, seed=8)
    if walls:
        u[:, 0] = 0
        u[:, -1] = 0
    pops = ora.equilibrium(p, None, u)
    md = None
    if chains:
        md = ora.make_md(chains[0], chains[1], eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5)
    opos, omom, ofacc, broken = ora.couple(p, pops, pos, mom32, mass, gamma, dt=dt, n_substeps=nsub, seed=11,
                                           md_step0=40, md=md, noise_kind=noise_kind, kernel=kernel, fext=fext)
    assert broken == 0
    lat = L.Lattice(shape, kT=kT, seed=4, walls=walls, body_force=body_force)
    lat.init_equilibrium(None, dev(u))
    gpos = dev(pos)
    gmom = dev(mom32, torch.float32)
    parts = L.particles(pos.shape[0], gpos, gmom, mass0=mass, gamma0=gamma)
    cp = L.couple_params(n_substeps=nsub, dt=dt, seed=11, md_step0=40, noise_kind=noise_kind,
                         chain_len=chains[1] if chains else 0, use_wca=bool(chains), eps=0.01, sigma=1.0,
                         k_fene=0.3, r0=1.5, per_substep=per_substep, kernel=kernel, fext=fext)
    L.lb_couple_particles(lat.h, parts, cp)
    facc = torch.empty((3,) + tuple(shape[::-1]), dtype=torch.float32, device="cuda")
    L.lb_get_particle_forces(lat.h, facc)
    out = dict(p=p, pops=pops, opos=opos, omom=omom, ofacc=ofacc, lat=lat,
               gpos=gpos.cpu().numpy(), gmom=gmom.cpu().numpy().astype(np.float64),
               gfacc=facc.cpu().numpy().astype(np.float64))
    if lb_after:
        lat.step(1)
        out["want_next"] = ora.step(p, pops, ofacc.astype(np.float32).astype(np.float64), 0)
        out["got_next"] = lat.get_populations().cpu().numpy()
        out["tables"] = ora.tables()
    assert lat.sync() == (L.LB_OK, 0)
    return out


def _pos_err(a, b, shape):
    d = a - b
    Lb = np.array(shape, dtype=np.float64)
    d -= Lb * np.round(d / Lb)
    return np.abs(d).max()


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_free_particles_parity(ora, kT):
    shape = (12, 10, 9)
    pos = inputs.uniform_particles(300, shape, seed=1)
    mom = inputs.maxwell_momenta(300, 1.0, 1e-4, seed=2)
    r = _run(ora, shape, pos, mom, kT=kT)
    _check_run(r, shape, 1e-6)


@pytest.mark.parametrize("per_substep,kernel", [(False, 2), (True, 2), (False, 3)])
def test_external_force_parity(ora, per_substep, kernel):
    """A constant external force on every particle (part of F^c; the fluid
    gets only the drag and random impulses, Eq. (ftotal)), on both kernels
    of the coupling and with phi_3."""
    shape = (12, 10, 9)
    pos = inputs.uniform_particles(300, shape, seed=1)
    mom = inputs.maxwell_momenta(300, 1.0, 1e-4, seed=2)
    r = _run(ora, shape, pos, mom, kT=1e-4, per_substep=per_substep, kernel=kernel, fext=(3e-3, -2e-3, 1e-3))
    _check_run(r, shape, 1e-6)


def test_three_point_noise_parity(ora):
    shape = (8, 8, 8)
    pos = inputs.uniform_particles(200, shape, seed=3)
    mom = np.zeros((200, 3))
    r = _run(ora, shape, pos, mom, kT=1e-4, noise_kind=1, lb_after=False)
    check(tid() + " momenta", r["gmom"], r["omom"], *MOM)


def test_walls_particles_parity(ora):
    shape = (10, 8, 12)
    pos = inputs.uniform_particles(200, shape, seed=5, zrange=(1.0, 10.0))
    mom = inputs.maxwell_momenta(200, 1.0, 1e-2, seed=6)  # fast enough to reach the walls
    r = _run(ora, shape, pos, mom, kT=1e-4, walls=True, dt=0.5, body_force=(1e-5, 0, 0))
    _check_run(r, shape, 1e-6, next_bar=None)
    assert r["gpos"][:, 2].min() >= 1.0 and r["gpos"][:, 2].max() <= 10.0


@pytest.mark.parametrize("per_substep", [False, True])
def test_chains_parity(ora, per_substep):
    """Two FENE + WCA chains of 24 beads (bond 0.97) in a 16^3 thermal fluid,
    by the persistent kernel and by one launch per sub-step."""
    shape = (16, 16, 16)
    pos = inputs.random_walk_chains(2, 24, shape, seed=7)
    mom = inputs.maxwell_momenta(48, 1.0, 1e-4, seed=8)
    r = _run(ora, shape, pos, mom, kT=1e-4, chains=(2, 24), per_substep=per_substep)
    _check_run(r, shape, 1e-6, next_bar=None, mom=CHAIN_MOM, facc=CHAIN_FACC)


def test_wca_narrow_box_between_walls(ora):
    """WCA particles in a box 4 cells wide in x, where the cell list has only
    two cells (each visited once), between walls in z (cells not wrapped)."""
    shape = (4, 20, 14)
    n = 120
    pos = inputs.random_walk_chains(n, 1, (4, 20, 11), min_dist=1.0, seed=41)  # no overlaps
    pos[:, 2] += 1.0  # z in [1, 12) = [1, nz - 2)
    mom = inputs.maxwell_momenta(n, 1.0, 1e-3, seed=42)
    r = _run(ora, shape, pos, mom, kT=1e-4, walls=True, chains=(n, 1))
    _check_run(r, shape, 1.2e-6, next_bar=None, mom=(2.5e-6, 5e-6), facc=(1e-6, 2e-6))


@pytest.mark.parametrize("per_substep", [False, True])
def test_wca_chains_many(ora, per_substep):
    """100 FENE + WCA chains of 256 beads in a 48^3 box (200 blocks of the
    persistent kernel; or one launch per sub-step, each after a cell-list
    build)."""
    shape = (48, 48, 48)
    pos = inputs.random_walk_chains(100, 256, shape, seed=43)
    mom = inputs.maxwell_momenta(25600, 1.0, 1e-4, seed=44)
    r = _run(ora, shape, pos, mom, kT=1e-4, chains=(100, 256), nsub=3, lb_after=False, per_substep=per_substep)
    _check_run(r, shape, 1e-6, next_bar=None, mom=(1.1e-5, 1.4e-5), facc=(4e-6, 5e-6))


@pytest.mark.parametrize("kernel", [2, 3, 4])
def test_interpolation_parity(ora, kernel):
    shape = (9, 11, 7)
    p = ora.make_params(shape, kT=0.0)
    u = inputs.gaussian_field(shape, 3, 1e-2, seed=9)
    pops = ora.equilibrium(p, None, u)
    pos = inputs.uniform_particles(500, shape, seed=10)
    # positions on node planes, half-way between them and next to the box
    # edges, where phi_3 changes branch or the stencil wraps
    pos[:8] = [[0.0, 0.0, 0.0], [0.5, 1.5, 2.5], [8.999999, 10.5, 6.5], [4.0, 5.0, 6.0],
               [0.25, 10.75, 0.5], [3.5, 3.5, 3.5], [8.5, 0.5, 6.999], [1e-9, 2.0, 3.0]]
    want = ora.interpolate(p, pops, pos, kernel=kernel)
    lat = L.Lattice(shape)
    lat.init_equilibrium(None, dev(u))
    out = torch.empty((500, 3), dtype=torch.float32, device="cuda")
    if kernel == 2:
        L.lb_interpolate(lat.h, 500, dev(pos), out)
    else:
        L.lb_interpolate_phi(lat.h, kernel, 500, dev(pos), out)
    assert rel(out.cpu().numpy().astype(np.float64), want) < 1e-6
    assert np.abs(out.cpu().numpy() - want).max() < 1e-8


@pytest.mark.parametrize("kernel", [3, 4])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_phi_kernel_free_particles_parity(ora, kernel, kT):
    """phi_3 / phi_4 stencils (27 / 64 nodes) in the coupling and the LB step
    that applies their impulses."""
    shape = (12, 10, 9)
    pos = inputs.uniform_particles(300, shape, seed=1)
    mom = inputs.maxwell_momenta(300, 1.0, 1e-4, seed=2)
    r = _run(ora, shape, pos, mom, kT=kT, kernel=kernel)
    _check_run(r, shape, 1e-6)


@pytest.mark.parametrize("kernel", [3, 4])
def test_phi_kernel_walls_parity(ora, kernel):
    """Between walls the particles stay K/2 from the solid planes; no impulse
    reaches a solid plane."""
    shape = (10, 8, 12)
    b = kernel / 2
    pos = inputs.uniform_particles(200, shape, seed=5, zrange=(b, shape[2] - 1 - b))
    mom = inputs.maxwell_momenta(200, 1.0, 1e-2, seed=6)  # fast enough to reach the walls
    r = _run(ora, shape, pos, mom, kT=1e-4, walls=True, dt=0.5, body_force=(1e-5, 0, 0), kernel=kernel)
    _check_run(r, shape, 1.2e-6)
    assert r["gpos"][:, 2].min() >= b and r["gpos"][:, 2].max() <= shape[2] - 1 - b
    assert np.all(r["gfacc"][:, 0] == 0) and np.all(r["gfacc"][:, -1] == 0)


@pytest.mark.parametrize("kernel", [3, 4])
@pytest.mark.parametrize("per_substep", [False, True])
def test_phi_kernel_chains_parity(ora, kernel, per_substep):
    """FENE + WCA chains with the wide stencils: the persistent kernel (its
    start-of-call gather through the block's node table) and the
    per-sub-step kernels."""
    shape = (16, 16, 16)
    pos = inputs.random_walk_chains(2, 24, shape, seed=7)
    mom = inputs.maxwell_momenta(48, 1.0, 1e-4, seed=8)
    r = _run(ora, shape, pos, mom, kT=1e-4, chains=(2, 24), kernel=kernel, per_substep=per_substep)
    _check_run(r, shape, 1e-6, next_bar=None, mom=CHAIN_MOM, facc=CHAIN_FACC)


@pytest.mark.parametrize("kernel", [3, 4])
def test_phi_node_cache_moving_chains(ora, kernel):
    """Chains of 64 monomers launched fast: stencil origins move every few
    sub-steps (new stencils gathered inside the grid barrier), three blocks
    sharing the start-of-call node tables."""
    shape = (24, 20, 22)
    pos = inputs.random_walk_chains(6, 64, shape, min_dist=1.0, seed=17)
    mom = inputs.maxwell_momenta(pos.shape[0], 1.0, 2e-2, seed=18)
    r = _run(ora, shape, pos, mom, kT=1e-4, chains=(6, 64), kernel=kernel)
    _check_run(r, shape, 1.2e-6, next_bar=None, mom=CHAIN_MOM, facc=CHAIN_FACC)


@pytest.mark.parametrize("kernel", [3, 4])
def test_phi_node_cache_dimers_walls(ora, kernel):
    """Fast dimers (chains of two) between walls on the persistent wide
    kernel: centres on a grid of spacing 2 inside the band K/2 + 1 from the
    solid planes, bonds of 0.97 in random directions, 14 blocks."""
    shape = (24, 20, 22)
    b = kernel // 2 + 1
    g = np.stack(np.meshgrid(np.arange(1.0, 24.0, 2.0), np.arange(1.0, 20.0, 2.0),
                             np.arange(b + 1.0, shape[2] - b - 1.0, 2.0), indexing="ij"), -1).reshape(-1, 3)
    e = np.random.default_rng(27).normal(size=g.shape)
    e /= np.linalg.norm(e, axis=1)[:, None]
    pos = np.stack([g - 0.485 * e, g + 0.485 * e], axis=1).reshape(-1, 3) % np.array(shape, dtype=np.float64)
    n = pos.shape[0]
    mom = inputs.maxwell_momenta(n, 1.0, 2e-2, seed=28)
    r = _run(ora, shape, pos, mom, kT=1e-4, walls=True, chains=(n // 2, 2), kernel=kernel, body_force=(1e-5, 0, 0))
    _check_run(r, shape, 1.2e-6, next_bar=None, mom=CHAIN_MOM, facc=CHAIN_FACC)
    assert r["gpos"][:, 2].min() >= kernel / 2 and r["gpos"][:, 2].max() <= shape[2] - 1 - kernel / 2


@pytest.mark.parametrize("kernel", [3, 4])
def test_phi_node_cache_full(ora, kernel):
    """WCA particles scattered through a 64^3 box: the 128 particles of a
    block share no stencil nodes, more than the block's start-of-call node
    table holds (2304 / 5461 slots), so the nodes that find no slot are
    gathered by their particles directly; the results still match the
    oracle."""
    shape = (64, 64, 64)
    rng = np.random.default_rng(29)
    pts = []
    while len(pts) < 512:  # at least 2.5 apart (periodic)
        c = rng.uniform(0.0, 64.0, 3)
        if all(np.linalg.norm((c - d + 32.0) % 64.0 - 32.0) >= 2.5 for d in pts):
            pts.append(c)
    pos = np.array(pts)
    # distinct stencil nodes of the first block's 128 particles: more than the table holds
    o = np.floor(pos[:128] + (0.5 if kernel == 3 else 0.0)).astype(int) - 1
    d = np.stack(np.meshgrid(*[np.arange(kernel)] * 3, indexing="ij"), -1).reshape(-1, 3)
    nodes = {tuple(x) for x in ((o[:, None, :] + d[None]) % 64).reshape(-1, 3)}
    assert len(nodes) > (2304 if kernel == 3 else 5461)
    mom = inputs.maxwell_momenta(pos.shape[0], 1.0, 1e-4, seed=28)
    r = _run(ora, shape, pos, mom, kT=1e-4, chains=(512, 1), kernel=kernel, nsub=4, lb_after=False)
    _check_run(r, shape, 1e-6, next_bar=None)


def test_phi3_many_particles_parity(ora):
    """200000 particles with phi_3 in a 32^3 box: many particles per node,
    every stencil shape (both phi_3 branches on every axis)."""
    shape = (32, 32, 32)
    pos = inputs.uniform_particles(200000, shape, seed=21)
    mom = inputs.maxwell_momenta(200000, 1.0, 1e-4, seed=22)
    r = _run(ora, shape, pos, mom, kT=1e-4, nsub=3, kernel=3)
    _check_run(r, shape, 1e-6, next_bar=None)


def test_phi_kernel_rejections():
    """Both stencil bits, a channel narrower than the stencil needs, and the
    reverse pass with a wide stencil are refused."""
    lat = L.Lattice((8, 8, 4), walls=True)
    lat.init_equilibrium()
    pos = dev(np.array([[1.0, 1.0, 1.5]]))
    mom = dev(np.zeros((1, 3)), torch.float32)
    parts = L.particles(1, pos, mom, mass0=1.0, gamma0=1.0)
    cp = L.couple_params(n_substeps=1, dt=0.1)
    cp.flags = L.LB_COUPLE_PHI3 | L.LB_COUPLE_PHI4
    with pytest.raises(L.LBError) as ei:
        L.lb_couple_particles(lat.h, parts, cp)
    assert ei.value.status == L.LB_EINVAL
    with pytest.raises(L.LBError) as ei:  # nz = 4 < 4 + 1
        L.lb_couple_particles(lat.h, parts, L.couple_params(n_substeps=1, dt=0.1, kernel=4))
    assert ei.value.status == L.LB_EINVAL
    L.lb_couple_particles(lat.h, parts, L.couple_params(n_substeps=1, dt=0.1, kernel=3))  # nz = 4 fits phi_3
    with pytest.raises(L.LBError) as ei:
        L.lb_interpolate_phi(lat.h, 5, 1, pos, torch.empty((1, 3), device="cuda"))
    assert ei.value.status == L.LB_EINVAL
    assert lat.sync() == (L.LB_OK, 0)


def test_coupled_momentum_conservation_gpu(ora):
    """Particles + fluid momentum is conserved through coupling and the LB step."""
    shape = (16, 16, 16)
    pos = inputs.random_walk_chains(4, 16, shape, seed=12)
    mom = inputs.maxwell_momenta(64, 1.0, 1e-4, seed=13)
    lat = L.Lattice(shape, kT=1e-4, seed=1)
    lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
    gpos, gmom = dev(pos), dev(mom, torch.float32)
    parts = L.particles(64, gpos, gmom, mass0=1.0, gamma0=2.0)

    def total():
        _, _, _, s = lat.moments(want_rho=False, want_j=False, want_pi=False, want_sums=True)
        return s.cpu().numpy()[1:4] + gmom.double().sum(0).cpu().numpy()

    P0 = total()
    for t in range(5):
        cp = L.couple_params(n_substeps=10, dt=0.1, seed=3, md_step0=10 * t, chain_len=16, use_wca=True,
                             eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5)
        L.lb_couple_particles(lat.h, parts, cp)
        lat.step(1)
    P1 = total()
    assert np.allclose(P1, P0, atol=2e-5), (P0, P1)
    assert lat.sync() == (L.LB_OK, 0)


@pytest.mark.parametrize("per_substep", [False, True])
def test_many_free_particles(ora, per_substep):
    """200000 free particles (several per node): the one-launch free-particle
    kernel (no grid barrier, so no residency limit), and the per-sub-step
    kernels (LB_COUPLE_PER_SUBSTEP)."""
    shape = (32, 32, 32)
    pos = inputs.uniform_particles(200000, shape, seed=21)
    mom = inputs.maxwell_momenta(200000, 1.0, 1e-4, seed=22)
    r = _run(ora, shape, pos, mom, kT=1e-4, nsub=3, per_substep=per_substep)
    _check_run(r, shape, 1e-6, next_bar=None)


@pytest.mark.parametrize("per_substep", [False, True])
def test_fast_wca_particles_rebuild_lists(ora, per_substep):
    """WCA particles moving ~0.5 sigma per call (more than half the Verlet
    skin) force list rebuilds inside and between calls; three calls in a row,
    each followed by an LB step, against the oracle's brute-force pairs."""
    # heavy particles (m = 10) launched fast (|v| ~ 0.27) in a cold fluid: they
    # keep moving ~0.3 sigma per call while WCA collisions stay integrable
    shape = (14, 14, 14)
    n = 600
    pos = inputs.random_walk_chains(n, 1, shape, min_dist=1.0, seed=31)  # no overlaps
    kT, m = 1e-4, 10.0
    mom = inputs.maxwell_momenta(n, m, 0.25, seed=32).astype(np.float32).astype(np.float64)
    p = ora.make_params(shape, kT=kT, seed=4)
    pops = ora.equilibrium(p)
    md = ora.make_md(0, 0, eps=0.01, sigma=1.0, use_wca=True)
    lat = L.Lattice(shape, kT=kT, seed=4)
    lat.init_equilibrium()
    gpos, gmom = dev(pos), dev(mom, torch.float32)
    parts = L.particles(n, gpos, gmom, mass0=m, gamma0=2.0)
    opos, omom = pos.copy(), mom.copy()
    for t in range(3):
        opos, omom, facc, _ = ora.couple(p, pops, opos, omom, m, 2.0, dt=0.1, n_substeps=10, seed=9,
                                         md_step0=10 * t, md=md)
        pops = ora.step(p, pops, facc.astype(np.float32).astype(np.float64), t)
        cp = L.couple_params(n_substeps=10, dt=0.1, seed=9, md_step0=10 * t, use_wca=True, eps=0.01, sigma=1.0,
                             per_substep=per_substep)
        L.lb_couple_particles(lat.h, parts, cp)
        lat.step(1)
    assert lat.sync() == (L.LB_OK, 0)
    check_pos(tid() + " positions", gpos.cpu().numpy(), opos, shape, 2.2e-6)
    check(tid() + " momenta", gmom.cpu().numpy().astype(np.float64), omom, 2e-6, 5e-6)


def _coupled_run(shape, *, walls, overlap, steps=4, join_early=False, kernel=2, dtype=L.LB_F32):
    """`steps` rounds of couple + step in a thermal fluid: FENE + WCA chains
    (periodic box) or single WCA particles between walls."""
    if walls:  # z in [1, nz - 2): no bond may cross the walls
        n_ch, clen = 192, 1
        pos = inputs.random_walk_chains(n_ch, 1, (shape[0], shape[1], shape[2] - 3), min_dist=1.0, seed=51)
        pos[:, 2] += 1.0
    else:
        n_ch, clen = 6, 32
        pos = inputs.random_walk_chains(n_ch, clen, shape, seed=51)
    n = pos.shape[0]
    mom = inputs.maxwell_momenta(n, 1.0, 2e-3, seed=52).astype(np.float32)  # fast: cells change
    lat = L.Lattice(shape, kT=1e-4, seed=6, walls=walls, body_force=(1e-5, 0.0, 0.0), dtype=dtype)
    lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
    gpos, gmom = dev(pos), dev(mom, torch.float32)
    parts = L.particles(n, gpos, gmom, mass0=1.0, gamma0=2.0)
    forces = []
    for t in range(steps):
        cp = L.couple_params(n_substeps=10, dt=0.1, seed=3, md_step0=10 * t, chain_len=clen, use_wca=True,
                             eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, overlap=overlap, kernel=kernel)
        L.lb_couple_particles(lat.h, parts, cp)
        if join_early:
            f = torch.empty((3,) + tuple(shape[::-1]), dtype=torch.float32, device="cuda")
            L.lb_get_particle_forces(lat.h, f)
            forces.append(f.cpu().numpy())
        lat.step(1)
    assert lat.sync() == (L.LB_OK, 0)
    return lat.get_populations().cpu().numpy(), gpos.cpu().numpy(), gmom.cpu().numpy(), forces


@pytest.mark.parametrize("walls,kernel", [(False, 2), (True, 2), (False, 4), (True, 3)])
def test_overlapped_coupling_matches_serial(walls, kernel):
    """LB_COUPLE_OVERLAP: the step's update of all nodes without the impulses
    (concurrent with the coupling) plus the re-update of the visited stencil
    nodes gives the serial result (up to the order of the impulse atomics);
    for phi_3 / phi_4 the re-update covers the 4^3 nodes around each cell."""
    shape = (20, 18, 16)
    a = _coupled_run(shape, walls=walls, overlap=False, kernel=kernel)
    b = _coupled_run(shape, walls=walls, overlap=True, kernel=kernel)
    # FP32 deviations ~1e-2: a few ulps where the impulse sums (and, for FP32
    # storage, the correction of the stored result) round differently; the
    # particles follow the fluid to a few ulps of their FP32 cell offsets
    assert np.abs(a[0] - b[0]).max() < 1e-7
    assert _pos_err(a[1], b[1], shape) < 1e-6
    assert np.abs(a[2] - b[2]).max() < 1e-6


def test_two_coupling_calls_per_step_with_overlap():
    """Two coupling calls before one step (5 + 5 sub-steps): the second
    overlapped call runs in the serial order, so the impulses of both calls
    reach the fluid; same result as two serial calls."""
    shape = (20, 18, 16)
    out = []
    for overlap in (False, True):
        pos = inputs.random_walk_chains(6, 32, shape, seed=51)
        mom = inputs.maxwell_momenta(192, 1.0, 2e-3, seed=52).astype(np.float32)
        lat = L.Lattice(shape, kT=1e-4, seed=6, body_force=(1e-5, 0.0, 0.0))
        lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
        gpos, gmom = dev(pos), dev(mom, torch.float32)
        parts = L.particles(192, gpos, gmom, mass0=1.0, gamma0=2.0)
        for t in range(3):
            for half in range(2):
                cp = L.couple_params(n_substeps=5, dt=0.1, seed=3, md_step0=10 * t + 5 * half, chain_len=32,
                                     use_wca=True, eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, overlap=overlap)
                L.lb_couple_particles(lat.h, parts, cp)
            lat.step(1)
        assert lat.sync() == (L.LB_OK, 0)
        out.append((lat.get_populations().cpu().numpy(), gpos.cpu().numpy()))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-7
    assert _pos_err(out[0][1], out[1][1], shape) < 1e-6


@pytest.mark.parametrize("dtype,walls,kernel", [(L.LB_F16, False, 3), (L.LB_BF16, True, 2)])
def test_overlapped_coupling_reduced_precision(dtype, walls, kernel):
    """FP16 / BF16 storage: the overlapped step re-updates the impulse nodes
    with the full update (not the FP32 correction), over the 4^3 block for
    phi_3; same result as the serial order up to storage roundings where the
    impulse sums (atomics) round differently.  One unit of the stored value
    (deviation x 2^10, |deviation| < 2e-3) is ~1e-6 in FP16 and ~8e-6 in BF16;
    the bar is about ten units after four steps."""
    shape = (20, 18, 16)
    a = _coupled_run(shape, walls=walls, overlap=False, kernel=kernel, dtype=dtype)
    b = _coupled_run(shape, walls=walls, overlap=True, kernel=kernel, dtype=dtype)
    d = np.abs(a[0] - b[0])
    unit = 1e-6 if dtype == L.LB_F16 else 8e-6
    assert d.max() < 10 * unit and d.mean() < unit, (d.max(), d.mean())
    assert _pos_err(a[1], b[1], shape) < 1e-5


@pytest.mark.parametrize("shape,kernel", [((3, 3, 3), 4), ((2, 5, 3), 3)])
def test_stencil_wider_than_box(ora, shape, kernel):
    """Boxes narrower than the stencil: periodic images of a node receive the
    weights of every stencil node that wraps onto them (as the oracle
    does)."""
    pos = inputs.uniform_particles(20, shape, seed=9)
    mom = inputs.maxwell_momenta(20, 1.0, 1e-4, seed=10)
    r = _run(ora, shape, pos, mom, kT=1e-4, nsub=4, kernel=kernel)
    _check_run(r, shape, 1e-6, next_bar=None)


def test_no_particles_is_a_no_op():
    lat = L.Lattice((8, 8, 8), kT=1e-4, seed=2)
    lat.init_equilibrium()
    ref = L.Lattice((8, 8, 8), kT=1e-4, seed=2)
    ref.init_equilibrium()
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    parts = L.particles(0, empty, empty.float(), mass0=1.0, gamma0=1.0)
    for overlap in (False, True):
        L.lb_couple_particles(lat.h, parts, L.couple_params(n_substeps=3, dt=0.1, overlap=overlap, kernel=3))
        lat.step(1)
        ref.step(1)
    assert lat.sync() == (L.LB_OK, 0)
    assert torch.equal(lat.get_populations(), ref.get_populations())


def test_overlapped_coupling_joined_by_another_call():
    """A call between the overlapped coupling and lb_step (here
    lb_get_particle_forces) waits for the coupling; the step then applies
    the impulses in its single pass."""
    shape = (20, 18, 16)
    a = _coupled_run(shape, walls=False, overlap=False, join_early=True)
    b = _coupled_run(shape, walls=False, overlap=True, join_early=True)
    for fa, fb in zip(a[3], b[3]):
        assert np.abs(fa - fb).max() < 1e-9 and np.abs(fa).max() > 0
    assert np.abs(a[0] - b[0]).max() < 1e-7


def test_step_sums_with_overlapped_coupling():
    """The sums of lb_step_sums come from the launch that runs beside an
    overlapped coupling (forces do not enter them) and equal lb_moments'."""
    shape = (20, 18, 16)
    pos = inputs.random_walk_chains(6, 32, shape, seed=61)
    mom = inputs.maxwell_momenta(192, 1.0, 1e-4, seed=62).astype(np.float32)
    lat = L.Lattice(shape, kT=1e-4, seed=6)
    lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
    parts = L.particles(192, dev(pos), dev(mom, torch.float32), mass0=1.0, gamma0=2.0)
    want = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    got = torch.empty_like(want)
    for t in range(3):
        cp = L.couple_params(n_substeps=10, dt=0.1, seed=3, md_step0=10 * t, chain_len=32, use_wca=True,
                             eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, overlap=True)
        L.lb_moments(lat.h, None, None, None, want)
        L.lb_couple_particles(lat.h, parts, cp)
        L.lb_step_sums(lat.h, 1, got)
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - w).max() < 1e-6 * np.abs(w).max()
    assert lat.sync() == (L.LB_OK, 0)


@pytest.mark.parametrize("kernel,walls", [(2, False), (4, False), (3, True)])
def test_free_particles_overlap_matches_serial(kernel, walls):
    """Free particles on the one-launch kernel with LB_COUPLE_OVERLAP: the
    re-update of the nodes its stencil records list gives the serial result
    (up to the order of the impulse atomics), over four coupled steps with
    particles fast enough to change cells."""
    shape = (20, 18, 16)
    out = []
    for overlap in (False, True):
        zr = (kernel / 2, shape[2] - 1 - kernel / 2) if walls else None
        pos = inputs.uniform_particles(3000, shape, seed=71, zrange=zr) if walls else \
            inputs.uniform_particles(3000, shape, seed=71)
        mom = inputs.maxwell_momenta(3000, 1.0, 2e-3, seed=72).astype(np.float32)
        lat = L.Lattice(shape, kT=1e-4, seed=6, walls=walls, body_force=(1e-5, 0.0, 0.0))
        u = inputs.shear_wave(shape, 0.01)
        if walls:
            u[:, 0] = 0
            u[:, -1] = 0
        lat.init_equilibrium(None, dev(u))
        gpos, gmom = dev(pos), dev(mom, torch.float32)
        parts = L.particles(3000, gpos, gmom, mass0=1.0, gamma0=2.0)
        for t in range(4):
            cp = L.couple_params(n_substeps=10, dt=0.1, seed=3, md_step0=10 * t, overlap=overlap, kernel=kernel)
            L.lb_couple_particles(lat.h, parts, cp)
            lat.step(1)
        assert lat.sync() == (L.LB_OK, 0)
        out.append((lat.get_populations().cpu().numpy(), gpos.cpu().numpy(), gmom.cpu().numpy()))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-7
    assert _pos_err(out[0][1], out[1][1], shape) < 1e-6
    assert np.abs(out[0][2] - out[1][2]).max() < 1e-6


@pytest.mark.parametrize("overlap", [False, True])
def test_couple_async_events_match(overlap):
    """lb_couple_particles_async: each call's particle state read back on a
    copy stream as soon as the call's done event fires and uploaded again as
    the next call's input (the host returns the state it read), the next
    coupling ordered after the upload by its ready event; the results are the
    same bits as lb_couple_particles with the state left on the device."""
    shape = (24, 24, 24)
    pos = inputs.random_walk_chains(6, 32, shape, seed=51)
    n = pos.shape[0]
    mom = inputs.maxwell_momenta(n, 1.0, 2e-3, seed=52).astype(np.float32)
    out = []
    for use_async in (False, True):
        lat = L.Lattice(shape, kT=1e-4, seed=6)
        lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
        gpos, gmom = dev(pos), dev(mom, torch.float32)
        hpos = torch.empty(gpos.shape, dtype=gpos.dtype, pin_memory=True)
        hmom = torch.empty(gmom.shape, dtype=gmom.dtype, pin_memory=True)
        parts = L.particles(n, gpos, gmom, mass0=1.0, gamma0=2.0)
        copy, ready, cdone = torch.cuda.Stream(), torch.cuda.Event(), torch.cuda.Event()
        torch.cuda.synchronize()
        for t in range(6):
            cp = L.couple_params(n_substeps=10, dt=0.1, seed=3, md_step0=10 * t, chain_len=32, use_wca=True,
                                 eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, overlap=overlap)
            if use_async:
                with torch.cuda.stream(copy):
                    if t:
                        copy.wait_event(cdone)
                    hpos.copy_(gpos, non_blocking=True)
                    hmom.copy_(gmom, non_blocking=True)
                    gpos.copy_(hpos, non_blocking=True)
                    gmom.copy_(hmom, non_blocking=True)
                    ready.record(copy)
                L.lb_couple_particles_async(lat.h, parts, cp, ready, cdone)
            else:
                L.lb_couple_particles(lat.h, parts, cp)
            lat.step(1)
        assert lat.sync() == (L.LB_OK, 0)
        out.append((gpos.cpu().numpy(), gmom.cpu().numpy(), lat.get_populations().cpu().numpy()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
