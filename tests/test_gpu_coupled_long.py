"""Coupled parity over 200 LB steps of 10 MD sub-steps each (Sec. 4.5, Eqs.
langevin_momentum_update and ftotal; Sec. 4.6, Eq. Delta; Sec. 3): the GPU
path (coupling overlapped with the LB update, as the workload runs it)
against the FP64 oracle run alone from the same start, the oracle's own FP64
impulses feeding its LB steps, so that the comparison measures how far the
FP32 particle state and fluid drift from the oracle over a long run.

Two workloads on a thermal 32^3 box (kT = 1e-4, the seeded noise shared by
both sides through the counter-based generator):
  - chains: 4 FENE + WCA chains of 24 beads, periodic;
  - walls: 64 free particles between the walls, a body force driving
    Poiseuille flow.
Snapshots after 50, 100 and 200 steps report the growth of the errors; the
asserts apply to all of them.  Measured on a GB300 after 200 steps (positions
absolute; momenta and populations n - a rho0 as relative L2 / worst element):
  chains: positions 3.7e-6, momenta 9.5e-6 / 1.2e-5, populations 2.5e-7 / 9.7e-7;
  walls:  positions 4.5e-6, momenta 1.8e-6 / 3.0e-6, populations 2.2e-7 / 4.3e-7.
The errors do not grow with the run: the friction ties the particles to the
fluid, and the fluid's FP32 rounding stays at the one-step level.  The
position error grows slowly (~2e-8 per step, the FP32 offsets' rounding); the
chain momenta carry the steep WCA force's amplification of it.  The bars
are about three times the measured errors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check, check_pos, tid  # noqa: E402

SHAPE = (32, 32, 32)
STEPS = 200
SNAPS = (50, 100, 200)
KT = 1e-4

# (positions absolute, momenta (rel, max), populations n - a rho0 (rel, max))
BARS = {
    "chains": (1.2e-5, (3.5e-5, 4e-5), (8e-7, 3e-6)),
    "walls": (1.4e-5, (6e-6, 1e-5), (7e-7, 1.4e-6)),
}


def dev(x, dt=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dt is not None:
        t = t.to(dt)
    return t.cuda()


def _setup(case):
    if case == "chains":
        n_ch, clen = 4, 24
        pos = inputs.random_walk_chains(n_ch, clen, SHAPE, seed=71)
        walls, body = False, (0.0, 0.0, 0.0)
    else:
        n_ch, clen = 0, 0
        pos = inputs.uniform_particles(64, SHAPE, seed=73, zrange=(2.0, SHAPE[2] - 3.0))
        walls, body = True, (1e-5, 0.0, 0.0)
    mom = inputs.maxwell_momenta(pos.shape[0], 1.0, KT, seed=72).astype(np.float32).astype(np.float64)
    u = inputs.shear_wave(SHAPE, 0.01)
    if walls:
        u[:, 0] = 0
        u[:, -1] = 0
    return pos, mom, u, walls, body, n_ch, clen


def _md_kw(clen):
    return dict(chain_len=clen, use_wca=clen > 0, eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5)


@pytest.mark.parametrize("case", ["chains", "walls"])
def test_coupled_200_steps_parity(ora, case):
    pos, mom, u, walls, body, n_ch, clen = _setup(case)
    n = pos.shape[0]
    nsub, dt, gamma, mass = 10, 0.1, 2.0, 1.0

    lat = L.Lattice(SHAPE, kT=KT, seed=12, walls=walls, body_force=body)
    lat.init_equilibrium(None, dev(u))
    gpos, gmom = dev(pos), dev(mom, torch.float32)
    parts = L.particles(n, gpos, gmom, mass0=mass, gamma0=gamma)
    got = {}
    for t in range(STEPS):
        cp = L.couple_params(n_substeps=nsub, dt=dt, seed=5, md_step0=nsub * t, overlap=True, **_md_kw(clen))
        L.lb_couple_particles(lat.h, parts, cp)
        lat.step(1)
        if t + 1 in SNAPS:
            got[t + 1] = (gpos.cpu().numpy(), gmom.cpu().numpy().astype(np.float64),
                          lat.get_populations().cpu().numpy())
    assert lat.sync() == (L.LB_OK, 0)

    p = ora.make_params(SHAPE, kT=KT, seed=12, walls=walls, body_force=body)
    pops = ora.equilibrium(p, None, u)
    md = ora.make_md(n_ch, clen, eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5) if clen else None
    opos, omom = pos.copy(), mom.copy()
    a = ora.tables()[1][:, None, None, None]
    pos_bar, mom_bar, pop_bar = BARS[case]
    for t in range(STEPS):
        opos, omom, facc, broken = ora.couple(p, pops, opos, omom, mass, gamma, dt=dt, n_substeps=nsub, seed=5,
                                              md_step0=nsub * t, md=md)
        assert broken == 0
        pops = ora.step(p, pops, facc, t)
        if t + 1 in SNAPS:
            g_pos, g_mom, g_pops = got[t + 1]
            tag = "%s t=%d" % (tid(), t + 1)
            check_pos(tag + " positions", g_pos, opos, SHAPE, pos_bar)
            check(tag + " momenta", g_mom, omom, *mom_bar)
            check(tag + " populations", g_pops - a, pops - a, *pop_bar)
