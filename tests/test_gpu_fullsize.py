"""Parity at the full benchmark size, in the launch configuration bench.py
times: 256^3 fluctuating FP32 fluid (kT = 1e-4) with 64 FENE/WCA chains x
256 beads, 10 MD sub-steps per LB step, the coupling overlapped with the LB
update on the cooperative kernel.  After two coupled steps on the GPU, a
third one is checked against the FP64 oracle:

- every particle's position and momentum, the oracle running the whole
  coupling call from the GPU's state (momenta ~1e-5 relative, the FP32
  rounding of the positions amplified by the steep WCA force);
- the post-step populations at sampled nodes, which the oracle evaluates one
  by one (step_nodes), at nodes without particle impulses and at impulse
  nodes, where the FP32 impulses enter through the force term.

Each check asserts the relative L2 error and the worst element at about
three times the errors measured on a GB300 (positions 3.9e-7; momenta
9.5e-6 / 1.4e-5; populations 1.7e-7 / 1.8e-7 without and 8.3e-7 / 1.3e-6
with impulses).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check, check_pos  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_bench_workload_parity(ora):
    shape = (256, 256, 256)
    n_ch, clen, nsub, kT = 64, 256, 10, 1e-4
    mass, gamma, dt = 1.0, 2.0, 0.1
    md_kw = dict(eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5)
    lat = L.Lattice(shape, kT=kT, seed=0, replica=0)
    lat.init_equilibrium()
    pos0 = inputs.random_walk_chains(n_ch, clen, shape, seed=0)
    mom0 = inputs.maxwell_momenta(n_ch * clen, mass, kT, seed=1000)
    gpos = torch.as_tensor(pos0).cuda()
    gmom = torch.as_tensor(mom0, dtype=torch.float32).cuda()
    parts = L.particles(n_ch * clen, gpos, gmom, mass0=mass, gamma0=gamma)
    cp = L.couple_params(n_substeps=nsub, dt=dt, seed=7, chain_len=clen, use_wca=True, overlap=True, **md_kw)
    for t in range(2):
        cp.md_step0 = nsub * t
        L.lb_couple_particles(lat.h, parts, cp)
        lat.step(1)
    torch.cuda.synchronize()
    state = lat.get_populations().cpu().numpy()
    pos, mom = gpos.cpu().numpy(), gmom.cpu().numpy().astype(np.float64)
    cp.md_step0 = nsub * 2
    L.lb_couple_particles(lat.h, parts, cp)
    lat.step(1)
    assert lat.sync() == (L.LB_OK, 0)

    p = ora.make_params(shape, kT=kT, seed=0)
    md = ora.make_md(n_ch, clen, **md_kw)
    opos, omom, facc, broken = ora.couple(p, state, pos, mom, mass, gamma, dt=dt, n_substeps=nsub, seed=7,
                                          md_step0=nsub * 2, md=md)
    assert broken == 0
    check_pos("fullsize positions", gpos.cpu().numpy(), opos, shape, 1.2e-6)
    check("fullsize momenta", gmom.cpu().numpy().astype(np.float64), omom, 3e-5, 4.5e-5)

    f32 = facc.astype(np.float32).astype(np.float64)
    hit = np.flatnonzero(np.abs(f32).sum(0).ravel() > 0)
    rng = np.random.default_rng(5)
    quiet = rng.choice(np.setdiff1d(rng.integers(0, 256 ** 3, 2000), hit), 400, replace=False)
    busy = rng.choice(hit, 400, replace=False)
    c, a, e, w, opp = ora.tables()
    got = lat.get_populations().cpu().numpy().reshape(19, -1)
    for tag, idx, bar in (("quiet", quiet, (5e-7, 6e-7)), ("busy", busy, (2.5e-6, 4e-6))):
        want = ora.step_nodes(p, state, idx, f32, 2)
        check("fullsize populations at %s nodes" % tag, got[:, idx].T - a, want - a, *bar)
