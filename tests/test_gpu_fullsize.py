"""Parity at the full benchmark size, in the launch configuration bench.py
times: 256^3 fluctuating FP32 fluid (kT = 1e-4) with 64 FENE/WCA chains x
256 beads, 10 MD sub-steps per LB step, the coupling overlapped with the LB
update on the cooperative kernel.  After two coupled steps on the GPU, a
third one is checked against the FP64 oracle:

- every particle's position (1e-6 absolute) and momentum (2e-4 relative),
  the oracle running the whole coupling call from the GPU's state;
- the post-step populations at sampled nodes, which the oracle evaluates one
  by one (step_nodes): 2e-6 relative at nodes without particle impulses, and
  2e-4 at impulse nodes, where the FP32 impulses (about 1e-4 relative from
  the oracle's) enter through the force term.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402


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
    d = gpos.cpu().numpy() - opos
    d -= 256.0 * np.round(d / 256.0)
    assert np.abs(d).max() < 1e-6
    assert rel(gmom.cpu().numpy().astype(np.float64), omom) < 2e-4

    f32 = facc.astype(np.float32).astype(np.float64)
    hit = np.flatnonzero(np.abs(f32).sum(0).ravel() > 0)
    rng = np.random.default_rng(5)
    quiet = rng.choice(np.setdiff1d(rng.integers(0, 256 ** 3, 2000), hit), 400, replace=False)
    busy = rng.choice(hit, 400, replace=False)
    c, a, e, w, opp = ora.tables()
    got = lat.get_populations().cpu().numpy().reshape(19, -1)
    for idx, tol in ((quiet, 2e-6), (busy, 2e-4)):
        want = ora.step_nodes(p, state, idx, f32, 2)
        assert rel(got[:, idx].T - a, want - a) < tol, (tol, rel(got[:, idx].T - a, want - a))
