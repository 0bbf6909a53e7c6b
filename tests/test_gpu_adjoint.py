"""GPU parity of the hand-written adjoint (kT = 0) against the FP64 oracle's
reverse pass, through the C ABI, plus the autograd wrapper.

Tolerances (FP32 adjoint against the FP64 reverse pass): one adjoint step to
1e-5 relative L2; whole reverse passes to 1e-3 relative per significant entry
and cosine similarity >= 0.99999.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import adjoint, inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check  # noqa: E402

GAM = dict(gamma_shear=0.2, gamma_bulk=-0.3, gamma_odd=0.4, gamma_even=-0.1)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


def dev(x, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dt).cuda()


def _lam_dev(lat, lam):
    """(19, nz, ny, nx) host array -> padded [19][pitch] device FP32 buffer."""
    pitch = L.lb_plane_pitch(lat.params)
    t = torch.zeros((19, pitch), dtype=torch.float32, device="cuda")
    t[:, :lat.n_nodes] = dev(lam.reshape(19, -1))
    return t


def _lam_host(lat, t):
    return t[:, :lat.n_nodes].cpu().numpy().astype(np.float64).reshape((19,) + lat.shape[::-1])


@pytest.mark.parametrize("walls", [False, True])
def test_one_adjoint_step_parity(ora, walls):
    shape = (7, 5, 9)
    bf = (2e-4, -1e-4, 0.0 if walls else 1e-4)
    u = inputs.gaussian_field(shape, 3, 5e-3, seed=1)
    f = inputs.gaussian_field(shape, 3, 1e-3, seed=2).astype(np.float32)
    lam = inputs.gaussian_field(shape, 19, 1.0, seed=3)
    if walls:
        u[:, 0] = u[:, -1] = 0
        f[:, 0] = f[:, -1] = 0
        lam[:, 0] = lam[:, -1] = 0
    p = ora.make_params(shape, walls=walls, body_force=bf, **GAM)
    s0 = ora.equilibrium(p, None, u)
    want_lam, want_g = ora.adjoint_step(p, s0, lam, f.astype(np.float64))
    ft = dev(f)
    lat = L.Lattice(shape, walls=walls, body_force=bf, force=ft, **GAM)
    lat.set_populations(dev(s0, torch.float64))
    cur, _ = L.lb_state_buffers(lat.h)
    lin = _lam_dev(lat, lam)
    lout = torch.zeros_like(lin)
    g = torch.zeros((3,) + shape[::-1], dtype=torch.float32, device="cuda")
    L.lb_adjoint_step(lat.h, cur, lin, lout, g)
    got_lam = _lam_host(lat, lout)
    fl = slice(1, shape[2] - 1) if walls else slice(None)
    check("adjoint step walls=%d lambda" % walls, got_lam[:, fl], want_lam[:, fl], 1e-5, 5e-5)
    check("adjoint step walls=%d force gradient" % walls, g.cpu().numpy()[:, fl], want_g[:, fl], 1e-5, 5e-5)
    lat.sync()


def test_reverse_pass_parity_and_autograd(ora):
    """Kinetic energy of the central 8^3 of a 16^3 box after 40 steps from rest,
    f ~ N(0, 1e-5): library reverse pass (checkpoints every 10) vs the FP64
    oracle reverse pass (all states stored)."""
    shape, T, K = (16, 16, 16), 40, 10
    lo, hi = (4, 4, 4), (12, 12, 12)
    f = inputs.gaussian_field(shape, 3, 1e-5, seed=0).astype(np.float32)
    p = ora.make_params(shape)
    s0 = ora.equilibrium(p)
    Lw, gw = ora.kinetic_energy_and_grad(p, s0, f.astype(np.float64), T, lo, hi)
    ft = torch.zeros((3,) + shape[::-1], dtype=torch.float32, device="cuda")
    lat = L.Lattice(shape, force=ft)
    lat.init_equilibrium()
    x = dev(f).requires_grad_(True)
    loss = adjoint.kinetic_energy(x, lat, T, lo, hi, K)
    loss.backward()
    g = x.grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() / Lw - 1) < 1e-4
    assert cos(g, gw) > 0.99999
    big = np.abs(gw) > 1e-3 * np.abs(gw).max()
    assert np.max(np.abs(g[big] - gw[big]) / np.abs(gw[big])) < 1e-3
    assert lat.step_index == T
    lat.sync()


def test_adjoint_forward_backward_split():
    """lb_adjoint_forward + lb_adjoint_backward give lb_adjoint_kinetic's loss
    and gradient, also when the lattice moves on in between; the backward
    runs once per forward; after the first call the reverse-mode arena is
    reused (no further device allocation)."""
    shape, T, K = (12, 10, 8), 12, 5
    lo, hi = (2, 2, 2), (9, 8, 6)
    ft = dev(inputs.gaussian_field(shape, 3, 1e-5, seed=3).astype(np.float32))
    lat = L.Lattice(shape, force=ft)
    g = torch.empty_like(ft)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def one(split):
        lat.init_equilibrium()
        lat.step_index = 0
        g.fill_(float("nan"))
        if split:
            L.lb_adjoint_forward(lat.h, T, K, lo, hi, loss)
            lat.step(3)
            L.lb_adjoint_backward(lat.h, g)
        else:
            L.lb_adjoint_kinetic(lat.h, T, K, lo, hi, g, loss)
        torch.cuda.synchronize()
        return loss.item(), g.cpu().numpy().astype(np.float64)

    la, ga = one(False)
    free0 = torch.cuda.mem_get_info()[0]
    lb, gb = one(True)
    lc, gc = one(True)
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.isfinite(ga).all() and np.abs(ga).max() > 0
    for l_, g_ in ((lb, gb), (lc, gc)):
        assert abs(l_ / la - 1) < 1e-12
        assert np.allclose(g_, ga, rtol=1e-6, atol=1e-9 * np.abs(ga).max())
    with pytest.raises(L.LBError) as ei:  # consumed by the last backward
        L.lb_adjoint_backward(lat.h, g)
    assert ei.value.status == L.LB_EINVAL
    assert lat.sync() == (L.LB_OK, 0)


def test_adjoint_requires_deterministic_run():
    lat = L.Lattice((8, 8, 8), kT=1e-4, force=torch.zeros((3, 8, 8, 8), device="cuda"))
    g = torch.zeros((3, 8, 8, 8), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as ei:
        L.lb_adjoint_kinetic(lat.h, 4, 2, (0, 0, 0), (8, 8, 8), g, loss)
    assert ei.value.status == L.LB_EUNSUPPORTED


@pytest.mark.slow
def test_config_64cubed_500_steps(ora):
    """The differentiable workload at full size: 64^3 periodic, kT = 0, learnable
    force field f ~ N(0, 1e-5), loss = kinetic energy of the central 16^3 after
    500 steps, checkpoints every 50.  Library gradient vs the FP64 oracle reverse
    pass (checkpointed), and vs central differences of the library's own
    forward (eps = 1e-3) on 32 random entries."""
    shape, T, K = (64, 64, 64), 500, 50
    lo, hi = (24, 24, 24), (40, 40, 40)
    f = inputs.gaussian_field(shape, 3, 1e-5, seed=0).astype(np.float32)
    p = ora.make_params(shape)
    s0 = ora.equilibrium(p)
    Lw, gw = ora.kinetic_energy_and_grad(p, s0, f.astype(np.float64), T, lo, hi, checkpoint_every=K)
    ft = torch.zeros((3,) + shape[::-1], dtype=torch.float32, device="cuda")
    lat = L.Lattice(shape, force=ft)

    def run(field, want_grad):
        lat.init_equilibrium()
        lat.step_index = 0
        ft.copy_(field)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        if not want_grad:  # the forward half alone (checkpoints and L)
            L.lb_adjoint_forward(lat.h, T, K, lo, hi, loss)
            return loss.item(), None
        g = torch.empty_like(ft)
        L.lb_adjoint_kinetic(lat.h, T, K, lo, hi, g, loss)
        return loss.item(), g.cpu().numpy().astype(np.float64)

    Lg, g = run(dev(f), True)
    print("64^3 adjoint: L gpu %.6e oracle %.6e, cosine %.7f" % (Lg, Lw, cos(g, gw)))
    assert abs(Lg / Lw - 1) < 1e-4
    assert cos(g, gw) > 0.99999
    big = np.abs(gw) > 1e-3 * np.abs(gw).max()
    assert np.max(np.abs(g[big] - gw[big]) / np.abs(gw[big])) < 1e-3
    rng = np.random.default_rng(1)
    eps = 1e-3
    errs = []
    for _ in range(32):
        c, z, y, x = (int(rng.integers(0, 3)), int(rng.integers(16, 48)), int(rng.integers(16, 48)),
                      int(rng.integers(16, 48)))
        fp, fm = f.copy(), f.copy()
        fp[c, z, y, x] += eps
        fm[c, z, y, x] -= eps
        fd = (run(dev(fp), False)[0] - run(dev(fm), False)[0]) / (2 * eps)
        errs.append(abs(fd - gw[c, z, y, x]) / max(abs(gw[c, z, y, x]), 1e-3 * np.abs(gw).max()))
    print("64^3 finite differences: max rel err %.2e" % max(errs))
    assert max(errs) < 1e-2


@pytest.mark.parametrize("walls", [False, True])
def test_coupled_reverse_pass_parity(ora, walls):
    """Reverse pass through coupled steps (free particles at kT = 0, 5
    sub-steps per LB step, 8 LB steps, checkpoints every 3): the library's
    dL/dforce, dL/d(initial positions) and dL/d(initial momenta) against the
    FP64 oracle's reverse pass (Sec. 4.5 with Eqs. Delta, 2point)."""
    shape, T, K = (12, 10, 12), 8, 3
    lo, hi = (2, 2, 2), (10, 8, 10)
    rng = np.random.default_rng(21)
    f = inputs.gaussian_field(shape, 3, 1e-4, seed=22).astype(np.float32)
    u0 = inputs.shear_wave(shape, 0.02) + inputs.gaussian_field(shape, 3, 2e-3, seed=23)
    if walls:
        f[:, 0] = f[:, -1] = 0
        u0[:, 0] = u0[:, -1] = 0
    n = 24
    pos = rng.uniform(0.0, 1.0, (n, 3)) * np.array(shape, dtype=float)
    if walls:
        pos[:, 2] = rng.uniform(1.2, shape[2] - 2.2, n)
        pos[0, 2] = 1.05
        pos[1, 2] = shape[2] - 2.05
    mom = rng.normal(0.0, 0.03, (n, 3)).astype(np.float32).astype(np.float64)
    if walls:  # two of them head into the walls
        mom[0, 2], mom[1, 2] = -0.25, 0.25
    p = ora.make_params(shape, walls=walls)
    s0 = ora.equilibrium(p, None, u0)
    L_want, g_want, lp_want, lm_want = ora.coupled_kinetic_energy_and_grad(
        p, s0, f.astype(np.float64), pos, mom, 1.0, 2.0, dt=0.1, n_substeps=5, nsteps=T, lo=lo, hi=hi)

    lat = L.Lattice(shape, walls=walls, force=dev(f))
    lat.set_populations(dev(s0, torch.float64))
    gpos, gmom = dev(pos, torch.float64), dev(mom)
    parts = L.particles(n, gpos, gmom, mass0=1.0, gamma0=2.0)
    cp = L.couple_params(n_substeps=5, dt=0.1)
    g = torch.empty((3,) + shape[::-1], dtype=torch.float32, device="cuda")
    gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gm = torch.empty_like(gp)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    L.lb_adjoint_kinetic_coupled(lat.h, parts, cp, T, K, lo, hi, g, gp, gm, loss)
    assert lat.sync() == (L.LB_OK, 0)
    assert float(loss.item()) == pytest.approx(L_want, rel=1e-4)
    fl = slice(1, shape[2] - 1) if walls else slice(None)
    gg = g.cpu().numpy().astype(np.float64)
    assert cos(gg[:, fl], g_want[:, fl]) > 0.99999
    assert rel(gg[:, fl], g_want[:, fl]) < 2e-3
    for got, want in ((gp, lp_want), (gm, lm_want)):
        got = got.cpu().numpy().astype(np.float64)
        assert cos(got, want) > 0.99999
        assert rel(got, want) < 2e-3
    # the forward part advanced the particles as lb_couple_particles does
    want_pos = pos.copy()
    opos, omom, st = pos.copy(), mom.copy(), s0
    for t in range(T):
        opos, omom, facc, _ = ora.couple(p, st, opos, omom, 1.0, 2.0, dt=0.1, n_substeps=5, seed=0,
                                         force=f.astype(np.float64))
        st = ora.step(p, st, f.astype(np.float64) + facc, t)
    d = gpos.cpu().numpy() - opos
    d -= np.array(shape) * np.round(d / np.array(shape))
    assert np.abs(d).max() < 1e-5, want_pos


def test_coupled_reverse_rejects_noise_and_chains():
    shape = (8, 8, 8)
    lat = L.Lattice(shape, kT=1e-4)
    g = torch.zeros((3, 8, 8, 8), dtype=torch.float32, device="cuda")
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda") + 2.5
    mom = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    parts = L.particles(4, pos, mom, mass0=1.0, gamma0=2.0)
    gp, gm = torch.zeros_like(mom), torch.zeros_like(mom)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as e:
        L.lb_adjoint_kinetic_coupled(lat.h, parts, L.couple_params(n_substeps=2, dt=0.1), 2, 1, (0, 0, 0),
                                     (8, 8, 8), g, gp, gm, loss)
    assert e.value.status == L.LB_EUNSUPPORTED
    lat2 = L.Lattice(shape)
    with pytest.raises(L.LBError) as e:
        L.lb_adjoint_kinetic_coupled(lat2.h, parts, L.couple_params(n_substeps=2, dt=0.1, chain_len=4,
                                                                    use_wca=True, r0=1.5, sigma=1.0), 2, 1,
                                     (0, 0, 0), (8, 8, 8), g, gp, gm, loss)
    assert e.value.status == L.LB_EUNSUPPORTED


def test_coupled_autograd_matches_library_gradients():
    """adjoint.coupled_kinetic_energy hands the library's gradients to
    autograd (force field, initial positions and momenta)."""
    shape, T = (10, 8, 10), 4
    lo, hi = (2, 2, 2), (8, 6, 8)
    rng = np.random.default_rng(31)
    f = dev(inputs.gaussian_field(shape, 3, 1e-4, seed=32))
    u0 = inputs.shear_wave(shape, 0.02)
    n = 6
    pos0 = rng.uniform(0.0, 1.0, (n, 3)) * np.array(shape, dtype=float)
    mom0 = rng.normal(0.0, 0.03, (n, 3))
    cp = L.couple_params(n_substeps=4, dt=0.1)
    grads = []
    for use_autograd in (False, True):
        lat = L.Lattice(shape, force=torch.zeros_like(f))
        lat.init_equilibrium(None, dev(u0, torch.float64))
        pos, mom = dev(pos0, torch.float64), dev(mom0)
        if use_autograd:
            fr = f.clone().requires_grad_(True)
            pr = pos.clone().requires_grad_(True)
            mr = mom.clone().requires_grad_(True)
            loss = adjoint.coupled_kinetic_energy(fr, pr, mr, lat, cp, T, lo, hi, mass0=1.0, gamma0=2.0,
                                                  checkpoint_every=2)
            loss.backward()
            grads.append((fr.grad, pr.grad.float(), mr.grad))
        else:
            lat.force.copy_(f)
            parts = L.particles(n, pos, mom, mass0=1.0, gamma0=2.0)
            g = torch.empty_like(f)
            gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
            gm = torch.empty_like(gp)
            ls = torch.empty(1, dtype=torch.float64, device="cuda")
            L.lb_adjoint_kinetic_coupled(lat.h, parts, cp, T, 2, lo, hi, g, gp, gm, ls)
            grads.append((g, gp, gm))
    for a, b in zip(*grads):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-9)  # atomics sum in a different order
