"""GPU parity of the fused stream-collide kernel against the FP64 oracle.

All calls go through the C ABI (via the ctypes binding).  Inputs are seeded
and synthetic (paper_0803_2826_gb300.inputs).  Tolerances:
  - one step, FP32 storage: relative L2 error <= 2e-6 (FP32 rounding of
    O(1e-2) deviations);
  - 1000 steps of the 32^3 fluctuating shear wave: <= 1e-5 relative for
    n - a rho0, rho - rho0, j and pi - pi^eq (the stated target);
  - FP16 / BF16 storage: bounded by their rounding (2^-11, 2^-8 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


NAMES = ["n - a rho0", "rho - rho0", "j", "pi - pi_eq"]
GAMMAS = dict(gamma_shear=0.2, gamma_bulk=-0.3, gamma_odd=0.4, gamma_even=-0.1)


def _pair(ora, shape, nsteps, *, u=None, rho=None, field=None, dtype=L.LB_F32, **kw):
    """Run the oracle and the GPU from the same equilibrium for nsteps."""
    okw = {k: v for k, v in kw.items()}
    p = ora.make_params(shape, **okw)
    f64 = None if field is None else field.astype(np.float32).astype(np.float64)
    pops = ora.equilibrium(p, rho, u)
    pops = ora.run(p, pops, nsteps, f64)
    ft = None if field is None else dev(field.astype(np.float32))
    lat = L.Lattice(shape, force=ft, dtype=dtype, **kw)
    lat.init_equilibrium(None if rho is None else dev(rho), None if u is None else dev(u))
    lat.step(nsteps)
    got = host(lat.get_populations())
    lat.sync()
    return p, pops, got, lat, f64


def _fields(ora, p, pops, force):
    c, a, e, w, opp = ora.tables()
    rho, j, pi = ora.moments(p, pops, force)
    u = j / rho
    eye = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]
    pieq = np.stack([rho * ((1 / 3) if a_ == b_ else 0) + rho * u[a_] * u[b_] for a_, b_ in eye])
    dn = pops - (a * p.rho0)[:, None, None, None]
    return dn, rho - p.rho0, j, pi - pieq


@pytest.mark.parametrize("shape", [(6, 5, 7), (130, 3, 4), (1, 1, 8), (32, 2, 3)])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_one_step_parity(ora, shape, kT):
    u = inputs.shear_wave(shape, 0.02) + inputs.gaussian_field(shape, 3, 1e-3, seed=1)
    rho = 1.0 + inputs.gaussian_field(shape, 1, 1e-3, seed=2)[0]
    field = inputs.gaussian_field(shape, 3, 1e-4, seed=3)
    p, want, got, lat, f64 = _pair(ora, shape, 1, u=u, rho=rho, field=field, kT=kT, seed=5,
                                   body_force=(1e-5, -2e-5, 3e-6), **GAMMAS)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    tag = "one step %s kT=%g" % (shape, kT)
    check(tag + " n - a rho0", got - aa, want - aa, 2e-6, 5e-6)
    for nm, x, y in zip(NAMES, _fields(ora, p, got, f64), _fields(ora, p, want, f64)):
        check(tag + " " + nm, x, y, 5e-6, 2e-5)


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_walls_parity(ora, kT):
    shape = (7, 6, 9)
    u = inputs.gaussian_field(shape, 3, 1e-3, seed=4)
    u[:, 0] = 0
    u[:, -1] = 0
    p, want, got, lat, _ = _pair(ora, shape, 5, u=u, kT=kT, seed=9, walls=True,
                                 body_force=(1e-5, 0.0, 0.0), **GAMMAS)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    fl = slice(1, shape[2] - 1)
    check("walls kT=%g n - a rho0" % kT, got[:, fl] - aa, want[:, fl] - aa, 5e-6, 2e-5)


@pytest.mark.parametrize("ge", [0.5, -0.5])
def test_two_rate_poiseuille_gpu(ora, ge):
    """Two relaxation rates with (tau_e - 1/2)(tau_o - 1/2) = 3/16 (the
    relation for which the oracle's Poiseuille profile is the exact parabola
    with half-way no-slip planes): the GPU's steady profile after 20000 steps
    matches the parabola to FP32 accuracy (2e-5 of the peak), and with
    gamma_o = 0 it matches the oracle's slipping profile to the same bar."""
    nz, g = 12, 1e-5
    te = 1.0 / (1.0 - ge)
    go = 1.0 - 1.0 / (0.5 + (3.0 / 16.0) / (te - 0.5))
    nu = (1 + ge) / (6 * (1 - ge))
    z = np.arange(1, nz - 1)
    ua = g / (2 * nu) * (z - 0.5) * (nz - 1.5 - z)
    for gam_o in (go, 0.0):
        kw = dict(walls=True, body_force=(g, 0.0, 0.0), gamma_shear=ge, gamma_bulk=ge, gamma_even=ge,
                  gamma_odd=gam_o)
        lat = L.Lattice((4, 4, nz), **kw)
        lat.init_equilibrium()
        lat.step(20000)
        rho, j, _, _ = lat.moments(want_pi=False)
        ux = (j[0] / rho)[1:-1].mean(dim=(1, 2)).double().cpu().numpy()
        assert lat.sync() == (L.LB_OK, 0)
        if gam_o == go:
            want = ua
        else:
            p = ora.make_params((1, 1, nz), **kw)
            rr, jj, _ = ora.moments(p, ora.run(p, ora.equilibrium(p), 20000))
            want = (jj[0] / rr)[1:-1, 0, 0]
            assert np.abs(want - ua).max() > 1e-3 * ua.max()  # the slip is there
        # FP32 steady state: the rounding of the O(1e-3) deviations each step
        # (~1e-10) against the O(1e-5) force per step biases the balance by
        # ~1e-5 of the peak (measured 1.05e-5 with gamma_o = 0)
        assert np.abs(ux - want).max() < 2e-5 * ua.max(), (gam_o, np.abs(ux - want).max() / ua.max())


@pytest.mark.parametrize("shape", [(9, 8, 10), (10, 8, 9)])
@pytest.mark.parametrize("kT,walls", [(0.0, False), (1e-4, False), (1e-4, True)])
def test_exponential_equilibrium_parity(ora, kT, walls, shape):
    """lb_params.equilibrium = 1 (Sec. 3.6, Eq. equildist_lagrange): 20
    steps with a force field against the oracle, velocities up to 0.1 (the
    exponential and quadratic forms differ there by ~1e-4 of a population);
    odd nx runs one node per thread, even nx two in packed FP32."""
    u = inputs.gaussian_field(shape, 3, 0.04, seed=11)
    if walls:
        u[:, 0] = 0
        u[:, -1] = 0
    field = inputs.gaussian_field(shape, 3, 1e-4, seed=12)
    kw = dict(kT=kT, seed=5, walls=walls, equilibrium=1, **GAMMAS)
    p, want, got, lat, f64 = _pair(ora, shape, 20, u=u, field=field, **kw)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    fl = slice(1, shape[2] - 1) if walls else slice(None)
    check("exponential equilibrium %s kT=%g walls=%d" % (shape, kT, walls), got[:, fl] - aa, want[:, fl] - aa, 5e-6,
          2e-5)
    # and it is not the quadratic update
    pq, want_q, _, _, _ = _pair(ora, shape, 20, u=u, field=field, **dict(kw, equilibrium=0))
    assert rel(want_q[:, fl] - aa, want[:, fl] - aa) > 20 * rel(got[:, fl] - aa, want[:, fl] - aa)


def test_exponential_equilibrium_rejections():
    lat = L.Lattice((8, 8, 8), equilibrium=1)
    lat.init_equilibrium()
    sums = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as ei:
        L.lb_step_sums(lat.h, 1, sums)
    assert ei.value.status == L.LB_EUNSUPPORTED
    g = torch.zeros((3, 8, 8, 8), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as ei:
        L.lb_adjoint_kinetic(lat.h, 2, 1, (2, 2, 2), (6, 6, 6), g, loss)
    assert ei.value.status == L.LB_EUNSUPPORTED
    with pytest.raises(L.LBError) as ei:
        L.Lattice((8, 8, 8), equilibrium=2)
    assert ei.value.status == L.LB_EINVAL


def test_shear_wave_1000_steps(ora):
    """The 32^3 fluctuating shear-wave workload: rho0 = 1, gamma_s = gamma_v = 0
    (nu = 1/6), kT = 1e-4, seed 0, u_x = 0.01 sin(2 pi z / 32), 1000 steps."""
    shape = (32, 32, 32)
    u = inputs.shear_wave(shape, 0.01)
    p, want, got, lat, _ = _pair(ora, shape, 1000, u=u, kT=1e-4, seed=0)
    for nm, x, y in zip(NAMES, _fields(ora, p, got, None), _fields(ora, p, want, None)):
        check("1000 steps 32^3 " + nm, x, y, 1e-5, 1e-5)
    # the GPU's own moment kernel agrees with the oracle's moments too
    rho, j, pi, sums = lat.moments(want_sums=True)
    orho, oj, opi = ora.moments(p, want)
    check("1000 steps 32^3 lb_moments rho - rho0", host(rho) - 1.0, orho - 1.0, 1e-5, 1e-5)
    check("1000 steps 32^3 lb_moments j", host(j), oj, 1e-5, 1e-5)


@pytest.mark.parametrize("dtype,tol", [(L.LB_F16, 3e-3), (L.LB_BF16, 2.5e-2)])
def test_reduced_precision_storage(ora, dtype, tol):
    shape = (12, 10, 8)
    u = inputs.shear_wave(shape, 0.01)
    p, want, got, lat, _ = _pair(ora, shape, 20, u=u, kT=1e-4, seed=3, dtype=dtype)
    c, a, e, w, opp = ora.tables()
    aa = a[:, None, None, None]
    check("20 steps storage %d" % dtype, got - aa, want - aa, tol, 4 * tol)


def test_noise_words_bitwise(ora):
    n = 257
    words = torch.empty((n, 4, 4), dtype=torch.int32, device="cuda")
    gauss = torch.empty((n, 4, 4), dtype=torch.float32, device="cuda")
    seed = 0xDEADBEEF12345
    L.lb_noise_words(seed, 3, 77, 0, 1000, n, 4, words, gauss)
    torch.cuda.synchronize()
    W = words.cpu().numpy().view(np.uint32)
    G = gauss.cpu().numpy().astype(np.float64)
    for q in range(0, n, 16):
        want = ora.raw_words(seed, 1000 + q, 77, domain=0, replica=3, nblocks=4)
        assert np.array_equal(W[q].ravel(), want)
        g = ora.gaussians(seed, 1000 + q, 77, domain=0, replica=3, nblocks=4)
        # FP32 logarithm and hardware sine / cosine (absolute error < 2^-21
        # on the centred angle) times a radius of at most ~5.8
        assert np.allclose(G[q].ravel(), g, rtol=0, atol=4e-6)
    # particle domain, one block
    L.lb_noise_words(5, 0, 9, 1, 0, n, 1, words, None)
    torch.cuda.synchronize()
    W = words.cpu().numpy().view(np.uint32)
    for q in (0, 1, 100, 256):
        assert np.array_equal(W.reshape(-1)[4 * q:4 * q + 4], ora.raw_words(5, q, 9, domain=1, nblocks=1))


def test_box_muller_all_uniforms(ora):
    """The kernels' Box-Muller map against the FP64 oracle for every one of
    the 2^23 values of the radial uniform v1 = (2k + 1) 2^-24 (random angle
    words): finite everywhere, including v1 = 1 - 2^-24, and within the bound
    of the FP32 logarithm (hardware log2 / series near 1), the rsqrt radius
    and the hardware sine / cosine times a radius of at most ~5.8."""
    rng = np.random.default_rng(17)
    n = 1 << 23
    w = np.empty(2 * n, dtype=np.uint32)
    w[0::2] = (np.arange(n, dtype=np.uint32) << 9) | rng.integers(0, 512, n, dtype=np.uint32)
    w[1::2] = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    dw = torch.from_numpy(w.view(np.int32)).cuda()
    dg = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    L.lb_box_muller(dw, n, dg)
    torch.cuda.synchronize()
    got = dg.cpu().numpy().astype(np.float64)
    want = ora.box_muller(w)
    assert np.isfinite(got).all()
    err = np.abs(got - want)
    assert err.max() < 4e-6, (err.max(), int(err.argmax()))
    # the radius in relative terms, also where it is tiny (v1 near 1):
    # g0^2 + g1^2 = -2 ln v1 up to the log2 bound (3.5e-6 relative at the
    # switch to the series) and the sine / cosine error
    r2 = got[0::2] ** 2 + got[1::2] ** 2
    want_r2 = -2.0 * np.log((2.0 * np.arange(n) + 1.0) * 2.0 ** -24)
    assert np.allclose(r2, want_r2, rtol=1e-5, atol=0)


def test_conservation_on_gpu(ora):
    """Mass constant; momentum grows by sum f per step (FP32 storage)."""
    shape = (16, 12, 10)
    f = np.array([1e-5, -2e-5, 5e-6])
    lat = L.Lattice(shape, kT=1e-4, seed=2, body_force=f, **GAMMAS)
    lat.init_equilibrium(None, dev(inputs.shear_wave(shape, 0.01)))
    _, j0, _, s0 = lat.moments(want_sums=True)
    lat.step(10)
    _, j1, _, s1 = lat.moments(want_sums=True)
    s0, s1 = s0.cpu().numpy(), s1.cpu().numpy()
    N = np.prod(shape)
    assert abs(s1[0] - s0[0]) < 1e-5 * N * 1e-3 + 1e-9
    dJ = s1[1:4] - s0[1:4]
    assert np.allclose(dJ, 10 * f * N, rtol=1e-3, atol=1e-6)
    assert lat.sync() == (L.LB_OK, 0)


def test_step_counter_and_resume(ora):
    """Counter-based noise makes a split run bit-identical to an uninterrupted one."""
    shape = (8, 8, 8)
    a = L.Lattice(shape, kT=1e-4, seed=7)
    b = L.Lattice(shape, kT=1e-4, seed=7)
    a.init_equilibrium()
    b.init_equilibrium()
    a.step(6)
    b.step(3)
    snap = b.get_populations()
    step = b.step_index
    c = L.Lattice(shape, kT=1e-4, seed=7)
    c.set_populations(snap)
    c.step_index = step
    c.step(3)
    assert torch.equal(a.get_populations(), c.get_populations())


@pytest.mark.parametrize("shape,walls,dtype", [((24, 10, 12), False, L.LB_F32), ((23, 9, 11), False, L.LB_F32),
                                                ((20, 8, 14), True, L.LB_F32), ((24, 10, 12), False, L.LB_F16)])
def test_step_sums_equal_moment_sums(shape, walls, dtype):
    """lb_step_sums: the sums its last stream-collide launch accumulates equal
    those of lb_moments on the state that step starts from (paired and
    single-node kernels, walls, FP16 storage); the state advances as lb_step."""
    kw = dict(kT=1e-4, seed=3, walls=walls, body_force=(1e-5, 0.0, 0.0), dtype=dtype)
    a, b = L.Lattice(shape, **kw), L.Lattice(shape, **kw)
    u = inputs.shear_wave(shape, 0.02) + inputs.gaussian_field(shape, 3, 1e-3, seed=4)
    if walls:
        u[:, 0] = 0
        u[:, -1] = 0
    for lat in (a, b):
        lat.init_equilibrium(None, torch.as_tensor(u).cuda())
    want = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    got = torch.empty_like(want)
    a.step(4)
    L.lb_moments(a.h, None, None, None, want)
    L.lb_step_sums(b.h, 5, got)
    a.step(1)
    torch.cuda.synchronize()
    w, g = want.cpu().numpy(), got.cpu().numpy()
    scale = np.abs(w).max()
    assert np.abs(g - w).max() < 1e-6 * scale, (g, w)
    assert np.array_equal(a.get_populations().cpu().numpy(), b.get_populations().cpu().numpy())
    assert a.sync() == (L.LB_OK, 0) and b.sync() == (L.LB_OK, 0)


def test_nonfinite_sums_reported():
    """A non-finite population (a NaN planted at one node) makes the moment
    sums non-finite: lb_moments and lb_step_sums set the device error word,
    lb_sync reports LB_ENONFINITE and clears it; no fault, no abort."""
    shape = (8, 6, 5)
    lat = L.Lattice(shape, kT=0.0, seed=1)
    lat.init_equilibrium()
    n = lat.get_populations()
    n[3, 2, 1, 4] = float("nan")
    lat.set_populations(n)
    _, _, _, sums = lat.moments(want_sums=True)
    with pytest.raises(L.LBError) as ei:
        lat.sync()
    assert ei.value.status == L.LB_ENONFINITE
    assert not np.isfinite(sums.cpu().numpy()).all()
    assert lat.sync() == (L.LB_OK, 0)
    got = torch.empty(L.LB_NSUMS, dtype=torch.float64, device="cuda")
    L.lb_step_sums(lat.h, 1, got)
    st, bits = L.lb_sync(lat.h, raise_on_error=False)
    assert st == L.LB_ENONFINITE and bits & L.LB_DERR_NONFINITE
    assert lat.sync() == (L.LB_OK, 0)
