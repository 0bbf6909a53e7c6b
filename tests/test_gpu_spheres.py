"""GPU parity of the solid spheres with moving link bounce-back (Sec. 4.1,
4.2) against the FP64 oracle, through the C ABI.

Tolerances: solid maps equal node for node; fluid populations to 2e-6
relative (as the plain step: FP32 deviations and collision); sphere
velocities to 1e-5 relative and centres to 1e-6 absolute (F0 and zeta are
FP32 sums over a few hundred links, the velocity update runs in FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0803_2826_gb300 import inputs  # noqa: E402
from paper_0803_2826_gb300 import lbfluct as L  # noqa: E402
from parity_util import check, tid  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _gpu_run(shape, pops0, R, U, rad, mass, steps, *, fc=None, omega=None, **kw):
    lat = L.Lattice(shape, **kw)
    lat.set_populations(torch.as_tensor(pops0).cuda())
    pos = torch.as_tensor(np.array(R, dtype=np.float64)).cuda()
    vel = torch.as_tensor(np.array(U, dtype=np.float64)).cuda()
    m = torch.as_tensor(np.array(mass, dtype=np.float64)).cuda()
    f = None if fc is None else torch.as_tensor(np.array(fc, dtype=np.float64)).cuda()
    om = None if omega is None else torch.as_tensor(np.array(omega, dtype=np.float64)).cuda()
    s = L.spheres(len(mass), pos, vel, rad, mass=m, force=f, omega=om)
    L.lb_spheres_place(lat.h, s)
    for _ in range(steps):
        L.lb_step_spheres(lat.h, s)
    own = torch.empty(lat.n_nodes, dtype=torch.int32, device="cuda")
    L.lb_get_solid_map(lat.h, own)
    st = lat.sync()
    out = (lat.get_populations().cpu().numpy(), own.cpu().numpy().reshape(shape[::-1]), pos.cpu().numpy(),
           vel.cpu().numpy(), st, lat)
    return out if om is None else out + (om.cpu().numpy(),)


def _ora_run(ora, p, pops, R, U, rad, mass, steps, fc=None, omega=None):
    owner = ora.sphere_owner(p, R, rad)
    for t in range(steps):
        pops, owner, R, U, omega, ut, st = ora.step_spheres(p, pops, owner, R, U, rad, mass, fc=fc, step=t,
                                                            omega=omega)
        assert st == 0
    return pops, owner, R, U, omega


@pytest.mark.parametrize("kT,shape", [(0.0, (16, 16, 16)), (1e-4, (16, 16, 16)), (1e-4, (17, 16, 15))])
def test_moving_spheres_parity(ora, kT, shape):
    """Even nx runs the paired kernel (far pairs take the plain update), odd
    nx the one-node kernel."""
    kw = dict(kT=kT, seed=3, gamma_shear=0.1)
    p = ora.make_params(shape, **kw)
    pops0 = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.01))
    R = np.array([[4.3, 5.1, 6.2], [11.2, 10.7, 9.9]])
    U = np.array([[0.05, -0.03, 0.02], [-0.04, 0.02, 0.06]])
    mass = [40.0, 60.0]
    fc = [[1e-3, 0.0, -2e-3], [0.0, 5e-4, 0.0]]
    want = _ora_run(ora, p, pops0, R, U, 2.6, mass, 12, fc=fc)
    got = _gpu_run(shape, pops0, R, U, 2.6, mass, 12, fc=fc, **kw)
    assert got[4] == (L.LB_OK, 0)
    assert np.array_equal(got[1], want[1])
    fl = want[1] < 0
    c, a, e, w, opp = ora.tables()
    aa = a[:, None]
    check(tid() + " populations", got[0][:, fl] - aa, want[0][:, fl] - aa, 2e-6, 1e-5)
    assert np.abs(got[2] - want[2]).max() < 1e-6
    check(tid() + " velocities", got[3], want[3], 1e-5, 2e-5)


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_rotating_spheres_parity(ora, kT):
    """Spheres with angular velocities (Eq. NodeVel): maps, populations,
    velocities and angular velocities against the oracle."""
    shape = (16, 16, 16)
    kw = dict(kT=kT, seed=3, gamma_shear=0.1)
    p = ora.make_params(shape, **kw)
    pops0 = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.01))
    R = np.array([[4.3, 5.1, 6.2], [11.2, 10.7, 9.9]])
    U = np.array([[0.05, -0.03, 0.02], [-0.04, 0.02, 0.06]])
    Om = np.array([[0.01, -0.02, 0.015], [0.0, 0.02, -0.01]])
    mass = [40.0, 60.0]
    want = _ora_run(ora, p, pops0, R, U, 2.6, mass, 12, omega=Om)
    got = _gpu_run(shape, pops0, R, U, 2.6, mass, 12, omega=Om, **kw)
    assert got[4] == (L.LB_OK, 0)
    assert np.array_equal(got[1], want[1])
    fl = want[1] < 0
    c, a, e, w, opp = ora.tables()
    aa = a[:, None]
    check("rotating spheres kT=%g populations" % kT, got[0][:, fl] - aa, want[0][:, fl] - aa, 2e-6, 1e-5)
    assert np.abs(got[2] - want[2]).max() < 1e-6
    check("rotating spheres kT=%g velocities" % kT, got[3], want[3], 1e-5, 2e-5)
    check("rotating spheres kT=%g angular velocities" % kT, got[6], want[4], 1e-5, 2e-5)
    assert np.abs(want[4] - Om).max() > 1e-4


def test_spheres_conserve_momentum_gpu(ora):
    shape = (24, 20, 22)
    c, a, e, w, opp = ora.tables()
    p = ora.make_params(shape)
    pops0 = ora.equilibrium(p, None, inputs.shear_wave(shape, 0.01))
    R = np.array([[5.3, 5.1, 6.2], [16.2, 12.7, 14.9], [12.0, 3.5, 17.0]])
    U = np.array([[0.05, -0.03, 0.02], [-0.04, 0.02, 0.06], [0.0, 0.03, -0.05]])
    mass = np.array([40.0, 60.0, 30.0])
    owner0 = ora.sphere_owner(p, R, 2.8)
    pops, owner, R1, U1, st, lat = _gpu_run(shape, pops0, R, U, 2.8, mass, 30)
    assert st == (L.LB_OK, 0)

    def total(pops, owner, U):
        fl = owner.reshape(-1) < 0
        return (pops.reshape(19, -1)[:, fl] - a[:, None]).sum(1) @ c + (mass[:, None] * U).sum(0)

    assert (owner != owner0).sum() > 10
    assert np.allclose(total(pops, owner, U1), total(pops0, owner0, U), rtol=0, atol=1e-5)


def test_fixed_sphere_array_drag_gpu(ora):
    """Steady flow through a fixed sphere array driven by a body force: the
    superficial velocity matches the oracle's (the drag pin of the oracle)."""
    L_, rad, g = 16, 3.5, 1e-6
    go = 1.0 - 1.0 / (0.5 + (3.0 / 16.0) / 0.5)
    kw = dict(body_force=(g, 0.0, 0.0), gamma_odd=go)
    p = ora.make_params((L_, L_, L_), **kw)
    pops0 = ora.equilibrium(p)
    R = np.array([[L_ / 2 + 0.1, L_ / 2 + 0.2, L_ / 2 + 0.3]])
    want = _ora_run(ora, p, pops0, R, np.zeros((1, 3)), rad, [0.0], 1500)
    got = _gpu_run((L_, L_, L_), pops0, R, np.zeros((1, 3)), rad, [0.0], 1500, **kw)
    fl = want[1] < 0
    c = ora.tables()[0]
    us_w = (want[0][:, fl].T @ c)[:, 0].sum()
    us_g = (got[0][:, fl].T @ c)[:, 0].sum()
    assert abs(us_g - us_w) < 1e-4 * abs(us_w), (us_g, us_w)


def test_comoving_uniform_state_is_stationary_gpu(ora):
    shape = (14, 14, 14)
    p = ora.make_params(shape)
    u0 = np.array([0.03, -0.02, 0.01])
    uu = np.zeros((3,) + shape[::-1])
    for d in range(3):
        uu[d] = u0[d]
    pops0 = ora.equilibrium(p, None, uu)
    got = _gpu_run(shape, pops0, [[7.2, 6.9, 7.4]], [u0], 3.1, [0.0], 5)
    fl = got[1] < 0
    assert np.abs(got[0][:, fl] - pops0[:, fl]).max() < 2e-7


def test_sphere_errors():
    lat = L.Lattice((16, 16, 16))
    lat.init_equilibrium()
    pos = torch.tensor([[5.0, 5.0, 5.0], [7.0, 5.0, 5.0]], dtype=torch.float64, device="cuda")
    vel = torch.zeros_like(pos)
    s = L.spheres(2, pos, vel, 2.5)
    with pytest.raises(L.LBError) as ei:  # not placed yet
        L.lb_step_spheres(lat.h, s)
    assert ei.value.status == L.LB_EINVAL
    L.lb_spheres_place(lat.h, s)  # the two spheres overlap
    st, bits = L.lb_sync(lat.h, raise_on_error=False)
    assert st == L.LB_EDEVICE and bits & L.LB_DERR_SPHERE
    with pytest.raises(L.LBError) as ei:
        L.lb_spheres_place(lat.h, L.spheres(1, pos, vel, 6.0))  # 2a + 5 > 16
    assert ei.value.status == L.LB_EINVAL
    for kw in (dict(walls=True), dict(dtype=L.LB_F16)):
        other = L.Lattice((16, 16, 16), **kw)
        with pytest.raises(L.LBError) as ei:
            L.lb_spheres_place(other.h, L.spheres(1, pos, vel, 2.5))
        assert ei.value.status == L.LB_EUNSUPPORTED
