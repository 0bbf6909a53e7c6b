"""Pins of the oracle's transverse velocity modes and their autocorrelation
(the observable of the batched replica workload).

- transverse_modes() of a planted single-harmonic velocity field returns the
  closed-form Fourier amplitude (A - i B) / 2 of u = A cos(k r) + B sin(k r).
- mode_autocorrelation() of e^{i w t} is cos(w tau) exactly.
- Sec. 3.6 and Sec. 3.4 (Eq. shearviscosity): in a thermal 8^3 box started
  from rest, the oracle's autocorrelation of the six transverse modes matches
  the exact linear theory of the fluctuating update (tests/lb_linear.py:
  equal-time variance kT / (rho0 V) once thermalised, decay by the shear
  eigenvalue per step) within five standard errors (batch means).
"""
import numpy as np
import pytest

from paper_0803_2826_gb300 import inputs
import lb_linear as LL  # noqa: E402


def test_transverse_modes_of_a_planted_harmonic(ora):
    """An equilibrium at rho = 1 with u_x = A cos(k z) + B sin(k z) and
    u_z = 2A cos(k' x) - B sin(k' x): moments() reads the state the next
    collision sees (streamed), and streaming the momentum part 3 a_i c_i.j of
    n^eq multiplies a transverse harmonic by 3 sum_i a_i c_ix^2 e^{-i k c_iz}
    = (2 + cos k) / 3 (the density is unchanged to O(u^2)); so the modes are
    (A - i B)/2 (2 + cos k)/3 and (2A + i B)/2 (2 + cos k')/3 up to O(u^2),
    and the other four vanish."""
    shape = (6, 5, 8)
    p = ora.make_params(shape)
    nx, ny, nz = shape
    A, B = 3e-3, -2e-3
    u = np.zeros((3, nz, ny, nx))
    z = np.arange(nz)[:, None, None] * np.ones((1, ny, nx))
    x = np.arange(nx)[None, None, :] * np.ones((nz, ny, 1))
    kz, kx = 2 * np.pi / nz, 2 * np.pi / nx
    u[0] = A * np.cos(kz * z) + B * np.sin(kz * z)       # mode 0: u_x at k_z
    u[2] = 2 * A * np.cos(kx * x) - B * np.sin(kx * x)   # mode 3: u_z at k_x
    got = ora.transverse_modes(p, ora.equilibrium(p, None, u))
    w0 = (A - 1j * B) / 2 * (2 + np.cos(kz)) / 3
    w3 = (2 * A + 1j * B) / 2 * (2 + np.cos(kx)) / 3
    assert abs(got[0] - w0) < 1e-4 * abs(w0), (got[0], w0)
    assert abs(got[3] - w3) < 1e-4 * abs(w3), (got[3], w3)
    for m in (1, 2, 4, 5):
        assert abs(got[m]) < 1e-12


def test_mode_autocorrelation_of_a_rotating_phase(ora):
    w = 0.37
    T = 60
    s = np.exp(1j * w * np.arange(T))[:, None] * np.ones((1, 6))
    c = ora.mode_autocorrelation(s, 5, T, 12)
    assert np.allclose(c, np.cos(w * np.arange(13)), rtol=0, atol=1e-14)


def _acf(s, tb, te, taus):
    return np.array([np.mean((s[tb + t:te] * np.conj(s[tb:te - t])).real) for t in taus])


def test_oracle_velocity_autocorrelation_matches_linear_theory(ora):
    L, kT, rho0, T, tb = 8, 1e-4, 1.0, 12000, 200
    p = ora.make_params((L, L, L), kT=kT, rho0=rho0, seed=5)
    pops = ora.equilibrium(p)
    series = np.zeros((T, 6), dtype=np.complex128)
    for t in range(T):
        series[t] = ora.transverse_modes(p, pops)
        pops = ora.step(p, pops, None, t)
    taus = [0, 1, 2, 3, 5, 8, 12, 20]
    tables = ora.tables()
    want = LL.transverse_acf(L, tables, kT, rho0, L ** 3, taus, tb, T)
    got = _acf(series, tb, T, taus)
    nb = 20
    blk = (T - tb) // nb
    est = np.array([_acf(series, tb + b * blk, tb + (b + 1) * blk, taus) for b in range(nb)])
    se = est.std(0, ddof=1) / np.sqrt(nb)
    z = (got - want) / se
    print("8^3 velocity autocorrelation / (kT / rho0 V):", np.round(got / (kT / (rho0 * L ** 3)), 4),
          "theory", np.round(want / (kT / (rho0 * L ** 3)), 4), "z", np.round(z, 2))
    assert np.all(np.abs(z) < 5), z
    # thermalised equal-time value and one-step decay, as the paper fixes them
    assert abs(want[0] / (kT / (rho0 * L ** 3)) - 1) < 1e-12
    lam = LL.shear_eigenvalue(L, tables).real
    assert abs(want[1] / want[0] - lam) < 5e-3
    # the looped definition of the oracle agrees with the vectorised estimate
    c = ora.mode_autocorrelation(series[:400], tb, 400, 3)
    assert np.allclose(c, _acf(series[:400], tb, 400, [0, 1, 2, 3]), rtol=1e-12, atol=0)
