"""Plain FP64 CPU oracle for the fluctuating D3Q19 lattice-Boltzmann update and
the frictional point-particle coupling of Duenweg & Ladd (arXiv 0803.2826).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_0803_2826_gb300`` and imports
nothing from it.

The arithmetic lives in ``lb_oracle.c`` (plain C, IEEE double, no fast-math);
this module compiles it with gcc on first use and wraps it with ctypes and
numpy.  Population arrays have shape ``(19, nz, ny, nx)`` and hold raw n_i.

Function -> passage it follows:
  tables()        Sec. 3.3 (D3Q19 weights), Sec. 3.4 Table 1 and Eq. (weights_unweighted)
  philox()        Philox4x32-10 of Salmon et al., SC'11 (noise source for Sec. 3.5)
  equilibrium()   Sec. 3.3, Eq. (original_equil_distrib)
  step(), step_nodes()  Eq. (LBE) streaming; Sec. 3.4-3.5 MRT collision with noise,
                  Eqs. (lco_update), (stochupdaterule1), (detailedbalance1);
                  Sec. 3.7 forcing; Sec. 4.1 Eq. (MBB) with u_b = 0 for walls
  moments()       Sec. 3.4 Eqs. (hmodes_beg)-(hmodes_end); Sec. 3.7 for j
  modes()         Sec. 3.4 Eq. (forward)
  md_forces()     Sec. 2.1 Eqs. (ulennardjones), (ufene)
  couple()        Sec. 4.5 Eqs. (fdrag), (ftotal), (langevin_momentum_update);
                  Sec. 4.6 Eqs. (ufluid_discrete), (Delta), (2point), (3point), (4point)
  interpolate()   Sec. 4.6 Eq. (ufluid_discrete)
  sphere_owner(), sphere_velocity(), step_spheres()  Sec. 4.1 Eq. (MBB); Sec. 4.2
                  Eqs. (EOMD-1)-(EOMD-3), (force0), (zeta), (EOMUsol) and the U~ equation
  effective_friction()  Sec. 4.5 drag experiment, Eqs. (dragexperiment_particle_equation),
                  (effsize), (aeff), (aeffcorr); Sec. 4.6 settling test
  adjoint_step()  reverse mode of step() at kT = 0, derived by hand in
                  population space (chain rule through Eq. (original_equil_distrib),
                  the MRT relaxation and Delta'' of Sec. 3.7, then the pull)
  kinetic_seed()  L = 1/2 sum |j|^2 / rho over a sub-box and dL/dstate
  kinetic_energy_and_grad()  forward + reverse pass of a whole run
  exp_equilibrium()  Sec. 3.6 Eq. (equildist_lagrange), the maximum-entropy equilibrium
                  (make_params(equilibrium=1) uses it in the collision)
  transverse_modes(), mode_autocorrelation()  Sec. 3.6 fluctuation spectrum and
                  Sec. 3.4 Eq. (shearviscosity): Fourier amplitudes of the transverse
                  velocity at the smallest wave vectors and their time autocorrelation
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "liblboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into liblboracle.so next to it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("walls", C.c_int), ("noise_rho0", C.c_int), ("equilibrium", C.c_int),
        ("rho0", C.c_double), ("kT", C.c_double),
        ("gamma_shear", C.c_double), ("gamma_bulk", C.c_double),
        ("gamma_odd", C.c_double), ("gamma_even", C.c_double),
        ("body_force", C.c_double * 3),
        ("seed", C.c_uint64), ("replica", C.c_uint32), ("pad2_", C.c_uint32),
    ]


class MD(C.Structure):
    _fields_ = [
        ("n_chains", C.c_int), ("chain_len", C.c_int), ("use_wca", C.c_int),
        ("pad_", C.c_int),
        ("eps", C.c_double), ("sigma", C.c_double),
        ("k_fene", C.c_double), ("r0", C.c_double),
    ]


class CoupleParams(C.Structure):
    _fields_ = [
        ("n_substeps", C.c_int), ("noise_kind", C.c_int),
        ("dt", C.c_double), ("seed", C.c_uint64),
        ("md_step0", C.c_uint32), ("kernel", C.c_uint32),
        ("fext", C.c_double * 3),
    ]


_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.ora_threads.restype = C.c_int
            lib.ora_tables.argtypes = [C.POINTER(C.c_int), _D, _D, _D, C.POINTER(C.c_int)]
            lib.ora_philox4x32_10.argtypes = [_U32, _U32, _U32]
            lib.ora_uniform.argtypes = [C.c_uint32]
            lib.ora_uniform.restype = C.c_double
            lib.ora_raw16.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_int, _U32]
            lib.ora_gaussians.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                          C.c_uint32, C.c_int, _D]
            lib.ora_box_muller.argtypes = [_U32, C.c_long, _D]
            P = C.POINTER(Params)
            lib.ora_equilibrium.argtypes = [P, _D, _D, _D]
            lib.ora_step.argtypes = [P, _D, _D, _D, C.c_uint32]
            lib.ora_moments.argtypes = [P, _D, _D, _D, _D, _D]
            lib.ora_modes.argtypes = [P, _D, _D]
            lib.ora_md_forces.argtypes = [P, C.POINTER(MD), C.c_int, _D, _D]
            lib.ora_md_forces.restype = C.c_int
            lib.ora_couple.argtypes = [P, _D, _D, C.c_int, _D, _D, _D, _D,
                                       C.POINTER(MD), C.POINTER(CoupleParams), _D]
            lib.ora_couple.restype = C.c_int
            lib.ora_couple_adjoint.argtypes = [P, _D, _D, C.c_int, _D, _D, _D, _D, C.POINTER(CoupleParams),
                                               _D, _D, _D, _D, _D]
            lib.ora_couple_adjoint.restype = C.c_int
            lib.ora_interpolate.argtypes = [P, _D, _D, C.c_int, _D, _D]
            lib.ora_interpolate_k.argtypes = [P, C.c_int, _D, _D, C.c_int, _D, _D]
            lib.ora_stencil.argtypes = [P, _D, C.POINTER(C.c_longlong), _D]
            lib.ora_stencil_k.argtypes = [P, C.c_int, _D, C.POINTER(C.c_longlong), _D]
            lib.ora_stencil_k.restype = C.c_int
            lib.ora_sphere_owner.argtypes = [P, C.c_int, _D, C.c_double, C.POINTER(C.c_int)]
            lib.ora_sphere_velocity.argtypes = [_D, C.c_double, _D, _D, _D, _D]
            lib.ora_step_spheres.argtypes = [P, _D, _D, _D, C.c_uint32, C.POINTER(C.c_int), C.c_int, C.c_double,
                                             _D, _D, _D, _D, _D, _D, _D]
            lib.ora_sphere_velocity6.argtypes = [_D, C.c_double, C.c_double, _D, _D, _D, _D]
            lib.ora_step_spheres.restype = C.c_int
            lib.ora_exp_equilibrium.argtypes = [C.c_double, _D, _D]
            lib.ora_step_nodes.argtypes = [P, _D, _D, C.c_uint32, C.c_int, C.POINTER(C.c_longlong), _D]
            lib.ora_phi.argtypes = [C.c_int, C.c_double]
            lib.ora_phi.restype = C.c_double
            lib.ora_adjoint_step.argtypes = [P, _D, _D, _D, _D, _D]
            lib.ora_kinetic_seed.argtypes = [P, _D, _D, C.POINTER(C.c_int), C.POINTER(C.c_int), _D, _D]
            lib.ora_kinetic_seed.restype = C.c_double
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def make_params(shape, *, rho0=1.0, kT=0.0, gamma_shear=0.0, gamma_bulk=0.0,
                gamma_odd=0.0, gamma_even=0.0, body_force=(0.0, 0.0, 0.0), seed=0,
                replica=0, walls=False, noise_rho0=False, equilibrium=0) -> Params:
    """shape = (nx, ny, nz); equilibrium: 0 the quadratic form of Eq.
    (original_equil_distrib), 1 the exponential form of Eq. (equildist_lagrange)
    in the collision."""
    p = Params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.walls = int(bool(walls))
    p.noise_rho0 = int(bool(noise_rho0))
    p.equilibrium = int(equilibrium)
    p.rho0 = rho0
    p.kT = kT
    p.gamma_shear, p.gamma_bulk = gamma_shear, gamma_bulk
    p.gamma_odd, p.gamma_even = gamma_odd, gamma_even
    for d in range(3):
        p.body_force[d] = float(body_force[d])
    p.seed = int(seed)
    p.replica = int(replica)
    return p


def threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(_load().ora_threads())


def tables():
    """(c[19,3] int, a[19], e[19,19] (row k), w[19], opp[19]) built from the paper."""
    lib = _load()
    c = np.zeros((Q, 3), dtype=np.int32)
    a = np.zeros(Q)
    e = np.zeros((Q, Q))
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib.ora_tables(c.ctypes.data_as(C.POINTER(C.c_int)), _dp(a), _dp(e), _dp(w),
                   opp.ctypes.data_as(C.POINTER(C.c_int)))
    return c.astype(np.int64), a, e, w, opp.astype(np.int64)


def philox(ctr, key):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib.ora_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(x: int) -> float:
    return _load().ora_uniform(int(x) & 0xffffffff)


def raw_words(seed, node, step, domain=0, replica=0, nblocks=4):
    lib = _load()
    o = (C.c_uint32 * 16)()
    lib.ora_raw16(int(seed), int(node), int(step), int(domain), int(replica), int(nblocks), o)
    return np.array([int(v) for v in o[:4 * nblocks]], dtype=np.uint32)


def gaussians(seed, node, step, domain=0, replica=0, nblocks=4):
    lib = _load()
    g = np.zeros(16)
    lib.ora_gaussians(int(seed), int(node), int(step), int(domain), int(replica),
                      int(nblocks), _dp(g))
    return g[:4 * nblocks]


def box_muller(words):
    """Box-Muller Gaussians of consecutive word pairs (uint32 array of even
    length), in the order the pairs come."""
    w = np.ascontiguousarray(words, dtype=np.uint32).ravel()
    assert w.size % 2 == 0
    g = np.zeros(w.size)
    _load().ora_box_muller(w.ctypes.data_as(_U32), w.size // 2, _dp(g))
    return g


def _nodes(p: Params):
    return p.nx * p.ny * p.nz


def equilibrium(p: Params, rho=None, u=None):
    """n^eq(rho, u) per node; rho shape (nz,ny,nx) or None (rho0); u (3,nz,ny,nx) or None."""
    lib = _load()
    pops = np.zeros((Q, p.nz, p.ny, p.nx))
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    lib.ora_equilibrium(C.byref(p), _dp(r), _dp(uu), _dp(pops))
    return pops


def step(p: Params, pops, force=None, step_index=0):
    """One stream+collide step; returns the new post-collision populations.
    force: optional (3, nz, ny, nx) field added to p.body_force."""
    lib = _load()
    src = np.ascontiguousarray(pops, dtype=np.float64)
    dst = np.empty_like(src)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    lib.ora_step(C.byref(p), _dp(src), _dp(dst), _dp(f), int(step_index) & 0xffffffff)
    return dst


def run(p: Params, pops, nsteps, force=None, step0=0):
    for t in range(nsteps):
        pops = step(p, pops, force, step0 + t)
    return pops


def moments(p: Params, pops, force=None):
    """(rho (nz,ny,nx), j (3,nz,ny,nx), pi (6,nz,ny,nx)) of the pre-collision state."""
    lib = _load()
    src = np.ascontiguousarray(pops, dtype=np.float64)
    rho = np.empty((p.nz, p.ny, p.nx))
    j = np.empty((3, p.nz, p.ny, p.nx))
    pi = np.empty((6, p.nz, p.ny, p.nx))
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    lib.ora_moments(C.byref(p), _dp(src), _dp(f), _dp(rho), _dp(j), _dp(pi))
    return rho, j, pi


def modes(p: Params, pops):
    """All 19 moments m_k of the pre-collision state, shape (19,nz,ny,nx)."""
    lib = _load()
    src = np.ascontiguousarray(pops, dtype=np.float64)
    m = np.empty((Q, p.nz, p.ny, p.nx))
    lib.ora_modes(C.byref(p), _dp(src), _dp(m))
    return m


def make_md(n_chains, chain_len, *, eps=0.01, sigma=1.0, k_fene=0.3, r0=1.5, use_wca=True) -> MD:
    md = MD()
    md.n_chains, md.chain_len, md.use_wca = int(n_chains), int(chain_len), int(bool(use_wca))
    md.eps, md.sigma, md.k_fene, md.r0 = eps, sigma, k_fene, r0
    return md


def md_forces(p: Params, md: MD, pos):
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    F = np.zeros_like(pos)
    broken = lib.ora_md_forces(C.byref(p), C.byref(md), pos.shape[0], _dp(pos), _dp(F))
    return F, broken


def couple(p: Params, pops, pos, mom, mass, gamma, *, dt, n_substeps, seed, md_step0=0,
           md: MD | None = None, force=None, noise_kind=0, kernel=2, fext=None):
    """One LB step's worth of particle sub-steps.  Returns (pos, mom, facc, broken);
    facc has shape (3, nz, ny, nx) and holds the spread impulses -J Delta.
    fext: constant external force on every particle (part of F^c)."""
    lib = _load()
    pos = np.array(pos, dtype=np.float64, order="C", copy=True)
    mom = np.array(mom, dtype=np.float64, order="C", copy=True)
    n = pos.shape[0]
    mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
    gamma = np.ascontiguousarray(np.broadcast_to(np.asarray(gamma, dtype=np.float64), (n,)))
    facc = np.zeros((3, p.nz, p.ny, p.nx))
    cp = CoupleParams()
    cp.n_substeps, cp.noise_kind, cp.dt = int(n_substeps), int(noise_kind), float(dt)
    cp.seed, cp.md_step0, cp.kernel = int(seed), int(md_step0), int(kernel)
    if fext is not None:
        for c in range(3):
            cp.fext[c] = float(fext[c])
    src = np.ascontiguousarray(pops, dtype=np.float64)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    broken = lib.ora_couple(C.byref(p), _dp(src), _dp(f), n, _dp(pos), _dp(mom), _dp(mass),
                            _dp(gamma), None if md is None else C.byref(md), C.byref(cp),
                            _dp(facc))
    return pos, mom, facc, broken


def couple_adjoint(p: Params, pops, pos0, mom0, mass, gamma, *, dt, n_substeps, lam_facc, lam_pos, lam_mom,
                   lam_pops, grad_f, force=None):
    """Reverse of couple() at kT = 0 for free particles (no md): from
    lam_facc = dL/dfacc and lam_pos / lam_mom = dL/d(state after the call),
    returns (dL/dpos0, dL/dmom0) and adds dL/dpops (through the interpolated
    u) into lam_pops and dL/dforce into grad_f (both in place)."""
    lib = _load()
    n = np.asarray(pos0).shape[0]
    pos0 = np.ascontiguousarray(pos0, dtype=np.float64)
    mom0 = np.ascontiguousarray(mom0, dtype=np.float64)
    mass = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
    gamma = np.ascontiguousarray(np.broadcast_to(np.asarray(gamma, dtype=np.float64), (n,)))
    lp = np.array(lam_pos, dtype=np.float64, order="C", copy=True)
    lm = np.array(lam_mom, dtype=np.float64, order="C", copy=True)
    cp = CoupleParams()
    cp.n_substeps, cp.noise_kind, cp.dt = int(n_substeps), 0, float(dt)
    src = np.ascontiguousarray(pops, dtype=np.float64)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    lf = np.ascontiguousarray(lam_facc, dtype=np.float64)
    assert lam_pops.flags.c_contiguous and lam_pops.dtype == np.float64
    assert grad_f.flags.c_contiguous and grad_f.dtype == np.float64
    st = lib.ora_couple_adjoint(C.byref(p), _dp(src), _dp(f), n, _dp(pos0), _dp(mom0), _dp(mass), _dp(gamma),
                                C.byref(cp), _dp(lf), _dp(lp), _dp(lm), _dp(lam_pops), _dp(grad_f))
    if st != 0:
        raise ValueError("couple_adjoint: a wall reflection with p_z = 0 (sign not recoverable)")
    return lp, lm


def coupled_kinetic_energy(p: Params, pops0, force, pos0, mom0, mass, gamma, *, dt, n_substeps, nsteps, lo, hi):
    """L after nsteps of (couple, step) from pops0 and the free particles
    (pos0, mom0), with the force field (forward only; kT = 0)."""
    pops = np.ascontiguousarray(pops0, dtype=np.float64)
    pos, mom = np.array(pos0, dtype=np.float64), np.array(mom0, dtype=np.float64)
    for t in range(nsteps):
        pos, mom, facc, _ = couple(p, pops, pos, mom, mass, gamma, dt=dt, n_substeps=n_substeps, seed=0,
                                   force=force)
        pops = step(p, pops, facc if force is None else force + facc, t)
    rho, j, _ = moments(p, pops, force)
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    return float(0.5 * np.sum((j[(slice(None),) + sl] ** 2).sum(0) / rho[sl]))


def coupled_kinetic_energy_and_grad(p: Params, pops0, force, pos0, mom0, mass, gamma, *, dt, n_substeps,
                                    nsteps, lo, hi):
    """(L, dL/dforce, dL/dpos0, dL/dmom0) of coupled_kinetic_energy by the
    reverse pass: per step in reverse, the stream-collide adjoint (which gives
    dL/df of that step, f = force + spread impulses), then the coupling
    adjoint driven by that dL/df as dL/dfacc."""
    force = np.zeros((3, p.nz, p.ny, p.nx)) if force is None else np.ascontiguousarray(force, dtype=np.float64)
    pops = np.ascontiguousarray(pops0, dtype=np.float64)
    pos, mom = np.array(pos0, dtype=np.float64), np.array(mom0, dtype=np.float64)
    hist = []
    for t in range(nsteps):
        hist.append((pops, pos, mom))
        pos, mom, facc, _ = couple(p, pops, pos, mom, mass, gamma, dt=dt, n_substeps=n_substeps, seed=0,
                                   force=force)
        pops = step(p, pops, force + facc, t)
        hist[-1] = hist[-1] + (facc,)
    L, lam, g = kinetic_seed(p, pops, lo, hi, force)
    lpos, lmom = np.zeros_like(pos), np.zeros_like(mom)
    for t in range(nsteps - 1, -1, -1):
        pops_t, pos_t, mom_t, facc_t = hist[t]
        gstep = np.zeros((3, p.nz, p.ny, p.nx))
        lam, gstep = adjoint_step(p, pops_t, lam, force + facc_t, gstep)
        g += gstep
        lpos, lmom = couple_adjoint(p, pops_t, pos_t, mom_t, mass, gamma, dt=dt, n_substeps=n_substeps,
                                    lam_facc=gstep, lam_pos=lpos, lam_mom=lmom, lam_pops=lam, grad_f=g,
                                    force=force)
    return L, g, lpos, lmom


def effective_friction(kernel, offset, *, L=16, steps=1500, F=1e-4, a0=1.0, mass=1.0, n_substeps=10,
                       dt=0.1, check_every=500, gamma_visc=0.0):
    """The settling test of Sec. 4.6 on couple() and step(): one particle held
    at the node L/2 plus `offset` (it is put back there before every LB step,
    so it does not move on the grid) in a periodic L^3 box at kT = 0 with
    shear and bulk eigenvalue gamma_visc (Eq. (shearviscosity): nu = (1 + gamma)
    / (6 (1 - gamma)), eta = rho0 nu; 1/6 for 0), pulled along x by the
    constant force F; a uniform force density -F/L^3 on the fluid makes the
    net force zero.  The bare friction is Gamma = 6 pi eta a0.  In the
    steady state the force balance of Eq. (dragexperiment_particle_equation)
    gives the particle velocity U = F/Gamma + u0, u0 the velocity the coupling
    interpolates at the particle; then 1/a = 6 pi eta U / F (Stokes) and
    Eq. (aeffcorr) gives g from 1/(g b) = 1/a + 2.84/L - 1/a0 (b = 1).
    Returns dict(u0, u0_prev, U, a, g): u0_prev is u0 `check_every` steps
    before the end (for a convergence check)."""
    eta = (1.0 + gamma_visc) / (6.0 * (1.0 - gamma_visc))
    gamma = 6.0 * np.pi * eta * a0
    p = make_params((L, L, L), body_force=(-F / L ** 3, 0.0, 0.0), gamma_shear=gamma_visc,
                    gamma_bulk=gamma_visc)
    pops = equilibrium(p)
    r0 = np.array([[L / 2 + offset[0], L / 2 + offset[1], L / 2 + offset[2]]], dtype=np.float64)
    mom = np.zeros((1, 3))
    u0_prev = None
    for t in range(steps):
        if t == steps - check_every:
            u0_prev = interpolate(p, pops, r0, kernel=kernel)[0, 0]
        _, mom, facc, _ = couple(p, pops, r0, mom, mass, gamma, dt=dt, n_substeps=n_substeps, seed=0,
                                 kernel=kernel, fext=(F, 0.0, 0.0))
        pops = step(p, pops, facc, t)
    u0 = interpolate(p, pops, r0, kernel=kernel)[0, 0]
    U = F / gamma + u0
    a = F / (6.0 * np.pi * eta * U)
    g = 1.0 / (1.0 / a + 2.84 / L - 1.0 / a0)
    return dict(u0=u0, u0_prev=u0_prev, U=U, a=a, g=g)


def step_nodes(p: Params, pops, idx, force=None, step_index=0):
    """step() evaluated at the listed fluid nodes only (linear indices):
    returns (len(idx), 19) post-collision populations."""
    lib = _load()
    src = np.ascontiguousarray(pops, dtype=np.float64)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((ix.shape[0], 19))
    lib.ora_step_nodes(C.byref(p), _dp(src), _dp(f), int(step_index) & 0xffffffff, ix.shape[0],
                       ix.ctypes.data_as(C.POINTER(C.c_longlong)), _dp(out))
    return out


def exp_equilibrium(rho, u):
    """n^eq of Eq. (equildist_lagrange) for density rho and velocity u (19 values)."""
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(19)
    lib.ora_exp_equilibrium(float(rho), _dp(uu), _dp(out))
    return out


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def sphere_owner(p: Params, R, a):
    """Solid map (nz, ny, nx): index of the sphere of radius a whose centre
    lies closer than a to the node (minimum image), -1 for fluid."""
    lib = _load()
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    owner = np.empty((p.nz, p.ny, p.nx), dtype=np.int32)
    lib.ora_sphere_owner(C.byref(p), R.shape[0], _dp(R), float(a), _ip(owner))
    return owner


def sphere_velocity(zeta, m, U, F):
    """(U(t+h), U~) of Eq. EOMUsol and the consistency equation for
    m dU/dt = -zeta U + F, zeta a symmetric 3x3 matrix."""
    lib = _load()
    z = np.ascontiguousarray(zeta, dtype=np.float64).reshape(9)
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    un, ut = np.empty(3), np.empty(3)
    lib.ora_sphere_velocity(_dp(z), float(m), _dp(U), _dp(F), _dp(un), _dp(ut))
    return un, ut


def sphere_velocity6(Z, m, inertia, V, F):
    """(V(t+h), V~) for M dV/dt = -Z V + F, V = (U, Omega), M = diag(m, m, m,
    I, I, I), Z a symmetric 6x6 matrix (Eq. EOMUsol and the U~ equation)."""
    lib = _load()
    z = np.ascontiguousarray(Z, dtype=np.float64).reshape(36)
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    vn, vt = np.empty(6), np.empty(6)
    lib.ora_sphere_velocity6(_dp(z), float(m), float(inertia), _dp(V), _dp(F), _dp(vn), _dp(vt))
    return vn, vt


def step_spheres(p: Params, pops, owner, R, U, a, mass, *, omega=None, fc=None, force=None, step=0, forces=None):
    """One LB step with solid spheres (moving link bounce-back, Sec. 4.1-4.2).
    Returns (pops, owner, R, U, omega, U~, status); the inputs are not
    modified.  omega: angular velocities [n][3], or None for spheres that do
    not rotate (then omega is returned as None); mass: per sphere (<= 0 holds
    it fixed); fc: external forces [n][3]; forces: an (n, 6) float64 array
    that receives the hydrodynamic force and torque of the step."""
    lib = _load()
    src = np.ascontiguousarray(pops, dtype=np.float64)
    dst = np.empty_like(src)
    own = np.array(owner, dtype=np.int32, order="C", copy=True)
    R = np.array(R, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
    U = np.array(U, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
    n = R.shape[0]
    Om = None if omega is None else np.array(omega, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)))
    f = None if fc is None else np.ascontiguousarray(fc, dtype=np.float64).reshape(-1, 3)
    ff = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    ut = np.empty((max(n, 1), 3))
    st = lib.ora_step_spheres(C.byref(p), _dp(src), _dp(dst), _dp(ff), int(step) & 0xffffffff, _ip(own), n,
                              float(a), _dp(R), _dp(U), _dp(Om), _dp(m), _dp(f), _dp(ut), _dp(forces))
    return dst, own, R, U, Om, ut[:n], st


def interpolate(p: Params, pops, pos, force=None, kernel=2):
    """u at the positions with interpolation function phi_kernel (2, 3, 4)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    up = np.empty_like(pos)
    src = np.ascontiguousarray(pops, dtype=np.float64)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    lib.ora_interpolate_k(C.byref(p), int(kernel), _dp(src), _dp(f), pos.shape[0], _dp(pos), _dp(up))
    return up


def stencil(p: Params, pos3, kernel=2):
    """The K^3 stencil nodes (linear indices) and weights of phi_kernel."""
    lib = _load()
    pp = np.ascontiguousarray(pos3, dtype=np.float64)
    node = (C.c_longlong * 64)()
    wt = np.zeros(64)
    nq = lib.ora_stencil_k(C.byref(p), int(kernel), _dp(pp), node, _dp(wt))
    return np.array(list(node)[:nq], dtype=np.int64), wt[:nq]


def phi(kernel, v):
    """The one-dimensional interpolation function phi_kernel(v)."""
    return _load().ora_phi(int(kernel), float(v))


def _quadratic_only(p: Params):
    if p.equilibrium != 0:
        raise ValueError("the reverse pass is derived for the quadratic equilibrium")


def adjoint_step(p: Params, state, lam_in, force=None, grad_f=None):
    """dL/dn*(t) from dL/dn*(t+1) for the step leaving `state`; adds dL/df to grad_f."""
    _quadratic_only(p)
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float64)
    li = np.ascontiguousarray(lam_in, dtype=np.float64)
    lo = np.empty_like(st)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    if grad_f is None:
        grad_f = np.zeros((3, p.nz, p.ny, p.nx))
    lib.ora_adjoint_step(C.byref(p), _dp(st), _dp(f), _dp(li), _dp(lo), _dp(grad_f))
    return lo, grad_f


def kinetic_seed(p: Params, state, lo, hi, force=None, grad_f=None):
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.float64)
    lam = np.empty_like(st)
    f = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    if grad_f is None:
        grad_f = np.zeros((3, p.nz, p.ny, p.nx))
    L = lib.ora_kinetic_seed(C.byref(p), _dp(st), _dp(f), (C.c_int * 3)(*lo), (C.c_int * 3)(*hi), _dp(lam),
                             _dp(grad_f))
    return L, lam, grad_f


def kinetic_energy(p: Params, pops0, force, nsteps, lo, hi):
    """L after nsteps from pops0 with the force field (forward only)."""
    pops = run(p, pops0, nsteps, force)
    rho, j, _ = moments(p, pops, force)
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    return float(0.5 * np.sum((j[(slice(None),) + sl] ** 2).sum(0) / rho[sl]))


def kinetic_energy_and_grad(p: Params, pops0, force, nsteps, lo, hi, checkpoint_every=None):
    """(L, dL/dforce) by the reverse pass.  Every state is kept, or with
    checkpoint_every = K only every K-th one, the others being recomputed
    segment by segment (same results, less host memory)."""
    K = nsteps if checkpoint_every is None else int(checkpoint_every)
    ckpt = {}
    s = np.ascontiguousarray(pops0, dtype=np.float64)
    for t in range(nsteps):
        if t % K == 0:
            ckpt[t] = s
        s = step(p, s, force, t)
    L, lam, g = kinetic_seed(p, s, lo, hi, force)
    for t0 in sorted(ckpt, reverse=True):
        t1 = min(nsteps, t0 + K)
        states = [ckpt[t0]]
        for t in range(t0, t1 - 1):
            states.append(step(p, states[-1], force, t))
        for t in range(t1 - 1, t0 - 1, -1):
            lam, g = adjoint_step(p, states[t - t0], lam, force, g)
    return L, g


# The six transverse velocity modes at the smallest wave vector of each axis:
# (velocity component, axis of the wave vector) in the order the batched
# records use.
TRANSVERSE_MODES = ((0, 2), (1, 2), (1, 0), (2, 0), (2, 1), (0, 1))


def transverse_modes(p: Params, pops, force=None):
    """Fourier amplitudes u^_m = (1/V) sum_r u_a(r) exp(-2 pi i r_b / L_b) of
    the velocity u = j / rho (Sec. 3.7 j, of the pre-collision state as
    moments() defines it) for the six transverse pairs (a, b) of
    TRANSVERSE_MODES; the modes whose equal-time variance Sec. 3.6 fixes
    (kT / (rho0 V)) and whose decay per step is the shear eigenvalue of
    Sec. 3.4 (Eq. shearviscosity).  Returns complex [6]."""
    rho, j, _ = moments(p, pops, force)
    u = j / rho
    V = float(p.nx * p.ny * p.nz)
    L = (p.nx, p.ny, p.nz)
    out = np.zeros(6, dtype=np.complex128)
    for m, (a, b) in enumerate(TRANSVERSE_MODES):
        r = np.arange(L[b], dtype=np.float64)
        ph = np.exp(-2j * np.pi * r / L[b])
        shape = [1, 1, 1]
        shape[2 - b] = L[b]  # arrays are (nz, ny, nx)
        out[m] = np.sum(u[a] * ph.reshape(shape)) / V
    return out


def mode_autocorrelation(series, t_begin, t_end, max_lag):
    """C(tau) = < Re u^_m(t0 + tau) conj(u^_m(t0)) > over t0 in
    [t_begin, t_end - tau) and the modes m, for tau = 0 .. max_lag, of a
    series [T][6] of transverse_modes (the definition, looped)."""
    s = np.asarray(series)
    out = np.zeros(max_lag + 1)
    for tau in range(max_lag + 1):
        acc, cnt = 0.0, 0
        for t0 in range(t_begin, t_end - tau):
            for m in range(s.shape[1]):
                acc += (s[t0 + tau, m] * np.conj(s[t0, m])).real
                cnt += 1
        out[tau] = acc / cnt if cnt else 0.0
    return out
