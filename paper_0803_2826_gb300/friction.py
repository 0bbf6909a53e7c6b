"""Effective friction of a coupled point particle: the drag / settling test
of Sec. 4.5-4.6, run on the CUDA library.

The bare friction Gamma of the coupling is not the long-time friction a
particle shows: the flow its own force induces lowers it,
1/Gamma_eff = 1/Gamma + mu_inf (Eq. (effsize)), and mu_inf depends on the
interpolation function and, for a point particle, on where the particle
sits in its cell.  ``effective_friction`` measures it the way Sec. 4.6
describes: one particle held at a grid position (put back there before each
LB step, so that it does not move on the grid), pulled by a constant force F
along x in a periodic L^3 box at kT = 0, with a uniform force density
-F/L^3 on the fluid so that the net force is zero.  In the steady state the
force balance F = Gamma (U - u0) (Eq. (dragexperiment_particle_equation))
gives the particle velocity U from the velocity u0 that the coupling
interpolates; Stokes' law gives the radius a = F / (6 pi eta U), and Eq.
(aeffcorr) the size parameter g, 1/(g b) = 1/a + 2.84/L - 1/a0, which does
not depend on L.  A caller that wants a given Gamma_eff picks Gamma from it
(Sec. 4.5: keep Gamma_eff fixed when the lattice is refined).

Every step runs in the library: ``lb_couple_particles`` (with the constant
force in ``fext``) and ``lb_step``; this module only resets the position
buffer and reads u0 with ``lb_interpolate_phi``.

``python -m paper_0803_2826_gb300.friction`` runs the 56 grid positions of
the paper's settling figure, (i, j, k)/10 with 0 <= i <= j <= k <= 5, for
phi_2, phi_3 and phi_4 and prints g per position and its spread.
"""
from __future__ import annotations

import math

from . import lbfluct as L


def grid_positions():
    """The 56 offsets (i/10, j/10, k/10), 0 <= i <= j <= k <= 5."""
    return [(i / 10, j / 10, k / 10) for k in range(6) for j in range(k + 1) for i in range(j + 1)]


def effective_friction(kernel, offset, *, L_box=16, steps=1500, F=1e-4, a0=1.0, mass=1.0, n_substeps=10,
                       dt=0.1, check_every=500, device="cuda"):
    """The drag test for one particle at node L/2 + offset with interpolation
    function phi_kernel.  Returns dict(u0, u0_prev, U, a, g, gamma_eff):
    u0_prev is u0 ``check_every`` steps before the end (convergence check).
    eta = 1/6 (all relaxation eigenvalues 0); Gamma = 6 pi eta a0."""
    import torch
    eta = 1.0 / 6.0
    gamma = 6.0 * math.pi * eta * a0
    n = L_box
    lat = L.Lattice((n, n, n), device=device, body_force=(-F / n ** 3, 0.0, 0.0))
    try:
        lat.init_equilibrium()
        r0 = torch.tensor([[n / 2 + offset[0], n / 2 + offset[1], n / 2 + offset[2]]], dtype=torch.float64,
                          device=device)
        pos = r0.clone()
        mom = torch.zeros((1, 3), dtype=torch.float32, device=device)
        parts = L.particles(1, pos, mom, mass0=mass, gamma0=gamma)
        cp = L.couple_params(n_substeps=n_substeps, dt=dt, kernel=kernel, fext=(F, 0.0, 0.0))
        u = torch.empty((1, 3), dtype=torch.float32, device=device)
        u0_prev = None
        for t in range(steps):
            if t == steps - check_every:
                L.lb_interpolate_phi(lat.h, kernel, 1, r0, u)
                u0_prev = float(u[0, 0])
            pos.copy_(r0)
            cp.md_step0 = n_substeps * t
            L.lb_couple_particles(lat.h, parts, cp)
            L.lb_step(lat.h, 1)
        L.lb_interpolate_phi(lat.h, kernel, 1, r0, u)
        u0 = float(u[0, 0])
        st, bits = lat.sync()
        if bits:
            raise L.LBError(L.LB_EDEVICE, "device error word 0x%x" % bits)
    finally:
        lat.close()
    U = F / gamma + u0
    a = F / (6.0 * math.pi * eta * U)
    g = 1.0 / (1.0 / a + 2.84 / n - 1.0 / a0)
    return dict(u0=u0, u0_prev=u0_prev, U=U, a=a, g=g, gamma_eff=F / U)


def sweep(kernels=(2, 3, 4), L_box=32, steps=3000):
    """g at the 56 grid positions for each kernel: {kernel: [g, ...]}."""
    out = {}
    for k in kernels:
        out[k] = [effective_friction(k, off, L_box=L_box, steps=steps)["g"] for off in grid_positions()]
    return out


def main():
    import argparse
    import time
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args()
    t0 = time.perf_counter()
    res = sweep(L_box=args.L, steps=args.steps)
    secs = time.perf_counter() - t0
    offs = grid_positions()
    print("n  offset           " + "  ".join("g(phi_%d)" % k for k in res))
    for i, off in enumerate(offs):
        print("%-2d %-16s " % (i, "(%.1f,%.1f,%.1f)" % off) + "  ".join("%8.5f" % res[k][i] for k in res))
    for k, gs in res.items():
        mean = sum(gs) / len(gs)
        print("phi_%d: mean g %.5f, min %.5f, max %.5f, (max-min)/(2 mean) = %.4f"
              % (k, mean, min(gs), max(gs), (max(gs) - min(gs)) / (2 * mean)))
    print("L = %d, %d steps per position, %.1f s" % (args.L, args.steps, secs))


if __name__ == "__main__":
    main()
