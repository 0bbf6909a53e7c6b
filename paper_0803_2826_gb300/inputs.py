"""Seeded synthetic inputs for the fluctuating D3Q19 lattice-Boltzmann workloads.

This module only draws and shapes numbers (velocity fields, random-walk chain
conformations, particle positions, sphere centres, replica sizes).  It holds none of the
lattice-Boltzmann arithmetic: both the CUDA library and the CPU oracle turn
these fields into populations themselves.  Every generator is deterministic in
its seed (numpy ``default_rng``).

Arrays follow the library's layouts: scalar fields ``(nz, ny, nx)``, vector
fields ``(3, nz, ny, nx)``, particle data ``(n, 3)``.
"""
from __future__ import annotations

import numpy as np

#: Edge lengths the batched-replica workload draws from.
REPLICA_EDGES = (16, 24, 32, 48, 64)


def shear_wave(shape, amplitude=0.01, wavelength=None):
    """Velocity field u_x = A sin(2 pi z / lambda), u_y = u_z = 0.

    shape = (nx, ny, nz); lambda defaults to nz (one period in the box);
    z is the integer node index.
    """
    nx, ny, nz = shape
    lam = nz if wavelength is None else wavelength
    z = np.arange(nz, dtype=np.float64)
    ux = amplitude * np.sin(2.0 * np.pi * z / lam)
    u = np.zeros((3, nz, ny, nx))
    u[0] = ux[:, None, None]
    return u


def gaussian_field(shape, ncomp, std, seed):
    """Independent N(0, std^2) values, shape (ncomp, nz, ny, nx)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, size=(ncomp, nz, ny, nx))


def standard_normal(shape, seed):
    """Independent N(0, 1) values of the given numpy shape."""
    return np.random.default_rng(seed).standard_normal(size=shape)


def random_walk_chains(n_chains, chain_len, box, *, bond=0.97, min_dist=1.0, seed=0,
                       max_tries=200):
    """Bead-spring chains as random walks of fixed bond length.

    Each chain starts at a uniform point of the periodic box ``box = (Lx, Ly,
    Lz)``; every further bead sits at distance ``bond`` from its predecessor in
    a uniformly random direction.  A step is redrawn (up to ``max_tries``
    times) when the new bead comes closer than ``min_dist`` to an earlier
    non-bonded bead, so that the first repulsive forces stay moderate; a walk
    that traps itself (no step found) is discarded and the chain regrown, so
    no two non-bonded beads are closer than ``min_dist``.  Returns float64
    positions (n_chains * chain_len, 3) in [0, L).
    """
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=np.float64)
    pos = np.zeros((n_chains * chain_len, 3))
    cell = 2.0
    grid = {}

    def key(p):
        return tuple((np.floor(p / cell).astype(np.int64)) % np.floor(L / cell).astype(np.int64))

    ncell = np.floor(L / cell).astype(np.int64)

    def too_close(p, skip):
        k = np.floor(p / cell).astype(np.int64)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = tuple((k + np.array([dx, dy, dz])) % ncell)
                    for j in grid.get(kk, ()):
                        if j == skip:
                            continue
                        d = p - pos[j]
                        d -= L * np.round(d / L)
                        if d @ d < min_dist * min_dist:
                            return True
        return False

    def place(p, i):
        pos[i] = p
        grid.setdefault(key(p), []).append(i)

    def grow(base):
        for t in range(max_tries):
            p0 = rng.uniform(0.0, 1.0, 3) * L
            if not too_close(p0, -1):
                break
        else:
            return 0
        place(p0, base)
        for b in range(1, chain_len):
            prev = pos[base + b - 1]
            for t in range(max_tries):
                v = rng.normal(size=3)
                v *= bond / np.linalg.norm(v)
                p = (prev + v) % L
                if not too_close(p, base + b - 1):
                    break
            else:
                return b
            place(p, base + b)
        return chain_len

    for c in range(n_chains):
        base = c * chain_len
        for attempt in range(max_tries):
            done = grow(base)
            if done == chain_len:
                break
            for i in range(base, base + done):  # take the trapped walk out again
                grid[key(pos[i])].remove(i)
        else:
            raise RuntimeError("random_walk_chains: could not place chain %d (box too crowded)" % c)
    return pos


def uniform_particles(n, box, seed, *, zrange=None):
    """n positions uniform in the box; with zrange=(lo, hi), z is uniform in it."""
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=np.float64)
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    if zrange is not None:
        pos[:, 2] = rng.uniform(zrange[0], zrange[1], size=n)
    return pos


def sphere_centres(n, box, radius, seed, *, gap=2.0, tries=100000):
    """n centres uniform in the periodic box, each at least 2 radius + gap
    from the others (minimum image), by random sequential addition; shape
    (n, 3).  Raises if the box cannot take them."""
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=np.float64)
    dmin = 2.0 * radius + gap
    out = np.empty((0, 3))
    for _ in range(tries):
        if out.shape[0] == n:
            return out
        c = rng.uniform(0.0, 1.0, 3) * L
        d = out - c
        d -= L * np.round(d / L)
        if out.shape[0] == 0 or (d * d).sum(1).min() >= dmin * dmin:
            out = np.vstack([out, c])
    if out.shape[0] == n:
        return out
    raise ValueError("could not place %d spheres of radius %g in box %s" % (n, radius, tuple(box)))


def maxwell_momenta(n, mass, kT, seed):
    """Momenta with independent N(0, m kT) components, shape (n, 3)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, np.sqrt(mass * kT), size=(n, 3)) if kT > 0 else np.zeros((n, 3))


def replica_edges(n_replicas=512, seed=7):
    """Edge lengths of the batched workload: uniform draws from REPLICA_EDGES."""
    idx = np.random.default_rng(seed).integers(0, len(REPLICA_EDGES), n_replicas)
    return [REPLICA_EDGES[i] for i in idx]


def poiseuille_velocity(shape, g, nu):
    """Analytic plane-Poiseuille profile between halfway walls at z = 0.5 and
    z = nz - 1.5, driven by a force density g (per unit mass density) along x:
    u_x(z) = g / (2 nu) (z - 0.5)(nz - 1.5 - z) in the fluid, 0 on the wall
    planes z = 0 and z = nz - 1.  Returns (3, nz, ny, nx)."""
    nx, ny, nz = shape
    z = np.arange(nz, dtype=np.float64)
    ux = g / (2.0 * nu) * (z - 0.5) * (nz - 1.5 - z)
    ux[0] = 0.0
    ux[-1] = 0.0
    u = np.zeros((3, nz, ny, nx))
    u[0] = ux[:, None, None]
    return u
