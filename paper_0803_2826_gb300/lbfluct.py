"""Thin Python binding of the C ABI in include/lbfluct.h.

Argument marshalling only: every step of the method runs in the CUDA library
liblbfluct.so.  Functions keep the C names (lb_create, lb_step, ...) and take
torch CUDA tensors (device memory) or raw integer device pointers; streams are
torch.cuda.Stream objects or raw cudaStream_t integers.  There is no CPU
fallback: if the library cannot be loaded, every call raises.

The ``Lattice`` class is a convenience owner of the two population buffers and
the handle; it allocates device memory with torch and passes pointers.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblbfluct.so")
BOUNDS_LIB_PATH = os.path.join(PKG, "liblbfluct_bounds.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_ETIMEOUT, LB_EUNSUPPORTED, LB_EDEVICE = range(8)
LB_F32, LB_F16, LB_BF16 = 0, 1, 2
LB_NSUMS = 38
LB_DERR_FENE_BROKEN, LB_DERR_NLIST_FULL, LB_DERR_NONFINITE, LB_DERR_BARRIER = 1, 2, 4, 8
LB_DERR_PARTICLE_RANGE = 16
LB_DERR_SPHERE = 32
LB_DERR_BOUNDS = 64
LB_COUPLE_PER_SUBSTEP, LB_COUPLE_OVERLAP, LB_COUPLE_PHI3, LB_COUPLE_PHI4 = 1, 2, 4, 8

STATUS_NAMES = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_ENONFINITE",
                5: "LB_ETIMEOUT", 6: "LB_EUNSUPPORTED", 7: "LB_EDEVICE"}

#: Symbols declared in include/lbfluct.h (checked by the ABI tests).
EXPORTS = (
    "lb_plane_pitch", "lb_population_bytes", "lb_create", "lb_destroy", "lb_last_error",
    "lb_sync", "lb_get_step", "lb_set_step", "lb_state_buffers", "lb_init_equilibrium",
    "lb_set_populations", "lb_get_populations", "lb_step", "lb_moments",
    "lb_couple_particles", "lb_couple_particles_async", "lb_interpolate", "lb_interpolate_phi", "lb_get_particle_forces",
    "lb_spheres_place", "lb_step_spheres", "lb_get_solid_map", "lb_noise_words", "lb_box_muller",
    "lb_set_timing", "lb_get_timing", "lb_step_sums", "lb_adjoint_step_impulse", "lb_adjoint_couple",
    "lb_adjoint_kinetic_coupled",
    "lb_get_launch_count", "lb_moment_sums_static", "lb_step_from", "lb_adjoint_step",
    "lb_adjoint_seed_kinetic", "lb_adjoint_kinetic", "lb_adjoint_forward", "lb_adjoint_backward",
    "lb_batch_population_bytes", "lb_batch_create", "lb_batch_destroy", "lb_batch_step", "lb_batch_sync",
    "lb_batch_autotune", "lb_batch_set_config", "lb_batch_get_config", "lb_batch_set_barrier_limit",
    "lb_batch_get_step", "lb_batch_get_launch_count", "lb_batch_init_equilibrium", "lb_batch_set_populations",
    "lb_batch_get_populations", "lb_batch_moments", "lb_batch_record_modes", "lb_batch_mode_acf", "lb_version",
)


class lb_batch_config(C.Structure):
    _fields_ = [("threads", C.c_int), ("tile_nodes", C.c_int), ("blocks_per_sm", C.c_int), ("grid", C.c_int)]


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class lb_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dtype", C.c_int), ("walls", C.c_int), ("noise_rho0", C.c_int),
        ("rho0", C.c_double), ("kT", C.c_double),
        ("gamma_shear", C.c_double), ("gamma_bulk", C.c_double),
        ("gamma_odd", C.c_double), ("gamma_even", C.c_double),
        ("body_force", C.c_double * 3),
        ("seed", C.c_uint64), ("replica", C.c_uint32), ("equilibrium", C.c_uint32),
        ("pop_scale", C.c_double),
    ]


class lb_particles(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("reserved", C.c_int),
        ("pos", C.c_void_p), ("mom", C.c_void_p), ("mass", C.c_void_p), ("gamma", C.c_void_p),
        ("mass0", C.c_double), ("gamma0", C.c_double),
    ]


class lb_spheres(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("reserved", C.c_int), ("radius", C.c_double),
        ("pos", C.c_void_p), ("vel", C.c_void_p), ("mass", C.c_void_p), ("mass0", C.c_double),
        ("force", C.c_void_p), ("omega", C.c_void_p),
    ]


class lb_couple_params(C.Structure):
    _fields_ = [
        ("n_substeps", C.c_int), ("noise_kind", C.c_int),
        ("dt", C.c_double), ("seed", C.c_uint64), ("md_step0", C.c_uint32),
        ("chain_len", C.c_int), ("use_wca", C.c_int), ("flags", C.c_int),
        ("eps", C.c_double), ("sigma", C.c_double), ("k_fene", C.c_double), ("r0", C.c_double),
        ("fext", C.c_double * 3),
    ]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblbfluct.so (building it first if it is missing); raise if
    impossible.  With LB_DEBUG_BOUNDS=1 in the environment the index-checking
    build liblbfluct_bounds.so is loaded instead (built on first use)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        bounds = os.environ.get("LB_DEBUG_BOUNDS", "") not in ("", "0")
        p = path or (BOUNDS_LIB_PATH if bounds else LIB_PATH)
        if not os.path.exists(p) or (bounds and path is None):
            from . import build as _build
            _build.build(debug_bounds=bounds)
        try:
            lib = C.CDLL(p)
        except OSError as e:  # no silent fallback
            raise RuntimeError("%s could not be loaded (%s); the CUDA library is required" % (os.path.basename(p), e))
        vp, i, u32, u64 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64
        P = C.POINTER(lb_params)
        H = C.c_void_p
        sig = {
            "lb_plane_pitch": (C.c_size_t, [P]),
            "lb_population_bytes": (C.c_size_t, [P]),
            "lb_create": (i, [P, vp, vp, vp, vp, C.POINTER(H)]),
            "lb_destroy": (i, [H]),
            "lb_last_error": (C.c_char_p, []),
            "lb_sync": (i, [H, C.POINTER(u32)]),
            "lb_get_step": (i, [H, C.POINTER(u32)]),
            "lb_set_step": (i, [H, u32]),
            "lb_state_buffers": (i, [H, C.POINTER(vp), C.POINTER(vp)]),
            "lb_init_equilibrium": (i, [H, vp, vp]),
            "lb_set_populations": (i, [H, vp]),
            "lb_get_populations": (i, [H, vp]),
            "lb_step": (i, [H, i]),
            "lb_moments": (i, [H, vp, vp, vp, vp]),
            "lb_couple_particles": (i, [H, C.POINTER(lb_particles), C.POINTER(lb_couple_params)]),
            "lb_couple_particles_async": (i, [H, C.POINTER(lb_particles), C.POINTER(lb_couple_params), vp, vp]),
            "lb_interpolate": (i, [H, i, vp, vp]),
            "lb_interpolate_phi": (i, [H, i, i, vp, vp]),
            "lb_get_particle_forces": (i, [H, vp]),
            "lb_spheres_place": (i, [H, C.POINTER(lb_spheres)]),
            "lb_step_spheres": (i, [H, C.POINTER(lb_spheres)]),
            "lb_get_solid_map": (i, [H, vp]),
            "lb_noise_words": (i, [u64, u32, u32, u32, u32, i, i, vp, vp, vp]),
            "lb_box_muller": (i, [vp, i, vp, vp]),
            "lb_set_timing": (i, [H, i]),
            "lb_step_sums": (i, [H, i, vp]),
            "lb_adjoint_step_impulse": (i, [H, vp, vp, vp, vp, vp]),
            "lb_adjoint_couple": (i, [H, vp, C.POINTER(lb_particles), C.POINTER(lb_couple_params), vp, vp, vp,
                                      vp, vp]),
            "lb_adjoint_kinetic_coupled": (i, [H, C.POINTER(lb_particles), C.POINTER(lb_couple_params), i, i,
                                               C.POINTER(i), C.POINTER(i), vp, vp, vp, vp]),
            "lb_get_timing": (i, [H, C.POINTER(C.c_double), C.POINTER(i), C.POINTER(C.c_double), C.POINTER(i)]),
            "lb_get_launch_count": (i, [H, C.POINTER(u64)]),
            "lb_moment_sums_static": (i, [P, vp, vp, vp]),
            "lb_step_from": (i, [H, vp, vp, u32]),
            "lb_adjoint_step": (i, [H, vp, vp, vp, vp]),
            "lb_adjoint_seed_kinetic": (i, [H, vp, C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp, vp]),
            "lb_adjoint_kinetic": (i, [H, i, i, C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp]),
            "lb_adjoint_forward": (i, [H, i, i, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]),
            "lb_adjoint_backward": (i, [H, vp]),
            "lb_batch_population_bytes": (C.c_size_t, [P, i]),
            "lb_batch_create": (i, [P, i, vp, vp, vp, C.POINTER(H)]),
            "lb_batch_destroy": (i, [H]),
            "lb_batch_step": (i, [H, i, i]),
            "lb_batch_sync": (i, [H, C.POINTER(u32)]),
            "lb_batch_autotune": (i, [H, i, C.POINTER(lb_batch_config), C.POINTER(C.c_double)]),
            "lb_batch_set_config": (i, [H, C.POINTER(lb_batch_config)]),
            "lb_batch_get_config": (i, [H, C.POINTER(lb_batch_config)]),
            "lb_batch_set_barrier_limit": (i, [H, u32]),
            "lb_batch_get_step": (i, [H, C.POINTER(u32)]),
            "lb_batch_get_launch_count": (i, [H, C.POINTER(u64)]),
            "lb_batch_init_equilibrium": (i, [H, i, vp, vp]),
            "lb_batch_set_populations": (i, [H, i, vp]),
            "lb_batch_get_populations": (i, [H, i, vp]),
            "lb_batch_moments": (i, [H, i, vp, vp, vp, vp]),
            "lb_batch_record_modes": (i, [H, vp, i]),
            "lb_batch_mode_acf": (i, [H, vp, i, i, i, i, vp]),
            "lb_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(x):
    """Device pointer of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor, got a %s tensor" % x.device)
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError("cannot take a device pointer of %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st):
    if st != LB_OK:
        raise LBError(st, load().lb_last_error().decode())


def make_params(shape, *, dtype=LB_F32, rho0=1.0, kT=0.0, gamma_shear=0.0, gamma_bulk=0.0,
                gamma_odd=0.0, gamma_even=0.0, body_force=(0.0, 0.0, 0.0), seed=0, replica=0,
                walls=False, noise_rho0=False, pop_scale=0.0, equilibrium=0) -> lb_params:
    """shape = (nx, ny, nz); equilibrium 1 selects the exponential equilibrium."""
    p = lb_params()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.dtype = int(dtype)
    p.walls = int(bool(walls))
    p.noise_rho0 = int(bool(noise_rho0))
    p.rho0, p.kT = float(rho0), float(kT)
    p.gamma_shear, p.gamma_bulk = float(gamma_shear), float(gamma_bulk)
    p.gamma_odd, p.gamma_even = float(gamma_odd), float(gamma_even)
    for d in range(3):
        p.body_force[d] = float(body_force[d])
    p.seed, p.replica, p.equilibrium = int(seed), int(replica), int(equilibrium)
    p.pop_scale = float(pop_scale)
    return p


# ---- one function per C entry point ------------------------------------------

def lb_plane_pitch(p: lb_params) -> int:
    return load().lb_plane_pitch(C.byref(p))


def lb_population_bytes(p: lb_params) -> int:
    return load().lb_population_bytes(C.byref(p))


def lb_create(p: lb_params, pops_a, pops_b, force=None, stream=None):
    h = C.c_void_p()
    _check(load().lb_create(C.byref(p), _ptr(pops_a), _ptr(pops_b), _ptr(force), _stream(stream),
                            C.byref(h)))
    return h


def lb_destroy(h):
    _check(load().lb_destroy(h))


def lb_last_error() -> str:
    return load().lb_last_error().decode()


def lb_sync(h, raise_on_error=True):
    bits = C.c_uint32(0)
    st = load().lb_sync(h, C.byref(bits))
    if raise_on_error:
        _check(st)
    return st, bits.value


def lb_get_step(h) -> int:
    v = C.c_uint32()
    _check(load().lb_get_step(h, C.byref(v)))
    return v.value


def lb_set_step(h, step: int):
    _check(load().lb_set_step(h, int(step) & 0xffffffff))


def lb_state_buffers(h):
    cur, oth = C.c_void_p(), C.c_void_p()
    _check(load().lb_state_buffers(h, C.byref(cur), C.byref(oth)))
    return cur.value, oth.value


def lb_init_equilibrium(h, rho=None, u=None):
    _check(load().lb_init_equilibrium(h, _ptr(rho), _ptr(u)))


def lb_set_populations(h, n):
    _check(load().lb_set_populations(h, _ptr(n)))


def lb_get_populations(h, n):
    _check(load().lb_get_populations(h, _ptr(n)))


def lb_step(h, nsteps=1):
    _check(load().lb_step(h, int(nsteps)))


def lb_moments(h, rho=None, j=None, pi=None, sums=None):
    _check(load().lb_moments(h, _ptr(rho), _ptr(j), _ptr(pi), _ptr(sums)))


def lb_couple_particles(h, parts: lb_particles, cp: lb_couple_params):
    _check(load().lb_couple_particles(h, C.byref(parts), C.byref(cp)))


def lb_couple_particles_async(h, parts: lb_particles, cp: lb_couple_params, ready_event=None, done_event=None):
    """ready_event: a recorded torch.cuda.Event (or a raw cudaEvent_t) after
    the work that wrote the particle inputs; done_event: a torch.cuda.Event
    (or raw cudaEvent_t) that the call records once pos / mom hold its
    result.  Either may be None.  torch creates an event's CUDA handle at its
    first record: an event never recorded is first recorded on the current
    stream (for ready_event: the inputs are taken as ready there)."""
    def raw(ev):
        if ev is None or isinstance(ev, int):
            return ev
        if ev.cuda_event == 0:  # torch creates its events lazily
            import torch
            ev.record(torch.cuda.current_stream())
        return ev.cuda_event
    _check(load().lb_couple_particles_async(h, C.byref(parts), C.byref(cp), raw(ready_event), raw(done_event)))


def lb_interpolate(h, n, pos, u_out):
    _check(load().lb_interpolate(h, int(n), _ptr(pos), _ptr(u_out)))


def lb_interpolate_phi(h, kernel, n, pos, u_out):
    _check(load().lb_interpolate_phi(h, int(kernel), int(n), _ptr(pos), _ptr(u_out)))


def lb_get_particle_forces(h, out):
    _check(load().lb_get_particle_forces(h, _ptr(out)))


def spheres(n, pos, vel, radius, *, mass=None, mass0=1.0, force=None, omega=None) -> lb_spheres:
    """The sphere set the library updates in place (pos, vel, omega: device
    FP64 [n][3], omega None for spheres that do not rotate; mass: FP64 [n] or
    None; force: FP64 [n][3] or None); the struct keeps the tensors alive."""
    s = lb_spheres()
    s.n, s.reserved, s.radius = int(n), 0, float(radius)
    s.pos, s.vel, s.mass, s.force = _ptr(pos), _ptr(vel), _ptr(mass), _ptr(force)
    s.omega = _ptr(omega)
    s.mass0 = float(mass0)
    s._arrays = (pos, vel, mass, force, omega)
    return s


def lb_spheres_place(h, s):
    _check(load().lb_spheres_place(h, C.byref(s)))


def lb_step_spheres(h, s):
    _check(load().lb_step_spheres(h, C.byref(s)))


def lb_get_solid_map(h, out):
    _check(load().lb_get_solid_map(h, _ptr(out)))


def lb_noise_words(seed, replica, step, domain, index0, count, nblocks, words, gauss=None, stream=None):
    _check(load().lb_noise_words(int(seed), int(replica), int(step), int(domain), int(index0), int(count),
                                 int(nblocks), _ptr(words), _ptr(gauss), _stream(stream)))


def lb_box_muller(words, npairs, gauss, stream=None):
    _check(load().lb_box_muller(_ptr(words), int(npairs), _ptr(gauss), _stream(stream)))


def lb_adjoint_step_impulse(h, state, impulse, lam_in, lam_out, grad_force=None):
    _check(load().lb_adjoint_step_impulse(h, _ptr(state), _ptr(impulse), _ptr(lam_in), _ptr(lam_out),
                                          _ptr(grad_force)))


def lb_adjoint_couple(h, state, start, cp, lam_facc, lam_pos, lam_mom, lam_pops, grad_force=None):
    _check(load().lb_adjoint_couple(h, _ptr(state), C.byref(start), C.byref(cp), _ptr(lam_facc), _ptr(lam_pos),
                                    _ptr(lam_mom), _ptr(lam_pops), _ptr(grad_force)))


def lb_adjoint_kinetic_coupled(h, parts, cp, nsteps, checkpoint_every, lo, hi, grad_force, grad_pos, grad_mom,
                               loss):
    L3 = C.c_int * 3
    _check(load().lb_adjoint_kinetic_coupled(h, C.byref(parts), C.byref(cp), int(nsteps), int(checkpoint_every),
                                             L3(*lo), L3(*hi), _ptr(grad_force), _ptr(grad_pos), _ptr(grad_mom),
                                             _ptr(loss)))


def lb_step_sums(h, nsteps, sums):
    _check(load().lb_step_sums(h, int(nsteps), _ptr(sums)))


def lb_set_timing(h, capacity):
    _check(load().lb_set_timing(h, int(capacity)))


def lb_get_timing(h):
    """(ms summed over stream-collide launches, their count, ms over coupling calls, their count)."""
    a, b = C.c_double(), C.c_double()
    na, nb = C.c_int(), C.c_int()
    _check(load().lb_get_timing(h, C.byref(a), C.byref(na), C.byref(b), C.byref(nb)))
    return a.value, na.value, b.value, nb.value


def lb_get_launch_count(h) -> int:
    v = C.c_uint64()
    _check(load().lb_get_launch_count(h, C.byref(v)))
    return v.value


def lb_moment_sums_static(p: lb_params, pops, sums, stream=None):
    """Moment sums of a population buffer without a handle and without any
    device allocation (see the header for who needs this)."""
    _check(load().lb_moment_sums_static(C.byref(p), _ptr(pops), _ptr(sums), _stream(stream)))


def lb_step_from(h, src, dst, step):
    _check(load().lb_step_from(h, _ptr(src), _ptr(dst), int(step) & 0xffffffff))


def lb_adjoint_step(h, state, lambda_in, lambda_out, grad_force=None):
    _check(load().lb_adjoint_step(h, _ptr(state), _ptr(lambda_in), _ptr(lambda_out), _ptr(grad_force)))


def _int3(v):
    return (C.c_int * 3)(*[int(x) for x in v])


def lb_adjoint_seed_kinetic(h, state, lo, hi, lambda_out, grad_force, loss):
    _check(load().lb_adjoint_seed_kinetic(h, _ptr(state), _int3(lo), _int3(hi), _ptr(lambda_out),
                                          _ptr(grad_force), _ptr(loss)))


def lb_adjoint_kinetic(h, nsteps, checkpoint_every, lo, hi, grad_force, loss):
    _check(load().lb_adjoint_kinetic(h, int(nsteps), int(checkpoint_every), _int3(lo), _int3(hi),
                                     _ptr(grad_force), _ptr(loss)))


def lb_adjoint_forward(h, nsteps, checkpoint_every, lo, hi, loss):
    _check(load().lb_adjoint_forward(h, int(nsteps), int(checkpoint_every), _int3(lo), _int3(hi), _ptr(loss)))


def lb_adjoint_backward(h, grad_force):
    _check(load().lb_adjoint_backward(h, _ptr(grad_force)))


def _params_array(plist):
    arr = (lb_params * len(plist))()
    for k, p in enumerate(plist):
        arr[k] = p
    return arr


def lb_batch_population_bytes(plist) -> int:
    return load().lb_batch_population_bytes(_params_array(plist), len(plist))


def lb_batch_create(plist, pops_a, pops_b, stream=None):
    b = C.c_void_p()
    _check(load().lb_batch_create(_params_array(plist), len(plist), _ptr(pops_a), _ptr(pops_b), _stream(stream),
                                  C.byref(b)))
    return b


def lb_batch_destroy(b):
    _check(load().lb_batch_destroy(b))


def lb_batch_step(b, nsteps, use_graph=True):
    _check(load().lb_batch_step(b, int(nsteps), int(bool(use_graph))))


def lb_batch_sync(b, raise_on_error=True):
    bits = C.c_uint32(0)
    st = load().lb_batch_sync(b, C.byref(bits))
    if raise_on_error:
        _check(st)
    return st, bits.value


def lb_batch_autotune(b, trial_steps=5):
    cfg = lb_batch_config()
    ms = C.c_double()
    _check(load().lb_batch_autotune(b, int(trial_steps), C.byref(cfg), C.byref(ms)))
    return cfg, ms.value


def lb_batch_set_config(b, threads, tile_nodes, blocks_per_sm):
    cfg = lb_batch_config(int(threads), int(tile_nodes), int(blocks_per_sm), 0)
    _check(load().lb_batch_set_config(b, C.byref(cfg)))


def lb_batch_get_config(b):
    cfg = lb_batch_config()
    _check(load().lb_batch_get_config(b, C.byref(cfg)))
    return cfg


def lb_batch_set_barrier_limit(b, spins):
    _check(load().lb_batch_set_barrier_limit(b, int(spins)))


def lb_batch_get_step(b) -> int:
    v = C.c_uint32()
    _check(load().lb_batch_get_step(b, C.byref(v)))
    return v.value


def lb_batch_get_launch_count(b) -> int:
    v = C.c_uint64()
    _check(load().lb_batch_get_launch_count(b, C.byref(v)))
    return v.value


def lb_batch_init_equilibrium(b, replica=-1, rho=None, u=None):
    _check(load().lb_batch_init_equilibrium(b, int(replica), _ptr(rho), _ptr(u)))


def lb_batch_set_populations(b, replica, n):
    _check(load().lb_batch_set_populations(b, int(replica), _ptr(n)))


def lb_batch_get_populations(b, replica, n):
    _check(load().lb_batch_get_populations(b, int(replica), _ptr(n)))


def lb_batch_moments(b, replica, rho=None, j=None, pi=None, sums=None):
    _check(load().lb_batch_moments(b, int(replica), _ptr(rho), _ptr(j), _ptr(pi), _ptr(sums)))


def lb_batch_record_modes(b, modes, capacity):
    """modes: device float64 [n][capacity][12] (or None to stop recording)."""
    _check(load().lb_batch_record_modes(b, _ptr(modes), int(capacity)))


def lb_batch_mode_acf(b, modes, capacity, t_begin, t_end, max_lag, acf):
    """acf: device float64 [n][max_lag + 1]."""
    _check(load().lb_batch_mode_acf(b, _ptr(modes), int(capacity), int(t_begin), int(t_end), int(max_lag),
                                    _ptr(acf)))


class Batch:
    """Owns the two batch population buffers (torch uint8 device tensors) and a batch handle."""

    def __init__(self, shapes, *, seeds=None, replicas=None, device="cuda", stream=None, **kw):
        import torch
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        n = len(self.shapes)
        seeds = list(range(n)) if seeds is None else list(seeds)
        replicas = list(range(n)) if replicas is None else list(replicas)
        self.params = [make_params(s, seed=seeds[k], replica=replicas[k], **kw) for k, s in enumerate(self.shapes)]
        nbytes = lb_batch_population_bytes(self.params)
        if nbytes == 0:
            raise LBError(LB_EINVAL, lb_last_error())
        self.device = torch.device(device)
        self._bufs = [torch.empty(nbytes, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.b = lb_batch_create(self.params, self._bufs[0], self._bufs[1], stream)

    def close(self):
        if getattr(self, "b", None) is not None:
            lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_populations(self, r):
        import torch
        nx, ny, nz = self.shapes[r]
        out = torch.empty((19, nz, ny, nx), dtype=torch.float64, device=self.device)
        lb_batch_get_populations(self.b, r, out)
        return out

    def moments(self, r):
        import torch
        nx, ny, nz = self.shapes[r]
        rho = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        j = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=self.device)
        lb_batch_moments(self.b, r, rho, j)
        return rho, j


def lb_version() -> str:
    return load().lb_version().decode()


# ---- convenience owner ---------------------------------------------------------

class Lattice:
    """Owns two population buffers (torch uint8 device tensors) and a handle."""

    def __init__(self, shape, *, device="cuda", stream=None, force=None, **kw):
        import torch
        self.params = make_params(shape, **kw)
        self.shape = tuple(int(v) for v in shape)
        self.n_nodes = self.shape[0] * self.shape[1] * self.shape[2]
        nbytes = lb_population_bytes(self.params)
        if nbytes == 0:
            raise LBError(LB_EINVAL, lb_last_error())
        self.device = torch.device(device)
        self._bufs = [torch.empty(nbytes, dtype=torch.uint8, device=self.device) for _ in range(2)]
        self.force = force
        self.stream = stream
        self.h = lb_create(self.params, self._bufs[0], self._bufs[1], force, stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state
    def init_equilibrium(self, rho=None, u=None):
        lb_init_equilibrium(self.h, rho, u)

    def set_populations(self, n):
        lb_set_populations(self.h, n)

    def get_populations(self):
        import torch
        n = torch.empty((19,) + self.shape[::-1], dtype=torch.float64, device=self.device)
        lb_get_populations(self.h, n)
        return n

    def step(self, nsteps=1):
        lb_step(self.h, nsteps)

    def moments(self, want_rho=True, want_j=True, want_pi=True, want_sums=False):
        import torch
        sh = self.shape[::-1]
        rho = torch.empty(sh, dtype=torch.float32, device=self.device) if want_rho else None
        j = torch.empty((3,) + sh, dtype=torch.float32, device=self.device) if want_j else None
        pi = torch.empty((6,) + sh, dtype=torch.float32, device=self.device) if want_pi else None
        sums = torch.empty(LB_NSUMS, dtype=torch.float64, device=self.device) if want_sums else None
        lb_moments(self.h, rho, j, pi, sums)
        return rho, j, pi, sums

    def sync(self):
        return lb_sync(self.h)

    @property
    def step_index(self):
        return lb_get_step(self.h)

    @step_index.setter
    def step_index(self, v):
        lb_set_step(self.h, v)


def particles(n, pos, mom, mass=None, gamma=None, mass0=1.0, gamma0=1.0) -> lb_particles:
    """The particle set the library updates in place; the struct keeps the
    tensors alive (it holds only their device pointers otherwise)."""
    s = lb_particles()
    s.n, s.reserved = int(n), 0
    s.pos, s.mom = _ptr(pos), _ptr(mom)
    s.mass, s.gamma = _ptr(mass), _ptr(gamma)
    s.mass0, s.gamma0 = float(mass0), float(gamma0)
    s._arrays = (pos, mom, mass, gamma)
    return s


def couple_params(*, n_substeps, dt, seed=0, md_step0=0, noise_kind=0, chain_len=0, use_wca=False,
                  eps=0.0, sigma=1.0, k_fene=0.0, r0=1.5, per_substep=False,
                  overlap=False, kernel=2, fext=(0.0, 0.0, 0.0)) -> lb_couple_params:
    """kernel: interpolation function phi_2 (default), phi_3 or phi_4;
    fext: constant external force on every particle."""
    if kernel not in (2, 3, 4):
        raise ValueError("kernel must be 2, 3 or 4")
    c = lb_couple_params()
    c.n_substeps, c.noise_kind, c.dt = int(n_substeps), int(noise_kind), float(dt)
    c.seed, c.md_step0 = int(seed), int(md_step0) & 0xffffffff
    c.chain_len, c.use_wca = int(chain_len), int(bool(use_wca))
    c.flags = ((LB_COUPLE_PER_SUBSTEP if per_substep else 0) | (LB_COUPLE_OVERLAP if overlap else 0) |
               {2: 0, 3: LB_COUPLE_PHI3, 4: LB_COUPLE_PHI4}[kernel])
    c.eps, c.sigma, c.k_fene, c.r0 = float(eps), float(sigma), float(k_fene), float(r0)
    for k in range(3):
        c.fext[k] = float(fext[k])
    return c
