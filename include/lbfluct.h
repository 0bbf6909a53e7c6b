/*
 * lbfluct.h -- C ABI of the GB300 (sm_103a) fluctuating D3Q19 lattice-Boltzmann
 * library with frictional point-particle coupling.
 *
 * Method: Duenweg & Ladd, "Lattice Boltzmann simulations of soft matter
 * systems" (arXiv 0803.2826).  Section numbers below refer to that paper:
 *   Sec. 3.3  D3Q19 equilibrium, Eq. (original_equil_distrib)
 *   Sec. 3.4  MRT collision in the Table 1 moment basis, Eq. (lco_update)
 *   Sec. 3.5  thermal noise on the non-conserved modes, Eq. (stochupdaterule1)
 *   Sec. 3.7  external forces (half-force velocity, Sigma), Eq. (moment_two_external_force)
 *   Sec. 4.1  link bounce-back, Eq. (MBB) with u_b = 0
 *   Sec. 4.5  force coupling and the Langevin integrator, Eq. (langevin_momentum_update)
 *   Sec. 4.6  linear interpolation, Eqs. (Delta), (2point)
 *   Sec. 2.1  Kremer-Grest WCA and FENE potentials, Eqs. (ulennardjones), (ufene)
 *
 * Conventions shared by every call
 *  - Lattice units b = h = 1, c_s^2 = 1/3, nodes at integer coordinates.
 *  - Velocity order: i = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 =
 *    (1,1,0),(1,-1,0),(-1,1,0),(-1,-1,0),(0,1,1),(0,1,-1),(0,-1,1),(0,-1,-1),
 *    (1,0,1),(1,0,-1),(-1,0,1),(-1,0,-1).
 *  - Node index s = x + nx*(y + ny*z).  Field arrays are structure-of-arrays:
 *    scalar [N], vector [3][N], stress [6][N] in the order xx,yy,zz,xy,yz,zx,
 *    populations [19][N]; N = nx*ny*nz.
 *  - The library's population buffers hold the POST-collision state n*_i(r)
 *    as deviations n_i - a_i rho0 (FP32), or as those deviations times
 *    pop_scale rounded to nearest-even FP16 / BF16.  One lb_step is "pull
 *    stream, then collide".  Plane i starts at byte offset
 *    i * lb_plane_pitch(p) * element size.
 *  - Every pointer argument named "device" must point to GPU memory of the
 *    current device; the library never frees caller memory (borrowed).
 *    Memory the library allocates itself (error word, reduction scratch,
 *    particle accumulators, neighbour lists) is released by lb_destroy.
 *  - Every call is asynchronous on the handle's stream unless it says it
 *    synchronises.  Device-side errors (a broken FENE bond, a neighbour-list
 *    overflow, non-finite sums, a batched-barrier timeout) are recorded in an
 *    error word and reported by the next synchronising call.
 *  - No call aborts or throws; every call returns an lb_status, and
 *    lb_last_error() gives a message for the last failure on this thread.
 */
#ifndef LBFLUCT_H
#define LBFLUCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_EINVAL = 1,        /* bad argument (size, null pointer, parameter range)  */
    LB_ENOMEM = 2,        /* a library-internal device allocation failed         */
    LB_ECUDA = 3,         /* a CUDA runtime call failed                          */
    LB_ENONFINITE = 4,    /* non-finite values detected in reduced moments       */
    LB_ETIMEOUT = 5,      /* a bounded device-side wait gave up                  */
    LB_EUNSUPPORTED = 6,  /* combination of options not supported                */
    LB_EDEVICE = 7        /* device error word set (bits returned by lb_sync)    */
} lb_status;

typedef enum { LB_F32 = 0, LB_F16 = 1, LB_BF16 = 2 } lb_dtype;

/* Device error-word bits (returned by lb_sync). */
#define LB_DERR_FENE_BROKEN   0x1u   /* a FENE bond reached r >= R0            */
#define LB_DERR_NLIST_FULL    0x2u   /* a particle had too many neighbours      */
#define LB_DERR_NONFINITE     0x4u   /* non-finite moment sum                   */
#define LB_DERR_BARRIER       0x8u   /* batched kernel: grid barrier timed out  */
#define LB_DERR_PARTICLE_RANGE 0x10u /* a particle position outside the box or not
                                        finite (its stencil was clamped)         */
#define LB_DERR_SPHERE        0x20u  /* spheres: a node claimed by two spheres, or
                                        a sphere moved more than one node a step */
#define LB_DERR_BOUNDS        0x40u  /* a library built with LB_DEBUG_BOUNDS found an
                                        element index outside its array (the access
                                        was skipped)                               */

#define LB_NSUMS 38  /* lb_moments sums: [0..18] sum_r dm_k, [19..37] sum_r dm_k^2 */

typedef struct {
    int nx, ny, nz;        /* box size in nodes; each >= 1 (>= 3 along z with walls)   */
    int dtype;             /* lb_dtype of the stored populations                     */
    int walls;             /* 0: periodic; 1: solid planes z = 0 and z = nz-1 with
                              link bounce-back (Sec. 4.1, Eq. (MBB), u_b = 0)          */
    int noise_rho0;        /* 0: noise amplitude sqrt(w_k mu rho) with the local rho;
                              1: with rho0 (Sec. 3.5, Eq. (normalized_mk))            */
    double rho0;           /* reference density (> 0)                               */
    double kT;             /* k_B T >= 0; mu = kT / c_s^2 (Sec. 3.5)                */
    double gamma_shear;    /* gamma_s, modes 5..9, |gamma| < 1 (Sec. 3.4)            */
    double gamma_bulk;     /* gamma_v, mode 4                                       */
    double gamma_odd;      /* gamma_3a = gamma_3b, kinetic modes 10..15             */
    double gamma_even;     /* gamma_4a = gamma_4b, kinetic modes 16..18             */
    double body_force[3];  /* uniform force density f added at every fluid node     */
    uint64_t seed;         /* Philox key of the fluid noise                          */
    uint32_t replica;      /* fourth Philox counter word (replica index)            */
    uint32_t equilibrium;  /* equilibrium of the collision: 0 the quadratic form of
                              Eq. (original_equil_distrib); 1 the exponential form of
                              Eq. (equildist_lagrange), the maximum-entropy populations
                              at given rho and j (Sec. 3.6) -- lb_step and lb_step_from
                              only (no step sums, reverse mode, batches or spheres;
                              couplings run in the serial order)                      */
    double pop_scale;      /* FP16/BF16 storage scale (0 selects 1024)              */
} lb_params;

typedef struct lb_handle lb_handle;

/* ---- sizes ------------------------------------------------------------- */

/* Elements per population plane (N rounded up to a multiple of 64). */
size_t lb_plane_pitch(const lb_params *p);
/* Bytes of one population buffer: 19 * lb_plane_pitch * element size. */
size_t lb_population_bytes(const lb_params *p);

/* ---- life cycle ---------------------------------------------------------- */

/* Create a handle over two caller-owned device population buffers (each
 * lb_population_bytes(p) bytes, 256-byte aligned) and an optional device
 * force-density field force[3][N] (FP32; NULL for none), added to
 * p->body_force at every step.  stream: a cudaStream_t (NULL = legacy default).
 * The handle starts with the state in pops_a and step counter 0.  Buffers are
 * not initialised: call lb_init_equilibrium or lb_set_populations.
 * Errors: LB_EINVAL (bad params / pointers), LB_ENOMEM, LB_ECUDA. */
lb_status lb_create(const lb_params *p, void *pops_a, void *pops_b, float *force,
                    void *stream, lb_handle **out);

/* Release library-owned memory; never touches the borrowed buffers.  NULL is a no-op. */
lb_status lb_destroy(lb_handle *h);

/* Message for the last failing call on this thread (never NULL). */
const char *lb_last_error(void);

/* Synchronise the handle's stream, read and clear the device error word.
 * Returns LB_EDEVICE (bits in *bits if non-NULL) when it was set. */
lb_status lb_sync(lb_handle *h, uint32_t *bits);

/* Step counter (the Philox "step" word of the next lb_step). */
lb_status lb_get_step(const lb_handle *h, uint32_t *step);
lb_status lb_set_step(lb_handle *h, uint32_t step);

/* Number of kernels this handle has launched so far (for launch accounting). */
lb_status lb_get_launch_count(const lb_handle *h, uint64_t *count);

/* Device pointer of the buffer that holds the current state, and of the other one. */
lb_status lb_state_buffers(const lb_handle *h, void **current, void **other);

/* ---- state ------------------------------------------------------------- */

/* Set the stored state to the equilibrium of Eq. (original_equil_distrib) for
 * device fields rho[N] and u[3][N] (FP64; either may be NULL: rho0, zero). */
lb_status lb_init_equilibrium(lb_handle *h, const double *rho, const double *u);

/* Copy raw populations n_i (device FP64 [19][N]) into / out of the stored
 * state, converting to / from the storage format.  With walls the solid
 * planes z = 0 and nz-1 hold no state: lb_get_populations reports the rest
 * state a_i rho0 there. */
lb_status lb_set_populations(lb_handle *h, const double *n);
lb_status lb_get_populations(const lb_handle *h, double *n);

/* ---- the LB step (hot path) ---------------------------------------------- */

/* Advance nsteps >= 0 steps.  Each step pulls n_i(r) = n*_i(r - c_i)
 * (Eq. (LBE); bounced back at walls), forms rho, j = sum n c + f/2,
 * u = j / rho (Eq. (special_choice_momentum_density)), relaxes the moments of
 * Table 1 (Eq. (lco_update), gamma_0..3 = 1), adds the force moments of
 * Sec. 3.7 and, for kT > 0, the noise sqrt(w_k mu rho)(1 - gamma_k^2)^(1/2) r_k
 * on modes 4..18 (Eqs. (stochupdaterule1), (detailedbalance1)), transforms
 * back (Eq. (back_transformation), q = a) and stores n*.  r_4..r_18 are the
 * first 15 Box-Muller Gaussians of Philox4x32-10 with key (seed lo, seed hi)
 * and counters (s, step, b, replica), b = 0..3.  f = body_force + force field
 * + the impulses spread by the last lb_couple_particles (applied once).
 * Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_step(lb_handle *h, int nsteps);

/* lb_step for nsteps >= 1 steps, whose last stream-collide launch also
 * accumulates the LB_NSUMS moment sums of lb_moments (sum over fluid nodes
 * of dm_k and dm_k^2, dm_k = sum_i e_ki (n_i - a_i rho0), Table 1) of the
 * state that last step starts from -- the values lb_moments(..., sums) would
 * give just before it -- into `sums` (device FP64 [LB_NSUMS]), without a
 * separate pass over the populations.  Per-block partial sums in library
 * scratch are reduced in a fixed order, so the result is reproducible
 * (it differs from lb_moments' in summation order only).  The paper has no
 * counterpart (a monitoring shortcut).  Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA;
 * non-finite sums set LB_DERR_NONFINITE. */
lb_status lb_step_sums(lb_handle *h, int nsteps, double *sums);

/* Hydrodynamic moments of the pre-collision state (pull of the stored state):
 * rho[N], j[3][N] = sum n c + f_ext/2, pi[6][N] = sum n c c (Eqs. (hmodes_beg)-
 * (hmodes_end)); f_ext = body_force + force field.  sums (device FP64
 * [LB_NSUMS]): sum over fluid nodes of dm_k and dm_k^2, dm_k = sum_i e_ki
 * (n_i - a_i rho0) with the basis of Table 1; computed by a deterministic
 * two-pass reduction in library scratch.  Any output may be NULL.  Solid
 * nodes give rho0 and zeros.  Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_moments(lb_handle *h, float *rho, float *j, float *pi, double *sums);

/* The sums of lb_moments (LB_NSUMS doubles into device `sums`) for the
 * state in the device population buffer `pops` (storage format and layout of
 * p), without a handle and without allocating anything.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * (a host application whose device memory another framework reserved up
 * front, or a monitoring loop that must not block on or fail in an allocation
 * mid-run), which also rules out lb_create.  Its reduction scratch is a
 * static 1.2 MiB device array that every GPU loading the library keeps until
 * exit.  Boxes of more than 2^28 nodes are rejected with LB_EINVAL.  The first
 * call on a device (and the first after its context changed, e.g. after
 * cudaDeviceReset) looks up that array's device address, so make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU (different streams or threads) race and must be
 * serialised by the caller.  stream: a cudaStream_t.  No force field is
 * involved (the sums use sum n c without f/2).  Errors: LB_EINVAL, LB_ECUDA,
 * LB_EUNSUPPORTED (device index >= 64). */
lb_status lb_moment_sums_static(const lb_params *p, const void *pops, double *sums, void *stream);

/* ---- point particles (Sec. 4.5, 4.6) ------------------------------------ */

typedef struct {
    int n;               /* number of particles (>= 0)                              */
    int reserved;        /* must be 0                                               */
    double *pos;         /* device [n][3], positions in [0, L); updated in place    */
    float *mom;          /* device [n][3], momenta; updated in place                */
    const float *mass;   /* device [n] or NULL (use mass0)                          */
    const float *gamma;  /* device [n] or NULL (use gamma0): friction Gamma         */
    double mass0, gamma0;
} lb_particles;

typedef struct {
    int n_substeps;      /* particle steps per LB step (>= 1)                        */
    int noise_kind;      /* 0: Gaussian theta; 1: three-point theta (Sec. 4.5)       */
    double dt;           /* particle time step in LB steps                           */
    uint64_t seed;       /* Philox key of the particle noise (domain 1)              */
    uint32_t md_step0;   /* Philox step word of the first sub-step                   */
    int chain_len;       /* > 1: particles k*chain_len..(k+1)*chain_len-1 are a FENE chain */
    int use_wca;         /* purely repulsive LJ between all pairs                    */
    int flags;           /* 0, or LB_COUPLE_* bits below                             */
    double eps, sigma;   /* WCA parameters                                           */
    double k_fene, r0;   /* FENE parameters                                          */
    double fext[3];      /* constant external force on every particle, added to F^c  */
                         /* (gravity, or the applied force F of the drag experiment  */
                         /* of Sec. 4.5); the fluid receives it only through the     */
                         /* friction; 0 for none                                     */
} lb_couple_params;

/* lb_couple_params.flags: run one kernel launch per sub-step instead of one
 * cooperative launch for the whole call (for callers that cannot guarantee
 * that the cooperative grid becomes co-resident, e.g. when other work shares
 * the GPU).  Results agree with the default path to FP32 rounding.  Without
 * the flag, that path is also taken when the particles do not fit one
 * co-resident grid. */
#define LB_COUPLE_PER_SUBSTEP 0x1

/* lb_couple_params.flags: run the coupling on a high-priority library stream
 * while the next lb_step updates every node without its impulses, then that
 * lb_step updates again, with the impulses, the nodes of the stencils the
 * particles visited (the update of a node depends only on the pre-step
 * state, its forces and the counter-based noise, so the result is the one a
 * single update with the impulses gives) and clears their impulses.  The
 * call returns with the coupling queued after all work on the handle's
 * stream; the next lb_step, or any other call on the handle, orders the
 * handle's stream after the coupling.  Until then the caller must not read
 * pos / mom itself (lb_couple_particles_async gives an event for that).  A call made while impulses of an earlier call still
 * wait for a step runs in the serial order (the flag is ignored). */
#define LB_COUPLE_OVERLAP 0x2

/* lb_couple_params.flags: interpolate and spread with the three-point
 * function phi_3 (Sec. 4.6, Eq. (3point)) or the four-point phi_4
 * (Eq. (4point)) instead of the linear phi_2: 27 or 64 nodes per particle
 * instead of 8.  Both satisfy the moment conditions C1-C3 (sum phi^2 = 1/2
 * and 3/8 wherever the particle is), so the friction a particle feels does
 * not depend on its position within a cell.  With walls a particle is kept
 * K/2 lattice units from the solid planes (K = 3 or 4, the stencil width;
 * 1 for phi_2), so nz must be at least K + 1.  Free particles take the
 * one-launch kernel, pair forces a cooperative kernel with each particle's
 * stencil velocities and impulse sums cached in shared memory (per-sub-step
 * kernels when its grid cannot be resident); at most one of the two bits may
 * be set; the reverse-mode entry points reject them. */
#define LB_COUPLE_PHI3 0x4
#define LB_COUPLE_PHI4 0x8

/* One LB step's worth of particle motion.  The fluid velocity
 * u = (sum n c + f_ext/2)/rho of the current state is held fixed; for each
 * sub-step: half drift; conservative forces F^c (FENE + WCA); u_p =
 * sum Delta(r - r_p) u(r) with Delta = phi_2 phi_2 phi_2 over 8 nodes (or
 * phi_3 / phi_4 over 27 / 64, see LB_COUPLE_PHI3); exact OU update
 * p' = C1 p + C2 (F^c + Gamma u_p) + C3 theta; the impulse of the drag and
 * random forces over the sub-step, J = p' - p - dt F^c (Eq. (ftotal); F^c,
 * fext included, is constant during the update), is spread as
 * -J Delta(r - r_p) into a library accumulator that the next
 * lb_step applies once; half drift.  Positions wrap periodically (x, y; z
 * without walls) or reflect specularly into z in [1, nz-2] with walls (the
 * band is K/2 from the solid planes for a stencil K nodes wide).
 * theta: Philox domain 1, counters (p, md_step0 + s, 1<<8, replica), key seed.
 * The caller's pos and mom are updated in place.  Errors: LB_EINVAL,
 * LB_ENOMEM, LB_ECUDA; broken bonds and neighbour overflow set device bits. */
lb_status lb_couple_particles(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp);

/* lb_couple_particles for callers that move the particle state with other
 * work, e.g. copies on a copy stream; either event may be NULL.
 * ready_event: a cudaEvent_t recorded after the work that wrote the
 * particle inputs (pos, mom, optional per-particle arrays).  With
 * LB_COUPLE_OVERLAP only the coupling, on the library stream, waits for it,
 * so the stream-collide launch of the next lb_step does not wait for the
 * copy; without it the handle's stream waits.
 * done_event: recorded where pos and mom hold this call's result (on the
 * library stream with LB_COUPLE_OVERLAP, else on the handle's stream; at
 * once for n = 0); a caller's stream that waits for it may read them before
 * the next lb_step, while the impulses still wait for that step.
 * The caller keeps the events alive until the work has used them.  Nothing is
 * recorded when the call fails.  Errors: those of lb_couple_particles. */
lb_status lb_couple_particles_async(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp,
                                    void *ready_event, void *done_event);

/* Interpolated fluid velocity u_p (device FP32 [n][3]) at device positions
 * pos[n][3] (Eq. (ufluid_discrete) with the linear stencil). */
lb_status lb_interpolate(lb_handle *h, int n, const double *pos, float *u_out);

/* The same with interpolation function phi_kernel, kernel = 2, 3 or 4
 * (Sec. 4.6, Eqs. (2point), (3point), (4point)); lb_interpolate is
 * kernel 2.  Positions must lie in the box.  Errors: LB_EINVAL. */
lb_status lb_interpolate_phi(lb_handle *h, int kernel, int n, const double *pos, float *u_out);

/* Kernel timers for profiling: after lb_set_timing(h, capacity) the library
 * records CUDA events around each stream-collide launch of lb_step (with
 * LB_COUPLE_OVERLAP: the update of all nodes, not the re-update of the
 * impulse nodes) and around the GPU work of each lb_couple_particles, on the
 * stream that work runs on, for the first `capacity` of each; capacity 0
 * stops and releases them.  lb_get_timing waits for the recorded work and
 * returns the summed milliseconds and the counts (any pointer may be NULL).
 * The paper has no counterpart.  Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA. */
lb_status lb_set_timing(lb_handle *h, int capacity);
lb_status lb_get_timing(lb_handle *h, double *ms_step, int *n_step, double *ms_couple, int *n_couple);

/* Copy the impulses the next lb_step will apply (device FP32 [3][N] out;
 * zeros when none are pending). */
lb_status lb_get_particle_forces(lb_handle *h, float *out);

/* ---- extended particles: solid spheres with moving bounce-back ------------- */

/* Spheres of one radius that translate and, with angular velocities, rotate
 * (Sec. 4.1 Eq. NodeVel; Sec. 4.2 writes the linear update, the rotational
 * one follows the same steps).  All pointers are device memory owned by the
 * caller. */
typedef struct {
    int n;                /* number of spheres (>= 0)                                */
    int reserved;         /* must be 0                                               */
    double radius;        /* a: a node closer than a to a centre is solid            */
    double *pos;          /* [n][3] centres R in [0, L), updated in place            */
    double *vel;          /* [n][3] velocities U, updated in place                   */
    const double *mass;   /* [n] or NULL (mass0); a mass <= 0 holds a sphere fixed:  */
                          /* R and U stay, its surface moves with U                   */
    double mass0;
    const double *force;  /* [n][3] external forces F^c, or NULL                     */
    double *omega;        /* [n][3] angular velocities, updated in place, or NULL    */
                          /* for spheres that do not rotate (moment of inertia       */
                          /* 2/5 m a^2; u_b = U + Omega x (r_b - R), Eq. NodeVel)    */
} lb_spheres;

/* Build the solid map of the spheres at their current centres (no exchange
 * with the fluid): call once before the first lb_step_spheres, and again
 * whenever the set of spheres changes.  Requires a periodic box (no walls)
 * and FP32 storage (LB_EUNSUPPORTED otherwise); spheres must not overlap
 * (LB_DERR_SPHERE).  The populations of solid nodes are ignored.  Errors:
 * LB_EINVAL, LB_EUNSUPPORTED, LB_ENOMEM, LB_ECUDA. */
lb_status lb_spheres_place(lb_handle *h, const lb_spheres *s);

/* One LB step with the spheres (h = 1; Sec. 4.1 Eq. (MBB), Sec. 4.2):
 *  1. R(t+h/2) = R + U/2 (Eq. EOMD-1); the solid map moves with the
 *     centres: a covered fluid node gives its momentum sum n c (and its
 *     moment about the centre) to its sphere, an uncovered node starts from
 *     n^eq(rho0, u) with u = U(t) (+ Omega(t) x (r - R)) and the sphere loses
 *     rho0 u;
 *  2. over the boundary links b (fluid node r, r + c_b solid):
 *     F0 = sum 2 n*_b c_b, zeta = (2 rho0 / c_s^2) sum a_b c_b c_b^T
 *     (Eqs. force0, zeta); with rotation also the torque and the coupled
 *     6 x 6 friction of g = (c_b, (r_b - R) x c_b), r_b = r + c_b/2;
 *  3. U(t+h) = e^-A U + zeta^-1 (1 - e^-A)(F0 + F^c), A = zeta / m
 *     (Eq. EOMUsol in zeta's eigenbasis), and U~ of the consistency
 *     equation, so that m (U(t+h) - U(t)) = F0 + F^c - zeta U~ (with
 *     rotation the same for (U, Omega) with the 6 x 6 friction and
 *     M = diag(m, m, m, I, I, I));
 *  4. stream and collide the fluid nodes; a population whose source node is
 *     solid returns as n_i(r) = n*_-i(r) + 2 a_i rho0 u_b.c_i / c_s^2 with
 *     u_b = U~ (+ Omega~ x (r_b - R)) (Eqs. MBB, NodeVel);
 *  5. R(t+h) = R(t+h/2) + U(t+h)/2 (Eq. EOMD-3).
 * Total momentum of fluid and spheres is conserved (plus the external
 * forces).  Sphere velocities must stay below one node per step.  Point
 * particles are not coupled in the same step (LB_EUNSUPPORTED while
 * impulses are pending).  Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ECUDA;
 * LB_DERR_SPHERE on the device. */
lb_status lb_step_spheres(lb_handle *h, const lb_spheres *s);

/* Copy the solid map (device int [N] out: sphere index or -1 for fluid). */
lb_status lb_get_solid_map(lb_handle *h, int *owner_out);

/* ---- reverse mode (deterministic runs, kT = 0) ------------------------------- */

/* One forward step from the state in `src` into `dst` (device buffers in the
 * storage format, lb_population_bytes each) with Philox step word `step`;
 * the handle's own state and step counter are not touched.  Used to
 * recompute states inside a checkpoint segment.  Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_step_from(lb_handle *h, const void *src, void *dst, uint32_t step);

/* Adjoint of one step (the transposed Jacobian of pull + collide, Sec. 3.4 and
 * 3.7, evaluated at the state `state` the step starts from): lambda_out =
 * dL/dstate_t from lambda_in = dL/dstate_{t+1} (device FP32, [19][pitch], the
 * population layout; entries of solid nodes must be zero and stay zero), and
 * dL/df of this step added into grad_force (device FP32 [3][N], may be NULL).
 * f = body_force + force field; particle impulses are not differentiated.
 * Requires kT = 0 (LB_EUNSUPPORTED otherwise).  Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_adjoint_step(lb_handle *h, const void *state, const float *lambda_in, float *lambda_out,
                          float *grad_force);

/* Seed of the reverse pass for L = 1/2 sum over nodes in [lo, hi) (host int[3]
 * each) of |j|^2 / rho, with j = sum n c + f/2 of the state pulled from
 * `state`: writes lambda_out = dL/dstate (FP32 [19][pitch]), adds dL/df into
 * grad_force (may be NULL) and stores L in *loss (device double). */
lb_status lb_adjoint_seed_kinetic(lb_handle *h, const void *state, const int lo[3], const int hi[3],
                                  float *lambda_out, float *grad_force, double *loss);

/* Forward half of the reverse pass of "advance nsteps, then L of the
 * sub-box" (L as in lb_adjoint_seed_kinetic): runs nsteps forward steps
 * from the current state (which advances, as lb_step would), keeping a
 * checkpoint every `checkpoint_every` steps, and at the final state forms L
 * (*loss, device double) and its seed dL/dstate.  The checkpoints, segment
 * buffers and adjoint buffers live in a device arena the handle owns: the
 * first call (or one needing more room) allocates it, later calls reuse it
 * without allocating, lb_destroy frees it.  Asynchronous on the handle's
 * stream.  Requires kT = 0.  Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ENOMEM,
 * LB_ECUDA. */
lb_status lb_adjoint_forward(lb_handle *h, int nsteps, int checkpoint_every, const int lo[3], const int hi[3],
                             double *loss);

/* Reverse half: walks the segments of the last lb_adjoint_forward backwards,
 * recomputing each segment's states from its checkpoint and applying
 * lb_adjoint_step (Sec. 3.4 and 3.7 transposed), and writes dL/d(force field)
 * into grad_force (device FP32 [3][N]; the field the handle was created
 * with).  Does not touch the handle's state, so the lattice may have moved
 * on.  Once per forward (another lb_adjoint_forward or
 * lb_adjoint_kinetic_coupled in between makes it LB_EINVAL).  Asynchronous,
 * no allocation.  Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ECUDA. */
lb_status lb_adjoint_backward(lb_handle *h, float *grad_force);

/* lb_adjoint_forward followed by lb_adjoint_backward: L into *loss and
 * dL/d(force field) into grad_force.  Errors: as those two. */
lb_status lb_adjoint_kinetic(lb_handle *h, int nsteps, int checkpoint_every, const int lo[3], const int hi[3],
                             float *grad_force, double *loss);

/* lb_adjoint_step for a step that also applied particle impulses: impulse
 * (device FP32 [3][pitch], the layout of the library's accumulator; NULL =
 * none) is added to f = body_force + force field.  grad_force receives
 * dL/df of the total f (so also dL/d(impulse)).  Requires kT = 0. */
lb_status lb_adjoint_step_impulse(lb_handle *h, const void *state, const float *impulse, const float *lambda_in,
                                  float *lambda_out, float *grad_force);

/* Reverse of one lb_couple_particles call (Sec. 4.5 with the stencil of
 * Eqs. (Delta), (2point)) for free particles at kT = 0 (chain_len <= 1, no
 * WCA; LB_EUNSUPPORTED otherwise; n_substeps <= 64).  Per particle the
 * sub-steps are replayed from `start` (the particle state before the call,
 * not modified) against the populations `state` (storage format) of that
 * step, then walked back: half drifts (with the sign flips of wall
 * reflections), the exact Ornstein-Uhlenbeck update, the spreading of
 * -J Delta and the interpolation of u.  lambda_facc: dL/d(impulse field)
 * of the step (device FP32 [3][N], e.g. grad_force of
 * lb_adjoint_step_impulse); lambda_pos / lambda_mom: device FP32 [n][3],
 * dL/d(state after the call) in, dL/d(state before it) out.  Adds dL/dstate
 * through u = (sum n c + f/2)/rho into lambda_pops (FP32 [19][pitch]) and
 * dL/d(force field) into grad_force ([3][N], may be NULL).
 * Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ENOMEM, LB_ECUDA. */
lb_status lb_adjoint_couple(lb_handle *h, const void *state, const lb_particles *start, const lb_couple_params *cp,
                            const float *lambda_facc, float *lambda_pos, float *lambda_mom, float *lambda_pops,
                            float *grad_force);

/* The reverse pass of "advance nsteps coupled steps (lb_couple_particles,
 * then lb_step) from the current state and the particles `parts`, then L of
 * the sub-box" (L as in lb_adjoint_seed_kinetic): the forward steps run as
 * usual (state and particles advance), with the populations and the
 * particle state kept every `checkpoint_every` steps; each segment is
 * recomputed (particle impulses into per-step buffers) and walked back with
 * lb_adjoint_step_impulse and lb_adjoint_couple.  Writes dL/d(force field)
 * (device FP32 [3][N]), dL/d(initial positions) and dL/d(initial momenta)
 * (device FP32 [n][3]) and L (*loss, device double).  Free particles at
 * kT = 0 only.  Temporaries come from the handle's reverse-mode arena (see
 * lb_adjoint_forward): allocated on the first call, reused after.
 * Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ENOMEM, LB_ECUDA. */
lb_status lb_adjoint_kinetic_coupled(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp, int nsteps,
                                     int checkpoint_every, const int lo[3], const int hi[3], float *grad_force,
                                     float *grad_pos, float *grad_mom, double *loss);

/* ---- batched replicas: one persistent launch over many boxes ---------------- */

/* Many independent periodic boxes (replicas) of different sizes advanced
 * together: replica r is the box per_replica[r] (its nx, ny, nz, seed and
 * replica counter word; dtype and all physics parameters must equal those of
 * replica 0; walls are not supported; each replica has fewer than 2^24 nodes).
 * Population buffer layout: replica r occupies 19 * lb_plane_pitch(&per_replica[r])
 * elements starting right after replica r-1, planes as for one box.  Every
 * replica follows exactly the single-box update of lb_step with its own
 * parameters, so replica r of a batch reproduces a single box created from
 * per_replica[r]. */
typedef struct lb_batch lb_batch;

/* Launch shape of the persistent kernel: threads per block, nodes per tile
 * (a run of consecutive nodes of one replica), blocks per SM; grid is an
 * output (resident blocks).  Chosen by lb_batch_autotune or set directly. */
typedef struct {
    int threads;
    int tile_nodes;
    int blocks_per_sm;
    int grid;
} lb_batch_config;

/* Bytes of one batch population buffer (0 on invalid parameters). */
size_t lb_batch_population_bytes(const lb_params *per_replica, int n);

/* Create a batch over two caller-owned device buffers of
 * lb_batch_population_bytes bytes (256-byte aligned).  The state starts in
 * pops_a at step 0.  Errors: LB_EINVAL, LB_EUNSUPPORTED, LB_ENOMEM, LB_ECUDA. */
lb_status lb_batch_create(const lb_params *per_replica, int n, void *pops_a, void *pops_b, void *stream,
                          lb_batch **out);
lb_status lb_batch_destroy(lb_batch *b);

/* Advance every replica nsteps steps in ONE cooperative persistent launch:
 * resident blocks take tiles in a strided order, then meet at a grid barrier
 * per step.  The barrier spins at most lb_batch_set_barrier_limit times
 * (default 2^22 polls) and then stops the run, which lb_batch_sync reports as
 * LB_ETIMEOUT.  use_graph != 0 records the launch in a CUDA graph (once per
 * nsteps value) and replays it.  Asynchronous. */
lb_status lb_batch_step(lb_batch *b, int nsteps, int use_graph);

/* Synchronise; report (and clear) the device error word: LB_ETIMEOUT after a
 * barrier timeout (the populations are then undefined), LB_EDEVICE else. */
lb_status lb_batch_sync(lb_batch *b, uint32_t *bits);

/* Time trial_steps steps for every launch shape of a small grid (threads
 * 128/256/512, tiles 512..8192 nodes, 1..8 blocks per SM) with CUDA events
 * and keep the fastest; the trial steps advance the state like lb_batch_step.
 * Synchronises.  Returns the chosen shape and its time per step. */
lb_status lb_batch_autotune(lb_batch *b, int trial_steps, lb_batch_config *chosen, double *best_ms_per_step);
lb_status lb_batch_set_config(lb_batch *b, const lb_batch_config *c);
lb_status lb_batch_get_config(const lb_batch *b, lb_batch_config *c);
lb_status lb_batch_set_barrier_limit(lb_batch *b, uint32_t spins);
lb_status lb_batch_get_step(const lb_batch *b, uint32_t *step);
lb_status lb_batch_get_launch_count(const lb_batch *b, uint64_t *count);

/* Transverse velocity modes of every replica, recorded by the batched run
 * (Sec. 3.6: in equilibrium each Fourier component of u has variance
 * kT / (rho0 V); Sec. 3.4, Eq. (shearviscosity): a transverse mode decays by
 * the shear eigenvalue of the linearised step per step).  From the next
 * lb_batch_step on, step t (counted from this call, t < capacity) adds to
 * device modes[r][t][0..11] (FP64, layout [n][capacity][12], caller-owned,
 * cleared here on the batch's stream) the sums over replica r's nodes of
 *   u_x e^{-i k_z z}, u_y e^{-i k_z z}, u_y e^{-i k_x x}, u_z e^{-i k_x x},
 *   u_z e^{-i k_y y}, u_x e^{-i k_y y}     (real part, then imaginary part),
 * k_b = 2 pi / L_b, u = (sum n c + f/2) / rho of the state that step
 * collides (its moments as lb_batch_moments defines them, taken inside the
 * step's own update; FP32 per tile, FP64 accumulation).  Steps past
 * capacity are not recorded.  modes = NULL stops recording.  Switching
 * recording on or off may change the grid (the configuration is re-applied
 * and a captured graph dropped), so call this after lb_batch_autotune; a
 * new buffer or capacity drops a captured graph; calling again with the same
 * buffer and capacity restarts the records at the next step and keeps the
 * graph (the start step lives in device memory).  The library allocates the
 * phase tables on the first call.
 * Errors: LB_EINVAL (capacity < 1, misaligned), LB_ENOMEM, LB_ECUDA. */
lb_status lb_batch_record_modes(lb_batch *b, double *modes, int capacity);

/* Per-replica autocorrelation of recorded modes (device modes as above with
 * the same capacity) into device acf[n][max_lag + 1] (FP64):
 *   acf[r][tau] = mean over t0 in [t_begin, t_end - tau) and the six modes of
 *                 Re u^(t0 + tau) conj(u^(t0)),   u^ = record / V_r,
 * the velocity autocorrelation whose equal-time value is kT / (rho0 V) and
 * whose decay is the shear eigenvalue per step.  Asynchronous on the batch's
 * stream.  Errors: LB_EINVAL (need 0 <= t_begin < t_end <= capacity and
 * 0 <= max_lag < t_end - t_begin), LB_ECUDA. */
lb_status lb_batch_mode_acf(lb_batch *b, const double *modes, int capacity, int t_begin, int t_end, int max_lag,
                            double *acf);

/* Per-replica state access and moments (replica = -1 in init: all replicas,
 * with rho / u then NULL); layouts as for one box of that replica's size. */
lb_status lb_batch_init_equilibrium(lb_batch *b, int replica, const double *rho, const double *u);
lb_status lb_batch_set_populations(lb_batch *b, int replica, const double *n);
lb_status lb_batch_get_populations(lb_batch *b, int replica, double *n);
lb_status lb_batch_moments(lb_batch *b, int replica, float *rho, float *j, float *pi, double *sums);

/* ---- noise streams (for verification) --------------------------------------- */

/* Raw Philox4x32-10 words and their Box-Muller Gaussians as the kernels draw
 * them (the noise source of Sec. 3.5 and Sec. 4.5).  For q = 0..count-1 and
 * block b = 0..nblocks-1 (nblocks 1..4) the counter is
 * (index0 + q, step, domain<<8 | b, replica) and the key (seed lo, seed hi).
 * words: device uint32 [count][nblocks][4]; gauss: device FP32 of the same
 * shape (or NULL), pairs (w0, w1) and (w2, w3) of a block mapped to
 * sqrt(-2 ln v1) (cos, sin)(2 pi v2) with v = (2 (w >> 9) + 1) 2^-24.
 * stream: a cudaStream_t.  Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_noise_words(uint64_t seed, uint32_t replica, uint32_t step, uint32_t domain, uint32_t index0,
                         int count, int nblocks, uint32_t *words, float *gauss, void *stream);

/* The Box-Muller map of lb_noise_words on caller-given word pairs: for
 * q < npairs, (gauss[2q], gauss[2q+1]) from (words[2q], words[2q+1]), as the
 * kernels compute it (for exhaustive checks over all 2^23 uniforms).
 * words: device uint32 [2 npairs]; gauss: device FP32 [2 npairs].
 * stream: a cudaStream_t.  Errors: LB_EINVAL, LB_ECUDA. */
lb_status lb_box_muller(const uint32_t *words, int npairs, float *gauss, void *stream);

/* ---- library information ------------------------------------------------- */

/* "lbfluct <version> sm_103a" */
const char *lb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBFLUCT_H */
