// lbf_internal.h -- handle layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "d3q19.cuh"
#include "lbfluct.h"
#include "step_args.h"

namespace lbi {

struct Particles;  // defined in particles.cu

// NVTX range around a host call (visible to profilers that attach an NVTX
// tool; a no-op otherwise, the header-only NVTX loads no library by itself).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace lbi

struct lb_handle {
    lb_params p;
    size_t n_nodes;
    size_t pitch;
    size_t elem;          // bytes per stored population value
    void *pops[2];        // borrowed
    int cur;              // pops[cur] holds the current state
    float *force;         // borrowed, nullable
    cudaStream_t stream;
    uint32_t step;
    // library-owned
    unsigned int *d_err;  // device error word
    double *d_partials;   // reduction scratch [nblocks][LB_NSUMS]
    int red_blocks;
    float *facc;          // particle impulse accumulator [3][pitch]
    int facc_dirty;       // facc holds impulses the next lb_step applies
    int facc_stale;       // facc holds applied impulses not yet cleared
    uint64_t launches;    // kernels launched through this handle
    lbi::Particles *parts;
    // an overlapped coupling (LB_COUPLE_OVERLAP) runs on `aux` while the next
    // lb_step updates all nodes without its impulses, then re-updates the
    // nodes of its stencil records with them
    cudaStream_t aux;     // high-priority stream, created on first use
    cudaEvent_t ev_main, ev_couple;
    int overlap_pending;  // a coupling on aux the next lb_step (or any other call) joins
    const int *patch_rec; // its stencil records [patch_nsub][patch_n]
    int patch_n, patch_nsub;
    int patch_span;       // nodes per axis around a recorded cell: 2 (phi_2) or 4 (phi_3, phi_4)
    unsigned int *claim;  // [n_nodes] tag of the last re-update of each node
    float *lam_u;         // [3][pitch] dL/du at the nodes (coupling reverse pass), kept zero between calls
    unsigned int claim_tag;
    float *sc_partials;   // lb_step_sums: [blocks][38] per-block sums, then reduction scratch
    size_t sc_partials_len;
    // kernel timers (lb_set_timing): event pairs around stream-collide
    // launches [0] and coupling calls [1]
    int timer_cap;
    int timer_n[2];
    cudaEvent_t *timer_ev[2];  // [2 * timer_cap] each
    // solid spheres (lb_spheres_place / lb_step_spheres)
    int *sph_owner;       // [n_nodes] sphere index or -1
    float *sph_acc;       // [sph_cap][12]: F0 (3), covering momentum (3), zeta (6)
    double *sph_rh;       // [sph_cap][3] half-step centres
    float4 *sph_ut;       // [sph_cap] U~
    float4 *sph_uw;       // [sph_cap] Omega~ (0 for spheres that do not rotate)
    int *sph_list;        // near fluid nodes of the current step (linear indices)
    size_t sph_list_cap;
    unsigned int *sph_count;  // entries in sph_list
    int sph_cap;
    int sph_n;            // spheres of the current solid map (-1: none placed)
    double sph_a;
    // reverse mode: one device arena for the checkpoints, segment states and
    // adjoint buffers of lb_adjoint_forward / _backward / _kinetic_coupled,
    // grown on demand and kept until lb_destroy
    char *arena;
    size_t arena_bytes;
    // the run lb_adjoint_forward checkpointed (for lb_adjoint_backward)
    int adj_ready;        // 1 from a forward until its backward (or another reverse-mode driver)
    int adj_nsteps, adj_K;
    uint32_t adj_step0;
};

namespace lbi {

void set_error(const char *fmt, ...);
lb_status cuda_fail(const char *what, cudaError_t e);
StepArgs make_args(const lb_handle *h);
int device_sm_count();

// stream_collide.cu
cudaError_t launch_stream_collide(const lb_handle *h, const void *src, void *dst, const float *facc);
// exp_eq.cu: the update with the exponential equilibrium (lb_params.equilibrium = 1)
cudaError_t launch_stream_collide_exp(const lb_handle *h, const void *src, void *dst, const float *facc);
// moments.cu
cudaError_t launch_init_equilibrium(const lb_handle *h, void *dst, const double *rho, const double *u);
cudaError_t launch_set_populations(const lb_handle *h, void *dst, const double *n);
cudaError_t launch_get_populations(const lb_handle *h, const void *src, double *n);
cudaError_t launch_moments(const lb_handle *h, const void *src, float *rho, float *j, float *pi,
                           double *sums);
// particles.cu
lb_status couple_particles(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp,
                          void *ready = nullptr, void *done = nullptr);
lb_status interpolate(lb_handle *h, int kernel, int n, const double *pos, float *u_out);
cudaError_t clear_particle_forces(lb_handle *h);
void join_overlap(const lb_handle *h);  // order h->stream after a pending overlapped coupling
// step_sums.cu
size_t sc_block_count(const lb_handle *h);
size_t step_sums_scratch(size_t nblocks);
cudaError_t reduce_step_sums(const lb_handle *h, const float *partials, size_t nblocks, float *scratch,
                             double *sums);
void timer_mark(lb_handle *h, int which, int end, cudaStream_t s);  // record a timer event
cudaError_t reset_particle_barrier(lb_handle *h);
// Forget the stencil records of applied impulses that are already cleared.
void drop_particle_records(lb_handle *h);
bool adjoint_couple_ok(const lb_handle *h, const lb_particles *pp, const lb_couple_params *cp, const char *who);
lb_status couple_adjoint(lb_handle *h, const void *state, const lb_particles *pp, const lb_couple_params *cp,
                         const float *lam_facc, float *lam_pos, float *lam_mom, float *lam_u);
lb_status couple_on(lb_handle *h, const void *state, const lb_particles *pp, const lb_couple_params *cp,
                    float *facc_out);
void destroy_particles(lb_handle *h);
// spheres.cu
void destroy_spheres(lb_handle *h);

}  // namespace lbi
