// api.cu -- the C ABI of lbfluct.h: handle life cycle, argument checks,
// error reporting and the step loop.  Kernels live in stream_collide.cuh,
// moments.cu and particles.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "lbf_internal.h"

namespace lbi {

template <int DT>
cudaError_t launch_stream_collide_dt(const lb_handle *h, const void *src, void *dst, const float *facc, float *partials);
extern template cudaError_t launch_stream_collide_dt<0>(const lb_handle *, const void *, void *, const float *, float *);
extern template cudaError_t launch_stream_collide_dt<1>(const lb_handle *, const void *, void *, const float *, float *);
extern template cudaError_t launch_stream_collide_dt<2>(const lb_handle *, const void *, void *, const float *, float *);
template <int DT>
cudaError_t launch_patch_dt(const lb_handle *h, const void *src, void *dst, float *facc, const int *records,
                            int n, int nsub, int span, unsigned int *claim, unsigned int tag);
extern template cudaError_t launch_patch_dt<0>(const lb_handle *, const void *, void *, float *, const int *,
                                               int, int, int, unsigned int *, unsigned int);
extern template cudaError_t launch_patch_dt<1>(const lb_handle *, const void *, void *, float *, const int *,
                                               int, int, int, unsigned int *, unsigned int);
extern template cudaError_t launch_patch_dt<2>(const lb_handle *, const void *, void *, float *, const int *,
                                               int, int, int, unsigned int *, unsigned int);

namespace {
thread_local char g_msg[512] = "no error";
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}

lb_status cuda_fail(const char *what, cudaError_t e)
{
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return LB_ECUDA;
}

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    return n;
}

StepArgs make_args(const lb_handle *h)
{
    const lb_params &p = h->p;
    StepArgs a;
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.z0 = p.walls ? 1 : 0;
    a.z1 = p.walls ? p.nz - 1 : p.nz;
    a.pitch = h->pitch;
    a.nn = h->n_nodes;
    a.rho0 = (float)p.rho0;
    a.kT = (float)p.kT;
    a.mu = (float)(p.kT * 3.0);
    a.g_shear = (float)p.gamma_shear;
    a.g_bulk = (float)p.gamma_bulk;
    a.g_odd = (float)p.gamma_odd;
    a.g_even = (float)p.gamma_even;
    a.phi_shear = (float)std::sqrt(1.0 - p.gamma_shear * p.gamma_shear);
    a.phi_bulk = (float)std::sqrt(1.0 - p.gamma_bulk * p.gamma_bulk);
    a.phi_odd = (float)std::sqrt(1.0 - p.gamma_odd * p.gamma_odd);
    a.phi_even = (float)std::sqrt(1.0 - p.gamma_even * p.gamma_even);
    for (int k = 4; k < 19; ++k) {
        const double phi = k == 4 ? std::sqrt(1.0 - p.gamma_bulk * p.gamma_bulk)
                           : k < 10 ? std::sqrt(1.0 - p.gamma_shear * p.gamma_shear)
                           : k < 16 ? std::sqrt(1.0 - p.gamma_odd * p.gamma_odd)
                                    : std::sqrt(1.0 - p.gamma_even * p.gamma_even);
        a.amp[k - 4] = (float)(phi * (double)lbd::sqrt_inv_w(k));
    }
    a.fx = (float)p.body_force[0];
    a.fy = (float)p.body_force[1];
    a.fz = (float)p.body_force[2];
    const double sc = (p.dtype == LB_F32) ? 1.0 : (p.pop_scale > 0.0 ? p.pop_scale : 1024.0);
    a.scale = (float)sc;
    a.inv_scale = (float)(1.0 / sc);
    a.noise_rho0 = p.noise_rho0;
    a.key0 = (uint32_t)(p.seed & 0xffffffffu);
    a.key1 = (uint32_t)(p.seed >> 32);
    a.replica = p.replica;
    a.step = h->step;
    a.rk = lbd::make_round_keys(p.seed);
    a.err = h->d_err;
    return a;
}

// An overlapped coupling is joined by the next lb_step; every other call on
// the handle first orders its stream after it (the impulses then stay pending
// and the next lb_step applies them in its single pass).
void join_overlap(const lb_handle *hc)
{
    lb_handle *h = const_cast<lb_handle *>(hc);
    if (!h || !h->overlap_pending) return;
    cudaStreamWaitEvent(h->stream, h->ev_couple, 0);
    h->overlap_pending = 0;
}

void timer_mark(lb_handle *h, int which, int end, cudaStream_t s)
{
    if (!h->timer_cap || h->timer_n[which] >= h->timer_cap) return;
    cudaEventRecord(h->timer_ev[which][2 * h->timer_n[which] + end], s);
    if (end) h->timer_n[which] += 1;
}

}  // namespace lbi

using namespace lbi;

namespace {

size_t elem_size(int dtype) { return dtype == LB_F32 ? 4 : 2; }

bool check_params(const lb_params *p)
{
    if (!p) {
        set_error("lb_params is NULL");
        return false;
    }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) {
        set_error("box %d x %d x %d: every edge must be >= 1", p->nx, p->ny, p->nz);
        return false;
    }
    const double n = (double)p->nx * p->ny * p->nz;
    if (n > 2147483647.0) {
        set_error("box of %.0f nodes exceeds 2^31 - 1 nodes", n);
        return false;
    }
    if (p->dtype < LB_F32 || p->dtype > LB_BF16) {
        set_error("dtype %d is not one of LB_F32, LB_F16, LB_BF16", p->dtype);
        return false;
    }
    if (p->walls != 0 && p->walls != 1) {
        set_error("walls must be 0 or 1");
        return false;
    }
    if (p->walls && p->nz < 3) {
        set_error("walls need nz >= 3 (two solid planes and one fluid plane)");
        return false;
    }
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) {
        set_error("rho0 must be finite and > 0");
        return false;
    }
    if (!(p->kT >= 0.0) || !std::isfinite(p->kT)) {
        set_error("kT must be finite and >= 0");
        return false;
    }
    const double g[4] = {p->gamma_shear, p->gamma_bulk, p->gamma_odd, p->gamma_even};
    for (double v : g) {
        if (!(v > -1.0 && v < 1.0)) {
            set_error("relaxation eigenvalues must satisfy |gamma| < 1 (got %g)", v);
            return false;
        }
    }
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(p->body_force[d])) {
            set_error("body_force must be finite");
            return false;
        }
    }
    if (p->pop_scale < 0.0 || !std::isfinite(p->pop_scale)) {
        set_error("pop_scale must be >= 0 (0 selects 1024)");
        return false;
    }
    if (p->equilibrium > 1) {
        set_error("lb_params.equilibrium must be 0 (quadratic) or 1 (exponential)");
        return false;
    }
    return true;
}

bool aligned256(const void *ptr) { return ((uintptr_t)ptr & 255u) == 0; }

void free_timers(lb_handle *h)
{
    for (int w = 0; w < 2; ++w) {
        if (!h->timer_ev[w]) continue;
        for (int i = 0; i < 2 * h->timer_cap; ++i)
            if (h->timer_ev[w][i]) cudaEventDestroy(h->timer_ev[w][i]);
        free(h->timer_ev[w]);
        h->timer_ev[w] = nullptr;
        h->timer_n[w] = 0;
    }
    h->timer_cap = 0;
}

// One step; with partials != NULL the stream-collide launch also writes its
// per-block moment sums there.
lb_status step_once(lb_handle *h, float *partials)
{
    const void *src = h->pops[h->cur];
    void *dst = h->pops[1 - h->cur];
    cudaError_t e;
    if (h->overlap_pending) {
        // all nodes without the impulses while the coupling runs on aux,
        // then the nodes it spread impulses to, again with them
        timer_mark(h, 0, 0, h->stream);
        switch (h->p.dtype) {
        case LB_F32: e = launch_stream_collide_dt<0>(h, src, dst, nullptr, partials); break;
        case LB_F16: e = launch_stream_collide_dt<1>(h, src, dst, nullptr, partials); break;
        default: e = launch_stream_collide_dt<2>(h, src, dst, nullptr, partials); break;
        }
        timer_mark(h, 0, 1, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_couple, 0);
        h->overlap_pending = 0;
        if (++h->claim_tag == 0u) {  // wrapped: start the tags again from 1
            if (e == cudaSuccess) e = cudaMemsetAsync(h->claim, 0, h->n_nodes * sizeof(unsigned int), h->stream);
            h->claim_tag = 1u;
        }
        if (e == cudaSuccess) {
            switch (h->p.dtype) {
            case LB_F32: e = launch_patch_dt<0>(h, src, dst, h->facc, h->patch_rec, h->patch_n, h->patch_nsub, h->patch_span,
                                                  h->claim, h->claim_tag);
                break;
            case LB_F16: e = launch_patch_dt<1>(h, src, dst, h->facc, h->patch_rec, h->patch_n, h->patch_nsub, h->patch_span,
                                                  h->claim, h->claim_tag);
                break;
            default: e = launch_patch_dt<2>(h, src, dst, h->facc, h->patch_rec, h->patch_n, h->patch_nsub, h->patch_span,
                                                  h->claim, h->claim_tag);
                break;
            }
        }
        if (e != cudaSuccess) return cuda_fail("lb_step", e);
        h->launches += 2;
        h->facc_dirty = 0;
        h->facc_stale = 0;  // the patch cleared every impulse node it applied
        drop_particle_records(h);
        h->cur = 1 - h->cur;
        h->step += 1;
        return LB_OK;
    }
    const float *facc = h->facc_dirty ? h->facc : nullptr;
    timer_mark(h, 0, 0, h->stream);
    if (h->p.equilibrium) {
        e = launch_stream_collide_exp(h, src, dst, facc);
    } else {
        switch (h->p.dtype) {
        case LB_F32: e = launch_stream_collide_dt<0>(h, src, dst, facc, partials); break;
        case LB_F16: e = launch_stream_collide_dt<1>(h, src, dst, facc, partials); break;
        default: e = launch_stream_collide_dt<2>(h, src, dst, facc, partials); break;
        }
    }
    timer_mark(h, 0, 1, h->stream);
    if (e != cudaSuccess) return cuda_fail("lb_step", e);
    h->launches += 1;
    if (facc) {  // applied once; cleared by the next lb_couple_particles
        h->facc_dirty = 0;
        h->facc_stale = 1;
    }
    h->cur = 1 - h->cur;
    h->step += 1;
    return LB_OK;
}
}  // namespace

extern "C" {

const char *lb_last_error(void) { return g_msg; }

const char *lb_version(void) { return "lbfluct 0.1.0 sm_103a"; }

size_t lb_plane_pitch(const lb_params *p)
{
    if (!check_params(p)) return 0;
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    return (n + 63) / 64 * 64;
}

size_t lb_population_bytes(const lb_params *p)
{
    const size_t pitch = lb_plane_pitch(p);
    return pitch ? 19 * pitch * elem_size(p->dtype) : 0;
}

lb_status lb_create(const lb_params *p, void *pops_a, void *pops_b, float *force, void *stream,
                    lb_handle **out)
{
    if (!out) {
        set_error("lb_create: out is NULL");
        return LB_EINVAL;
    }
    *out = nullptr;
    if (!check_params(p)) return LB_EINVAL;
    if (!pops_a || !pops_b || pops_a == pops_b) {
        set_error("lb_create: need two distinct population buffers");
        return LB_EINVAL;
    }
    if (!aligned256(pops_a) || !aligned256(pops_b)) {
        set_error("lb_create: population buffers must be 256-byte aligned");
        return LB_EINVAL;
    }
    if (force && ((uintptr_t)force & 3u)) {
        set_error("lb_create: force field must be 4-byte aligned");
        return LB_EINVAL;
    }
    lb_handle *h = (lb_handle *)calloc(1, sizeof(lb_handle));
    if (!h) {
        set_error("lb_create: host allocation failed");
        return LB_ENOMEM;
    }
    h->p = *p;
    h->n_nodes = (size_t)p->nx * p->ny * p->nz;
    h->pitch = lb_plane_pitch(p);
    h->elem = elem_size(p->dtype);
    h->pops[0] = pops_a;
    h->pops[1] = pops_b;
    h->cur = 0;
    h->force = force;
    h->stream = (cudaStream_t)stream;
    h->step = 0;
    h->sph_n = -1;
    h->red_blocks = 4 * device_sm_count();
    cudaError_t e = cudaMalloc((void **)&h->d_err, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_partials, sizeof(double) * LB_NSUMS * h->red_blocks);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream);
    if (e != cudaSuccess) {
        lb_destroy(h);
        set_error("lb_create: device allocation failed (%s)", cudaGetErrorString(e));
        return LB_ENOMEM;
    }
    *out = h;
    return LB_OK;
}

lb_status lb_set_timing(lb_handle *h, int capacity)
{
    if (!h || capacity < 0) {
        set_error("lb_set_timing: need a handle and capacity >= 0");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (h->aux) cudaStreamSynchronize(h->aux);
    cudaStreamSynchronize(h->stream);
    free_timers(h);
    if (capacity == 0) return LB_OK;
    for (int w = 0; w < 2; ++w) {
        h->timer_ev[w] = (cudaEvent_t *)calloc(2 * (size_t)capacity, sizeof(cudaEvent_t));
        if (!h->timer_ev[w]) {
            free_timers(h);
            set_error("lb_set_timing: host allocation failed");
            return LB_ENOMEM;
        }
        for (int i = 0; i < 2 * capacity; ++i) {
            if (cudaEventCreate(&h->timer_ev[w][i]) != cudaSuccess) {
                h->timer_cap = capacity;
                free_timers(h);
                set_error("lb_set_timing: event creation failed");
                return LB_ECUDA;
            }
        }
    }
    h->timer_cap = capacity;
    return LB_OK;
}

lb_status lb_get_timing(lb_handle *h, double *ms_step, int *n_step, double *ms_couple, int *n_couple)
{
    if (!h) {
        set_error("lb_get_timing: handle is NULL");
        return LB_EINVAL;
    }
    double sum[2] = {0.0, 0.0};
    for (int w = 0; w < 2; ++w) {
        for (int i = 0; i < h->timer_n[w]; ++i) {
            float ms = 0.0f;
            cudaError_t e = cudaEventSynchronize(h->timer_ev[w][2 * i + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->timer_ev[w][2 * i], h->timer_ev[w][2 * i + 1]);
            if (e != cudaSuccess) return cuda_fail("lb_get_timing", e);
            sum[w] += ms;
        }
    }
    if (ms_step) *ms_step = sum[0];
    if (n_step) *n_step = h->timer_n[0];
    if (ms_couple) *ms_couple = sum[1];
    if (n_couple) *n_couple = h->timer_n[1];
    return LB_OK;
}

lb_status lb_destroy(lb_handle *h)
{
    if (!h) return LB_OK;
    free_timers(h);
    if (h->aux) cudaStreamSynchronize(h->aux);
    join_overlap(h);
    destroy_particles(h);
    destroy_spheres(h);
    if (h->claim) cudaFree(h->claim);
    if (h->lam_u) cudaFree(h->lam_u);
    if (h->arena) cudaFree(h->arena);
    if (h->sc_partials) cudaFree(h->sc_partials);
    if (h->ev_main) cudaEventDestroy(h->ev_main);
    if (h->ev_couple) cudaEventDestroy(h->ev_couple);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->facc) cudaFree(h->facc);
    free(h);
    return LB_OK;
}

lb_status lb_sync(lb_handle *h, uint32_t *bits)
{
    if (!h) {
        set_error("lb_sync: handle is NULL");
        return LB_EINVAL;
    }
    join_overlap(h);
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->d_err, sizeof(v), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail("lb_sync", e);
    if (bits) *bits = v;
    if (v) {
        e = cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), h->stream);
        if (e == cudaSuccess && (v & LB_DERR_BARRIER)) e = reset_particle_barrier(h);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail("lb_sync", e);
        set_error("device error word 0x%x%s%s%s%s", v, (v & LB_DERR_FENE_BROKEN) ? " [FENE bond broken]" : "",
                  (v & LB_DERR_NLIST_FULL) ? " [neighbour list full]" : "",
                  (v & LB_DERR_NONFINITE) ? " [non-finite sums]" : "",
                  (v & LB_DERR_BARRIER) ? " [grid barrier timeout]" : "");
        if (v & LB_DERR_NONFINITE) return LB_ENONFINITE;
        if (v & LB_DERR_BARRIER) return LB_ETIMEOUT;
        return LB_EDEVICE;
    }
    return LB_OK;
}

lb_status lb_get_step(const lb_handle *h, uint32_t *step)
{
    if (!h || !step) {
        set_error("lb_get_step: NULL argument");
        return LB_EINVAL;
    }
    *step = h->step;
    return LB_OK;
}

lb_status lb_set_step(lb_handle *h, uint32_t step)
{
    if (!h) {
        set_error("lb_set_step: handle is NULL");
        return LB_EINVAL;
    }
    h->step = step;
    return LB_OK;
}

lb_status lb_state_buffers(const lb_handle *h, void **current, void **other)
{
    if (!h) {
        set_error("lb_state_buffers: handle is NULL");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (current) *current = h->pops[h->cur];
    if (other) *other = h->pops[1 - h->cur];
    return LB_OK;
}

lb_status lb_init_equilibrium(lb_handle *h, const double *rho, const double *u)
{
    if (!h) {
        set_error("lb_init_equilibrium: handle is NULL");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = launch_init_equilibrium(h, h->pops[h->cur], rho, u);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_init_equilibrium", e);
}

lb_status lb_set_populations(lb_handle *h, const double *n)
{
    if (!h || !n) {
        set_error("lb_set_populations: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = launch_set_populations(h, h->pops[h->cur], n);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_set_populations", e);
}

lb_status lb_get_launch_count(const lb_handle *h, uint64_t *count)
{
    if (!h || !count) {
        set_error("lb_get_launch_count: NULL argument");
        return LB_EINVAL;
    }
    *count = h->launches;
    return LB_OK;
}

lb_status lb_get_populations(const lb_handle *h, double *n)
{
    if (!h || !n) {
        set_error("lb_get_populations: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = launch_get_populations(h, h->pops[h->cur], n);
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_get_populations", e);
}

lb_status lb_step(lb_handle *h, int nsteps)
{
    const lbi::NvtxRange range("lb_step");
    if (!h) {
        set_error("lb_step: handle is NULL");
        return LB_EINVAL;
    }
    if (nsteps < 0) {
        set_error("lb_step: nsteps = %d < 0", nsteps);
        return LB_EINVAL;
    }
    for (int t = 0; t < nsteps; ++t) {
        const lb_status st = step_once(h, nullptr);
        if (st != LB_OK) return st;
    }
    return LB_OK;
}

lb_status lb_step_sums(lb_handle *h, int nsteps, double *sums)
{
    const lbi::NvtxRange range("lb_step_sums");
    if (!h || !sums || nsteps < 1) {
        set_error("lb_step_sums: need a handle, a sums buffer and nsteps >= 1");
        return LB_EINVAL;
    }
    if (h->p.equilibrium) {
        set_error("lb_step_sums: the sums come from the quadratic-equilibrium launch (use lb_step + lb_moments)");
        return LB_EUNSUPPORTED;
    }
    const size_t nb = sc_block_count(h);
    const size_t len = nb * 38 + step_sums_scratch(nb);
    if (h->sc_partials_len < len) {
        cudaFree(h->sc_partials);
        h->sc_partials = nullptr;
        h->sc_partials_len = 0;
        const cudaError_t e = cudaMalloc((void **)&h->sc_partials, len * sizeof(float));
        if (e != cudaSuccess) {
            set_error("lb_step_sums: scratch allocation failed (%s)", cudaGetErrorString(e));
            return LB_ENOMEM;
        }
        h->sc_partials_len = len;
    }
    for (int t = 0; t + 1 < nsteps; ++t) {
        const lb_status st = step_once(h, nullptr);
        if (st != LB_OK) return st;
    }
    const lb_status st = step_once(h, h->sc_partials);
    if (st != LB_OK) return st;
    const cudaError_t e = reduce_step_sums(h, h->sc_partials, nb, h->sc_partials + nb * 38, sums);
    if (e != cudaSuccess) return cuda_fail("lb_step_sums", e);
    h->launches += 2;
    return LB_OK;
}

lb_status lb_moments(lb_handle *h, float *rho, float *j, float *pi, double *sums)
{
    if (!h) {
        set_error("lb_moments: handle is NULL");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (!rho && !j && !pi && !sums) return LB_OK;
    cudaError_t e = launch_moments(h, h->pops[h->cur], rho, j, pi, sums);
    h->launches += sums ? 2 : 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_moments", e);
}

lb_status lb_couple_particles(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp)
{
    const lbi::NvtxRange range("lb_couple_particles");
    if (!h || !parts || !cp) {
        set_error("lb_couple_particles: NULL argument");
        return LB_EINVAL;
    }
    return couple_particles(h, parts, cp);
}

lb_status lb_couple_particles_async(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp,
                                    void *ready_event, void *done_event)
{
    const lbi::NvtxRange range("lb_couple_particles");
    if (!h || !parts || !cp) {
        set_error("lb_couple_particles_async: NULL argument");
        return LB_EINVAL;
    }
    return couple_particles(h, parts, cp, ready_event, done_event);
}

lb_status lb_interpolate(lb_handle *h, int n, const double *pos, float *u_out)
{
    return lb_interpolate_phi(h, 2, n, pos, u_out);
}

lb_status lb_interpolate_phi(lb_handle *h, int kernel, int n, const double *pos, float *u_out)
{
    if (!h || n < 0 || (n > 0 && (!pos || !u_out)) || kernel < 2 || kernel > 4) {
        set_error("lb_interpolate: bad argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    return interpolate(h, kernel, n, pos, u_out);
}

lb_status lb_get_particle_forces(lb_handle *h, float *out)
{
    if (!h || !out) {
        set_error("lb_get_particle_forces: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    const size_t N = h->n_nodes;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        if (h->facc && h->facc_dirty)
            e = cudaMemcpyAsync(out + d * N, h->facc + d * h->pitch, N * sizeof(float), cudaMemcpyDeviceToDevice,
                                h->stream);
        else
            e = cudaMemsetAsync(out + d * N, 0, N * sizeof(float), h->stream);
    }
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_get_particle_forces", e);
}

}  // extern "C"
