// batch.cu -- many independent periodic replica boxes of different sizes
// advanced by one persistent launch.
//
// Every replica is an ordinary fluctuating D3Q19 box (the update of
// stream_collide.cuh: pull, MRT collision with noise, Sec. 3.4-3.5) with its
// own geometry, Philox key and replica counter word.  The replicas' nodes are
// cut into tiles (runs of consecutive node indices inside one replica); one
// launch of k_batch runs `nsteps` steps: in each step the resident blocks take
// tiles in a strided order, then meet at a grid barrier before the buffers
// swap.  The launch is cooperative (all blocks resident), the barrier spins a
// bounded number of times and on expiry sets LB_DERR_BARRIER and makes every
// block return.  Loads across barriers bypass L1 (ld.global.cg) because a
// buffer read two steps ago may be cached there.  The step counter and the
// buffer parity live in device memory, so a captured graph of the launch can
// be replayed as is.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "d3q19.cuh"
#include "grid_barrier.cuh"
#include "lbf_internal.h"
#include "stream_collide.cuh"

namespace lbi {
namespace {

// Unsigned division by a run-time constant (round-up method of Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994).
struct Div {
    uint32_t m, s, d;  // d == 1: identity
};

Div make_div(uint32_t d)
{
    Div v;
    v.d = d;
    if (d <= 1) {
        v.m = 0;
        v.s = 0;
        return v;
    }
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    v.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    v.s = l - 1;
    return v;
}

__device__ __forceinline__ uint32_t divide(uint32_t n, const Div &v)
{
    if (v.d <= 1) return n;
    const uint32_t t = __umulhi(v.m, n);
    return (t + ((n - t) >> 1)) >> v.s;
}

struct BatchDesc {
    int nx, ny, nz;
    uint32_t nodes;
    uint64_t off;      // element offset of plane 0 of this replica
    uint32_t pitch;    // elements per plane
    uint32_t replica;  // Philox counter word 3
    Div dx, dxy;
    lbd::RoundKeys rk;
};

struct BatchTile {
    int rep;
    uint32_t begin, count;
};

struct BatchState {
    uint32_t step;  // Philox step word of the next step
    uint32_t cur;   // buffer holding the current state
};

struct BatchArgs {
    StepArgs phys;  // physics constants (geometry fields unused)
    const BatchDesc *desc;
    const BatchTile *tiles;
    int ntiles;
    void *pops[2];
    int nsteps;
    int nodes_per_thread;
    BatchState *state;
    unsigned int *bar;  // [0] arrivals, [1] generation, [2] abort
    unsigned int *err;
    unsigned int spin_limit;
};

// Bounded grid barrier (grid_barrier.cuh).  Returns false if the run must
// stop (a barrier timed out here or elsewhere).
__device__ __forceinline__ bool batch_barrier(const BatchArgs &a)
{
    return lbi::grid_barrier(a.bar, a.err, a.spin_limit);
}

template <int DT, bool NOISE>
__device__ __forceinline__ void batch_node(const BatchDesc &d, uint32_t s, const typename lbd::Store<DT>::T *src,
                                           typename lbd::Store<DT>::T *dst, const StepArgs &ph, uint32_t step)
{
    using S = lbd::Store<DT>;
    const uint32_t row = divide(s, d.dx);
    const int x = (int)(s - row * (uint32_t)d.nx);
    const uint32_t zz = divide(s, d.dxy);
    const int y = (int)(row - zz * (uint32_t)d.ny);
    const int z = (int)zz;
    const int xm = (x == 0) ? d.nx - 1 : x - 1, xp = (x == d.nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? d.ny - 1 : y - 1, yp = (y == d.ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? d.nz - 1 : z - 1, zp = (z == d.nz - 1) ? 0 : z + 1;
    const size_t P = d.pitch;
    const typename S::T *base = src + d.off;
    float n[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        const uint32_t off = (uint32_t)((sz * d.ny + sy) * d.nx + sx);
        n[i] = S::cvt(__ldcg(base + (size_t)i * P + off), ph.inv_scale);
    }
    StepArgs a = ph;
    a.step = step;
    float out[19];
    collide_node<NOISE>(n, ph.fx, ph.fy, ph.fz, a, d.rk, s, d.replica, out);
    typename S::T *o = dst + d.off;
#pragma unroll
    for (int i = 0; i < 19; ++i) o[(size_t)i * P + s] = S::pack(out[i], ph.scale);
}

template <int DT, bool NOISE>
__global__ void k_batch(BatchArgs a)
{
    using T = typename lbd::Store<DT>::T;
    uint32_t step = a.state->step;
    uint32_t cur = a.state->cur;
    for (int t = 0; t < a.nsteps; ++t) {
        const T *src = static_cast<const T *>(a.pops[cur]);
        T *dst = static_cast<T *>(a.pops[cur ^ 1u]);
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const BatchTile tl = a.tiles[tile];
            const BatchDesc &d = a.desc[tl.rep];
            for (uint32_t k = threadIdx.x; k < tl.count; k += blockDim.x)
                batch_node<DT, NOISE>(d, tl.begin + k, src, dst, a.phys, step);
        }
        if (!batch_barrier(a)) return;
        cur ^= 1u;
        step += 1u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.state->step = step;
        a.state->cur = cur;
    }
}

}  // namespace
}  // namespace lbi

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct lb_batch {
    lb_params phys;                 // shared physics (geometry fields of replica 0)
    int n;
    std::vector<lbi::BatchDesc> desc_h;
    std::vector<lb_params> rep_params;
    lbi::BatchDesc *desc = nullptr;
    lbi::BatchTile *tiles = nullptr;
    int ntiles = 0;
    void *pops[2];
    size_t total_elems = 0;
    size_t elem = 4;
    cudaStream_t stream;
    cudaStream_t capture_stream = nullptr;  // graphs are recorded here, launched on `stream`
    lbi::BatchState *state = nullptr;  // device
    unsigned int *bar = nullptr;       // device [3]
    unsigned int *err = nullptr;       // device
    double *partials = nullptr;        // moments scratch
    int red_blocks = 0;
    uint32_t step = 0;                 // host mirror
    int cur = 0;                       // host mirror
    lb_batch_config cfg;
    unsigned int spin_limit = 1u << 22;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    uint64_t launches = 0;
};

using namespace lbi;

namespace {

size_t esize(int dtype) { return dtype == LB_F32 ? 4 : 2; }

bool same_physics(const lb_params &a, const lb_params &b)
{
    return a.dtype == b.dtype && a.walls == b.walls && a.noise_rho0 == b.noise_rho0 && a.rho0 == b.rho0 &&
           a.kT == b.kT && a.gamma_shear == b.gamma_shear && a.gamma_bulk == b.gamma_bulk &&
           a.gamma_odd == b.gamma_odd && a.gamma_even == b.gamma_even && a.body_force[0] == b.body_force[0] &&
           a.body_force[1] == b.body_force[1] && a.body_force[2] == b.body_force[2] && a.pop_scale == b.pop_scale;
}

lb_status build_tiles(lb_batch *b, int tile_nodes)
{
    std::vector<BatchTile> tl;
    for (int r = 0; r < b->n; ++r) {
        const uint32_t nodes = b->desc_h[r].nodes;
        for (uint32_t s = 0; s < nodes; s += (uint32_t)tile_nodes)
            tl.push_back(BatchTile{r, s, std::min<uint32_t>((uint32_t)tile_nodes, nodes - s)});
    }
    // largest replicas' tiles first gives the strided schedule a balanced tail
    std::stable_sort(tl.begin(), tl.end(), [&](const BatchTile &x, const BatchTile &y) {
        return b->desc_h[x.rep].nodes > b->desc_h[y.rep].nodes;
    });
    cudaFree(b->tiles);
    b->tiles = nullptr;
    cudaError_t e = cudaMalloc((void **)&b->tiles, tl.size() * sizeof(BatchTile));
    if (e != cudaSuccess) {
        set_error("lb_batch: tile table allocation failed");
        return LB_ENOMEM;
    }
    e = cudaMemcpy(b->tiles, tl.data(), tl.size() * sizeof(BatchTile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail("lb_batch: tile upload", e);
    b->ntiles = (int)tl.size();
    return LB_OK;
}

StepArgs batch_phys(const lb_batch *b)
{
    lb_handle tmp{};
    tmp.p = b->phys;
    tmp.n_nodes = 1;
    tmp.pitch = 64;
    return make_args(&tmp);
}

template <int DT, bool NOISE>
void *kernel_ptr()
{
    return (void *)k_batch<DT, NOISE>;
}

void *pick_kernel(const lb_batch *b)
{
    const bool noise = b->phys.kT > 0.0;
    switch (b->phys.dtype) {
    case LB_F32: return noise ? kernel_ptr<0, true>() : kernel_ptr<0, false>();
    case LB_F16: return noise ? kernel_ptr<1, true>() : kernel_ptr<1, false>();
    default: return noise ? kernel_ptr<2, true>() : kernel_ptr<2, false>();
    }
}

// Resident blocks for a configuration (cooperative launches need all of them).
int resident_grid(const lb_batch *b, int threads, int blocks_per_sm)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(b), threads, 0) != cudaSuccess) return 0;
    const int use = std::min(per_sm, blocks_per_sm);
    return use * device_sm_count();
}

cudaError_t launch_batch(lb_batch *b, int nsteps)
{
    BatchArgs a;
    a.phys = batch_phys(b);
    a.desc = b->desc;
    a.tiles = b->tiles;
    a.ntiles = b->ntiles;
    a.pops[0] = b->pops[0];
    a.pops[1] = b->pops[1];
    a.nsteps = nsteps;
    a.nodes_per_thread = 1;
    a.state = b->state;
    a.bar = b->bar;
    a.err = b->err;
    a.spin_limit = b->spin_limit;
    const int grid = std::min(b->cfg.grid, b->ntiles);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid > 0 ? grid : 1);
    lc.blockDim = dim3(b->cfg.threads);
    lc.dynamicSmemBytes = 0;
    lc.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    void *args[] = {&a};
    b->launches += 1;
    return cudaLaunchKernelExC(&lc, pick_kernel(b), args);
}

lb_status apply_config(lb_batch *b, const lb_batch_config *c)
{
    if (c->threads < 32 || c->threads > 1024 || (c->threads % 32) || c->tile_nodes < 32 || c->blocks_per_sm < 1) {
        set_error("lb_batch: bad configuration (threads %d, tile %d, blocks/SM %d)", c->threads, c->tile_nodes,
                  c->blocks_per_sm);
        return LB_EINVAL;
    }
    const int grid = resident_grid(b, c->threads, c->blocks_per_sm);
    if (grid <= 0) {
        set_error("lb_batch: kernel cannot be resident with %d threads per block", c->threads);
        return LB_EUNSUPPORTED;
    }
    lb_status st = build_tiles(b, c->tile_nodes);
    if (st != LB_OK) return st;
    b->cfg = *c;
    b->cfg.grid = grid;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = 0;
    }
    return LB_OK;
}

// A fake single-box handle over replica r, for the per-replica helpers.
void replica_view(lb_batch *b, int r, lb_handle &h)
{
    memset(&h, 0, sizeof(h));
    h.p = b->rep_params[r];
    h.n_nodes = b->desc_h[r].nodes;
    h.pitch = b->desc_h[r].pitch;
    h.elem = b->elem;
    for (int k = 0; k < 2; ++k) h.pops[k] = (char *)b->pops[k] + b->desc_h[r].off * b->elem;
    h.cur = b->cur;
    h.stream = b->stream;
    h.step = b->step;
    h.d_err = b->err;
    h.d_partials = b->partials;
    h.red_blocks = b->red_blocks;
}

}  // namespace

extern "C" {

size_t lb_batch_population_bytes(const lb_params *per_replica, int n)
{
    if (!per_replica || n < 1) return 0;
    size_t total = 0;
    for (int r = 0; r < n; ++r) {
        const size_t pitch = lb_plane_pitch(&per_replica[r]);
        if (!pitch) return 0;
        total += 19 * pitch * esize(per_replica[0].dtype);
    }
    return total;
}

lb_status lb_batch_create(const lb_params *per_replica, int n, void *pops_a, void *pops_b, void *stream,
                          lb_batch **out)
{
    if (!out) {
        set_error("lb_batch_create: out is NULL");
        return LB_EINVAL;
    }
    *out = nullptr;
    if (!per_replica || n < 1 || !pops_a || !pops_b || pops_a == pops_b) {
        set_error("lb_batch_create: need n >= 1 replicas and two distinct buffers");
        return LB_EINVAL;
    }
    if (((uintptr_t)pops_a & 255u) || ((uintptr_t)pops_b & 255u)) {
        set_error("lb_batch_create: buffers must be 256-byte aligned");
        return LB_EINVAL;
    }
    for (int r = 0; r < n; ++r) {
        if (!lb_plane_pitch(&per_replica[r])) return LB_EINVAL;
        if (per_replica[r].walls || per_replica[r].equilibrium) {
            set_error("lb_batch_create: replicas must be periodic with the quadratic equilibrium");
            return LB_EUNSUPPORTED;
        }
        if (!same_physics(per_replica[r], per_replica[0])) {
            set_error("lb_batch_create: replica %d differs from replica 0 in dtype or physics parameters", r);
            return LB_EUNSUPPORTED;
        }
        const double nodes = (double)per_replica[r].nx * per_replica[r].ny * per_replica[r].nz;
        if (nodes >= 16777216.0) {
            set_error("lb_batch_create: replica %d has more than 2^24 - 1 nodes", r);
            return LB_EINVAL;
        }
    }
    lb_batch *b = new lb_batch();
    if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        set_error("lb_batch_create: stream creation failed");
        return LB_ECUDA;
    }
    b->phys = per_replica[0];
    b->n = n;
    b->elem = esize(per_replica[0].dtype);
    b->pops[0] = pops_a;
    b->pops[1] = pops_b;
    b->stream = (cudaStream_t)stream;
    b->rep_params.assign(per_replica, per_replica + n);
    size_t off = 0;
    for (int r = 0; r < n; ++r) {
        const lb_params &p = per_replica[r];
        BatchDesc d;
        d.nx = p.nx;
        d.ny = p.ny;
        d.nz = p.nz;
        d.nodes = (uint32_t)((size_t)p.nx * p.ny * p.nz);
        d.pitch = (uint32_t)lb_plane_pitch(&p);
        d.off = off;
        d.replica = p.replica;
        d.dx = make_div((uint32_t)p.nx);
        d.dxy = make_div((uint32_t)(p.nx * p.ny));
        d.rk = lbd::make_round_keys(p.seed);
        b->desc_h.push_back(d);
        off += 19 * (size_t)d.pitch;  // plane pitch is a multiple of 64 elements: 256-byte aligned blocks
    }
    b->total_elems = off;
    b->red_blocks = 4 * device_sm_count();
    cudaError_t e = cudaMalloc((void **)&b->desc, n * sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->state, sizeof(BatchState));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->bar, 3 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->err, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->partials, sizeof(double) * LB_NSUMS * b->red_blocks);
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        set_error("lb_batch_create: device allocation failed (%s)", cudaGetErrorString(e));
        return LB_ENOMEM;
    }
    BatchState s0{0u, 0u};
    e = cudaMemcpy(b->desc, b->desc_h.data(), n * sizeof(BatchDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->state, &s0, sizeof(s0), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->bar, 0, 3 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        return cuda_fail("lb_batch_create", e);
    }
    lb_batch_config c{256, 2048, 2, 0};
    lb_status st = apply_config(b, &c);
    if (st != LB_OK) {
        lb_batch_destroy(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch *b)
{
    if (!b) return LB_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    cudaFree(b->desc);
    cudaFree(b->tiles);
    cudaFree(b->state);
    cudaFree(b->bar);
    cudaFree(b->err);
    cudaFree(b->partials);
    delete b;
    return LB_OK;
}

lb_status lb_batch_set_config(lb_batch *b, const lb_batch_config *c)
{
    if (!b || !c) {
        set_error("lb_batch_set_config: NULL argument");
        return LB_EINVAL;
    }
    return apply_config(b, c);
}

lb_status lb_batch_get_config(const lb_batch *b, lb_batch_config *c)
{
    if (!b || !c) {
        set_error("lb_batch_get_config: NULL argument");
        return LB_EINVAL;
    }
    *c = b->cfg;
    return LB_OK;
}

lb_status lb_batch_set_barrier_limit(lb_batch *b, uint32_t spins)
{
    if (!b) {
        set_error("lb_batch_set_barrier_limit: NULL handle");
        return LB_EINVAL;
    }
    b->spin_limit = spins;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = 0;
    }
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int nsteps, int use_graph)
{
    if (!b || nsteps < 0) {
        set_error("lb_batch_step: bad argument");
        return LB_EINVAL;
    }
    if (nsteps == 0) return LB_OK;
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        if (!b->graph || b->graph_steps != nsteps) {
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            cudaGraph_t g = nullptr;
            const cudaStream_t user = b->stream;
            b->stream = b->capture_stream;
            e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = launch_batch(b, nsteps);
                b->launches -= 1;  // counted when the graph is launched
                e = cudaStreamEndCapture(b->capture_stream, &g);
                if (le != cudaSuccess) e = le;
            }
            b->stream = user;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                return cuda_fail("lb_batch_step (graph capture of the persistent launch)", e);
            }
            b->graph_steps = nsteps;
        }
        e = cudaGraphLaunch(b->graph, b->stream);
        b->launches += 1;
    } else {
        e = launch_batch(b, nsteps);
    }
    if (e != cudaSuccess) return cuda_fail("lb_batch_step", e);
    b->step += (uint32_t)nsteps;
    b->cur ^= (nsteps & 1);
    return LB_OK;
}

lb_status lb_batch_sync(lb_batch *b, uint32_t *bits)
{
    if (!b) {
        set_error("lb_batch_sync: NULL handle");
        return LB_EINVAL;
    }
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b->err, sizeof(v), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail("lb_batch_sync", e);
    if (bits) *bits = v;
    if (v) {
        // reset the error word, the barrier (abort flag, counters) and the
        // device step / buffer record to the host's for reuse; the populations
        // of a stopped run are undefined and must be set again
        BatchState s{b->step, (uint32_t)b->cur};
        e = cudaMemcpy(b->state, &s, sizeof(s), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(b->bar, 0, 3 * sizeof(unsigned int));
        if (e != cudaSuccess) return cuda_fail("lb_batch_sync", e);
        set_error("batched run stopped: device error word 0x%x%s", v,
                  (v & LB_DERR_BARRIER) ? " [grid barrier timeout]" : "");
        return (v & LB_DERR_BARRIER) ? LB_ETIMEOUT : LB_EDEVICE;
    }
    return LB_OK;
}

lb_status lb_batch_autotune(lb_batch *b, int trial_steps, lb_batch_config *chosen, double *best_ms_per_step)
{
    if (!b || trial_steps < 1) {
        set_error("lb_batch_autotune: bad argument");
        return LB_EINVAL;
    }
    const int threads_opts[] = {128, 256, 512};
    const int tile_opts[] = {512, 1024, 2048, 4096, 8192};
    const int bps_opts[] = {1, 2, 4, 8};
    lb_batch_config best{0, 0, 0, 0};
    double best_ms = 1e300;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int th : threads_opts)
        for (int tile : tile_opts)
            for (int bps : bps_opts) {
                if (th * bps > 2048) continue;
                lb_batch_config c{th, tile, bps, 0};
                if (apply_config(b, &c) != LB_OK) continue;
                if (lb_batch_step(b, 1, 0) != LB_OK) continue;  // warm-up
                cudaEventRecord(e0, b->stream);
                if (lb_batch_step(b, trial_steps, 0) != LB_OK) continue;
                cudaEventRecord(e1, b->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = ms / trial_steps;
                if (per < best_ms) {
                    best_ms = per;
                    best = b->cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    uint32_t bits = 0;
    lb_status st = lb_batch_sync(b, &bits);
    if (st != LB_OK) return st;
    if (best.threads == 0) {
        set_error("lb_batch_autotune: no configuration ran");
        return LB_ECUDA;
    }
    st = apply_config(b, &best);
    if (st != LB_OK) return st;
    if (chosen) *chosen = b->cfg;
    if (best_ms_per_step) *best_ms_per_step = best_ms;
    return LB_OK;
}

lb_status lb_batch_get_step(const lb_batch *b, uint32_t *step)
{
    if (!b || !step) {
        set_error("lb_batch_get_step: NULL argument");
        return LB_EINVAL;
    }
    *step = b->step;
    return LB_OK;
}

lb_status lb_batch_init_equilibrium(lb_batch *b, int replica, const double *rho, const double *u)
{
    if (!b || replica < -1 || replica >= b->n) {
        set_error("lb_batch_init_equilibrium: bad replica index");
        return LB_EINVAL;
    }
    const int r0 = replica < 0 ? 0 : replica, r1 = replica < 0 ? b->n : replica + 1;
    for (int r = r0; r < r1; ++r) {
        lb_handle h;
        replica_view(b, r, h);
        cudaError_t e = launch_init_equilibrium(&h, h.pops[h.cur], rho, u);
        b->launches += 1;
        if (e != cudaSuccess) return cuda_fail("lb_batch_init_equilibrium", e);
    }
    return LB_OK;
}

lb_status lb_batch_get_populations(lb_batch *b, int replica, double *n)
{
    if (!b || !n || replica < 0 || replica >= b->n) {
        set_error("lb_batch_get_populations: bad argument");
        return LB_EINVAL;
    }
    lb_handle h;
    replica_view(b, replica, h);
    cudaError_t e = launch_get_populations(&h, h.pops[h.cur], n);
    b->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_batch_get_populations", e);
}

lb_status lb_batch_set_populations(lb_batch *b, int replica, const double *n)
{
    if (!b || !n || replica < 0 || replica >= b->n) {
        set_error("lb_batch_set_populations: bad argument");
        return LB_EINVAL;
    }
    lb_handle h;
    replica_view(b, replica, h);
    cudaError_t e = launch_set_populations(&h, h.pops[h.cur], n);
    b->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_batch_set_populations", e);
}

lb_status lb_batch_moments(lb_batch *b, int replica, float *rho, float *j, float *pi, double *sums)
{
    if (!b || replica < 0 || replica >= b->n) {
        set_error("lb_batch_moments: bad replica index");
        return LB_EINVAL;
    }
    lb_handle h;
    replica_view(b, replica, h);
    cudaError_t e = launch_moments(&h, h.pops[h.cur], rho, j, pi, sums);
    b->launches += sums ? 2 : 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_batch_moments", e);
}

lb_status lb_batch_get_launch_count(const lb_batch *b, uint64_t *count)
{
    if (!b || !count) {
        set_error("lb_batch_get_launch_count: NULL argument");
        return LB_EINVAL;
    }
    *count = b->launches;
    return LB_OK;
}

}  // extern "C"
