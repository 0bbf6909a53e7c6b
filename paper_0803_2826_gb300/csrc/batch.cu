// batch.cu -- many independent periodic replica boxes of different sizes
// advanced by one persistent launch.
//
// Every replica is an ordinary fluctuating D3Q19 box (the update of
// stream_collide.cuh: pull, MRT collision with noise, Sec. 3.4-3.5) with its
// own geometry, Philox key and replica counter word.  The replicas' nodes are
// cut into tiles (runs of consecutive node indices inside one replica); one
// launch of k_batch runs `nsteps` steps: in each step the resident blocks take
// tiles in a strided order, then meet at a grid barrier before the buffers
// swap.  Optionally (lb_batch_record_modes) every step also records, per
// replica, the six transverse velocity modes u_a(k_b) at the smallest wave
// vector of each axis (Sec. 3.6 fluctuation spectrum; their decay per step is
// the shear eigenvalue of Sec. 3.4, Eq. shearviscosity): each warp sums
// u_a e^{-i k_b r_b} over its nodes of a tile and adds the twelve real parts
// to the replica's record with FP64 atomics; k_mode_acf forms the per-replica
// autocorrelation from the records afterwards.
// The launch is cooperative (all blocks resident), the barrier spins a
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
    uint32_t phase;    // offset of this replica's phase table (mode records)
    Div dx, dxy;
    lbd::RoundKeys rk;
    uint32_t key0, key1;  // the seed's two key words (the paired kernels form the round keys from them)
};

struct BatchTile {
    int rep;
    uint32_t begin, count;
};

struct BatchState {
    uint32_t step;       // Philox step word of the next step
    uint32_t cur;        // buffer holding the current state
    uint32_t rec_step0;  // step recorded at index 0 of the mode records
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
    // transverse-mode records (OBS kernels): modes[rep][t][12], t = step - state->rec_step0 < rec_cap;
    // phase[desc.phase + ...] = (cos, -sin)(2 pi r / L) for r along x, then y, then z
    double *modes;
    const float2 *phase;
    uint32_t rec_cap;
};

constexpr int kModeVals = 12;  // six complex transverse modes
// register caps of the paired kernels (no spills at these; caps of 88 to
// 102, which would let five 128-thread blocks share an SM, spill and
// measured slower: the autotuner keeps 512-thread blocks).  The paired
// kernels form each replica's Philox round keys from its two key words
// (lbp::RunningKeys) instead of holding the twenty precomputed ones: 1.5%
// faster at the same occupancy.
constexpr int kBatchPairMaxRegs = 128;
constexpr int kBatchPairObsMaxRegs = 128;

// Bounded grid barrier (grid_barrier.cuh).  Returns false if the run must
// stop (a barrier timed out here or elsewhere).
__device__ __forceinline__ bool batch_barrier(const BatchArgs &a)
{
    return lbi::grid_barrier(a.bar, a.err, a.spin_limit);
}

template <int DT, bool NOISE, bool OBS>
__device__ __forceinline__ void batch_node(const BatchDesc &d, uint32_t s, const typename lbd::Store<DT>::T *src,
                                           typename lbd::Store<DT>::T *dst, const StepArgs &ph, uint32_t step,
                                           const float2 *phase, float acc[kModeVals])
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
        n[i] = in_bounds((size_t)i * P + off, 19 * P, ph.err) ? S::cvt(__ldcg(base + (size_t)i * P + off), ph.inv_scale)
                                                             : 0.0f;
    }
    StepArgs a = ph;
    a.step = step;
    float m[19], out[19];
    lbd::forward(n, m);
    if (OBS) {  // u = (sum n c + f/2) / rho of the streamed state (Sec. 3.7)
        const float ir = 1.0f / (ph.rho0 + m[0]);
        const float ux = (m[1] + 0.5f * ph.fx) * ir, uy = (m[2] + 0.5f * ph.fy) * ir, uz = (m[3] + 0.5f * ph.fz) * ir;
        const float2 ex = __ldg(phase + d.phase + x);
        const float2 ey = __ldg(phase + d.phase + d.nx + y);
        const float2 ez = __ldg(phase + d.phase + d.nx + d.ny + z);
        acc[0] = fmaf(ux, ez.x, acc[0]);
        acc[1] = fmaf(ux, ez.y, acc[1]);
        acc[2] = fmaf(uy, ez.x, acc[2]);
        acc[3] = fmaf(uy, ez.y, acc[3]);
        acc[4] = fmaf(uy, ex.x, acc[4]);
        acc[5] = fmaf(uy, ex.y, acc[5]);
        acc[6] = fmaf(uz, ex.x, acc[6]);
        acc[7] = fmaf(uz, ex.y, acc[7]);
        acc[8] = fmaf(uz, ey.x, acc[8]);
        acc[9] = fmaf(uz, ey.y, acc[9]);
        acc[10] = fmaf(ux, ey.x, acc[10]);
        acc[11] = fmaf(ux, ey.y, acc[11]);
    }
    collide_moments<NOISE>(m, ph.fx, ph.fy, ph.fz, a, d.rk, s, d.replica, out);
    typename S::T *o = dst + d.off;
#pragma unroll
    for (int i = 0; i < 19; ++i)
        if (in_bounds((size_t)i * P + s, 19 * P, ph.err)) o[(size_t)i * P + s] = S::pack(out[i], ph.scale);
}

// Nodes s and s + 1 (s even, nx even: the same row) of replica d: the pair
// update of k_stream_collide2 -- one row address per plane for both nodes,
// 8-byte (FP32) / 4-byte (FP16, BF16) accesses where the pair moves
// together, and the collision of both nodes in packed FP32 (f32x2.cuh).
template <int DT>
__device__ __forceinline__ void ld_pair(const typename lbd::Store<DT>::T *p, float inv, float &a, float &b);
template <>
__device__ __forceinline__ void ld_pair<0>(const float *p, float, float &a, float &b)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}
template <>
__device__ __forceinline__ void ld_pair<1>(const __half *p, float inv, float &a, float &b)
{
    const __half2 v = __ldcg(reinterpret_cast<const __half2 *>(p));
    a = __low2float(v) * inv;
    b = __high2float(v) * inv;
}
template <>
__device__ __forceinline__ void ld_pair<2>(const __nv_bfloat16 *p, float inv, float &a, float &b)
{
    const __nv_bfloat162 v = __ldcg(reinterpret_cast<const __nv_bfloat162 *>(p));
    a = __low2float(v) * inv;
    b = __high2float(v) * inv;
}

template <int DT, bool NOISE, bool OBS>
__device__ __forceinline__ void batch_pair(const BatchDesc &d, uint32_t s, const typename lbd::Store<DT>::T *src,
                                           typename lbd::Store<DT>::T *dst, const StepArgs &ph, uint32_t step,
                                           const float2 *phase, float acc[kModeVals])
{
    using S = lbd::Store<DT>;
    const uint32_t row = divide(s, d.dx);
    const int x0 = (int)(s - row * (uint32_t)d.nx);
    const uint32_t zz = divide(s, d.dxy);
    const int y = (int)(row - zz * (uint32_t)d.ny);
    const int z = (int)zz;
    const int xm = (x0 == 0) ? d.nx - 1 : x0 - 1;   // source of node x0 for c_x = +1
    const int xp = (x0 + 2 == d.nx) ? 0 : x0 + 2;   // source of node x0 + 1 for c_x = -1
    const int ym = (y == 0) ? d.ny - 1 : y - 1, yp = (y == d.ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? d.nz - 1 : z - 1, zp = (z == d.nz - 1) ? 0 : z + 1;
    const uint32_t P = d.pitch;
    const typename S::T *base = src + d.off;
    lbp::F2 n[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        const uint32_t r = (uint32_t)i * P + (uint32_t)((sz * d.ny + sy) * d.nx);
        const size_t lim = 19 * (size_t)P;
        float v0 = 0.0f, v1 = 0.0f;  // stored values; FP16 / BF16 unscaled below by one packed multiply
        if (lbd::cx(i) == 0) {
            if (in_bounds(r + x0 + 1, lim, ph.err)) ld_pair<DT>(base + r + x0, 1.0f, v0, v1);
        } else if (lbd::cx(i) == 1) {
            if (in_bounds(r + xm, lim, ph.err) && in_bounds(r + x0, lim, ph.err)) {
                v0 = S::cvt(__ldcg(base + r + xm), 1.0f);
                v1 = S::cvt(__ldcg(base + r + x0), 1.0f);
            }
        } else {
            if (in_bounds(r + x0 + 1, lim, ph.err) && in_bounds(r + xp, lim, ph.err)) {
                v0 = S::cvt(__ldcg(base + r + x0 + 1), 1.0f);
                v1 = S::cvt(__ldcg(base + r + xp), 1.0f);
            }
        }
        n[i] = DT == 0 ? lbp::f2(v0, v1) : lbp::f2(v0, v1) * lbp::f2s(ph.inv_scale);
    }
    StepArgs a = ph;
    a.step = step;
    lbp::F2 m[19], out[19];
    lbp::forward2(n, m);
    const lbp::F2 fx = lbp::f2s(ph.fx), fy = lbp::f2s(ph.fy), fz = lbp::f2s(ph.fz);
    if (OBS) {  // u = (sum n c + f/2) / rho of the streamed state (Sec. 3.7)
        const lbp::F2 rho = lbp::f2s(ph.rho0) + m[0];
        float rl, rh;
        lbp::split(rho, rl, rh);
        const lbp::F2 ir = lbp::f2(__frcp_rn(rl), __frcp_rn(rh));
        const lbp::F2 half = lbp::f2s(0.5f);
        const lbp::F2 ux = lbp::fma2(half, fx, m[1]) * ir;
        const lbp::F2 uy = lbp::fma2(half, fy, m[2]) * ir;
        const lbp::F2 uz = lbp::fma2(half, fz, m[3]) * ir;
        const float2 ex0 = __ldg(phase + d.phase + x0), ex1 = __ldg(phase + d.phase + x0 + 1);
        const float2 ey = __ldg(phase + d.phase + d.nx + y);
        const float2 ez = __ldg(phase + d.phase + d.nx + d.ny + z);
        // scalar sums (twelve registers, not twenty-four): the y and z phases
        // are the same for both nodes of the pair, the x phases are not
        float uxl, uxh, uyl, uyh, uzl, uzh;
        lbp::split(ux, uxl, uxh);
        lbp::split(uy, uyl, uyh);
        lbp::split(uz, uzl, uzh);
        const float sx = uxl + uxh, sy = uyl + uyh, sz = uzl + uzh;
        acc[0] = fmaf(sx, ez.x, acc[0]);
        acc[1] = fmaf(sx, ez.y, acc[1]);
        acc[2] = fmaf(sy, ez.x, acc[2]);
        acc[3] = fmaf(sy, ez.y, acc[3]);
        acc[4] = fmaf(uyh, ex1.x, fmaf(uyl, ex0.x, acc[4]));
        acc[5] = fmaf(uyh, ex1.y, fmaf(uyl, ex0.y, acc[5]));
        acc[6] = fmaf(uzh, ex1.x, fmaf(uzl, ex0.x, acc[6]));
        acc[7] = fmaf(uzh, ex1.y, fmaf(uzl, ex0.y, acc[7]));
        acc[8] = fmaf(sz, ey.x, acc[8]);
        acc[9] = fmaf(sz, ey.y, acc[9]);
        acc[10] = fmaf(sx, ey.x, acc[10]);
        acc[11] = fmaf(sx, ey.y, acc[11]);
    }
    lbp::collide_moments2k<NOISE>(m, fx, fy, fz, a, lbp::RunningKeys{d.key0, d.key1}, s, d.replica, out);
    typename S::T *o = dst + d.off;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float o0, o1;
        lbp::split(DT == 0 ? out[i] : out[i] * lbp::f2s(ph.scale), o0, o1);
        if (in_bounds((uint32_t)i * P + s + 1, 19 * (size_t)P, ph.err)) Pair<DT>::store(o + (uint32_t)i * P + s, o0, o1, 1.0f);
    }
}

// The warp's mode sums of one tile (acc of every lane) added to the
// replica's record of this step: a butterfly reduce-scatter (12 -> 6 -> 3,
// padded to 4 -> 2 -> 1 values per lane, then the last pair of lanes), after
// which lane l holds the warp sum of value k = 6 b4 + 3 b3 + 2 b2 + b1 (b_i
// the bits of l; 2 b2 + b1 = 3 is padding), and the twelve even lanes with a
// value add it to the record (FP64 atomics; no block barrier).
__device__ __forceinline__ void record_warp(const float acc[kModeVals], double *rec)
{
    const int lane = threadIdx.x & 31;
    float b[6], c[3], d[4], e[2], f[1];
    butterfly_half<12>(acc, b, 16, lane & 16);
    butterfly_half<6>(b, c, 8, lane & 8);
    d[0] = c[0];
    d[1] = c[1];
    d[2] = c[2];
    d[3] = 0.0f;
    butterfly_half<4>(d, e, 4, lane & 4);
    butterfly_half<2>(e, f, 2, lane & 2);
    const float v = f[0] + __shfl_xor_sync(0xffffffffu, f[0], 1);
    const int pos = 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
    const int k = 6 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1) + pos;
    if (rec && !(lane & 1) && pos < 3) atomicAdd(rec + k, (double)v);
}

template <int DT, bool NOISE, bool OBS, bool PAIR>
__device__ __forceinline__ void batch_run(const BatchArgs &a)
{
    using T = typename lbd::Store<DT>::T;
    uint32_t step = a.state->step;
    uint32_t cur = a.state->cur;
    const uint32_t rec_step0 = a.state->rec_step0;
    for (int t = 0; t < a.nsteps; ++t) {
        const T *src = static_cast<const T *>(a.pops[cur]);
        T *dst = static_cast<T *>(a.pops[cur ^ 1u]);
        const uint32_t trec = step - rec_step0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const BatchTile tl = a.tiles[tile];
            const BatchDesc &d = a.desc[tl.rep];
            float acc[kModeVals];
            if (PAIR) {  // every replica has even nx: tiles hold whole pairs
#pragma unroll
                for (int q = 0; q < kModeVals; ++q) acc[q] = 0.0f;
                for (uint32_t k = 2 * threadIdx.x; k < tl.count; k += 2 * blockDim.x)
                    batch_pair<DT, NOISE, OBS>(d, tl.begin + k, src, dst, a.phys, step, a.phase, acc);
            } else {
#pragma unroll
                for (int q = 0; q < kModeVals; ++q) acc[q] = 0.0f;
                for (uint32_t k = threadIdx.x; k < tl.count; k += blockDim.x)
                    batch_node<DT, NOISE, OBS>(d, tl.begin + k, src, dst, a.phys, step, a.phase, acc);
            }
            if (OBS) {
                double *rec = trec < a.rec_cap ? a.modes + ((size_t)tl.rep * a.rec_cap + trec) * kModeVals : nullptr;
                record_warp(acc, rec);
            }
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

template <int DT, bool NOISE, bool OBS>
__global__ void k_batch(BatchArgs a)
{
    batch_run<DT, NOISE, OBS, false>(a);
}

template <int DT, bool NOISE>
__global__ void __maxnreg__(kBatchPairMaxRegs) k_batch_pair(BatchArgs a)
{
    batch_run<DT, NOISE, false, true>(a);
}

template <int DT, bool NOISE>
__global__ void __maxnreg__(kBatchPairObsMaxRegs) k_batch_pair_obs(BatchArgs a)
{
    batch_run<DT, NOISE, true, true>(a);
}

__global__ void k_set_rec_step0(BatchState *st, uint32_t v)
{
    st->rec_step0 = v;
}

// Autocorrelation of the recorded transverse modes of replica blockIdx.x at
// lag tau = blockIdx.y * blockDim.x + threadIdx.x:
//   C(tau) = (1 / (6 (t_end - t_begin - tau) V^2)) sum_{t0 = t_begin}^{t_end - tau - 1}
//            sum_q rec[t0 + tau][q] rec[t0][q],
// the mean over t0 and the six modes of Re u^(t0 + tau) conj(u^(t0)) with
// u^ = (record) / V.
__global__ void k_mode_acf(const double *modes, const BatchDesc *desc, int cap, int t_begin, int t_end,
                           int max_lag, double *acf)
{
    const int rep = blockIdx.x;
    const int tau = blockIdx.y * blockDim.x + threadIdx.x;
    if (tau > max_lag) return;
    const double *s = modes + (size_t)rep * cap * kModeVals;
    const int cnt = t_end - t_begin - tau;
    double acc = 0.0;
    for (int t0 = t_begin; t0 < t_end - tau; ++t0) {
        const double *x = s + (size_t)t0 * kModeVals, *y = s + (size_t)(t0 + tau) * kModeVals;
#pragma unroll
        for (int q = 0; q < kModeVals; ++q) acc = fma(x[q], y[q], acc);
    }
    const double V = (double)desc[rep].nodes;
    acf[(size_t)rep * (max_lag + 1) + tau] = cnt > 0 ? acc / (6.0 * (double)cnt * V * V) : 0.0;
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
    // transverse-mode records (lb_batch_record_modes)
    double *modes = nullptr;        // caller's [n][rec_cap][12], NULL: not recording
    int rec_cap = 0;
    uint32_t rec_step0 = 0;
    float2 *phase = nullptr;        // library: per-replica (cos, -sin) tables
    bool pairs = false;             // every replica has even nx: two nodes per thread
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

template <int DT, bool NOISE, bool OBS>
void *kernel_ptr(bool pair)
{
    if (!pair) return (void *)k_batch<DT, NOISE, OBS>;
    return OBS ? (void *)k_batch_pair_obs<DT, NOISE> : (void *)k_batch_pair<DT, NOISE>;
}

template <bool OBS>
void *pick_kernel_obs(const lb_batch *b)
{
    const bool noise = b->phys.kT > 0.0;
    const bool pr = b->pairs;
    switch (b->phys.dtype) {
    case LB_F32: return noise ? kernel_ptr<0, true, OBS>(pr) : kernel_ptr<0, false, OBS>(pr);
    case LB_F16: return noise ? kernel_ptr<1, true, OBS>(pr) : kernel_ptr<1, false, OBS>(pr);
    default: return noise ? kernel_ptr<2, true, OBS>(pr) : kernel_ptr<2, false, OBS>(pr);
    }
}

void *pick_kernel(const lb_batch *b)
{
    return b->modes ? pick_kernel_obs<true>(b) : pick_kernel_obs<false>(b);
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
    a.phys.err = b->err;
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
    a.modes = b->modes;
    a.phase = b->phase;
    a.rec_cap = (uint32_t)b->rec_cap;
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
    b->pairs = true;
    for (int r = 0; r < n; ++r) b->pairs = b->pairs && (per_replica[r].nx % 2 == 0);
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
        d.phase = 0;  // set by lb_batch_record_modes
        d.dx = make_div((uint32_t)p.nx);
        d.dxy = make_div((uint32_t)(p.nx * p.ny));
        d.rk = lbd::make_round_keys(p.seed);
        d.key0 = (uint32_t)(p.seed & 0xffffffffu);
        d.key1 = (uint32_t)(p.seed >> 32);
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
    BatchState s0{0u, 0u, 0u};
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
    cudaFree(b->phase);
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
    const NvtxRange range("lb_batch_step");
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
        BatchState s{b->step, (uint32_t)b->cur, b->rec_step0};
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

lb_status lb_batch_record_modes(lb_batch *b, double *modes, int capacity)
{
    if (!b || (modes && capacity < 1)) {
        set_error("lb_batch_record_modes: bad argument");
        return LB_EINVAL;
    }
    if (modes && ((uintptr_t)modes & 7u)) {
        set_error("lb_batch_record_modes: records must be 8-byte aligned");
        return LB_EINVAL;
    }
    cudaError_t e = cudaSuccess;
    if (modes && !b->phase) {
        // (cos, -sin)(2 pi r / L) for r along x, y, z of every replica, in FP64 rounded once
        std::vector<float2> tab;
        for (int r = 0; r < b->n; ++r) {
            BatchDesc &d = b->desc_h[r];
            d.phase = (uint32_t)tab.size();
            const int L3[3] = {d.nx, d.ny, d.nz};
            for (int ax = 0; ax < 3; ++ax)
                for (int q = 0; q < L3[ax]; ++q) {
                    const double ph = 2.0 * M_PI * (double)q / (double)L3[ax];
                    tab.push_back(make_float2((float)std::cos(ph), (float)-std::sin(ph)));
                }
        }
        e = cudaMalloc((void **)&b->phase, tab.size() * sizeof(float2));
        if (e != cudaSuccess) {
            b->phase = nullptr;
            set_error("lb_batch_record_modes: phase table allocation failed");
            return LB_ENOMEM;
        }
        e = cudaMemcpy(b->phase, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->desc, b->desc_h.data(), b->n * sizeof(BatchDesc), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail("lb_batch_record_modes (phase tables)", e);
    }
    if (modes) {
        e = cudaMemsetAsync(modes, 0, (size_t)b->n * capacity * kModeVals * sizeof(double), b->stream);
        if (e == cudaSuccess) {
            k_set_rec_step0<<<1, 1, 0, b->stream>>>(b->state, b->step);
            b->launches += 1;
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return cuda_fail("lb_batch_record_modes (clearing the records)", e);
    }
    const bool kernel_changes = (modes != nullptr) != (b->modes != nullptr);
    const bool args_change = modes != b->modes || (modes ? capacity : 0) != b->rec_cap;
    b->modes = modes;
    b->rec_cap = modes ? capacity : 0;
    b->rec_step0 = b->step;
    if (kernel_changes) {
        // the recording kernel may differ in occupancy: recompute the grid (this drops the graph)
        lb_batch_config c = b->cfg;
        return apply_config(b, &c);
    }
    if (args_change && b->graph) {  // the captured launch holds the old record arguments
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = 0;
    }
    return LB_OK;
}

lb_status lb_batch_mode_acf(lb_batch *b, const double *modes, int capacity, int t_begin, int t_end, int max_lag,
                            double *acf)
{
    if (!b || !modes || !acf || capacity < 1 || t_begin < 0 || t_end > capacity || t_begin >= t_end ||
        max_lag < 0 || max_lag >= t_end - t_begin) {
        set_error("lb_batch_mode_acf: bad argument (need 0 <= t_begin < t_end <= capacity, 0 <= max_lag < t_end - "
                  "t_begin)");
        return LB_EINVAL;
    }
    const int threads = 128;
    const dim3 grid((unsigned)b->n, (unsigned)((max_lag + threads) / threads));
    k_mode_acf<<<grid, threads, 0, b->stream>>>(modes, b->desc, capacity, t_begin, t_end, max_lag, acf);
    b->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_batch_mode_acf", e);
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
