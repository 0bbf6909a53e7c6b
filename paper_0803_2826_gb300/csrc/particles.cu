// particles.cu -- frictional point-particle coupling (Sec. 4.5) with the
// linear interpolation kernel of Sec. 4.6, and the Kremer-Grest forces of
// Sec. 2.1 for bead-spring chains.
//
// Per LB step the caller runs n_substeps particle steps against the frozen
// fluid velocity u = (sum n c + f_ext/2)/rho of the current state.  One
// kernel launch per sub-step does, for each particle (a group of 8 lanes):
//   forces      F^c from FENE bonds (chain neighbours p-1, p+1) and WCA pairs
//               from a Verlet list                          Eqs. (ufene), (ulennardjones)
//   interpolate u_p = sum_8 phi2 phi2 phi2 u(node)          Eqs. (ufluid_discrete), (Delta), (2point)
//   OU update   p' = C1 p + C2 (F^c + Gamma u_p) + C3 theta  Eq. (langevin_momentum_update)
//   spread      facc(node) -= J Delta(node - r_p), J = p' - p - C2 F^c   Eq. (ftotal)
//   drift       second half drift of this sub-step and first half drift of the next
//
// Positions are double in the caller's buffer, but inside a coupling call a
// position is an integer cell plus an FP32 offset in [0, 1) (a "shadow"
// float4, the cell packed in 10-bit fields), so the kernels do no FP64
// arithmetic except one conversion in and one out per call (GB300 runs FP64
// at a small fraction of its FP32 rate).  Shadows ping-pong between two
// buffers so every thread reads the positions of the same sub-step.
#include <algorithm>
#include <cstdio>

#include "d3q19.cuh"
#include "grid_barrier.cuh"
#include "lbf_internal.h"

namespace lbi {

constexpr int kMaxNb = 48;          // Verlet-list capacity per particle and chunk
constexpr int kChunks = 8;          // neighbour-list chunks = lanes per particle
constexpr float kSkin = 0.4f;       // Verlet skin in units of sigma
constexpr int kPartThreads = 128;
constexpr int kMaxCellDim = 1024;   // cells are packed in 10-bit fields

struct Particles {
    int cap = 0;
    float4 *shadow[2] = {nullptr, nullptr};  // [cap] cell + offset
    int *records = nullptr;      // base node of each (sub-step, particle) stencil
    size_t rec_cap = 0;
    size_t n_records = 0;
    int *nlist = nullptr;        // [cap][kChunks][kMaxNb]
    int *ncount = nullptr;       // [cap][kChunks]
    float4 *ref = nullptr;       // [cap] shadow positions at the last build
    unsigned int *flags = nullptr;  // two rebuild-request slots
    uint32_t sub_counter = 0;
    int nlist_n = -1;            // particle count the list was built for
    size_t rec_off = 0;          // offset of the live records in `records`
    int last_nsub = 0;           // sub-steps of the previous call
    bool persistent = true;      // use the persistent kernel when it fits
    unsigned int *bar = nullptr; // grid barrier words of the persistent kernel
};

namespace {

struct CoupleArgs {
    StepArgs g;
    int n;
    int chain_len;
    int use_wca;
    int noise_kind;
    float dt;
    float mass0, gamma0;
    int uniform_coef;      // no per-particle mass / gamma: C1..C3 below are valid
    float C1, C2, C3;
    float eps, sigma2, rc2, rlist2, k_fene, inv_r02, half_skin2;
    uint32_t pkey0, pkey1;
    uint32_t md_step;
    int last;              // last sub-step of this call
    uint32_t slot;         // rebuild slot written by this sub-step
};

// ---- cell + offset positions -----------------------------------------------

struct CPos {
    int c[3];
    float f[3];
};

__device__ __forceinline__ float4 pack(const CPos &q)
{
    const uint32_t w = (uint32_t)q.c[0] | ((uint32_t)q.c[1] << 10) | ((uint32_t)q.c[2] << 20);
    return make_float4(q.f[0], q.f[1], q.f[2], __uint_as_float(w));
}

__device__ __forceinline__ CPos unpack(float4 v)
{
    const uint32_t w = __float_as_uint(v.w);
    CPos q;
    q.c[0] = (int)(w & 1023u);
    q.c[1] = (int)((w >> 10) & 1023u);
    q.c[2] = (int)((w >> 20) & 1023u);
    q.f[0] = v.x;
    q.f[1] = v.y;
    q.f[2] = v.z;
    return q;
}

__device__ __forceinline__ double join1(int c, float f) { return (double)c + (double)f; }

// Put a double position into the box (periodic wrap; specular reflection
// into z in [1, nz-2] with walls, flipping p_z) -- the definition the
// FP32 path below follows.
__device__ void confine_d(double r[3], float p[3], const StepArgs &g)
{
    const double L[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
    const bool walls = g.z0 > 0;
    for (int c = 0; c < 3; ++c) {
        if (c == 2 && walls) {
            const double lo = 1.0, hi = (double)(g.nz - 2);
            if (r[2] < lo) { r[2] = 2.0 * lo - r[2]; p[2] = -p[2]; }
            if (r[2] > hi) { r[2] = 2.0 * hi - r[2]; p[2] = -p[2]; }
        } else {
            r[c] -= L[c] * floor(r[c] / L[c]);
            if (r[c] >= L[c]) r[c] -= L[c];
        }
    }
}

// Split a double position (already in the box) into cell + offset.  Returns
// false (and a clamped position) for positions outside the box or not finite.
__device__ __forceinline__ bool split(const double r[3], const StepArgs &g, CPos &q)
{
    const int L[3] = {g.nx, g.ny, g.nz};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = r[k];
        if (!(v >= 0.0 && v < (double)L[k])) {
            ok = false;
            v = 0.0;
        }
        int c = (int)floor(v);
        c = c < 0 ? 0 : (c > L[k] - 1 ? L[k] - 1 : c);
        q.c[k] = c;
        float f = (float)(v - (double)c);
        q.f[k] = f < 1.0f ? f : 0.99999994f;
    }
    return ok;
}

// r += h p (FP32 offset), then wrap / reflect as confine_d does.  A step of
// more than a few cells, or a non-finite one, is not a valid particle move:
// the position is clamped into the box and false is returned.
__device__ __forceinline__ bool drift(CPos &q, float p[3], float h, const StepArgs &g)
{
    const int L[3] = {g.nx, g.ny, g.nz};
    const bool walls = g.z0 > 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float f = fmaf(h, p[k], q.f[k]);
        if (!(f > -4.0f && f < 5.0f)) {  // also catches NaN
            ok = false;
            f = q.f[k];
        }
        const float fl = floorf(f);
        q.c[k] += (int)fl;
        q.f[k] = f - fl;
        if (q.f[k] >= 1.0f) {  // rounding of f - fl up to 1
            q.f[k] = 0.0f;
            q.c[k] += 1;
        }
        if (!(k == 2 && walls)) q.c[k] = ((q.c[k] % L[k]) + L[k]) % L[k];
    }
    if (walls) {
        const int hi = g.nz - 2;
        if (q.c[2] < 1 || q.c[2] > hi || (q.c[2] == hi && q.f[2] > 0.0f)) {
            double r[3] = {join1(q.c[0], q.f[0]), join1(q.c[1], q.f[1]), join1(q.c[2], q.f[2])};
            confine_d(r, p, g);
            if (!split(r, g, q)) ok = false;  // split clamps into the box
        }
    }
    return ok;
}

// Minimum-image separation a - b in FP32 from cell + offset positions.
__device__ __forceinline__ void separation(const CPos &a, const CPos &b, const StepArgs &g, float d[3])
{
    const int L[3] = {g.nx, g.ny, g.nz};
    const bool walls = g.z0 > 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int dc = a.c[k] - b.c[k];
        if (!(k == 2 && walls)) {
            if (2 * dc > L[k]) dc -= L[k];
            else if (2 * dc < -L[k]) dc += L[k];
        }
        d[k] = (float)dc + (a.f[k] - b.f[k]);
    }
}

// Fluid velocity at node (x, y, z): pull-gather of the stored state,
// u = (sum n c + f_ext/2) / rho.  Solid nodes give 0.
template <int DT>
__device__ __forceinline__ void node_velocity(const typename lbd::Store<DT>::T *__restrict__ src,
                                              const float *__restrict__ ffield, int x, int y, int z,
                                              const StepArgs &a, float u[3])
{
    using S = lbd::Store<DT>;
    if (z < a.z0 || z >= a.z1) {
        u[0] = u[1] = u[2] = 0.0f;
        return;
    }
    const bool walls = a.z0 > 0;
    const int xm = (x == 0) ? a.nx - 1 : x - 1, xp = (x == a.nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? a.ny - 1 : y - 1, yp = (y == a.ny - 1) ? 0 : y + 1;
    int zm, zp;
    if (walls) {
        zm = z - 1;
        zp = z + 1;
    } else {
        zm = (z == 0) ? a.nz - 1 : z - 1;
        zp = (z == a.nz - 1) ? 0 : z + 1;
    }
    const size_t self = ((size_t)z * a.ny + y) * a.nx + x;
    float rho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        const bool bounce = walls && lbd::cz(i) != 0 && (sz == 0 || sz == a.nz - 1);
        const size_t off = bounce ? ((size_t)lbd::opposite(i) * a.pitch + self)
                                  : ((size_t)i * a.pitch + ((size_t)sz * a.ny + sy) * a.nx + sx);
        const float v = S::cvt(src[off], a.inv_scale);
        rho += v;
        if (lbd::cx(i)) jx += lbd::cx(i) * v;
        if (lbd::cy(i)) jy += lbd::cy(i) * v;
        if (lbd::cz(i)) jz += lbd::cz(i) * v;
    }
    rho += a.rho0;
    float fx = a.fx, fy = a.fy, fz = a.fz;
    if (ffield) {
        fx += ffield[self];
        fy += ffield[a.nn + self];
        fz += ffield[2 * a.nn + self];
    }
    const float ir = 1.0f / rho;
    u[0] = (jx + 0.5f * fx) * ir;
    u[1] = (jy + 0.5f * fy) * ir;
    u[2] = (jz + 0.5f * fz) * ir;
}

// Stencil node q (0..7) of the cell containing position pos: coordinates and
// linear weight phi2(x) phi2(y) phi2(z).
__device__ __forceinline__ float stencil_node(const CPos &pos, int q, const StepArgs &g, int &x, int &y, int &z)
{
    const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
    const float w = (dx ? pos.f[0] : 1.0f - pos.f[0]) * (dy ? pos.f[1] : 1.0f - pos.f[1]) *
                    (dz ? pos.f[2] : 1.0f - pos.f[2]);
    x = pos.c[0] + dx;
    y = pos.c[1] + dy;
    z = pos.c[2] + dz;
    if (x >= g.nx) x -= g.nx;
    if (y >= g.ny) y -= g.ny;
    if (z >= g.nz) z = (g.z0 > 0) ? g.nz - 1 : z - g.nz;
    return w;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// First half drift of a call: double positions in, shadow out.
__global__ void k_half_drift(const double *pos, float *mom, const float *mass, float4 *shadow, unsigned int *err,
                             CoupleArgs c)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    const float m = mass ? mass[p] : c.mass0;
    double r[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    float pm[3] = {mom[3 * p], mom[3 * p + 1], mom[3 * p + 2]};
    const double h = 0.5 * (double)c.dt / (double)m;
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] += h * (double)pm[k];
    confine_d(r, pm, c.g);
    CPos q;
    if (!split(r, c.g, q)) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    shadow[p] = pack(q);
    mom[3 * p] = pm[0];
    mom[3 * p + 1] = pm[1];
    mom[3 * p + 2] = pm[2];
}

// Verlet-list build over all pairs.  Particles j are split into kChunks
// chunks by j mod kChunks; block (bi, c) tests 128 particles i against chunk c
// (tiled through shared memory) and writes the partial list of (i, c), so no
// atomics or clearing are needed and the sub-step kernel's lane c reads
// chunk c.  Returns at once unless a rebuild was requested in slot `rd`.
constexpr int kTile = 128;

__global__ void __launch_bounds__(kTile) k_build_nlist(const float4 *shadow, int *nlist, int *ncount, float4 *ref,
                                                       const unsigned int *flags, unsigned int *err, CoupleArgs c,
                                                       uint32_t rd)
{
    if (flags[rd] == 0u) return;
    __shared__ float4 sp[kTile];
    const int i = blockIdx.x * kTile + threadIdx.x;
    const int chunk = blockIdx.y;  // particles j with j % kChunks == chunk (neighbours of a
                                   // chain spread evenly over the 8 lanes that read them)
    const int per = (c.n - chunk + kChunks - 1) / kChunks;
    CPos pi{};
    float4 raw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < c.n) {
        raw = shadow[i];
        pi = unpack(raw);
    }
    int cnt = 0;
    bool full = false;
    int *mine = nlist + ((size_t)i * kChunks + chunk) * kMaxNb;
    for (int base = 0; base < per; base += kTile) {
        const int t = base + threadIdx.x;
        if (t < per) sp[threadIdx.x] = shadow[chunk + kChunks * t];
        __syncthreads();
        const int lim = min(kTile, per - base);
        if (i < c.n) {
            for (int q = 0; q < lim; ++q) {
                const int jj = chunk + kChunks * (base + q);
                if (jj == i) continue;
                float d[3];
                separation(pi, unpack(sp[q]), c.g, d);
                const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 < c.rlist2) {
                    if (cnt < kMaxNb) mine[cnt] = jj;
                    else full = true;
                    ++cnt;
                }
            }
        }
        __syncthreads();
    }
    if (i < c.n) {
        ncount[(size_t)i * kChunks + chunk] = cnt < kMaxNb ? cnt : kMaxNb;
        if (chunk == 0) ref[i] = raw;
        if (full) atomicOr(err, LB_DERR_NLIST_FULL);
    }
}

// One particle sub-step; eight lanes per particle.  Lane q gathers the fluid
// velocity of stencil node q (19 loads) and spreads the impulse there; the
// lanes split the neighbour list (lane q reads chunk q) and the two FENE
// bonds, and shuffle-reduce u_p and F^c.  Every lane then holds the same
// u_p, F^c and theta and does the (cheap) momentum update; lane 0 writes.
template <int DT>
__global__ void __launch_bounds__(kPartThreads)
    k_substep(const typename lbd::Store<DT>::T *__restrict__ src, const float *__restrict__ ffield,
              const float4 *__restrict__ sh_in, float4 *__restrict__ sh_out, double *pos_out, float *mom,
              const float *mass, const float *gamma, const int *nlist, const int *ncount, const float4 *ref,
              float *facc, int *records, unsigned int *flags, unsigned int *err, CoupleArgs c,
              uint32_t clear_slot)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && c.use_wca) flags[clear_slot] = 0u;  // the list build has run
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid >> 3;
    const int q = tid & 7;
    if (p >= c.n) return;  // whole groups of eight leave together
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    const StepArgs &g = c.g;
    const CPos me = unpack(sh_in[p]);
    float pm[3] = {mom[3 * p], mom[3 * p + 1], mom[3 * p + 2]};

    // conservative forces at the half-step positions, split over the lanes
    float F[3] = {0.f, 0.f, 0.f};
    if (c.use_wca) {
        const size_t li = (size_t)p * kChunks + q;
        const int nc = ncount[li];
        const int *lst = nlist + li * kMaxNb;
        for (int k = 0; k < nc; ++k) {
            float d[3];
            separation(me, unpack(sh_in[lst[k]]), g, d);
            const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < c.rc2) {
                const float sr2 = c.sigma2 / r2;
                const float sr6 = sr2 * sr2 * sr2;
                const float mag = 24.0f * c.eps * (2.0f * sr6 * sr6 - sr6) / r2;
                F[0] += mag * d[0];
                F[1] += mag * d[1];
                F[2] += mag * d[2];
            }
        }
    }
    if (c.chain_len > 1 && q < 2) {
        const int k = p % c.chain_len;
        const int j = q == 0 ? p - 1 : p + 1;
        const bool bonded = (q == 0) ? (k > 0) : (k < c.chain_len - 1 && j < c.n);
        if (bonded) {
            float d[3];
            separation(me, unpack(sh_in[j]), g, d);
            const float x = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * c.inv_r02;
            if (x >= 1.0f) {
                atomicOr(err, LB_DERR_FENE_BROKEN);
            } else {
                const float mag = -c.k_fene / (1.0f - x);
                F[0] += mag * d[0];
                F[1] += mag * d[1];
                F[2] += mag * d[2];
            }
        }
    }

    // fluid velocity at the particle: lane q takes stencil node q
    int x, y, z;
    const float w = stencil_node(me, q, g, x, y, z);
    float un[3];
    node_velocity<DT>(src, ffield, x, y, z, g, un);
    float up[3] = {w * un[0], w * un[1], w * un[2]};
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            up[k] += __shfl_xor_sync(gmask, up[k], o);
            F[k] += __shfl_xor_sync(gmask, F[k], o);
        }
    }

    // exact Ornstein-Uhlenbeck momentum update (same in every lane)
    const float m = mass ? mass[p] : c.mass0;
    const float G = gamma ? gamma[p] : c.gamma0;
    float C1 = c.C1, C2 = c.C2, C3 = c.C3;
    if (!c.uniform_coef) {
        const float x1 = G * c.dt / m;
        C1 = expf(-x1);
        C2 = (m / G) * (-expm1f(-x1));
        C3 = sqrtf(m * g.kT * (-expm1f(-2.0f * x1)));
    }
    float th[3] = {0.f, 0.f, 0.f};
    if (g.kT > 0.0f) {
        const lbd::U4 wv = lbd::philox10(lbd::U4{(uint32_t)p, c.md_step, (1u << 8) | 0u, g.replica}, c.pkey0, c.pkey1);
        if (c.noise_kind == 1) {
            const uint32_t ws[3] = {wv.x, wv.y, wv.z};
            const float s3 = 1.7320508075688772f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint64_t kk = 2ull * (uint64_t)(ws[k] >> 9) + 1ull;  // uniform = kk / 2^24
                th[k] = (6ull * kk < (1ull << 24)) ? -s3 : ((6ull * kk > 5ull * (1ull << 24)) ? s3 : 0.0f);
            }
        } else {
            float g3;
            lbd::box_muller(wv.x, wv.y, th[0], th[1]);
            lbd::box_muller(wv.z, wv.w, th[2], g3);
        }
    }
    float pn[3], J[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pn[k] = C1 * pm[k] + C2 * (F[k] + G * up[k]) + C3 * th[k];
        J[k] = pn[k] - pm[k] - C2 * F[k];
    }

    // spread -J Delta: lane q into its own node
    {
        const size_t P = g.pitch;
        const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
        atomicAdd(facc + s, -J[0] * w);
        atomicAdd(facc + P + s, -J[1] * w);
        atomicAdd(facc + 2 * P + s, -J[2] * w);
    }
    if (q != 0) return;
    if (records) records[p] = (int)(((size_t)me.c[2] * g.ny + me.c[1]) * g.nx + me.c[0]);

    // second half drift of this sub-step, then the first of the next one
    const float h = 0.5f * c.dt / m;
    CPos nx = me;
    bool ok = drift(nx, pn, h, g);
    if (c.last) {
        pos_out[3 * p] = join1(nx.c[0], nx.f[0]);
        pos_out[3 * p + 1] = join1(nx.c[1], nx.f[1]);
        pos_out[3 * p + 2] = join1(nx.c[2], nx.f[2]);
    } else {
        ok = drift(nx, pn, h, g) && ok;
    }
    if (!ok) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    sh_out[p] = pack(nx);
    mom[3 * p] = pn[0];
    mom[3 * p + 1] = pn[1];
    mom[3 * p + 2] = pn[2];
    if (ref) {
        float d[3];
        separation(nx, unpack(ref[p]), g, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] > c.half_skin2) flags[c.slot] = 1u;
    }
}

// Zero the eight accumulator nodes around each recorded stencil base.
__global__ void k_clear_records(float *facc, const int *records, size_t n, StepArgs g)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int base = records[q];
        const int x0 = base % g.nx;
        const int y0 = (base / g.nx) % g.ny;
        const int z0 = base / (g.nx * g.ny);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int x = x0 + (k & 1), y = y0 + ((k >> 1) & 1), z = z0 + (k >> 2);
            if (x >= g.nx) x -= g.nx;
            if (y >= g.ny) y -= g.ny;
            if (z >= g.nz) z = (g.z0 > 0) ? g.nz - 1 : z - g.nz;
            const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
            facc[s] = 0.0f;
            facc[g.pitch + s] = 0.0f;
            facc[2 * g.pitch + s] = 0.0f;
        }
    }
}

// Interpolated velocity at caller positions; eight lanes per position.
template <int DT>
__global__ void k_interpolate(const typename lbd::Store<DT>::T *__restrict__ src, const float *__restrict__ ffield,
                              const double *pos, float *u_out, int n, unsigned int *err, StepArgs g)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid >> 3, q = tid & 7;
    if (p >= n) return;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    double r[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    CPos me;
    if (!split(r, g, me) && q == 0) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    int x, y, z;
    const float w = stencil_node(me, q, g, x, y, z);
    float un[3];
    node_velocity<DT>(src, ffield, x, y, z, g, un);
    float up[3] = {w * un[0], w * un[1], w * un[2]};
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) up[k] += __shfl_xor_sync(gmask, up[k], o);
    if (q == 0) {
        u_out[3 * p] = up[0];
        u_out[3 * p + 1] = up[1];
        u_out[3 * p + 2] = up[2];
    }
}

void free_parts(Particles *P)
{
    if (!P) return;
    cudaFree(P->shadow[0]);
    cudaFree(P->shadow[1]);
    cudaFree(P->records);
    cudaFree(P->nlist);
    cudaFree(P->ncount);
    cudaFree(P->ref);
    cudaFree(P->flags);
    cudaFree(P->bar);
    delete P;
}

lb_status ensure_buffers(lb_handle *h, int n, int nsub)
{
    if (!h->facc) {
        cudaError_t e = cudaMalloc((void **)&h->facc, 3 * h->pitch * sizeof(float));
        if (e != cudaSuccess) {
            set_error("lb_couple_particles: accumulator allocation failed (%s)", cudaGetErrorString(e));
            return LB_ENOMEM;
        }
        e = cudaMemsetAsync(h->facc, 0, 3 * h->pitch * sizeof(float), h->stream);
        if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
    }
    if (!h->parts) h->parts = new Particles();
    Particles *P = h->parts;
    if (P->cap < n) {
        cudaFree(P->shadow[0]);
        cudaFree(P->shadow[1]);
        cudaFree(P->nlist);
        cudaFree(P->ncount);
        cudaFree(P->ref);
        P->shadow[0] = P->shadow[1] = nullptr;
        P->nlist = nullptr;
        P->ncount = nullptr;
        P->ref = nullptr;
        cudaError_t e = cudaMalloc((void **)&P->shadow[0], (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->shadow[1], (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->nlist, (size_t)n * kChunks * kMaxNb * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->ncount, (size_t)n * kChunks * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->ref, (size_t)n * sizeof(float4));
        if (e != cudaSuccess) {
            P->cap = 0;
            set_error("lb_couple_particles: particle buffer allocation failed (%s)", cudaGetErrorString(e));
            return LB_ENOMEM;
        }
        P->cap = n;
        P->nlist_n = -1;
    }
    if (!P->flags) {
        // [0], [1]: rebuild slots of the multi-kernel path; [2], [3]: build
        // request and rebuild epoch of the persistent path
        cudaError_t e = cudaMalloc((void **)&P->flags, 4 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->bar, 3 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(P->flags, 0, 4 * sizeof(unsigned int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(P->bar, 0, 3 * sizeof(unsigned int), h->stream);
        if (e != cudaSuccess) {
            set_error("lb_couple_particles: flag allocation failed");
            return LB_ENOMEM;
        }
    }
    const size_t need = (size_t)n * (size_t)nsub;
    if (P->rec_cap < P->rec_off + P->n_records + need || P->rec_cap < 2 * need) {
        // grow, keeping the records not yet cleared (moved to offset 0)
        int *nr = nullptr;
        const size_t cap = std::max((P->n_records + need) * 2, 2 * need);
        cudaError_t e = cudaMalloc((void **)&nr, cap * sizeof(int));
        if (e != cudaSuccess) {
            set_error("lb_couple_particles: record allocation failed");
            return LB_ENOMEM;
        }
        if (P->n_records) {
            e = cudaMemcpyAsync(nr, P->records + P->rec_off, P->n_records * sizeof(int), cudaMemcpyDeviceToDevice,
                                h->stream);
            if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
            e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
        }
        cudaFree(P->records);
        P->records = nr;
        P->rec_cap = cap;
        P->rec_off = 0;
    }
    return LB_OK;
}

// ---------------------------------------------------------------------------
// Persistent variant: one cooperative launch runs all sub-steps of a call.
// Each group of 8 lanes owns one particle for the whole call (position,
// momentum and the fluid velocity of its 8 stencil nodes stay in registers;
// the velocities are re-gathered only when the particle changes cell).  Sub-
// steps are separated by the bounded grid barrier.  The Verlet list is built
// by k_build_nlist before the launch when the previous call asked for it; if a
// particle still moves more than half the skin during the call, every group
// rebuilds its own list in place (a slower scan, no barrier needed).
// ---------------------------------------------------------------------------
struct PersistArgs {
    CoupleArgs c;
    int nsub;
    const void *src;
    const float *ffield;
    double *pos;
    float *mom;
    const float *mass, *gamma;
    float4 *sh[2];
    int *nlist, *ncount;
    float4 *ref;
    float *facc;
    int *records;            // this call: [nsub][n]
    const int *stale;        // previous call's records to clear: [nstale_sub][n], or NULL
    int nstale_sub;
    unsigned int *flags;     // [0] build before the next call, [1] rebuild epoch request
    uint32_t epoch0;         // epoch of this call's first sub-step
    unsigned int *bar;
    unsigned int *err;
    unsigned int spin_limit;
};

// Shadow positions from the caller's double positions, when a list build is
// requested (the positions may have been changed between calls).
__global__ void k_shadow_from_pos(const double *pos, float4 *shadow, const unsigned int *flag, unsigned int *err,
                                  CoupleArgs c)
{
    if (*flag == 0u) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    const double r[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    CPos q;
    if (!split(r, c.g, q)) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    shadow[p] = pack(q);
}

__device__ __forceinline__ void rebuild_own_list(const PersistArgs &a, int p, int q, const CPos &me,
                                                 const float4 *sh)
{
    const int n = a.c.n;
    int *mine = a.nlist + ((size_t)p * kChunks + q) * kMaxNb;
    int cnt = 0;
    bool full = false;
    for (int j = q; j < n; j += kChunks) {  // the chunk k_build_nlist assigns to lane q
        if (j == p) continue;
        float d[3];
        separation(me, unpack(sh[j]), a.c.g, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < a.c.rlist2) {
            if (cnt < kMaxNb) mine[cnt] = j;
            else full = true;
            ++cnt;
        }
    }
    a.ncount[(size_t)p * kChunks + q] = cnt < kMaxNb ? cnt : kMaxNb;
    if (full) atomicOr(a.err, LB_DERR_NLIST_FULL);
    if (q == 0) a.ref[p] = pack(me);
}

template <int DT>
__global__ void __launch_bounds__(kPartThreads, 8) k_couple_persistent(PersistArgs a)
{
    using S = lbd::Store<DT>;
    const CoupleArgs &c = a.c;
    const StepArgs &g = c.g;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid >> 3, q = tid & 7;
    const bool active = p < c.n;
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    const typename S::T *src = static_cast<const typename S::T *>(a.src);
    if (c.use_wca && blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = 0u;  // the pre-launch build has run

    // phase 0: clear the previous call's impulses, first half drift
    CPos me{};
    float pm[3] = {0.f, 0.f, 0.f};
    float m = 1.f, G = 1.f, C1 = c.C1, C2 = c.C2, C3 = c.C3;
    if (active) {
        for (int s = 0; s < a.nstale_sub; ++s) {
            const int base = a.stale[(size_t)s * c.n + p];
            CPos bq{};
            bq.c[0] = base % g.nx;
            bq.c[1] = (base / g.nx) % g.ny;
            bq.c[2] = base / (g.nx * g.ny);
            int x, y, z;
            (void)stencil_node(bq, q, g, x, y, z);
            const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
            a.facc[node] = 0.0f;
            a.facc[g.pitch + node] = 0.0f;
            a.facc[2 * g.pitch + node] = 0.0f;
        }
        m = a.mass ? a.mass[p] : c.mass0;
        G = a.gamma ? a.gamma[p] : c.gamma0;
        if (!c.uniform_coef) {
            const float x1 = G * c.dt / m;
            C1 = expf(-x1);
            C2 = (m / G) * (-expm1f(-x1));
            C3 = sqrtf(m * g.kT * (-expm1f(-2.0f * x1)));
        }
        double r[3] = {a.pos[3 * p], a.pos[3 * p + 1], a.pos[3 * p + 2]};
        pm[0] = a.mom[3 * p];
        pm[1] = a.mom[3 * p + 1];
        pm[2] = a.mom[3 * p + 2];
        const double h = 0.5 * (double)c.dt / (double)m;
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] += h * (double)pm[k];
        confine_d(r, pm, g);
        if (!split(r, g, me) && q == 0) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
        if (q == 0) a.sh[0][p] = pack(me);
    }
    if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;

    int cache_cell = -1;
    float uc[3] = {0.f, 0.f, 0.f};
    const float h = 0.5f * c.dt / m;
    for (int s = 0; s < a.nsub; ++s) {
        const float4 *shin = a.sh[s & 1];
        float4 *shout = a.sh[(s + 1) & 1];
        if (active) {
            if (c.use_wca && ((volatile unsigned int *)a.flags)[1] == a.epoch0 + (uint32_t)s)
                rebuild_own_list(a, p, q, me, shin);

            float F[3] = {0.f, 0.f, 0.f};
            if (c.use_wca) {
                const size_t li = (size_t)p * kChunks + q;
                const int nc = a.ncount[li];
                const int *lst = a.nlist + li * kMaxNb;
                for (int k = 0; k < nc; ++k) {
                    float d[3];
                    separation(me, unpack(shin[lst[k]]), g, d);
                    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 < c.rc2) {
                        const float sr2 = c.sigma2 / r2;
                        const float sr6 = sr2 * sr2 * sr2;
                        const float mag = 24.0f * c.eps * (2.0f * sr6 * sr6 - sr6) / r2;
                        F[0] += mag * d[0];
                        F[1] += mag * d[1];
                        F[2] += mag * d[2];
                    }
                }
            }
            if (c.chain_len > 1 && q < 2) {
                const int k = p % c.chain_len;
                const int j = q == 0 ? p - 1 : p + 1;
                const bool bonded = (q == 0) ? (k > 0) : (k < c.chain_len - 1 && j < c.n);
                if (bonded) {
                    float d[3];
                    separation(me, unpack(shin[j]), g, d);
                    const float x = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * c.inv_r02;
                    if (x >= 1.0f) {
                        atomicOr(a.err, LB_DERR_FENE_BROKEN);
                    } else {
                        const float mag = -c.k_fene / (1.0f - x);
                        F[0] += mag * d[0];
                        F[1] += mag * d[1];
                        F[2] += mag * d[2];
                    }
                }
            }

            // fluid velocity: lane q caches node q of the current cell
            int x, y, z;
            const float w = stencil_node(me, q, g, x, y, z);
            const int cell = (me.c[2] * g.ny + me.c[1]) * g.nx + me.c[0];
            if (cell != cache_cell) {
                node_velocity<DT>(src, a.ffield, x, y, z, g, uc);
                cache_cell = cell;
            }
            float up[3] = {w * uc[0], w * uc[1], w * uc[2]};
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    up[k] += __shfl_xor_sync(gmask, up[k], o);
                    F[k] += __shfl_xor_sync(gmask, F[k], o);
                }
            }

            float th[3] = {0.f, 0.f, 0.f};
            if (g.kT > 0.0f) {
                const lbd::U4 wv = lbd::philox10(
                    lbd::U4{(uint32_t)p, c.md_step + (uint32_t)s, (1u << 8) | 0u, g.replica}, c.pkey0, c.pkey1);
                if (c.noise_kind == 1) {
                    const uint32_t ws[3] = {wv.x, wv.y, wv.z};
                    const float s3 = 1.7320508075688772f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const uint64_t kk = 2ull * (uint64_t)(ws[k] >> 9) + 1ull;
                        th[k] = (6ull * kk < (1ull << 24)) ? -s3 : ((6ull * kk > 5ull * (1ull << 24)) ? s3 : 0.0f);
                    }
                } else {
                    float g3;
                    lbd::box_muller(wv.x, wv.y, th[0], th[1]);
                    lbd::box_muller(wv.z, wv.w, th[2], g3);
                }
            }
            float pn[3], J[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pn[k] = C1 * pm[k] + C2 * (F[k] + G * up[k]) + C3 * th[k];
                J[k] = pn[k] - pm[k] - C2 * F[k];
            }
            {
                const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
                atomicAdd(a.facc + node, -J[0] * w);
                atomicAdd(a.facc + g.pitch + node, -J[1] * w);
                atomicAdd(a.facc + 2 * g.pitch + node, -J[2] * w);
            }
            if (q == 0) a.records[(size_t)s * c.n + p] = cell;

            // drift (every lane computes the same new position)
            const bool last = (s == a.nsub - 1);
            bool ok = drift(me, pn, h, g);
            if (last) {
                if (q == 0) {
                    a.pos[3 * p] = join1(me.c[0], me.f[0]);
                    a.pos[3 * p + 1] = join1(me.c[1], me.f[1]);
                    a.pos[3 * p + 2] = join1(me.c[2], me.f[2]);
                    a.mom[3 * p] = pn[0];
                    a.mom[3 * p + 1] = pn[1];
                    a.mom[3 * p + 2] = pn[2];
                }
            } else {
                ok = drift(me, pn, h, g) && ok;
            }
            if (!ok && q == 0) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
            pm[0] = pn[0];
            pm[1] = pn[1];
            pm[2] = pn[2];
            if (q == 0) {
                shout[p] = pack(me);
                if (c.use_wca) {
                    float d[3];
                    separation(me, unpack(a.ref[p]), g, d);
                    const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (!last && d2 > c.half_skin2) atomicMax(&a.flags[1], a.epoch0 + (uint32_t)s + 1u);
                    if (last && d2 > 0.25f * c.half_skin2) a.flags[0] = 1u;  // build before the next call
                }
            }
        }
        if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
    }
}

template <int DT>
cudaError_t run_substeps(lb_handle *h, const lb_particles *pp, const lb_couple_params *cp)
{
    Particles *P = h->parts;
    const int n = pp->n;
    CoupleArgs c;
    c.g = make_args(h);
    c.n = n;
    c.chain_len = cp->chain_len;
    c.use_wca = cp->use_wca;
    c.noise_kind = cp->noise_kind;
    c.dt = (float)cp->dt;
    c.mass0 = (float)pp->mass0;
    c.gamma0 = (float)pp->gamma0;
    c.uniform_coef = (pp->mass == nullptr && pp->gamma == nullptr);
    {
        const double x1 = pp->gamma0 * cp->dt / pp->mass0;
        c.C1 = (float)std::exp(-x1);
        c.C2 = (float)(pp->mass0 / pp->gamma0 * (-std::expm1(-x1)));
        c.C3 = (float)std::sqrt(pp->mass0 * h->p.kT * (-std::expm1(-2.0 * x1)));
    }
    c.eps = (float)cp->eps;
    c.sigma2 = (float)(cp->sigma * cp->sigma);
    c.rc2 = (float)(cp->sigma * cp->sigma * 1.2599210498948732);  // (2^(1/6) sigma)^2
    const double rl = 1.122462048309373 * cp->sigma + kSkin * cp->sigma;
    c.rlist2 = (float)(rl * rl);
    c.half_skin2 = (float)(0.25 * kSkin * kSkin * cp->sigma * cp->sigma);
    c.k_fene = (float)cp->k_fene;
    c.inv_r02 = (float)(cp->r0 > 0 ? 1.0 / (cp->r0 * cp->r0) : 0.0);
    c.pkey0 = (uint32_t)(cp->seed & 0xffffffffu);
    c.pkey1 = (uint32_t)(cp->seed >> 32);
    c.last = 0;
    c.md_step = cp->md_step0;
    c.slot = 0;
    const int blocks = (n + kPartThreads - 1) / kPartThreads;
    using T = typename lbd::Store<DT>::T;
    const T *src = static_cast<const T *>(h->pops[h->cur]);
    const bool need_nlist = cp->use_wca != 0;

    // persistent path when every particle group can be resident at once
    const int pblocks = (int)(((size_t)n * 8 + kPartThreads - 1) / kPartThreads);
    int per_sm = 0;
    if (P->persistent && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_couple_persistent<DT>,
                                                                       kPartThreads, 0) == cudaSuccess &&
        pblocks <= per_sm * device_sm_count()) {
        cudaError_t e = cudaSuccess;
        if (need_nlist && P->nlist_n != n) {
            const unsigned int init[4] = {0u, 0u, 1u, 0u};  // [2]: build before the launch, [3]: epoch
            e = cudaMemcpyAsync(P->flags, init, sizeof(init), cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return e;
            P->nlist_n = n;
        }
        const bool fold_clear = h->facc_stale && P->n_records == (size_t)n * (size_t)P->last_nsub &&
                                P->n_records <= P->rec_cap / 2 && (size_t)n * cp->n_substeps <= P->rec_cap / 2;
        if (h->facc_stale && !fold_clear) {
            e = clear_particle_forces(h);
            if (e != cudaSuccess) return e;
            h->facc_stale = 0;
        }
        if (need_nlist) {
            k_shadow_from_pos<<<blocks, kPartThreads, 0, h->stream>>>(pp->pos, P->shadow[1], P->flags + 2, h->d_err,
                                                                       c);
            dim3 bgrid((n + kTile - 1) / kTile, kChunks);
            k_build_nlist<<<bgrid, kTile, 0, h->stream>>>(P->shadow[1], P->nlist, P->ncount, P->ref, P->flags,
                                                          h->d_err, c, 2u);
            h->launches += 2;
        }
        PersistArgs a;
        a.c = c;
        a.nsub = cp->n_substeps;
        a.src = src;
        a.ffield = h->force;
        a.pos = pp->pos;
        a.mom = pp->mom;
        a.mass = pp->mass;
        a.gamma = pp->gamma;
        a.sh[0] = P->shadow[0];
        a.sh[1] = P->shadow[1];
        a.nlist = P->nlist;
        a.ncount = P->ncount;
        a.ref = P->ref;
        a.facc = h->facc;
        // the record buffer has two halves: the stale records (cleared in the
        // kernel's first phase) stay in one, this call's go to the other
        const size_t half = P->rec_cap / 2;
        const size_t new_off = fold_clear ? (P->rec_off == 0 ? half : 0) : P->rec_off + P->n_records;
        a.stale = fold_clear ? P->records + P->rec_off : nullptr;
        a.nstale_sub = fold_clear ? P->last_nsub : 0;
        a.records = P->records + new_off;
        a.flags = P->flags + 2;
        a.epoch0 = P->sub_counter + 1u;
        a.bar = P->bar;
        a.err = h->d_err;
        a.spin_limit = 1u << 22;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(pblocks);
        lc.blockDim = dim3(kPartThreads);
        lc.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        void *args[] = {&a};
        e = cudaLaunchKernelExC(&lc, (const void *)k_couple_persistent<DT>, args);
        if (e != cudaSuccess) return e;
        h->launches += 1;
        if (fold_clear) {
            P->rec_off = new_off;
            P->n_records = (size_t)n * (size_t)cp->n_substeps;
            h->facc_stale = 0;
        } else {
            P->n_records += (size_t)n * (size_t)cp->n_substeps;
        }
        P->sub_counter += (uint32_t)cp->n_substeps;
        P->last_nsub = cp->n_substeps;
        return cudaGetLastError();
    }

    if (h->facc_stale) {
        cudaError_t e = clear_particle_forces(h);
        if (e != cudaSuccess) return e;
        h->facc_stale = 0;
    }
    if (need_nlist && P->nlist_n != n) {
        cudaError_t e = cudaMemsetAsync(P->flags, 0xff, 2 * sizeof(unsigned int), h->stream);
        if (e != cudaSuccess) return e;
        P->nlist_n = n;
    }
    k_half_drift<<<blocks, kPartThreads, 0, h->stream>>>(pp->pos, pp->mom, pp->mass, P->shadow[0], h->d_err, c);
    h->launches += 1;
    for (int s = 0; s < cp->n_substeps; ++s) {
        const uint32_t rd = P->sub_counter & 1u, wr = rd ^ 1u;
        if (need_nlist) {
            dim3 bgrid((n + kTile - 1) / kTile, kChunks);
            k_build_nlist<<<bgrid, kTile, 0, h->stream>>>(P->shadow[s & 1], P->nlist, P->ncount, P->ref, P->flags,
                                                          h->d_err, c, rd);
            h->launches += 1;
        }
        c.md_step = cp->md_step0 + (uint32_t)s;
        c.last = (s == cp->n_substeps - 1);
        c.slot = wr;
        int *rec = P->records + P->rec_off + P->n_records;
        const int sblocks = (int)(((size_t)n * 8 + kPartThreads - 1) / kPartThreads);
        k_substep<DT><<<sblocks, kPartThreads, 0, h->stream>>>(
            src, h->force, P->shadow[s & 1], P->shadow[(s + 1) & 1], pp->pos, pp->mom, pp->mass, pp->gamma,
            P->nlist, P->ncount, need_nlist ? P->ref : nullptr, h->facc, rec, P->flags, h->d_err, c, rd);
        P->n_records += (size_t)n;
        P->sub_counter += 1;
        h->launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace

lb_status couple_particles(lb_handle *h, const lb_particles *pp, const lb_couple_params *cp)
{
    if (pp->n < 0 || pp->reserved != 0 || cp->reserved != 0) {
        set_error("lb_couple_particles: bad particle count or reserved field");
        return LB_EINVAL;
    }
    if (pp->n == 0) return LB_OK;
    if (!pp->pos || !pp->mom) {
        set_error("lb_couple_particles: pos and mom are required");
        return LB_EINVAL;
    }
    if (h->p.nx > kMaxCellDim || h->p.ny > kMaxCellDim || h->p.nz > kMaxCellDim) {
        set_error("lb_couple_particles: particles need box edges <= %d", kMaxCellDim);
        return LB_EINVAL;
    }
    if (cp->n_substeps < 1 || !(cp->dt > 0.0) || cp->noise_kind < 0 || cp->noise_kind > 1) {
        set_error("lb_couple_particles: need n_substeps >= 1, dt > 0, noise_kind 0 or 1");
        return LB_EINVAL;
    }
    if ((!pp->mass && !(pp->mass0 > 0.0)) || (!pp->gamma && !(pp->gamma0 > 0.0))) {
        set_error("lb_couple_particles: mass0 and gamma0 must be > 0 when no per-particle arrays are given");
        return LB_EINVAL;
    }
    if (cp->chain_len > 1 && !(cp->r0 > 0.0)) {
        set_error("lb_couple_particles: FENE chains need r0 > 0");
        return LB_EINVAL;
    }
    if (cp->use_wca && !(cp->sigma > 0.0)) {
        set_error("lb_couple_particles: WCA needs sigma > 0");
        return LB_EINVAL;
    }
    if (cp->use_wca && (1.122462048309373 + kSkin) * cp->sigma * 2.0 >= (double)std::min(h->p.nx, h->p.ny)) {
        set_error("lb_couple_particles: box too small for the WCA neighbour search");
        return LB_EINVAL;
    }
    if (((uintptr_t)pp->pos & 7u) || ((uintptr_t)pp->mom & 3u)) {
        set_error("lb_couple_particles: misaligned pos or mom");
        return LB_EINVAL;
    }
    lb_status st = ensure_buffers(h, pp->n, cp->n_substeps);
    if (st != LB_OK) return st;
    cudaError_t e;
    // impulses of the previous call that lb_step already applied are cleared
    // inside run_substeps (by the persistent kernel, or by k_clear_records)
    switch (h->p.dtype) {
    case LB_F32: e = run_substeps<0>(h, pp, cp); break;
    case LB_F16: e = run_substeps<1>(h, pp, cp); break;
    default: e = run_substeps<2>(h, pp, cp); break;
    }
    if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
    h->facc_dirty = 1;
    return LB_OK;
}

cudaError_t clear_particle_forces(lb_handle *h)
{
    Particles *P = h->parts;
    if (!P || !h->facc) return cudaSuccess;
    if (P->n_records) {
        const StepArgs g = make_args(h);
        int blocks = (int)std::min<size_t>((P->n_records + 255) / 256, (size_t)8 * device_sm_count());
        k_clear_records<<<blocks, 256, 0, h->stream>>>(h->facc, P->records + P->rec_off, P->n_records, g);
        h->launches += 1;
        P->n_records = 0;
        P->rec_off = 0;
    }
    return cudaGetLastError();
}

lb_status interpolate(lb_handle *h, int n, const double *pos, float *u_out)
{
    if (n == 0) return LB_OK;
    const StepArgs g = make_args(h);
    const int blocks = (int)(((size_t)n * 8 + kPartThreads - 1) / kPartThreads);
    switch (h->p.dtype) {
    case LB_F32:
        k_interpolate<0><<<blocks, kPartThreads, 0, h->stream>>>(static_cast<const float *>(h->pops[h->cur]),
                                                                  h->force, pos, u_out, n, h->d_err, g);
        break;
    case LB_F16:
        k_interpolate<1><<<blocks, kPartThreads, 0, h->stream>>>(static_cast<const __half *>(h->pops[h->cur]),
                                                                  h->force, pos, u_out, n, h->d_err, g);
        break;
    default:
        k_interpolate<2><<<blocks, kPartThreads, 0, h->stream>>>(
            static_cast<const __nv_bfloat16 *>(h->pops[h->cur]), h->force, pos, u_out, n, h->d_err, g);
        break;
    }
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_interpolate", e);
}

void destroy_particles(lb_handle *h)
{
    free_parts(h->parts);
    h->parts = nullptr;
}

}  // namespace lbi
