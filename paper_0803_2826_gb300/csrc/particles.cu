// particles.cu -- frictional point-particle coupling (Sec. 4.5) with the
// interpolation functions phi_2, phi_3, phi_4 of Sec. 4.6, and the
// Kremer-Grest forces of Sec. 2.1 for bead-spring chains.
//
// Per LB step the caller runs n_substeps particle steps against the frozen
// fluid velocity u = (sum n c + f_ext/2)/rho of the current state.  One
// kernel launch per sub-step does, for each particle (a group of 8 lanes):
//   forces      F^c from FENE bonds (chain neighbours p-1, p+1), WCA pairs
//               from a Verlet list and a constant external force   Eqs. (ufene), (ulennardjones)
//   interpolate u_p = sum phi phi phi u(node) over the K^3 stencil  Eqs. (ufluid_discrete), (Delta)
//   OU update   p' = C1 p + C2 (F^c + Gamma u_p) + C3 theta  Eq. (langevin_momentum_update)
//   spread      facc(node) -= J Delta(node - r_p), J = p' - p - dt F^c, the
//               impulse of the drag and random forces (F^c is constant
//               during the update)                         Eq. (ftotal)
//   drift       second half drift of this sub-step and first half drift of the next
//
// Free particles (no FENE / WCA) take k_couple_free instead: one launch for
// all sub-steps of a call (each particle's sub-steps depend on no other
// particle), with the stencil's node velocities and impulse sums in registers.
//
// Positions are double in the caller's buffer, but inside a coupling call a
// position is an integer cell plus an FP32 offset in [0, 1) (a "shadow"
// float4, the cell packed in 10-bit fields), so the kernels do no FP64
// arithmetic except one conversion in and one out per call (GB300 runs FP64
// at a small fraction of its FP32 rate).  Shadows ping-pong between two
// buffers so every thread reads the positions of the same sub-step.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "d3q19.cuh"
#include "grid_barrier.cuh"
#include "lbf_internal.h"

namespace lbi {

constexpr int kMaxNb = 64;          // Verlet-list capacity per particle
constexpr int kChunks = 8;          // lanes per particle in the per-sub-step kernels
constexpr float kSkin = 0.4f;       // Verlet skin in units of sigma
constexpr int kPartThreads = 128;
constexpr int kMaxCellDim = 1024;   // cells are packed in 10-bit fields
constexpr int kFlagWords = 5;       // [0], [1]: per-sub-step kernels; [2..4]: persistent kernel

struct Particles {
    int cap = 0;
    float4 *shadow[2] = {nullptr, nullptr};  // [cap] cell + offset
    int *records = nullptr;      // base node of each (sub-step, particle) stencil
    size_t rec_cap = 0;
    size_t n_records = 0;
    int *nlist = nullptr;        // [cap][kMaxNb], ascending
    int *ncount = nullptr;       // [cap]
    float4 *ref = nullptr;       // [cap] shadow positions at the last build
    unsigned int *flags = nullptr;  // rebuild requests (kFlagWords words)
    uint32_t sub_counter = 0;
    int nlist_n = -1;            // particle count the list was built for
    size_t rec_off = 0;          // offset of the live records in `records`
    int last_nsub = 0;           // sub-steps of the previous call
    unsigned int *bar = nullptr; // grid barrier words of the persistent kernel
    // cell list of the Verlet-list build: particles binned into cells of edge
    // >= r_list, cells hashed into `nbuckets` linked-list buckets
    int *head = nullptr;         // [nbuckets] first particle of a bucket, -1 = empty
    int *next = nullptr;         // [cap] next particle in the same bucket
    int *bucket_of = nullptr;    // [cap] bucket of each particle (to empty it again)
    int nb_log2 = 0;             // log2 nbuckets
    int rec_span = 2;            // nodes per axis the live records' stencils touch (2, or 4 for phi_3 / phi_4)
    int rec_n = 0;               // particles per sub-step of the live records (-1: calls with different counts)
    // fluid velocities at the stencil nodes of each particle, kept over the
    // sub-steps of a call (the fluid is frozen during a call): [cap][64]
    // float4, valid while the particle's stencil origin and the call epoch
    // match its tag
    float4 *ucache = nullptr;
    int2 *utag = nullptr;        // [cap] (packed stencil origin, epoch)
    int ucache_cap = 0;
    uint32_t epoch = 0;          // coupling calls that used the cache
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
    int ncell[3];          // cell-list cells per axis (edge L / ncell >= r_list)
    float cinv[3];         // ncell / L
    int nb_log2;           // log2 of the bucket count
    int kw;                // interpolation stencil width: 2 (phi_2), 3 (phi_3), 4 (phi_4)
    float fext[3];         // constant external force on every particle (part of F^c)
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

// Put a double position into the box (periodic wrap; with walls, specular
// reflection into the band z in [kw/2, nz-1-kw/2], flipping p_z, so that a
// stencil kw nodes wide touches fluid nodes only) -- the definition the FP32
// path below follows.
__device__ void confine_d(double r[3], float p[3], const StepArgs &g, int kw = 2)
{
    const double L[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
    const bool walls = g.z0 > 0;
    for (int c = 0; c < 3; ++c) {
        if (c == 2 && walls) {
            const double lo = 0.5 * kw, hi = (double)(g.nz - 1) - lo;
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

// Whether a cell + offset position lies outside the wall band of a stencil
// kw nodes wide, z in [kw/2, nz-1-kw/2] (exact: the band edges are whole or
// half-integer).
__device__ __forceinline__ bool outside_band(const CPos &q, const StepArgs &g, int kw)
{
    const int c = q.c[2];
    const float f = q.f[2];
    if (kw & 1) {
        const int lo = kw >> 1, hi = g.nz - 2 - (kw >> 1);
        return c < lo || (c == lo && f < 0.5f) || c > hi || (c == hi && f > 0.5f);
    }
    const int lo = kw >> 1, hi = g.nz - 1 - (kw >> 1);
    return c < lo || c > hi || (c == hi && f > 0.0f);
}

// r += h p (FP32 offset), then wrap / reflect as confine_d does.  A step of
// more than a few cells, or a non-finite one, is not a valid particle move:
// the position is clamped into the box and false is returned.
__device__ __forceinline__ bool drift(CPos &q, float p[3], float h, const StepArgs &g, int kw = 2)
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
        if (!(k == 2 && walls)) {
            int v = q.c[k];
            if (v < 0) v += L[k];
            else if (v >= L[k]) v -= L[k];
            if ((unsigned)v >= (unsigned)L[k]) v = ((v % L[k]) + L[k]) % L[k];  // boxes narrower than a step
            q.c[k] = v;
        }
    }
    if (walls) {
        if (outside_band(q, g, kw)) {
            double r[3] = {join1(q.c[0], q.f[0]), join1(q.c[1], q.f[1]), join1(q.c[2], q.f[2])};
            confine_d(r, p, g, kw);
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

// One axis of the stencil of phi_KW (Sec. 4.6) for the position c + f:
// first node o and the KW weights of nodes o, o + 1, ...  phi_2: 1 - f, f.
// phi_3 (Eq. 3point): with n the nearest node and d = c + f - n in
// [-1/2, 1/2), the middle weight is (1 + sqrt(1 - 3 d^2)) / 3 and C1, C2
// give the outer two, (1 - w_0 -+ d) / 2.  phi_4 (Eq. 4point): the nodes
// c - 1 .. c + 2 carry (3 - 2f - S, 3 - 2f + S, 1 + 2f + S, 1 + 2f - S) / 8
// with S = sqrt(1 + 4 f (1 - f)), the two branches of phi_4 at the four
// distances.  Both forms are the paper's functions rewritten so that the
// weights sum to one and the small outer weights carry no cancellation of
// large terms.
template <int KW>
__device__ __forceinline__ int axis_weights(int c, float f, float w[KW])
{
    if constexpr (KW == 2) {
        w[0] = 1.0f - f;
        w[1] = f;
        return c;
    } else if constexpr (KW == 3) {
        const bool up = f >= 0.5f;
        const float d = up ? f - 1.0f : f;  // exact
        const float w0 = (1.0f + sqrtf(fmaf(-3.0f * d, d, 1.0f))) * (1.0f / 3.0f);
        w[0] = 0.5f * (1.0f - w0 - d);
        w[1] = w0;
        w[2] = 0.5f * (1.0f - w0 + d);
        return up ? c : c - 1;
    } else {
        const float S = sqrtf(fmaf(4.0f * f, 1.0f - f, 1.0f));
        const float a = 3.0f - 2.0f * f, b = 1.0f + 2.0f * f;
        w[0] = 0.125f * (a - S);
        w[1] = 0.125f * (a + S);
        w[2] = 0.125f * (b + S);
        w[3] = 0.125f * (b - S);
        return c - 1;
    }
}

template <int KW>
struct Stencil {
    int o[3];       // first node per axis (may lie outside the box before wrapping)
    float w[3][KW]; // weights per axis
};

template <int KW>
__device__ __forceinline__ void make_stencil(const CPos &pos, Stencil<KW> &s)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) s.o[k] = axis_weights<KW>(pos.c[k], pos.f[k], s.w[k]);
}

__device__ __forceinline__ int wrap_node(int v, int L)
{
    v = v < 0 ? v + L : (v >= L ? v - L : v);
    if ((unsigned)v >= (unsigned)L) v = ((v % L) + L) % L;  // boxes narrower than the stencil
    return v;
}

// Node q (0 .. KW^3 - 1, x fastest) of a stencil: coordinates and weight
// Delta = phi(x) phi(y) phi(z) (Eq. Delta).  For KW = 2 this is
// stencil_node() above, operation for operation.  With walls z is kept in
// the box (the band keeps the stencil off the solid planes).
template <int KW>
__device__ __forceinline__ float stencil_node_k(const Stencil<KW> &s, int q, const StepArgs &g, int &x, int &y,
                                                int &z)
{
    const int dx = q % KW, dy = (q / KW) % KW, dz = q / (KW * KW);
    float wx = s.w[0][0], wy = s.w[1][0], wz = s.w[2][0];
#pragma unroll
    for (int j = 1; j < KW; ++j) {  // selects, no indexed local arrays
        if (dx == j) wx = s.w[0][j];
        if (dy == j) wy = s.w[1][j];
        if (dz == j) wz = s.w[2][j];
    }
    x = wrap_node(s.o[0] + dx, g.nx);
    y = wrap_node(s.o[1] + dy, g.ny);
    z = s.o[2] + dz;
    if (g.z0 > 0) z = z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z);
    else z = wrap_node(z, g.nz);
    return wx * wy * wz;
}

template <int KW>
constexpr int free_lanes() { return KW == 2 ? 1 : 8; }

// Coordinates of node q of the stencil with first nodes o (stencil_node_k
// without the weight).
template <int KW>
__device__ __forceinline__ void stencil_coords(const int o[3], int q, const StepArgs &g, int &x, int &y, int &z)
{
    const int dx = q % KW, dy = (q / KW) % KW, dz = q / (KW * KW);
    x = wrap_node(o[0] + dx, g.nx);
    y = wrap_node(o[1] + dy, g.ny);
    z = o[2] + dz;
    if (g.z0 > 0) z = z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z);
    else z = wrap_node(z, g.nz);
}

// The record of a particle's sub-step, which the overlapped step's
// re-update and the clearing of applied impulses expand to a block of
// record_span^3 nodes: for phi_2 and phi_4 the linear index of the
// particle's cell (the block is the cell's corners, resp. one node further
// on each side: the stencil), for phi_3 the wrapped stencil origin (the
// block is the 27-node stencil itself, not the 64 nodes around the cell).
template <int KW>
constexpr int record_span() { return KW == 3 ? 3 : (KW == 4 ? 4 : 2); }

template <int KW>
__device__ __forceinline__ int stencil_record(const CPos &me, const StepArgs &g)
{
    if constexpr (KW == 3) {
        int o[3];
        const int L[3] = {g.nx, g.ny, g.nz};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = me.c[k] - 1 + (me.f[k] >= 0.5f ? 1 : 0);  // the origin of axis_weights<3>
            if (o[k] < 0) o[k] += L[k];
        }
        return (o[2] * g.ny + o[1]) * g.nx + o[0];
    } else {
        return (me.c[2] * g.ny + me.c[1]) * g.nx + me.c[0];
    }
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
    confine_d(r, pm, c.g, c.kw);
    CPos q;
    if (!split(r, c.g, q)) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    shadow[p] = pack(q);
    mom[3 * p] = pm[0];
    mom[3 * p + 1] = pm[1];
    mom[3 * p + 2] = pm[2];
}

// Verlet-list build from a cell list.  The box is cut into ncell[k] cells per
// axis of edge >= r_list, so every pair closer than r_list lies in the same or
// adjacent cells (periodically adjacent, except across the walls); cells are
// hashed into 2^nb_log2 buckets, each a linked list (head / next) filled with
// atomicExch.  Particle p is served by 8 lanes that split the (up to 27)
// cells around p and append every j within r_list to one shared-memory list;
// lane 0 sorts it and drops duplicates (two cells may share a bucket): the
// same list as a test of all pairs, in O(n) work.
__device__ __forceinline__ void cell_of(const CPos &q, const CoupleArgs &c, int cc[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int v = (int)(((float)q.c[k] + q.f[k]) * c.cinv[k]);
        cc[k] = min(max(v, 0), c.ncell[k] - 1);
    }
}

// Fibonacci hashing of the linear cell index.
__device__ __forceinline__ int bucket_of_cell(int x, int y, int z, const CoupleArgs &c)
{
    const uint32_t lin = ((uint32_t)z * (uint32_t)c.ncell[1] + (uint32_t)y) * (uint32_t)c.ncell[0] + (uint32_t)x;
    return (int)((lin * 2654435761u) >> (32 - c.nb_log2));
}

// Cells adjacent to cell v along one axis (itself included), each once.
__device__ __forceinline__ int adjacent_cells(int v, int nc, bool wall, int out[3])
{
    if (wall) {
        int m = 0;
        if (v > 0) out[m++] = v - 1;
        out[m++] = v;
        if (v < nc - 1) out[m++] = v + 1;
        return m;
    }
    if (nc < 3) {
        out[0] = 0;
        out[1] = 1;
        return nc;
    }
    out[0] = v == 0 ? nc - 1 : v - 1;
    out[1] = v;
    out[2] = v == nc - 1 ? 0 : v + 1;
    return 3;
}

// Put particle p (cell + offset q) into its bucket.
__device__ __forceinline__ void bin_particle(int p, const CPos &q, const CoupleArgs &c, int *head, int *next,
                                             int *bucket_of)
{
    int cc[3];
    cell_of(q, c, cc);
    const int b = bucket_of_cell(cc[0], cc[1], cc[2], c);
    bucket_of[p] = b;
    next[p] = atomicExch(head + b, p);
}

// Binning of the shadows a build will read (the multi-kernel path; the
// persistent path bins in k_shadow_from_pos).
__global__ void k_bin(const float4 *shadow, int *head, int *next, int *bucket_of, const unsigned int *flags,
                      CoupleArgs c, uint32_t rd)
{
    if (flags[rd] == 0u) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    bin_particle(p, unpack(shadow[p]), c, head, next, bucket_of);
}

// The buckets are emptied again by the kernel that consumes the lists (each
// particle resets the head of its own bucket), so no clearing pass is needed.
__device__ __forceinline__ void unbin_particle(int p, int *head, const int *bucket_of) { head[bucket_of[p]] = -1; }

__global__ void __launch_bounds__(kPartThreads) k_build_nlist(const float4 *shadow, const int *head,
                                                              const int *next, int *nlist, int *ncount, float4 *ref,
                                                              const unsigned int *flags, unsigned int *err,
                                                              CoupleArgs c, uint32_t rd)
{
    if (flags[rd] == 0u) return;
    constexpr int kGroups = kPartThreads / kChunks;
    __shared__ int lst[kMaxNb][kGroups];  // column per particle: conflict-free
    __shared__ int fill[kGroups];
    const int t = threadIdx.x, grp = t >> 3;
    const int tid = blockIdx.x * blockDim.x + t;
    const int p = tid >> 3, q = tid & 7;
    if (p >= c.n) return;  // whole groups of eight leave together
    const unsigned gmask = 0xFFu << (t & 24);
    if (q == 0) fill[grp] = 0;
    __syncwarp(gmask);
    const float4 raw = shadow[p];
    const CPos me = unpack(raw);
    int cc[3], cx[3], cy[3], cz[3];
    cell_of(me, c, cc);
    const int mx = adjacent_cells(cc[0], c.ncell[0], false, cx);
    const int my = adjacent_cells(cc[1], c.ncell[1], false, cy);
    const int mz = adjacent_cells(cc[2], c.ncell[2], c.g.z0 > 0, cz);
    bool full = false, broken = false;
    for (int k = q; k < mx * my * mz; k += kChunks) {
        const int ix = k % mx, iy = (k / mx) % my, iz = k / (mx * my);
        int hops = 0;
        for (int j = head[bucket_of_cell(cx[ix], cy[iy], cz[iz], c)]; j >= 0; j = next[j]) {
            if (j >= c.n || ++hops > c.n) {  // cannot happen for a consistent list
                broken = true;
                break;
            }
            if (j == p) continue;
            float d[3];
            separation(me, unpack(shadow[j]), c.g, d);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= c.rlist2) continue;
            const int slot = atomicAdd(&fill[grp], 1);
            if (slot < kMaxNb) lst[slot][grp] = j;
            else full = true;
        }
    }
    __syncwarp(gmask);
    if (q == 0) {  // insertion sort, duplicates dropped
        const int m = min(fill[grp], kMaxNb);
        int cnt = 0;
        for (int k = 0; k < m; ++k) {
            const int j = lst[k][grp];
            int at = cnt;
            while (at > 0 && lst[at - 1][grp] > j) {
                lst[at][grp] = lst[at - 1][grp];
                --at;
            }
            if (at > 0 && lst[at - 1][grp] == j) {  // duplicate: undo the shift
                for (int r = at; r < cnt; ++r) lst[r][grp] = lst[r + 1][grp];
                continue;
            }
            lst[at][grp] = j;
            ++cnt;
        }
        fill[grp] = cnt;
        ncount[p] = cnt;
        ref[p] = raw;
    }
    __syncwarp(gmask);
    const int cnt = fill[grp];
    int *mine = nlist + (size_t)p * kMaxNb;
    for (int k = q; k < cnt; k += kChunks) mine[k] = lst[k][grp];
    if (full || broken) atomicOr(err, LB_DERR_NLIST_FULL);
}

// The same list for one particle, built by one thread (the persistent
// kernel's rebuild inside a call), sorted in place in `mine`.
__device__ int build_own_list(int p, const CPos &me, const float4 *shadow, const int *head, const int *next,
                              const CoupleArgs &c, int *mine, unsigned int *err)
{
    int cc[3], cx[3], cy[3], cz[3];
    cell_of(me, c, cc);
    const int mx = adjacent_cells(cc[0], c.ncell[0], false, cx);
    const int my = adjacent_cells(cc[1], c.ncell[1], false, cy);
    const int mz = adjacent_cells(cc[2], c.ncell[2], c.g.z0 > 0, cz);
    int cnt = 0;
    bool full = false, broken = false;
    for (int k = 0; k < mx * my * mz; ++k) {
        const int ix = k % mx, iy = (k / mx) % my, iz = k / (mx * my);
        int hops = 0;
        for (int j = head[bucket_of_cell(cx[ix], cy[iy], cz[iz], c)]; j >= 0; j = next[j]) {
            if (j >= c.n || ++hops > c.n) {
                broken = true;
                break;
            }
            if (j == p) continue;
            float d[3];
            separation(me, unpack(shadow[j]), c.g, d);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= c.rlist2) continue;
            int at = cnt;
            while (at > 0 && mine[at - 1] > j) --at;
            if (at > 0 && mine[at - 1] == j) continue;
            if (cnt == kMaxNb) {
                full = true;
                continue;
            }
            for (int r = cnt; r > at; --r) mine[r] = mine[r - 1];
            mine[at] = j;
            ++cnt;
        }
    }
    if (full || broken) atomicOr(err, LB_DERR_NLIST_FULL);
    return cnt;
}

// WCA force of b on a (Eq. (ulennardjones), cut and shifted at 2^(1/6) sigma),
// added to F.
// `use` false adds nothing; the arithmetic has no branch, so that several
// pairs can be in flight at once.
__device__ __forceinline__ void wca_add(const CPos &a, const CPos &b, const CoupleArgs &c, float F[3],
                                        bool use = true)
{
    float d[3];
    separation(a, b, c.g, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float ir2 = __frcp_rn(r2);
    const float sr2 = c.sigma2 * ir2;
    const float sr6 = sr2 * sr2 * sr2;
    const float mag = (use && r2 < c.rc2) ? 24.0f * c.eps * (2.0f * sr6 * sr6 - sr6) * ir2 : 0.0f;
    F[0] = fmaf(mag, d[0], F[0]);
    F[1] = fmaf(mag, d[1], F[1]);
    F[2] = fmaf(mag, d[2], F[2]);
}

// FENE force of the bond to b on a (Eq. (ufene)), added to F; false (and no
// force) for a bond stretched to R0 or beyond.
__device__ __forceinline__ bool fene_add(const CPos &a, const CPos &b, const CoupleArgs &c, float F[3])
{
    float d[3];
    separation(a, b, c.g, d);
    const float x = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * c.inv_r02;
    if (x >= 1.0f) return false;
    const float mag = -c.k_fene / (1.0f - x);
    F[0] += mag * d[0];
    F[1] += mag * d[1];
    F[2] += mag * d[2];
    return true;
}

// The particle noise theta of Eq. (langevin_momentum_update): unit-variance
// Gaussians (two Box-Muller pairs) or the three-point distribution
// (-sqrt 3, 0, +sqrt 3 with probabilities 1/6, 2/3, 1/6) from one Philox
// block, counters (p, step, 1 << 8, replica).
__device__ __forceinline__ void particle_theta(uint32_t p, uint32_t step, const CoupleArgs &c, float th[3])
{
    const lbd::U4 wv = lbd::philox10(lbd::U4{p, step, (1u << 8) | 0u, c.g.replica}, c.pkey0, c.pkey1);
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

// One particle sub-step; eight lanes per particle.  Lane q gathers the fluid
// velocity of stencil node q (19 loads) and spreads the impulse there; the
// lanes split the neighbour list (lane q takes entries q, q + 8, ...) and the
// two FENE bonds, and shuffle-reduce u_p and F^c.  Every lane then holds the same
// u_p, F^c and theta and does the (cheap) momentum update; lane 0 writes.
template <int DT, int KW>
__global__ void __launch_bounds__(kPartThreads)
    k_substep(const typename lbd::Store<DT>::T *__restrict__ src, const float *__restrict__ ffield,
              const float4 *__restrict__ sh_in, float4 *__restrict__ sh_out, double *pos_out, float *mom,
              const float *mass, const float *gamma, const int *nlist, const int *ncount, const float4 *ref,
              int *head, const int *bucket_of, float *facc, int *records, unsigned int *flags,
              unsigned int *err, float4 *__restrict__ ucache, int2 *__restrict__ utag, int epoch,
              CoupleArgs c, uint32_t clear_slot)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && c.use_wca) flags[clear_slot] = 0u;  // the list build has run
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid >> 3;
    const int q = tid & 7;
    if (p >= c.n) return;  // whole groups of eight leave together
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);
    const StepArgs &g = c.g;
    if (c.use_wca && q == 0) unbin_particle(p, head, bucket_of);
    const CPos me = unpack(sh_in[p]);
    float pm[3] = {mom[3 * p], mom[3 * p + 1], mom[3 * p + 2]};

    // conservative forces at the half-step positions, split over the lanes
    // (lane 0 starts from the external force)
    float F[3] = {q == 0 ? c.fext[0] : 0.f, q == 0 ? c.fext[1] : 0.f, q == 0 ? c.fext[2] : 0.f};
    if (c.use_wca) {
        const int nc = ncount[p];
        const int *lst = nlist + (size_t)p * kMaxNb;
        for (int k = q; k < nc; k += kChunks) wca_add(me, unpack(sh_in[lst[k]]), c, F);
    }
    if (c.chain_len > 1 && q < 2) {
        const int k = p % c.chain_len;
        const int j = q == 0 ? p - 1 : p + 1;
        const bool bonded = (q == 0) ? (k > 0) : (k < c.chain_len - 1 && j < c.n);
        if (bonded && !fene_add(me, unpack(sh_in[j]), c, F)) atomicOr(err, LB_DERR_FENE_BROKEN);
    }

    // fluid velocity at the particle: lane q takes stencil nodes q, q + 8, ...
    // The node velocities of the particle's stencil are cached per call: a
    // particle keeps its stencil for many sub-steps, so the pull-gathers of
    // 19 populations per node run only when its stencil origin moves.
    constexpr int kNodes = KW * KW * KW, kPerLane = (kNodes + kChunks - 1) / kChunks;
    Stencil<KW> st;
    make_stencil<KW>(me, st);
    const int okey = wrap_node(st.o[0], g.nx) | (wrap_node(st.o[1], g.ny) << 10) |
                     ((g.z0 > 0 ? st.o[2] : wrap_node(st.o[2], g.nz)) << 20);
    int miss = 1;
    if (q == 0) {
        const int2 tag = utag[p];
        miss = !(tag.x == okey && tag.y == epoch);
    }
    // one decision for the group, taken before lane 0 may rewrite the tag
    const bool hit = __shfl_sync(gmask, miss, 0, kChunks) == 0;
    float4 *uc = ucache + (size_t)p * 64 + q;
    float up[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const int qq = q + kChunks * i;
        if (kNodes % kChunks == 0 || qq < kNodes) {
            int x, y, z;
            const float w = stencil_node_k<KW>(st, qq, g, x, y, z);
            float un[3];
            if (hit) {
                const float4 v = __ldcg(uc + kChunks * i);
                un[0] = v.x;
                un[1] = v.y;
                un[2] = v.z;
            } else {
                node_velocity<DT>(src, ffield, x, y, z, g, un);
                __stcg(uc + kChunks * i, make_float4(un[0], un[1], un[2], 0.0f));
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) up[k] = i == 0 ? w * un[k] : fmaf(w, un[k], up[k]);
        }
    }
    if (!hit && q == 0) utag[p] = make_int2(okey, epoch);
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
    if (g.kT > 0.0f) particle_theta((uint32_t)p, c.md_step, c, th);
    float pn[3], J[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pn[k] = C1 * pm[k] + C2 * (F[k] + G * up[k]) + C3 * th[k];
        J[k] = pn[k] - pm[k] - c.dt * F[k];
    }

    // spread -J Delta: lane q into its own nodes
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const int qq = q + kChunks * i;
        if (kNodes % kChunks == 0 || qq < kNodes) {
            int x, y, z;
            const float w = stencil_node_k<KW>(st, qq, g, x, y, z);
            const size_t P = g.pitch;
            const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
            if (in_bounds(s, g.nn, g.err)) {
                atomicAdd(facc + s, -J[0] * w);
                atomicAdd(facc + P + s, -J[1] * w);
                atomicAdd(facc + 2 * P + s, -J[2] * w);
            }
        }
    }
    if (q != 0) return;
    if (records) records[p] = stencil_record<KW>(me, g);

    // second half drift of this sub-step, then the first of the next one
    const float h = 0.5f * c.dt / m;
    CPos nx = me;
    bool ok = drift(nx, pn, h, g, KW);
    if (c.last) {
        pos_out[3 * p] = join1(nx.c[0], nx.f[0]);
        pos_out[3 * p + 1] = join1(nx.c[1], nx.f[1]);
        pos_out[3 * p + 2] = join1(nx.c[2], nx.f[2]);
    } else {
        ok = drift(nx, pn, h, g, KW) && ok;
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

// Zero the accumulator nodes around each recorded cell: [b, b + 1] per axis
// for span 2 (phi_2), [b - 1, b + 2] for span 4 (covers phi_3 and phi_4).
template <int SPAN>
__global__ void k_clear_records(float *facc, const int *records, size_t n, StepArgs g)
{
    constexpr int lo = SPAN == 4 ? -1 : 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int base = records[q];
        const int x0 = base % g.nx;
        const int y0 = (base / g.nx) % g.ny;
        const int z0 = base / (g.nx * g.ny);
#pragma unroll
        for (int k = 0; k < SPAN * SPAN * SPAN; ++k) {
            const int x = wrap_node(x0 + lo + k % SPAN, g.nx), y = wrap_node(y0 + lo + (k / SPAN) % SPAN, g.ny);
            int z = z0 + lo + k / (SPAN * SPAN);
            if (g.z0 > 0) z = z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z);
            else z = wrap_node(z, g.nz);
            const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
            facc[s] = 0.0f;
            facc[g.pitch + s] = 0.0f;
            facc[2 * g.pitch + s] = 0.0f;
        }
    }
}

// The same for live records laid out [nsub][n]: eight lanes per particle
// walk its cells, skip a cell equal to the one before (a particle keeps its
// cell for many sub-steps) and zero nodes q, q + 8, ... of the block.
template <int SPAN>
__global__ void k_clear_records_by_particle(float *facc, const int *records, int n, int nsub, StepArgs g)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * 8) return;
    const int p = (int)(t >> 3), q = (int)(t & 7);
    constexpr int lo = SPAN == 4 ? -1 : 0, nk = SPAN * SPAN * SPAN;
    int prev = -1;
    for (int s = 0; s < nsub; ++s) {
        const int base = records[(size_t)s * n + p];
        if (base == prev) continue;
        prev = base;
        const int x0 = base % g.nx, y0 = (base / g.nx) % g.ny, z0 = base / (g.nx * g.ny);
#pragma unroll
        for (int k = q; k < nk; k += 8) {
            const int x = wrap_node(x0 + lo + k % SPAN, g.nx), y = wrap_node(y0 + lo + (k / SPAN) % SPAN, g.ny);
            int z = z0 + lo + k / (SPAN * SPAN);
            if (g.z0 > 0) z = z < 0 ? 0 : (z >= g.nz ? g.nz - 1 : z);
            else z = wrap_node(z, g.nz);
            const size_t i = ((size_t)z * g.ny + y) * g.nx + x;
            facc[i] = 0.0f;
            facc[g.pitch + i] = 0.0f;
            facc[2 * g.pitch + i] = 0.0f;
        }
    }
}

// Interpolated velocity at caller positions with phi_KW; eight lanes per
// position, lane q takes stencil nodes q, q + 8, ...
template <int DT, int KW>
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
    constexpr int kNodes = KW * KW * KW, kPerLane = (kNodes + kChunks - 1) / kChunks;
    Stencil<KW> st;
    make_stencil<KW>(me, st);
    float up[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const int qq = q + kChunks * i;
        if (kNodes % kChunks == 0 || qq < kNodes) {
            int x, y, z;
            const float w = stencil_node_k<KW>(st, qq, g, x, y, z);
            float un[3];
            node_velocity<DT>(src, ffield, x, y, z, g, un);
#pragma unroll
            for (int k = 0; k < 3; ++k) up[k] = i == 0 ? w * un[k] : fmaf(w, un[k], up[k]);
        }
    }
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
    cudaFree(P->head);
    cudaFree(P->next);
    cudaFree(P->bucket_of);
    cudaFree(P->ucache);
    cudaFree(P->utag);
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
        cudaFree(P->next);
        cudaFree(P->bucket_of);
        P->shadow[0] = P->shadow[1] = nullptr;
        P->nlist = nullptr;
        P->ncount = nullptr;
        P->ref = nullptr;
        P->next = nullptr;
        P->bucket_of = nullptr;
        cudaError_t e = cudaMalloc((void **)&P->shadow[0], (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->shadow[1], (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->nlist, (size_t)n * kMaxNb * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->ncount, (size_t)n * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->ref, (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->next, (size_t)n * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->bucket_of, (size_t)n * sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(P->bucket_of, 0, (size_t)n * sizeof(int), h->stream);
        if (e != cudaSuccess) {
            P->cap = 0;
            set_error("lb_couple_particles: particle buffer allocation failed (%s)", cudaGetErrorString(e));
            return LB_ENOMEM;
        }
        P->cap = n;
        P->nlist_n = -1;
    }
    {
        // at least 2n buckets (a power of two): few cells share one
        int lg = 10;
        while ((1 << lg) < 2 * n && lg < 30) ++lg;
        if (lg > P->nb_log2) {
            cudaFree(P->head);
            P->head = nullptr;
            P->nb_log2 = 0;
            cudaError_t e = cudaMalloc((void **)&P->head, ((size_t)1 << lg) * sizeof(int));
            if (e != cudaSuccess) {
                set_error("lb_couple_particles: cell-list allocation failed (%s)", cudaGetErrorString(e));
                return LB_ENOMEM;
            }
            P->nb_log2 = lg;
            e = cudaMemsetAsync(P->head, 0xff, ((size_t)1 << lg) * sizeof(int), h->stream);  // all empty
            if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
        }
    }
    if (!P->flags) {
        // [0], [1]: rebuild slots of the multi-kernel path; [2]: build request
        // and [3], [4]: rebuild epochs (by sub-step parity) of the persistent path
        cudaError_t e = cudaMalloc((void **)&P->flags, kFlagWords * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->bar, 3 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(P->flags, 0, kFlagWords * sizeof(unsigned int), h->stream);
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
// Persistent variant: one cooperative launch runs all sub-steps of a call,
// one thread per particle, so a warp advances 32 particles with a single
// instruction stream.  For the cell a particle is in, its thread keeps the
// fluid velocity of the 8 stencil nodes (re-gathered only when the particle
// changes cell, by the whole warp: four particles at a time, one node per
// lane) and the impulses spread to those nodes, summed over the sub-steps
// spent in the cell and added to the accumulator when the particle leaves
// the cell or the call ends (the accumulator is read only by the next
// lb_step).  The first Verlet neighbours stay in registers.  Sub-steps are
// separated by the bounded grid barrier.  The list comes from k_build_nlist
// before the launch when the previous call asked for it; if a particle moves
// more than half the skin during the call, every thread re-bins its particle
// and rebuilds its list from the cell list at the next sub-step.
// ---------------------------------------------------------------------------
constexpr int kPThreads = 128;   // particles per block of the persistent kernel
constexpr int kNbReg = 8;        // Verlet neighbours held in registers
constexpr unsigned kFullMask = 0xffffffffu;

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
    int *head, *next, *bucket_of;  // cell list; every bucket is empty again when the kernel ends
    float *facc;
    int *records;            // this call: [nsub][n]
    const int *stale;        // previous call's records to clear: [nstale_sub][n], or NULL
    int nstale_sub;
    unsigned int *flags;     // [0] build before the next call, [1 + (s & 1)] rebuild epoch of sub-step s
    uint32_t epoch0;         // epoch of this call's first sub-step
    unsigned int *bar;
    unsigned int *err;
    unsigned int spin_limit;
};

// Shadow positions from the caller's double positions, binned into the cell
// list, when a list build is requested (the positions may have been changed
// between calls).
__global__ void k_shadow_from_pos(const double *pos, float4 *shadow, int *head, int *next, int *bucket_of,
                                  const unsigned int *flag, unsigned int *err, CoupleArgs c)
{
    if (*flag == 0u) return;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    const double r[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    CPos q;
    if (!split(r, c.g, q)) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    shadow[p] = pack(q);
    bin_particle(p, q, c, head, next, bucket_of);
}

// Fluid velocity u of the 8 stencil nodes of cell `cell` into uc, for every
// lane with `need`; the whole warp must call this together.  Each round takes
// up to four such lanes: lane 8 k + q gathers node q of the k-th one and the
// owners collect their 24 values by shuffles.
template <int DT>
__device__ __forceinline__ void warp_gather(bool need, const int cell[3], const typename lbd::Store<DT>::T *src,
                                            const float *ffield, const StepArgs &g, float uc[8][3])
{
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(kFullMask, need);
    while (m) {
        int o[4] = {-1, -1, -1, -1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (m) {
                o[k] = __ffs(m) - 1;
                m &= m - 1;
            }
        }
        const int slot = lane >> 3, q = lane & 7;
        const int owner = slot == 0 ? o[0] : (slot == 1 ? o[1] : (slot == 2 ? o[2] : o[3]));
        CPos nc{};
        nc.c[0] = __shfl_sync(kFullMask, cell[0], owner < 0 ? 0 : owner);
        nc.c[1] = __shfl_sync(kFullMask, cell[1], owner < 0 ? 0 : owner);
        nc.c[2] = __shfl_sync(kFullMask, cell[2], owner < 0 ? 0 : owner);
        float u[3] = {0.f, 0.f, 0.f};
        if (owner >= 0) {
            int x, y, z;
            (void)stencil_node(nc, q, g, x, y, z);
            node_velocity<DT>(src, ffield, x, y, z, g, u);
        }
        const int mine = lane == o[0] ? 0 : (lane == o[1] ? 1 : (lane == o[2] ? 2 : (lane == o[3] ? 3 : -1)));
        const int base = (mine < 0 ? 0 : mine) << 3;
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float v = __shfl_sync(kFullMask, u[k], base | qq);
                if (mine >= 0) uc[qq][k] = v;
            }
        }
    }
}

// The same for every lane of the warp at once (the start of a call): round r
// serves lanes 4 r .. 4 r + 3, and kRounds rounds keep their loads in flight
// together.
template <int DT>
__device__ __forceinline__ void warp_gather_all(bool active, const int cell[3],
                                                const typename lbd::Store<DT>::T *src, const float *ffield,
                                                const StepArgs &g, float uc[8][3])
{
    constexpr int kRounds = 4;
    const int lane = threadIdx.x & 31, slot = lane >> 3, q = lane & 7;
#pragma unroll 1
    for (int r0 = 0; r0 < 8; r0 += kRounds) {
        float u[kRounds][3];
#pragma unroll
        for (int i = 0; i < kRounds; ++i) {
            const int owner = 4 * (r0 + i) + slot;
            const int on = __shfl_sync(kFullMask, (int)active, owner);
            CPos nc{};
            nc.c[0] = __shfl_sync(kFullMask, cell[0], owner);
            nc.c[1] = __shfl_sync(kFullMask, cell[1], owner);
            nc.c[2] = __shfl_sync(kFullMask, cell[2], owner);
            u[i][0] = u[i][1] = u[i][2] = 0.0f;
            if (on) {
                int x, y, z;
                (void)stencil_node(nc, q, g, x, y, z);
                node_velocity<DT>(src, ffield, x, y, z, g, u[i]);
            }
        }
        const int from = (lane & 3) << 3;  // the slot that served this lane
#pragma unroll
        for (int i = 0; i < kRounds; ++i) {
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float v = __shfl_sync(kFullMask, u[i][k], from | qq);
                    if ((lane >> 2) == r0 + i) uc[qq][k] = v;
                }
            }
        }
    }
}

// Add the impulse sums of the 8 stencil nodes of `cell` to the accumulator
// and zero them.
__device__ __forceinline__ void flush_impulses(const int cell[3], float acc[8][3], float *facc, const StepArgs &g)
{
    CPos cq{};
    cq.c[0] = cell[0];
    cq.c[1] = cell[1];
    cq.c[2] = cell[2];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int x, y, z;
        (void)stencil_node(cq, q, g, x, y, z);
        const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
        if (in_bounds(node, g.nn, g.err)) {
            atomicAdd(facc + node, acc[q][0]);
            atomicAdd(facc + g.pitch + node, acc[q][1]);
            atomicAdd(facc + 2 * g.pitch + node, acc[q][2]);
        }
        acc[q][0] = acc[q][1] = acc[q][2] = 0.0f;
    }
}

template <int DT>
__device__ __forceinline__ void couple_persistent_run(const PersistArgs &a)
{
    using T = typename lbd::Store<DT>::T;
    __shared__ unsigned int ticket;  // arrival word of the split barrier
    const CoupleArgs &c = a.c;
    const StepArgs &g = c.g;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < c.n;
    const T *src = static_cast<const T *>(a.src);
    if (c.use_wca && blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = 0u;  // the pre-launch build has run

    // phase 0: clear the previous call's impulses, first half drift
    CPos me{}, refp{};
    float pm[3] = {0.f, 0.f, 0.f};
    float m = 1.f, G = 1.f, C1 = c.C1, C2 = c.C2, C3 = c.C3;
    // neighbour indices; unused slots (and the bonds of unbonded ends) point
    // at the particle itself (inactive lanes: particle 0), so that every load
    // of a sub-step is unconditional
    const int self = active ? p : 0;
    int nnb = 0;
    int nb[kNbReg];
#pragma unroll
    for (int k = 0; k < kNbReg; ++k) nb[k] = self;
    bool bond_lo = false, bond_hi = false;
    if (active) {
        if (c.use_wca) unbin_particle(p, a.head, a.bucket_of);
        int prev = -1;
        for (int s = 0; s < a.nstale_sub; ++s) {
            const int base = a.stale[(size_t)s * c.n + p];
            if (base == prev) continue;  // same cell as the sub-step before
            prev = base;
            CPos bq{};
            bq.c[0] = base % g.nx;
            bq.c[1] = (base / g.nx) % g.ny;
            bq.c[2] = base / (g.nx * g.ny);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int x, y, z;
                (void)stencil_node(bq, q, g, x, y, z);
                const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
                a.facc[node] = 0.0f;
                a.facc[g.pitch + node] = 0.0f;
                a.facc[2 * g.pitch + node] = 0.0f;
            }
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
        if (!split(r, g, me)) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
        a.sh[0][p] = pack(me);
        if (c.use_wca) {
            nnb = a.ncount[p];
            const int *lst = a.nlist + (size_t)p * kMaxNb;
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < nnb) nb[k] = lst[k];
            refp = unpack(a.ref[p]);
        }
        if (c.chain_len > 1) {
            const int k = p % c.chain_len;
            bond_lo = k > 0;
            bond_hi = k < c.chain_len - 1 && p + 1 < c.n;
        }
    }
    const int jlo = bond_lo ? p - 1 : self, jhi = bond_hi ? p + 1 : self;
    int kmax = __reduce_max_sync(kFullMask, min(nnb, kNbReg));  // register slots any lane of the warp uses
    // fluid velocity at the 8 nodes of the cell ccell, and the impulse sums there
    float uc[8][3], acc[8][3];
#pragma unroll
    for (int q = 0; q < 8; ++q) uc[q][0] = uc[q][1] = uc[q][2] = acc[q][0] = acc[q][1] = acc[q][2] = 0.0f;
    int ccell[3] = {me.c[0], me.c[1], me.c[2]};
    warp_gather_all<DT>(active, ccell, src, a.ffield, g, uc);
    if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;

    bool binned = false;
    const float h = 0.5f * c.dt / m;
    for (int s = 0; s < a.nsub; ++s) {
        const float4 *shin = a.sh[s & 1];
        float4 *shout = a.sh[(s + 1) & 1];
        // neighbour positions and the rebuild flag (written before the last
        // barrier; L1 is bypassed), then the work that needs only this
        // particle's own state (its noise and stencil weights) while they load
        float4 v[kNbReg];
#pragma unroll
        for (int k = 0; k < kNbReg; ++k)
            if (k < kmax) v[k] = __ldcg(shin + nb[k]);
        const float4 vlo = __ldcg(shin + jlo), vhi = __ldcg(shin + jhi);
        const unsigned int req = c.use_wca ? __ldcg(a.flags + 1 + (s & 1)) : 0u;
        float th[3] = {0.f, 0.f, 0.f};
        if (g.kT > 0.0f) particle_theta((uint32_t)p, c.md_step + (uint32_t)s, c, th);
        float w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int x, y, z;
            w[q] = stencil_node(me, q, g, x, y, z);
        }

        if (c.use_wca && req == a.epoch0 + (uint32_t)s) {
            // a particle moved more than half the skin: re-bin all, rebuild every list
            if (binned) {
                if (active) unbin_particle(p, a.head, a.bucket_of);
                if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
            }
            if (active) bin_particle(p, me, c, a.head, a.next, a.bucket_of);
            if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
            binned = true;
            if (active) {
                int *mine = a.nlist + (size_t)p * kMaxNb;
                nnb = build_own_list(p, me, shin, a.head, a.next, c, mine, a.err);
#pragma unroll
                for (int k = 0; k < kNbReg; ++k) nb[k] = k < nnb ? mine[k] : self;
                a.ncount[p] = nnb;
                a.ref[p] = pack(me);
                refp = me;
            }
            kmax = __reduce_max_sync(kFullMask, min(nnb, kNbReg));
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < kmax) v[k] = __ldcg(shin + nb[k]);
        }

        // conservative forces at the half-step positions, from the external force
        float F[3] = {c.fext[0], c.fext[1], c.fext[2]};
        if (c.use_wca) {
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < kmax) wca_add(me, unpack(v[k]), c, F, k < nnb);
            for (int k = kNbReg; k < nnb; ++k) wca_add(me, unpack(__ldcg(shin + a.nlist[(size_t)p * kMaxNb + k])), c, F);
        }
        if (c.chain_len > 1) {
            if (bond_lo && !fene_add(me, unpack(vlo), c, F)) atomicOr(a.err, LB_DERR_FENE_BROKEN);
            if (bond_hi && !fene_add(me, unpack(vhi), c, F)) atomicOr(a.err, LB_DERR_FENE_BROKEN);
        }

        // (uc already holds the fluid velocity of cell me.c: gathered before
        // the first sub-step or, after a cell change, inside the previous barrier)
        if (active) {
            float up[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                up[0] = fmaf(w[q], uc[q][0], up[0]);
                up[1] = fmaf(w[q], uc[q][1], up[1]);
                up[2] = fmaf(w[q], uc[q][2], up[2]);
            }
            float pn[3], J[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pn[k] = C1 * pm[k] + C2 * (F[k] + G * up[k]) + C3 * th[k];
                J[k] = pn[k] - pm[k] - c.dt * F[k];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                acc[q][0] = fmaf(-J[0], w[q], acc[q][0]);
                acc[q][1] = fmaf(-J[1], w[q], acc[q][1]);
                acc[q][2] = fmaf(-J[2], w[q], acc[q][2]);
            }
            a.records[(size_t)s * c.n + p] = (me.c[2] * g.ny + me.c[1]) * g.nx + me.c[0];

            // second half drift of this sub-step, then the first of the next one
            const bool last = (s == a.nsub - 1);
            bool ok = drift(me, pn, h, g);
            if (last) {
                a.pos[3 * p] = join1(me.c[0], me.f[0]);
                a.pos[3 * p + 1] = join1(me.c[1], me.f[1]);
                a.pos[3 * p + 2] = join1(me.c[2], me.f[2]);
                a.mom[3 * p] = pn[0];
                a.mom[3 * p + 1] = pn[1];
                a.mom[3 * p + 2] = pn[2];
            } else {
                ok = drift(me, pn, h, g) && ok;
            }
            if (!ok) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
            pm[0] = pn[0];
            pm[1] = pn[1];
            pm[2] = pn[2];
            shout[p] = pack(me);
            if (c.use_wca) {
                float d[3];
                separation(me, refp, g, d);
                const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!last && d2 > c.half_skin2) atomicMax(&a.flags[1 + ((s + 1) & 1)], a.epoch0 + (uint32_t)s + 1u);
                if (last && d2 > 0.25f * c.half_skin2) a.flags[0] = 1u;  // build before the next call
            }
        }
        // the barrier in two halves: between them, particles that change cell
        // for the next sub-step hand in their impulse sums and the warp gathers
        // their new cells (this reads only the frozen fluid and writes only
        // registers and the accumulator, which no block reads during the call)
        grid_arrive(a.bar, &ticket);
        if (s + 1 < a.nsub) {
            const bool moved = active && (me.c[0] != ccell[0] || me.c[1] != ccell[1] || me.c[2] != ccell[2]);
            if (__any_sync(kFullMask, moved)) {
                if (moved) {
                    flush_impulses(ccell, acc, a.facc, g);
                    ccell[0] = me.c[0];
                    ccell[1] = me.c[1];
                    ccell[2] = me.c[2];
                }
                warp_gather<DT>(moved, ccell, src, a.ffield, g, uc);
            }
        }
        if (!grid_wait(a.bar, a.err, a.spin_limit, &ticket)) return;
    }
    if (active) {
        flush_impulses(ccell, acc, a.facc, g);
        if (binned) unbin_particle(p, a.head, a.bucket_of);
    }
}

// The phi_2 persistent coupling, and the same code capped at 112 registers
// for large boxes: its blocks then leave room for five instead of four
// stream-collide blocks on the SMs they share while the two run side by side.
// The cap spills (the coupling takes ~0.37 instead of ~0.23 ms at 256^3,
// still shorter than the stream-collide launch beside it, 0.44 ms) and took
// the 256^3 step from 0.470 to 0.464 ms; in small boxes, where the coupling
// is the longer of the two, the uncapped kernel is faster.
template <int DT>
__global__ void __launch_bounds__(kPThreads) k_couple_persistent(PersistArgs a)
{
    couple_persistent_run<DT>(a);
}

template <int DT>
__global__ void __maxnreg__(112) k_couple_persistent_lean(PersistArgs a)
{
    couple_persistent_run<DT>(a);
}

// Boxes from this many nodes take k_couple_persistent_lean.
constexpr size_t kLeanCouplingNodes = (size_t)1 << 24;

// ---------------------------------------------------------------------------
// Persistent variant for the wide stencils (phi_3, phi_4: 27 / 64 nodes) of
// k_couple_persistent: the same sub-step loop, forces, list rebuilds and
// barriers, one thread per particle, but the fluid velocity at the stencil
// nodes and the impulse sums there live in the block's shared memory (the
// 27 / 64 nodes do not fit in registers): column t of sm[c][q][t], c = u_x,
// u_y, u_z, J_x, J_y, J_z, q the stencil node.  When a particle's stencil
// origin moves, its thread adds the impulse sums to the accumulator and the
// warp gathers the new stencil's velocities (four particles per round, the
// nodes spread over the lanes).  One block of kPThreads per SM (the cache
// takes 81 KB / 192 KB).
// ---------------------------------------------------------------------------
template <int KW>
constexpr size_t wide_smem_bytes() { return (size_t)6 * KW * KW * KW * kPThreads * sizeof(float); }

template <int KW>
__device__ __forceinline__ float &wide_cache(float *sm, int c, int q, int t)
{
    return sm[((size_t)c * (KW * KW * KW) + q) * kPThreads + t];
}

// Gather the fluid velocity of all stencil nodes of origin org into the
// cache column of every lane with `need`; the whole warp calls.
template <int DT, int KW>
__device__ __forceinline__ void warp_gather_wide(bool need, const int org[3], const typename lbd::Store<DT>::T *src,
                                                 const float *ffield, const StepArgs &g, float *sm)
{
    constexpr int kN = KW * KW * KW, kR = 4;                // owners per round
    constexpr int kSlots = (kR * kN + 31) / 32;             // nodes per lane per round
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    unsigned m = __ballot_sync(kFullMask, need);
    while (m) {
        int own[kR];
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            own[k] = -1;
            if (m) {
                own[k] = __ffs(m) - 1;
                m &= m - 1;
            }
        }
        int o[kR][3];
#pragma unroll
        for (int k = 0; k < kR; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) o[k][d] = __shfl_sync(kFullMask, org[d], own[k] < 0 ? 0 : own[k]);
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            const int item = lane + 32 * sl;
            if (item < kR * kN) {
                const int k = item / kN, q = item % kN;
                int ok = own[0];
                int oo[3] = {o[0][0], o[0][1], o[0][2]};
#pragma unroll
                for (int kk = 1; kk < kR; ++kk)
                    if (k == kk) {
                        ok = own[kk];
                        oo[0] = o[kk][0];
                        oo[1] = o[kk][1];
                        oo[2] = o[kk][2];
                    }
                if (ok >= 0) {
                    int x, y, z;
                    stencil_coords<KW>(oo, q, g, x, y, z);
                    float u[3];
                    node_velocity<DT>(src, ffield, x, y, z, g, u);
                    wide_cache<KW>(sm, 0, q, wbase + ok) = u[0];
                    wide_cache<KW>(sm, 1, q, wbase + ok) = u[1];
                    wide_cache<KW>(sm, 2, q, wbase + ok) = u[2];
                }
            }
        }
    }
    __syncwarp();
}

// Add this thread's impulse sums at origin org to the accumulator and zero them.
template <int KW>
__device__ __forceinline__ void flush_wide(const int org[3], float *sm, float *facc, const StepArgs &g)
{
    constexpr int kN = KW * KW * KW;
    const int t = threadIdx.x;
#pragma unroll 4
    for (int q = 0; q < kN; ++q) {
        int x, y, z;
        stencil_coords<KW>(org, q, g, x, y, z);
        const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
        float &jx = wide_cache<KW>(sm, 3, q, t), &jy = wide_cache<KW>(sm, 4, q, t), &jz = wide_cache<KW>(sm, 5, q, t);
        if (in_bounds(node, g.nn, g.err)) {
            atomicAdd(facc + node, jx);
            atomicAdd(facc + g.pitch + node, jy);
            atomicAdd(facc + 2 * g.pitch + node, jz);
        }
        jx = jy = jz = 0.0f;
    }
}

// Start of a call: the fluid velocity at every particle's stencil nodes,
// each distinct node gathered once by the whole block.  The particles of a
// block are usually consecutive monomers, whose stencils overlap (for the
// random-walk chains of the workload 128 monomers touch ~1000 distinct nodes
// with phi_3 and ~1600 with phi_4, against 3456 and 8192 stencil entries);
// the impulse columns, still empty, hold a hash table of the distinct nodes
// (open addressing, linear probing, inserted with atomicCAS): node index + 1
// as key, its velocity, and the list of slots in insertion order, from which
// all threads gather with several nodes' loads in flight.  Each particle then
// copies its nodes' velocities into its own columns, so the sub-steps read
// the same values, in the same layout, as with a gather per particle.  A node
// that finds no slot within kTableProbes probes is gathered by its particle
// directly.  All threads of the block call; on return the table is dead.
template <int KW>
constexpr int wide_table_cap()
{
    return (int)((size_t)3 * KW * KW * KW * kPThreads * sizeof(float) / 18);  // key 4 + velocity 12 + list 2 bytes
}
constexpr int kTableProbes = 32;

template <int DT, int KW>
__device__ __forceinline__ void block_gather_wide(bool active, const int org[3],
                                                  const typename lbd::Store<DT>::T *src, const float *ffield,
                                                  const StepArgs &g, float *sm, int *count)
{
    constexpr int kN = KW * KW * KW;
    constexpr uint32_t cap = (uint32_t)wide_table_cap<KW>();
    unsigned char *tb = reinterpret_cast<unsigned char *>(&wide_cache<KW>(sm, 3, 0, 0));
    unsigned int *key = reinterpret_cast<unsigned int *>(tb);
    float *tu = reinterpret_cast<float *>(tb + (size_t)cap * 4);
    unsigned short *list = reinterpret_cast<unsigned short *>(tb + (size_t)cap * 16);
    const int t = threadIdx.x;
    for (uint32_t i = t; i < cap; i += kPThreads) key[i] = 0u;
    if (t == 0) *count = 0;
    __syncthreads();
    if (active) {
#pragma unroll 1
        for (int q = 0; q < kN; ++q) {
            int x, y, z;
            stencil_coords<KW>(org, q, g, x, y, z);
            const uint32_t k = (uint32_t)(((size_t)z * g.ny + y) * g.nx + x) + 1u;
            uint32_t h = __umulhi(k * 2654435761u, cap);  // Fibonacci hashing onto [0, cap)
            int slot = -1;
            for (int probe = 0; probe < kTableProbes; ++probe) {
                const uint32_t old = atomicCAS(&key[h], 0u, k);
                if (old == 0u) {
                    list[atomicAdd(count, 1)] = (unsigned short)h;
                    slot = (int)h;
                    break;
                }
                if (old == k) {
                    slot = (int)h;
                    break;
                }
                h = (h + 1u == cap) ? 0u : h + 1u;
            }
            wide_cache<KW>(sm, 0, q, t) = __int_as_float(slot);  // the slot until the copy below
        }
    }
    __syncthreads();
    const int n = *count;
    const uint32_t nxy = (uint32_t)g.nx * (uint32_t)g.ny;
#pragma unroll 2
    for (int i = t; i < n; i += kPThreads) {
        const uint32_t h = list[i];
        const uint32_t node = key[h] - 1u;
        const uint32_t z = node / nxy, r = node - z * nxy;
        const uint32_t y = r / (uint32_t)g.nx, x = r - y * (uint32_t)g.nx;
        float u[3];
        node_velocity<DT>(src, ffield, (int)x, (int)y, (int)z, g, u);
        tu[h] = u[0];
        tu[cap + h] = u[1];
        tu[2 * cap + h] = u[2];
    }
    __syncthreads();
    if (active) {
#pragma unroll 1
        for (int q = 0; q < kN; ++q) {
            const int slot = __float_as_int(wide_cache<KW>(sm, 0, q, t));
            float u[3];
            if (slot >= 0) {
                u[0] = tu[slot];
                u[1] = tu[cap + slot];
                u[2] = tu[2 * cap + slot];
            } else {  // no room in the table
                int x, y, z;
                stencil_coords<KW>(org, q, g, x, y, z);
                node_velocity<DT>(src, ffield, x, y, z, g, u);
            }
            wide_cache<KW>(sm, 0, q, t) = u[0];
            wide_cache<KW>(sm, 1, q, t) = u[1];
            wide_cache<KW>(sm, 2, q, t) = u[2];
        }
    }
    __syncthreads();
}

template <int DT, int KW>
__global__ void __launch_bounds__(kPThreads) k_couple_persistent_wide(PersistArgs a)
{
    using T = typename lbd::Store<DT>::T;
    constexpr int kN = KW * KW * KW;
    extern __shared__ float wsm[];
    __shared__ unsigned int ticket;  // arrival word of the split barrier
    __shared__ int tcount;           // entries of the start-of-call node table
    const CoupleArgs &c = a.c;
    const StepArgs &g = c.g;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < c.n;
    const T *src = static_cast<const T *>(a.src);
    if (c.use_wca && blockIdx.x == 0 && threadIdx.x == 0) a.flags[0] = 0u;  // the pre-launch build has run

    // phase 0: first half drift, neighbours (the previous call's impulses were
    // cleared before the launch)
    CPos me{}, refp{};
    float pm[3] = {0.f, 0.f, 0.f};
    float m = 1.f, G = 1.f, C1 = c.C1, C2 = c.C2, C3 = c.C3;
    const int self = active ? p : 0;
    int nnb = 0;
    int nb[kNbReg];
#pragma unroll
    for (int k = 0; k < kNbReg; ++k) nb[k] = self;
    bool bond_lo = false, bond_hi = false;
    if (active) {
        if (c.use_wca) unbin_particle(p, a.head, a.bucket_of);
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
        const double hd = 0.5 * (double)c.dt / (double)m;
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] += hd * (double)pm[k];
        confine_d(r, pm, g, KW);
        if (!split(r, g, me)) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
        a.sh[0][p] = pack(me);
        if (c.use_wca) {
            nnb = a.ncount[p];
            const int *lst = a.nlist + (size_t)p * kMaxNb;
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < nnb) nb[k] = lst[k];
            refp = unpack(a.ref[p]);
        }
        if (c.chain_len > 1) {
            const int k = p % c.chain_len;
            bond_lo = k > 0;
            bond_hi = k < c.chain_len - 1 && p + 1 < c.n;
        }
    }
    const int jlo = bond_lo ? p - 1 : self, jhi = bond_hi ? p + 1 : self;
    int kmax = __reduce_max_sync(kFullMask, min(nnb, kNbReg));
    int org[3];
    {
        Stencil<KW> st;
        make_stencil<KW>(me, st);
        org[0] = st.o[0];
        org[1] = st.o[1];
        org[2] = st.o[2];
    }
    block_gather_wide<DT, KW>(active, org, src, a.ffield, g, wsm, &tcount);
    for (int q = 0; q < kN; ++q)
        wide_cache<KW>(wsm, 3, q, threadIdx.x) = wide_cache<KW>(wsm, 4, q, threadIdx.x) =
            wide_cache<KW>(wsm, 5, q, threadIdx.x) = 0.0f;
    if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;

    bool binned = false;
    const float h = 0.5f * c.dt / m;
    for (int s = 0; s < a.nsub; ++s) {
        const float4 *shin = a.sh[s & 1];
        float4 *shout = a.sh[(s + 1) & 1];
        float4 v[kNbReg];
#pragma unroll
        for (int k = 0; k < kNbReg; ++k)
            if (k < kmax) v[k] = __ldcg(shin + nb[k]);
        const float4 vlo = __ldcg(shin + jlo), vhi = __ldcg(shin + jhi);
        const unsigned int req = c.use_wca ? __ldcg(a.flags + 1 + (s & 1)) : 0u;
        float th[3] = {0.f, 0.f, 0.f};
        if (g.kT > 0.0f) particle_theta((uint32_t)p, c.md_step + (uint32_t)s, c, th);
        Stencil<KW> st;
        make_stencil<KW>(me, st);

        if (c.use_wca && req == a.epoch0 + (uint32_t)s) {
            // a particle moved more than half the skin: re-bin all, rebuild every list
            if (binned) {
                if (active) unbin_particle(p, a.head, a.bucket_of);
                if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
            }
            if (active) bin_particle(p, me, c, a.head, a.next, a.bucket_of);
            if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
            binned = true;
            if (active) {
                int *mine = a.nlist + (size_t)p * kMaxNb;
                nnb = build_own_list(p, me, shin, a.head, a.next, c, mine, a.err);
#pragma unroll
                for (int k = 0; k < kNbReg; ++k) nb[k] = k < nnb ? mine[k] : self;
                a.ncount[p] = nnb;
                a.ref[p] = pack(me);
                refp = me;
            }
            kmax = __reduce_max_sync(kFullMask, min(nnb, kNbReg));
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < kmax) v[k] = __ldcg(shin + nb[k]);
        }

        float F[3] = {c.fext[0], c.fext[1], c.fext[2]};
        if (c.use_wca) {
#pragma unroll
            for (int k = 0; k < kNbReg; ++k)
                if (k < kmax) wca_add(me, unpack(v[k]), c, F, k < nnb);
            for (int k = kNbReg; k < nnb; ++k) wca_add(me, unpack(__ldcg(shin + a.nlist[(size_t)p * kMaxNb + k])), c, F);
        }
        if (c.chain_len > 1) {
            if (bond_lo && !fene_add(me, unpack(vlo), c, F)) atomicOr(a.err, LB_DERR_FENE_BROKEN);
            if (bond_hi && !fene_add(me, unpack(vhi), c, F)) atomicOr(a.err, LB_DERR_FENE_BROKEN);
        }

        // (the stencil cache already holds origin st.o: gathered before the
        // first sub-step or, for a moved origin, inside the previous barrier)
        if (active) {
            float up[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                const float w = st.w[0][q % KW] * st.w[1][(q / KW) % KW] * st.w[2][q / (KW * KW)];
                up[0] = fmaf(w, wide_cache<KW>(wsm, 0, q, threadIdx.x), up[0]);
                up[1] = fmaf(w, wide_cache<KW>(wsm, 1, q, threadIdx.x), up[1]);
                up[2] = fmaf(w, wide_cache<KW>(wsm, 2, q, threadIdx.x), up[2]);
            }
            float pn[3], J[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pn[k] = C1 * pm[k] + C2 * (F[k] + G * up[k]) + C3 * th[k];
                J[k] = pn[k] - pm[k] - c.dt * F[k];
            }
#pragma unroll
            for (int q = 0; q < kN; ++q) {
                const float w = st.w[0][q % KW] * st.w[1][(q / KW) % KW] * st.w[2][q / (KW * KW)];
                float &jx = wide_cache<KW>(wsm, 3, q, threadIdx.x);
                float &jy = wide_cache<KW>(wsm, 4, q, threadIdx.x);
                float &jz = wide_cache<KW>(wsm, 5, q, threadIdx.x);
                jx = fmaf(-J[0], w, jx);
                jy = fmaf(-J[1], w, jy);
                jz = fmaf(-J[2], w, jz);
            }
            a.records[(size_t)s * c.n + p] = stencil_record<KW>(me, g);

            const bool last = (s == a.nsub - 1);
            bool ok = drift(me, pn, h, g, KW);
            if (last) {
                a.pos[3 * p] = join1(me.c[0], me.f[0]);
                a.pos[3 * p + 1] = join1(me.c[1], me.f[1]);
                a.pos[3 * p + 2] = join1(me.c[2], me.f[2]);
                a.mom[3 * p] = pn[0];
                a.mom[3 * p + 1] = pn[1];
                a.mom[3 * p + 2] = pn[2];
            } else {
                ok = drift(me, pn, h, g, KW) && ok;
            }
            if (!ok) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
            pm[0] = pn[0];
            pm[1] = pn[1];
            pm[2] = pn[2];
            shout[p] = pack(me);
            if (c.use_wca) {
                float d[3];
                separation(me, refp, g, d);
                const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!last && d2 > c.half_skin2) atomicMax(&a.flags[1 + ((s + 1) & 1)], a.epoch0 + (uint32_t)s + 1u);
                if (last && d2 > 0.25f * c.half_skin2) a.flags[0] = 1u;  // build before the next call
            }
        }
        // the barrier in two halves: between them, particles whose stencil
        // origin moves for the next sub-step hand in their impulse sums and the
        // warp gathers their new stencils (this reads only the frozen fluid and
        // writes only the block's cache and the accumulator, which no block
        // reads during the call)
        grid_arrive(a.bar, &ticket);
        if (s + 1 < a.nsub) {
            Stencil<KW> stn;
            make_stencil<KW>(me, stn);
            const bool moved = active && (stn.o[0] != org[0] || stn.o[1] != org[1] || stn.o[2] != org[2]);
            if (__any_sync(kFullMask, moved)) {
                if (moved) {
                    flush_wide<KW>(org, wsm, a.facc, g);
                    org[0] = stn.o[0];
                    org[1] = stn.o[1];
                    org[2] = stn.o[2];
                }
                warp_gather_wide<DT, KW>(moved, org, src, a.ffield, g, wsm);
            }
        }
        if (!grid_wait(a.bar, a.err, a.spin_limit, &ticket)) return;
    }
    if (active) {
        flush_wide<KW>(org, wsm, a.facc, g);
        if (binned) unbin_particle(p, a.head, a.bucket_of);
    }
}

// ---------------------------------------------------------------------------
// Free particles (no pair or bond forces): with the fluid frozen during a
// call, a particle's sub-steps depend on no other particle, so one launch
// runs all sub-steps of every particle with no grid barrier and no limit on
// the particle count.  A group of LANES threads serves a particle (one for
// phi_2, eight for phi_3 / phi_4); lane q keeps the fluid velocity of the
// stencil nodes q, q + LANES, ... of the particle's current stencil origin in
// registers, gathers them again only when the origin moves, and sums the
// impulses it spreads there over the sub-steps spent at that origin, adding
// them to the accumulator when the origin moves or the call ends.  Per
// sub-step: interpolation (Eqs. ufluid_discrete, Delta), the exact OU update
// (Eq. langevin_momentum_update), the impulse -J Delta with
// J = p' - p - dt F^c (Eq. ftotal; F^c the constant external force), the two
// half drifts.  Every lane of a group computes the same position and
// momentum; lane 0 writes them.
// ---------------------------------------------------------------------------
struct FreeArgs {
    CoupleArgs c;
    int nsub;
    const void *src;
    const float *ffield;
    double *pos;
    float *mom;
    const float *mass, *gamma;
    float *facc;
    int *records;  // [nsub][n] cell of each sub-step (the overlapped re-update's list)
    unsigned int *err;
};

template <int DT, int KW>
__global__ void __launch_bounds__(kPartThreads) k_couple_free(FreeArgs a)
{
    using T = typename lbd::Store<DT>::T;
    constexpr int LANES = free_lanes<KW>();
    constexpr int kNodes = KW * KW * KW, kPer = (kNodes + LANES - 1) / LANES;
    const CoupleArgs &c = a.c;
    const StepArgs &g = c.g;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = tid / LANES, q = tid % LANES;
    if (p >= c.n) return;  // whole groups leave together (LANES divides the block)
    const unsigned gmask = LANES == 1 ? 0xFFFFFFFFu : (0xFFu << (threadIdx.x & 24));
    const T *src = static_cast<const T *>(a.src);

    const float m = a.mass ? a.mass[p] : c.mass0;
    const float G = a.gamma ? a.gamma[p] : c.gamma0;
    float C1 = c.C1, C2 = c.C2, C3 = c.C3;
    if (!c.uniform_coef) {
        const float x1 = G * c.dt / m;
        C1 = expf(-x1);
        C2 = (m / G) * (-expm1f(-x1));
        C3 = sqrtf(m * g.kT * (-expm1f(-2.0f * x1)));
    }
    // first half drift in FP64 from the caller's position, then cell + offset
    float pm[3] = {a.mom[3 * p], a.mom[3 * p + 1], a.mom[3 * p + 2]};
    CPos me;
    {
        double r[3] = {a.pos[3 * p], a.pos[3 * p + 1], a.pos[3 * p + 2]};
        const double hd = 0.5 * (double)c.dt / (double)m;
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] += hd * (double)pm[k];
        confine_d(r, pm, g, KW);
        if (!split(r, g, me) && q == 0) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
    }

    float uc[kPer][3], acc[kPer][3];
#pragma unroll
    for (int i = 0; i < kPer; ++i) uc[i][0] = uc[i][1] = uc[i][2] = acc[i][0] = acc[i][1] = acc[i][2] = 0.0f;
    int org[3] = {INT_MIN, INT_MIN, INT_MIN};  // stencil origin of uc / acc (none yet)
    bool ok = true;
    const float h = 0.5f * c.dt / m;
    for (int s = 0; s < a.nsub; ++s) {
        Stencil<KW> st;
        make_stencil<KW>(me, st);
        if (st.o[0] != org[0] || st.o[1] != org[1] || st.o[2] != org[2]) {
            if (org[0] != INT_MIN) {  // hand in the impulses summed at the old origin
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int qq = q + LANES * i;
                    if (kNodes % LANES == 0 || qq < kNodes) {
                        int x, y, z;
                        stencil_coords<KW>(org, qq, g, x, y, z);
                        const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
                        if (in_bounds(node, g.nn, g.err)) {
                            atomicAdd(a.facc + node, acc[i][0]);
                            atomicAdd(a.facc + g.pitch + node, acc[i][1]);
                            atomicAdd(a.facc + 2 * g.pitch + node, acc[i][2]);
                        }
                        acc[i][0] = acc[i][1] = acc[i][2] = 0.0f;
                    }
                }
            }
            org[0] = st.o[0];
            org[1] = st.o[1];
            org[2] = st.o[2];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int qq = q + LANES * i;
                if (kNodes % LANES == 0 || qq < kNodes) {
                    int x, y, z;
                    stencil_coords<KW>(org, qq, g, x, y, z);
                    node_velocity<DT>(src, a.ffield, x, y, z, g, uc[i]);
                }
            }
        }
        float w[kPer];
        float up[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int qq = q + LANES * i;
            w[i] = 0.0f;
            if (kNodes % LANES == 0 || qq < kNodes) {
                int x, y, z;
                w[i] = stencil_node_k<KW>(st, qq, g, x, y, z);
                up[0] = fmaf(w[i], uc[i][0], up[0]);
                up[1] = fmaf(w[i], uc[i][1], up[1]);
                up[2] = fmaf(w[i], uc[i][2], up[2]);
            }
        }
        if (LANES > 1) {
#pragma unroll
            for (int o = 1; o < LANES; o <<= 1)
#pragma unroll
                for (int k = 0; k < 3; ++k) up[k] += __shfl_xor_sync(gmask, up[k], o);
        }
        float th[3] = {0.f, 0.f, 0.f};
        if (g.kT > 0.0f) particle_theta((uint32_t)p, c.md_step + (uint32_t)s, c, th);
        float pn[3], J[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            pn[k] = C1 * pm[k] + C2 * (c.fext[k] + G * up[k]) + C3 * th[k];
            J[k] = pn[k] - pm[k] - c.dt * c.fext[k];
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            acc[i][0] = fmaf(-J[0], w[i], acc[i][0]);
            acc[i][1] = fmaf(-J[1], w[i], acc[i][1]);
            acc[i][2] = fmaf(-J[2], w[i], acc[i][2]);
        }
        if (q == 0 && a.records) a.records[(size_t)s * c.n + p] = stencil_record<KW>(me, g);
        // second half drift of this sub-step, then the first of the next one
        ok = drift(me, pn, h, g, KW) && ok;
        if (s + 1 < a.nsub) ok = drift(me, pn, h, g, KW) && ok;
        pm[0] = pn[0];
        pm[1] = pn[1];
        pm[2] = pn[2];
    }
    if (org[0] != INT_MIN) {
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int qq = q + LANES * i;
            if (kNodes % LANES == 0 || qq < kNodes) {
                int x, y, z;
                stencil_coords<KW>(org, qq, g, x, y, z);
                const size_t node = ((size_t)z * g.ny + y) * g.nx + x;
                if (in_bounds(node, g.nn, g.err)) {
                    atomicAdd(a.facc + node, acc[i][0]);
                    atomicAdd(a.facc + g.pitch + node, acc[i][1]);
                    atomicAdd(a.facc + 2 * g.pitch + node, acc[i][2]);
                }
            }
        }
    }
    if (q != 0) return;
    if (!ok) atomicOr(a.err, LB_DERR_PARTICLE_RANGE);
    a.pos[3 * p] = join1(me.c[0], me.f[0]);
    a.pos[3 * p + 1] = join1(me.c[1], me.f[1]);
    a.pos[3 * p + 2] = join1(me.c[2], me.f[2]);
    a.mom[3 * p] = pm[0];
    a.mom[3 * p + 1] = pm[1];
    a.mom[3 * p + 2] = pm[2];
}

// Kernel arguments of a coupling call (everything but the cell list).
// Interpolation stencil width selected by lb_couple_params.flags.
int stencil_width(int flags)
{
    if (flags & LB_COUPLE_PHI3) return 3;
    if (flags & LB_COUPLE_PHI4) return 4;
    return 2;
}

CoupleArgs make_couple_args(const lb_handle *h, const lb_particles *pp, const lb_couple_params *cp)
{
    CoupleArgs c;
    c.g = make_args(h);
    c.n = pp->n;
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
    c.ncell[0] = c.ncell[1] = c.ncell[2] = 1;
    c.cinv[0] = c.cinv[1] = c.cinv[2] = 0.0f;
    c.nb_log2 = 0;
    c.kw = stencil_width(cp->flags);
    for (int k = 0; k < 3; ++k) c.fext[k] = (float)cp->fext[k];
    return c;
}

void note_records(Particles *P, int n, size_t count)
{
    if (P->n_records == 0) P->rec_n = n;
    else if (P->rec_n != n) P->rec_n = -1;
    P->n_records += count;
}

template <int DT>
cudaError_t run_substeps(lb_handle *h, const lb_particles *pp, const lb_couple_params *cp)
{
    Particles *P = h->parts;
    const int n = pp->n;
    CoupleArgs c = make_couple_args(h, pp, cp);
    const double rl = 1.122462048309373 * cp->sigma + kSkin * cp->sigma;
    {
        // cells of edge >= r_list (with a margin for the FP32 binning)
        const int L[3] = {h->p.nx, h->p.ny, h->p.nz};
        for (int k = 0; k < 3; ++k) {
            c.ncell[k] = std::max(1, (int)((double)L[k] / (1.001 * rl)));
            c.cinv[k] = (float)((double)c.ncell[k] / (double)L[k]);
        }
        c.nb_log2 = P->nb_log2;
    }
    const int blocks = (n + kPartThreads - 1) / kPartThreads;
    using T = typename lbd::Store<DT>::T;
    const T *src = static_cast<const T *>(h->pops[h->cur]);
    const bool need_nlist = cp->use_wca != 0;

    // free particles: one launch runs every sub-step, no grid barrier, any count
    if (!(cp->flags & LB_COUPLE_PER_SUBSTEP) && !need_nlist && c.chain_len <= 1) {
        if (h->facc_stale) {
            cudaError_t e = clear_particle_forces(h);
            if (e != cudaSuccess) return e;
            h->facc_stale = 0;
        }
        FreeArgs fa;
        fa.c = c;
        fa.nsub = cp->n_substeps;
        fa.src = src;
        fa.ffield = h->force;
        fa.pos = pp->pos;
        fa.mom = pp->mom;
        fa.mass = pp->mass;
        fa.gamma = pp->gamma;
        fa.facc = h->facc;
        fa.records = P->records + P->rec_off + P->n_records;
        fa.err = h->d_err;
        const int lanes = c.kw == 2 ? free_lanes<2>() : free_lanes<3>();
        const unsigned int fblocks = (unsigned int)(((size_t)n * lanes + kPartThreads - 1) / kPartThreads);
        if (c.kw == 3) k_couple_free<DT, 3><<<fblocks, kPartThreads, 0, h->stream>>>(fa);
        else if (c.kw == 4) k_couple_free<DT, 4><<<fblocks, kPartThreads, 0, h->stream>>>(fa);
        else k_couple_free<DT, 2><<<fblocks, kPartThreads, 0, h->stream>>>(fa);
        h->launches += 1;
        note_records(P, n, (size_t)n * (size_t)cp->n_substeps);
        P->rec_span = std::max(P->rec_span, c.kw == 3 ? 3 : (c.kw == 4 ? 4 : 2));
        P->sub_counter += (uint32_t)cp->n_substeps;
        P->last_nsub = cp->n_substeps;
        return cudaGetLastError();
    }

    // persistent path when every particle group can be resident at once
    const int gblocks = (int)(((size_t)n * kChunks + kPartThreads - 1) / kPartThreads);  // 8 lanes a particle
    const int pblocks = (n + kPThreads - 1) / kPThreads;                                   // one thread a particle
    int per_sm = 0;
    if (!(cp->flags & LB_COUPLE_PER_SUBSTEP) && c.kw > 2) {
        // phi_3 / phi_4: the persistent kernel with the stencil caches in shared memory
        const size_t smem = c.kw == 3 ? wide_smem_bytes<3>() : wide_smem_bytes<4>();
        const void *kfn = c.kw == 3 ? (const void *)k_couple_persistent_wide<DT, 3>
                                    : (const void *)k_couple_persistent_wide<DT, 4>;
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kPThreads, smem);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();  // no wide persistent kernel here: the per-sub-step path below
            per_sm = 0;
        }
        if (per_sm > 0 && pblocks <= per_sm * device_sm_count()) {
            if (need_nlist && P->nlist_n != n) {
                const unsigned int init[kFlagWords] = {0u, 0u, 1u, 0u, 0u};  // [2]: build before the launch
                e = cudaMemcpyAsync(P->flags, init, sizeof(init), cudaMemcpyHostToDevice, h->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                if (e != cudaSuccess) return e;
                P->nlist_n = n;
            }
            if (h->facc_stale) {
                e = clear_particle_forces(h);
                if (e != cudaSuccess) return e;
                h->facc_stale = 0;
            }
            if (need_nlist) {
                k_shadow_from_pos<<<blocks, kPartThreads, 0, h->stream>>>(pp->pos, P->shadow[1], P->head, P->next,
                                                                           P->bucket_of, P->flags + 2, h->d_err, c);
                k_build_nlist<<<gblocks, kPartThreads, 0, h->stream>>>(P->shadow[1], P->head, P->next, P->nlist,
                                                                       P->ncount, P->ref, P->flags, h->d_err, c, 2u);
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
            a.head = P->head;
            a.next = P->next;
            a.bucket_of = P->bucket_of;
            a.facc = h->facc;
            a.records = P->records + P->rec_off + P->n_records;
            a.stale = nullptr;
            a.nstale_sub = 0;
            a.flags = P->flags + 2;
            a.epoch0 = P->sub_counter + 1u;
            a.bar = P->bar;
            a.err = h->d_err;
            a.spin_limit = 1u << 22;
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(pblocks);
            lc.blockDim = dim3(kPThreads);
            lc.dynamicSmemBytes = smem;
            lc.stream = h->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            void *args[] = {&a};
            e = cudaLaunchKernelExC(&lc, kfn, args);
            if (e != cudaSuccess) return e;
            h->launches += 1;
            note_records(P, n, (size_t)n * (size_t)cp->n_substeps);
            P->rec_span = std::max(P->rec_span, c.kw == 3 ? 3 : 4);
            P->sub_counter += (uint32_t)cp->n_substeps;
            P->last_nsub = cp->n_substeps;
            return cudaGetLastError();
        }
    }
    if (!(cp->flags & LB_COUPLE_PER_SUBSTEP) && c.kw == 2 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)(h->n_nodes >= kLeanCouplingNodes ? k_couple_persistent_lean<DT> : k_couple_persistent<DT>), kPThreads, 0) == cudaSuccess &&
        pblocks <= per_sm * device_sm_count()) {
        cudaError_t e = cudaSuccess;
        if (need_nlist && P->nlist_n != n) {
            const unsigned int init[kFlagWords] = {0u, 0u, 1u, 0u, 0u};  // [2]: build before the launch
            e = cudaMemcpyAsync(P->flags, init, sizeof(init), cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return e;
            P->nlist_n = n;
        }
        const bool fold_clear = h->facc_stale && P->rec_span == 2 && P->n_records == (size_t)n * (size_t)P->last_nsub &&
                                P->n_records <= P->rec_cap / 2 && (size_t)n * cp->n_substeps <= P->rec_cap / 2;
        if (h->facc_stale && !fold_clear) {
            e = clear_particle_forces(h);
            if (e != cudaSuccess) return e;
            h->facc_stale = 0;
        }
        if (need_nlist) {
            k_shadow_from_pos<<<blocks, kPartThreads, 0, h->stream>>>(pp->pos, P->shadow[1], P->head, P->next,
                                                                       P->bucket_of, P->flags + 2, h->d_err, c);
            k_build_nlist<<<gblocks, kPartThreads, 0, h->stream>>>(P->shadow[1], P->head, P->next, P->nlist,
                                                                   P->ncount, P->ref, P->flags, h->d_err, c, 2u);
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
        a.head = P->head;
        a.next = P->next;
        a.bucket_of = P->bucket_of;
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
        lc.blockDim = dim3(kPThreads);
        lc.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        void *args[] = {&a};
        const void *kfn = h->n_nodes >= kLeanCouplingNodes ? (const void *)k_couple_persistent_lean<DT>
                                                           : (const void *)k_couple_persistent<DT>;
        e = cudaLaunchKernelExC(&lc, kfn, args);
        if (e != cudaSuccess) return e;
        h->launches += 1;
        if (fold_clear) {
            P->rec_off = new_off;
            P->n_records = 0;
            h->facc_stale = 0;
        }
        note_records(P, n, (size_t)n * (size_t)cp->n_substeps);
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
    if (P->ucache_cap < n) {  // node-velocity cache of the per-sub-step kernels
        cudaFree(P->ucache);
        cudaFree(P->utag);
        P->ucache = nullptr;
        P->utag = nullptr;
        P->ucache_cap = 0;
        cudaError_t e = cudaMalloc((void **)&P->ucache, (size_t)n * 64 * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&P->utag, (size_t)n * sizeof(int2));
        if (e == cudaSuccess) e = cudaMemsetAsync(P->utag, 0, (size_t)n * sizeof(int2), h->stream);
        if (e != cudaSuccess) return e;
        P->ucache_cap = n;
        P->epoch = 0;
    }
    if (++P->epoch >= 0x7fffffffu) {  // tags hold the epoch as int: start again from 1
        cudaError_t e = cudaMemsetAsync(P->utag, 0, (size_t)P->ucache_cap * sizeof(int2), h->stream);
        if (e != cudaSuccess) return e;
        P->epoch = 1;
    }
    k_half_drift<<<blocks, kPartThreads, 0, h->stream>>>(pp->pos, pp->mom, pp->mass, P->shadow[0], h->d_err, c);
    h->launches += 1;
    for (int s = 0; s < cp->n_substeps; ++s) {
        const uint32_t rd = P->sub_counter & 1u, wr = rd ^ 1u;
        const int sblocks = (int)(((size_t)n * 8 + kPartThreads - 1) / kPartThreads);
        if (need_nlist) {
            k_bin<<<blocks, kPartThreads, 0, h->stream>>>(P->shadow[s & 1], P->head, P->next, P->bucket_of,
                                                          P->flags, c, rd);
            k_build_nlist<<<sblocks, kPartThreads, 0, h->stream>>>(P->shadow[s & 1], P->head, P->next, P->nlist,
                                                                   P->ncount, P->ref, P->flags, h->d_err, c, rd);
            h->launches += 2;
        }
        c.md_step = cp->md_step0 + (uint32_t)s;
        c.last = (s == cp->n_substeps - 1);
        c.slot = wr;
        int *rec = P->records + P->rec_off + P->n_records;
#define LBI_SUBSTEP(KW)                                                                                          \
    k_substep<DT, KW><<<sblocks, kPartThreads, 0, h->stream>>>(                                                  \
        src, h->force, P->shadow[s & 1], P->shadow[(s + 1) & 1], pp->pos, pp->mom, pp->mass, pp->gamma, P->nlist, \
        P->ncount, need_nlist ? P->ref : nullptr, P->head, P->bucket_of, h->facc, rec, P->flags, h->d_err,         \
        P->ucache, P->utag, (int)P->epoch, c, rd)
        if (c.kw == 3) LBI_SUBSTEP(3);
        else if (c.kw == 4) LBI_SUBSTEP(4);
        else LBI_SUBSTEP(2);
#undef LBI_SUBSTEP
        note_records(P, n, (size_t)n);
        P->rec_span = std::max(P->rec_span, c.kw == 3 ? 3 : (c.kw == 4 ? 4 : 2));
        P->sub_counter += 1;
        h->launches += 1;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reverse mode of the coupling (kT = 0, free particles).  Each particle is
// independent: its thread replays the sub-steps with the arithmetic of the
// forward kernels (cell + FP32 offset positions), remembering per sub-step
// the half-drift position r_h, the momenta p~ (after the first confine) and
// p', and the z sign each confine applied; then it walks them back:
//   r' = s2 (r_h + a p'), p_stored = s2 p'          (z only for s2)
//   facc_q -= J w_q(r_h), J = p' - p~
//   p' = C1 p~ + C2 Gamma u_p, u_p = sum_q w_q(r_h) u_q
//   r_h = s1 (r + a p), p~ = s1 p
// adding dL/du_q into lam_u ([3][pitch], atomics); k_lambda_u_to_pops turns
// that into dL/dpopulations and dL/dforce.  (Sec. 4.5, Eqs. Delta, 2point.)
// ---------------------------------------------------------------------------
constexpr int kMaxAdjSub = 64;  // sub-steps a reverse call can replay

template <int DT>
__global__ void __launch_bounds__(kPartThreads)
    k_couple_adjoint(const typename lbd::Store<DT>::T *__restrict__ src, const float *__restrict__ ffield,
                     const double *pos0, const float *mom0, const float *mass, const float *gamma,
                     const float *__restrict__ lam_facc, float *lam_pos, float *lam_mom, float *lam_u,
                     unsigned int *err, CoupleArgs c, int nsub)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.n) return;
    const StepArgs &g = c.g;
    const float m = mass ? mass[p] : c.mass0;
    const float G = gamma ? gamma[p] : c.gamma0;
    float C1 = c.C1, C2 = c.C2;
    if (!c.uniform_coef) {
        const float x1 = G * c.dt / m;
        C1 = expf(-x1);
        C2 = (m / G) * (-expm1f(-x1));
    }
    const float a = 0.5f * c.dt / m;
    CPos rh[kMaxAdjSub];
    float pt[kMaxAdjSub][3], pn[kMaxAdjSub][3], s1[kMaxAdjSub], s2[kMaxAdjSub];

    // replay: first half drift in FP64 as the forward kernel does, then FP32
    CPos me;
    float q[3] = {mom0[3 * p], mom0[3 * p + 1], mom0[3 * p + 2]};
    {
        double r[3] = {pos0[3 * p], pos0[3 * p + 1], pos0[3 * p + 2]};
        const double h = 0.5 * (double)c.dt / (double)m;
        for (int k = 0; k < 3; ++k) r[k] += h * (double)q[k];
        const float before = q[2];
        confine_d(r, q, g);
        s1[0] = (before != 0.0f && q[2] == -before) ? -1.0f : 1.0f;
        if (!split(r, g, me)) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    }
    for (int s = 0; s < nsub; ++s) {
        float uc[8][3], w[8];
        for (int k = 0; k < 8; ++k) {
            int x, y, z;
            w[k] = stencil_node(me, k, g, x, y, z);
            node_velocity<DT>(src, ffield, x, y, z, g, uc[k]);
        }
        float up[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k)
            for (int d = 0; d < 3; ++d) up[d] = fmaf(w[k], uc[k][d], up[d]);
        rh[s] = me;
        for (int d = 0; d < 3; ++d) {
            pt[s][d] = q[d];
            q[d] = C1 * q[d] + C2 * G * up[d];
            pn[s][d] = q[d];
        }
        float before = q[2];
        bool ok = drift(me, q, a, g);  // second half drift of sub-step s
        s2[s] = (before != 0.0f && q[2] == -before) ? -1.0f : 1.0f;
        if (s + 1 < nsub) {
            before = q[2];
            ok = drift(me, q, a, g) && ok;  // first half drift of sub-step s + 1
            s1[s + 1] = (before != 0.0f && q[2] == -before) ? -1.0f : 1.0f;
        }
        if (!ok) atomicOr(err, LB_DERR_PARTICLE_RANGE);
    }

    // walk back
    float lr[3] = {lam_pos[3 * p], lam_pos[3 * p + 1], lam_pos[3 * p + 2]};
    float lp[3] = {lam_mom[3 * p], lam_mom[3 * p + 1], lam_mom[3 * p + 2]};
    for (int s = nsub - 1; s >= 0; --s) {
        float lrh[3], lpn[3], lJ[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < 3; ++d) {
            const float sg = d == 2 ? s2[s] : 1.0f;
            lrh[d] = sg * lr[d];
            lpn[d] = sg * fmaf(a, lr[d], lp[d]);
        }
        const CPos &r = rh[s];
        float J[3];
        for (int d = 0; d < 3; ++d) J[d] = pn[s][d] - pt[s][d];
        float uc[8][3], w[8], gw[8][3];
        size_t nodes[8];
        for (int k = 0; k < 8; ++k) {
            int x, y, z;
            w[k] = stencil_node(r, k, g, x, y, z);
            node_velocity<DT>(src, ffield, x, y, z, g, uc[k]);
            nodes[k] = ((size_t)z * g.ny + y) * g.nx + x;
            const int o[3] = {k & 1, (k >> 1) & 1, k >> 2};
            float ph[3], dph[3];
            for (int d = 0; d < 3; ++d) {
                ph[d] = o[d] ? r.f[d] : 1.0f - r.f[d];
                dph[d] = o[d] ? 1.0f : -1.0f;
            }
            gw[k][0] = dph[0] * ph[1] * ph[2];
            gw[k][1] = ph[0] * dph[1] * ph[2];
            gw[k][2] = ph[0] * ph[1] * dph[2];
        }
        // spread
        for (int k = 0; k < 8; ++k) {
            float lfJ = 0.0f;
            for (int d = 0; d < 3; ++d) {
                const float lf = lam_facc[d * g.nn + nodes[k]];
                lJ[d] = fmaf(-lf, w[k], lJ[d]);
                lfJ = fmaf(lf, J[d], lfJ);
            }
            for (int d = 0; d < 3; ++d) lrh[d] = fmaf(-lfJ, gw[k][d], lrh[d]);
        }
        // update p' = C1 p~ + C2 G u_p
        float lpt[3], lu[3];
        for (int d = 0; d < 3; ++d) {
            lpn[d] += lJ[d];
            lpt[d] = -lJ[d] + C1 * lpn[d];
            lu[d] = C2 * G * lpn[d];
        }
        // interpolation u_p = sum_q w_q u_q
        for (int k = 0; k < 8; ++k) {
            float udot = 0.0f;
            for (int d = 0; d < 3; ++d) {
                atomicAdd(lam_u + d * g.pitch + nodes[k], w[k] * lu[d]);
                udot = fmaf(uc[k][d], lu[d], udot);
            }
            for (int d = 0; d < 3; ++d) lrh[d] = fmaf(udot, gw[k][d], lrh[d]);
        }
        // first half drift
        for (int d = 0; d < 3; ++d) {
            const float sg = d == 2 ? s1[s] : 1.0f;
            lr[d] = sg * lrh[d];
            lp[d] = sg * fmaf(a, lrh[d], lpt[d]);
        }
    }
    for (int d = 0; d < 3; ++d) {
        lam_pos[3 * p + d] = lr[d];
        lam_mom[3 * p + d] = lp[d];
    }
}

}  // namespace

lb_status couple_particles(lb_handle *h, const lb_particles *pp, const lb_couple_params *cp, void *ready, void *done)
{
    const int known = LB_COUPLE_PER_SUBSTEP | LB_COUPLE_OVERLAP | LB_COUPLE_PHI3 | LB_COUPLE_PHI4;
    if (pp->n < 0 || pp->reserved != 0 || (cp->flags & ~known) != 0 ||
        (cp->flags & (LB_COUPLE_PHI3 | LB_COUPLE_PHI4)) == (LB_COUPLE_PHI3 | LB_COUPLE_PHI4)) {
        set_error("lb_couple_particles: bad particle count, reserved field or flags");
        return LB_EINVAL;
    }
    if (h->p.walls && h->p.nz < stencil_width(cp->flags) + 1) {
        set_error("lb_couple_particles: the channel is too narrow for the interpolation stencil");
        return LB_EINVAL;
    }
    if (pp->n == 0) {
        const cudaError_t e = done ? cudaEventRecord((cudaEvent_t)done, h->stream) : cudaSuccess;
        return e == cudaSuccess ? LB_OK : cuda_fail("lb_couple_particles", e);
    }
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
    join_overlap(h);  // a coupling of this step that has not been joined yet
    // impulses of an earlier call that no step has applied yet lie outside
    // this call's stencil records, which the overlapped step re-updates:
    // such a call runs in the serial order
    const bool overlap = (cp->flags & LB_COUPLE_OVERLAP) != 0 && !h->facc_dirty && h->p.equilibrium == 0;
    cudaStream_t main_stream = h->stream;
    if (overlap) {
        // run on the handle's high-priority stream after everything queued on
        // the main stream so far
        cudaError_t e = cudaSuccess;
        if (!h->aux) {
            int lo = 0, hi = 0;
            e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_couple, cudaEventDisableTiming);
        }
        if (e == cudaSuccess && !h->claim) {
            e = cudaMalloc((void **)&h->claim, h->n_nodes * sizeof(unsigned int));
            if (e == cudaSuccess) e = cudaMemsetAsync(h->claim, 0, h->n_nodes * sizeof(unsigned int), main_stream);
            h->claim_tag = 0u;
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_main, main_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_main, 0);
        // the caller's inputs: only the coupling waits for them
        if (e == cudaSuccess && ready) e = cudaStreamWaitEvent(h->aux, (cudaEvent_t)ready, 0);
        if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
        h->stream = h->aux;
    } else if (ready) {
        const cudaError_t e = cudaStreamWaitEvent(main_stream, (cudaEvent_t)ready, 0);
        if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
    }
    struct Restore {  // the main stream comes back on every return
        lb_handle *h;
        cudaStream_t s;
        ~Restore() { h->stream = s; }
    } restore{h, main_stream};
    lb_status st = ensure_buffers(h, pp->n, cp->n_substeps);
    if (st != LB_OK) return st;
    cudaError_t e;
    // impulses of the previous call that lb_step already applied are cleared
    // inside run_substeps (by the persistent kernel, or by k_clear_records)
    timer_mark(h, 1, 0, h->stream);
    switch (h->p.dtype) {
    case LB_F32: e = run_substeps<0>(h, pp, cp); break;
    case LB_F16: e = run_substeps<1>(h, pp, cp); break;
    default: e = run_substeps<2>(h, pp, cp); break;
    }
    timer_mark(h, 1, 1, h->stream);
    if (e == cudaSuccess && overlap) e = cudaEventRecord(h->ev_couple, h->aux);
    // the caller's event: pos and mom hold this call's result
    if (e == cudaSuccess && done) e = cudaEventRecord((cudaEvent_t)done, overlap ? h->aux : main_stream);
    if (e != cudaSuccess) return cuda_fail("lb_couple_particles", e);
    h->facc_dirty = 1;
    if (overlap) {
        Particles *P = h->parts;
        h->overlap_pending = 1;
        h->patch_n = pp->n;
        h->patch_nsub = cp->n_substeps;
        h->patch_rec = P->records + P->rec_off + P->n_records - (size_t)pp->n * (size_t)cp->n_substeps;
        h->patch_span = stencil_width(cp->flags);  // the record span: 2, 3 (origin records) or 4
    }
    return LB_OK;
}

cudaError_t clear_particle_forces(lb_handle *h)
{
    Particles *P = h->parts;
    if (!P || !h->facc) return cudaSuccess;
    if (P->n_records) {
        const StepArgs g = make_args(h);
        const int *rec = P->records + P->rec_off;
        if (P->rec_n > 0 && P->n_records % (size_t)P->rec_n == 0) {  // [nsub][n]: skip repeated cells
            const int nsub = (int)(P->n_records / (size_t)P->rec_n);
            const unsigned int blocks = (unsigned int)(((size_t)P->rec_n * 8 + 255) / 256);
            if (P->rec_span == 4)
                k_clear_records_by_particle<4><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->rec_n, nsub, g);
            else if (P->rec_span == 3)
                k_clear_records_by_particle<3><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->rec_n, nsub, g);
            else
                k_clear_records_by_particle<2><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->rec_n, nsub, g);
        } else {
            int blocks = (int)std::min<size_t>((P->n_records + 255) / 256, (size_t)8 * device_sm_count());
            if (P->rec_span == 4)
                k_clear_records<4><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->n_records, g);
            else if (P->rec_span == 3)
                k_clear_records<3><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->n_records, g);
            else
                k_clear_records<2><<<blocks, 256, 0, h->stream>>>(h->facc, rec, P->n_records, g);
        }
        h->launches += 1;
        P->n_records = 0;
        P->rec_off = 0;
        P->rec_span = 2;
    }
    return cudaGetLastError();
}

template <int DT>
void launch_interpolate(lb_handle *h, int kernel, int n, const double *pos, float *u_out)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs g = make_args(h);
    const int blocks = (int)(((size_t)n * 8 + kPartThreads - 1) / kPartThreads);
    const T *src = static_cast<const T *>(h->pops[h->cur]);
    if (kernel == 3)
        k_interpolate<DT, 3><<<blocks, kPartThreads, 0, h->stream>>>(src, h->force, pos, u_out, n, h->d_err, g);
    else if (kernel == 4)
        k_interpolate<DT, 4><<<blocks, kPartThreads, 0, h->stream>>>(src, h->force, pos, u_out, n, h->d_err, g);
    else
        k_interpolate<DT, 2><<<blocks, kPartThreads, 0, h->stream>>>(src, h->force, pos, u_out, n, h->d_err, g);
}

lb_status interpolate(lb_handle *h, int kernel, int n, const double *pos, float *u_out)
{
    if (n == 0) return LB_OK;
    switch (h->p.dtype) {
    case LB_F32: launch_interpolate<0>(h, kernel, n, pos, u_out); break;
    case LB_F16: launch_interpolate<1>(h, kernel, n, pos, u_out); break;
    default: launch_interpolate<2>(h, kernel, n, pos, u_out); break;
    }
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_interpolate", e);
}

// Checks shared by the reverse-mode entry points of the coupling.
bool adjoint_couple_ok(const lb_handle *h, const lb_particles *pp, const lb_couple_params *cp, const char *who)
{
    if (!pp || !cp || pp->n < 0 || pp->reserved != 0 || (pp->n > 0 && (!pp->pos || !pp->mom))) {
        set_error("%s: bad particle arguments", who);
        return false;
    }
    if (h->p.kT != 0.0 || cp->chain_len > 1 || cp->use_wca || h->p.equilibrium) {
        set_error("%s: the coupling reverse pass covers free particles at kT = 0 (quadratic equilibrium)", who);
        return false;
    }
    if (cp->flags & (LB_COUPLE_PHI3 | LB_COUPLE_PHI4)) {
        set_error("%s: the coupling reverse pass covers the phi_2 stencil", who);
        return false;
    }
    if (cp->fext[0] != 0.0 || cp->fext[1] != 0.0 || cp->fext[2] != 0.0) {
        set_error("%s: the coupling reverse pass covers particles without an external force", who);
        return false;
    }
    if (cp->n_substeps < 1 || cp->n_substeps > kMaxAdjSub || !(cp->dt > 0.0)) {
        set_error("%s: need 1 <= n_substeps <= %d and dt > 0", who, kMaxAdjSub);
        return false;
    }
    if ((!pp->mass && !(pp->mass0 > 0.0)) || (!pp->gamma && !(pp->gamma0 > 0.0))) {
        set_error("%s: mass0 and gamma0 must be > 0 when no per-particle arrays are given", who);
        return false;
    }
    return true;
}

lb_status couple_adjoint(lb_handle *h, const void *state, const lb_particles *pp, const lb_couple_params *cp,
                         const float *lam_facc, float *lam_pos, float *lam_mom, float *lam_u)
{
    if (!adjoint_couple_ok(h, pp, cp, "lb_adjoint_couple")) return LB_EUNSUPPORTED;
    if (pp->n == 0) return LB_OK;
    const CoupleArgs c = make_couple_args(h, pp, cp);
    const int blocks = (pp->n + kPartThreads - 1) / kPartThreads;
    switch (h->p.dtype) {
    case LB_F32:
        k_couple_adjoint<0><<<blocks, kPartThreads, 0, h->stream>>>(
            static_cast<const float *>(state), h->force, pp->pos, pp->mom, pp->mass, pp->gamma, lam_facc, lam_pos,
            lam_mom, lam_u, h->d_err, c, cp->n_substeps);
        break;
    case LB_F16:
        k_couple_adjoint<1><<<blocks, kPartThreads, 0, h->stream>>>(
            static_cast<const __half *>(state), h->force, pp->pos, pp->mom, pp->mass, pp->gamma, lam_facc, lam_pos,
            lam_mom, lam_u, h->d_err, c, cp->n_substeps);
        break;
    default:
        k_couple_adjoint<2><<<blocks, kPartThreads, 0, h->stream>>>(
            static_cast<const __nv_bfloat16 *>(state), h->force, pp->pos, pp->mom, pp->mass, pp->gamma, lam_facc,
            lam_pos, lam_mom, lam_u, h->d_err, c, cp->n_substeps);
        break;
    }
    h->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_couple", e);
}

// A coupling call against the populations `state` whose impulses go to
// facc_out ([3][pitch], zeroed here) instead of the handle's accumulator; the
// particles are updated in place.  The handle's accumulator must hold no
// uncleared impulses (its stencil records are reused here).
lb_status couple_on(lb_handle *h, const void *state, const lb_particles *pp, const lb_couple_params *cp,
                    float *facc_out)
{
    void *saved_pop = h->pops[h->cur];
    float *saved_facc = h->facc;
    const int saved_dirty = h->facc_dirty, saved_stale = h->facc_stale;
    h->pops[h->cur] = const_cast<void *>(state);
    h->facc = facc_out;
    h->facc_stale = 0;
    cudaError_t e = cudaMemsetAsync(facc_out, 0, 3 * h->pitch * sizeof(float), h->stream);
    lb_couple_params c2 = *cp;
    c2.flags &= ~LB_COUPLE_OVERLAP;
    lb_status st = e == cudaSuccess ? couple_particles(h, pp, &c2) : cuda_fail("lb_adjoint_kinetic_coupled", e);
    if (h->parts) {  // these records index facc_out
        h->parts->n_records = 0;
        h->parts->rec_off = 0;
        h->parts->rec_span = 2;
    }
    h->pops[h->cur] = saved_pop;
    h->facc = saved_facc;
    h->facc_dirty = saved_dirty;
    h->facc_stale = saved_stale;
    return st;
}

// After a grid-barrier timeout the arrival word is left mid-count; zero it
// (stream-ordered) so that the next persistent launch starts clean.
cudaError_t reset_particle_barrier(lb_handle *h)
{
    Particles *P = h->parts;
    if (!P || !P->bar) return cudaSuccess;
    return cudaMemsetAsync(P->bar, 0, 3 * sizeof(unsigned int), h->stream);
}

void drop_particle_records(lb_handle *h)
{
    Particles *P = h->parts;
    if (!P) return;
    P->n_records = 0;
    P->rec_off = 0;
    P->rec_span = 2;
}

void destroy_particles(lb_handle *h)
{
    free_parts(h->parts);
    h->parts = nullptr;
}

}  // namespace lbi
