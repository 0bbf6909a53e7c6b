// spheres.cu -- extended particles: solid spheres that translate through the
// lattice (and may rotate), coupled to the fluid by the moving link bounce-back of Sec. 4.1
// (Eq. MBB) and updated as in Sec. 4.2 (Eqs. EOMD-1..3, force0, zeta,
// EOMUsol and the consistency equation for the velocity U~).
//
// One lb_step_spheres call, all on the handle's stream:
//   k_sph_half     one thread per sphere: R(t+h/2) = R + U/2, accumulators zeroed
//   k_sph_map      per sphere, the nodes of a box around it: the solid map
//                  follows R(t+h/2); a covered fluid node gives its momentum
//                  to the sphere, an uncovered node starts from n^eq(rho0, U)
//                  and the sphere loses rho0 U
//   k_sph_links    per sphere, the fluid nodes of its box: F0 = sum 2 n*_b c_b
//                  and zeta = 6 rho0 sum a_b c_b c_b^T over the boundary links
//   k_sph_update   one thread per sphere: U(t+h) and U~ (zeta's eigenbasis
//                  by FP32 Jacobi rotations; U kept in FP64)
//   the plain stream-collide launch over every node (exact for fluid nodes
//                  without a solid neighbour), then
//   k_sph_near_nodes  the near fluid nodes (listed by k_sph_links) again: pull
//                  streaming in which a population whose source node is solid
//                  returns as n*_-i(r) + 6 a_i rho0 U~.c_i, then the same
//                  collision
//   k_sph_finish   one thread per sphere: R(t+h) = R(t+h/2) + U(t+h)/2
// The solid map holds the sphere index of a solid node, -2 for a fluid node
// with a solid neighbour (the only nodes whose pull needs the map) and -1
// for the other fluid nodes; k_sph_links sets the marks within a + 2.5 of
// each centre every step (a -2 left further out by a moved sphere is
// harmless: that node is recomputed with the same result).
// Spheres translate, and rotate when angular velocities are given (u_b = U +
// Omega x (r_b - R), Eq. NodeVel; moment of inertia 2/5 m a^2); rho in Eqs.
// MBB and zeta is rho0, and spheres must stay apart; positions and velocities are FP64 (a
// few values per sphere), the populations FP32 deviations n - a rho0 (the
// rho0 part of F0 sums to zero over a closed set of links and is left out).
#include <cmath>

#include "stream_collide.cuh"

namespace lbi {

extern template cudaError_t launch_stream_collide_dt<0>(const lb_handle *, const void *, void *, const float *,
                                                        float *);

namespace {

constexpr int kSphThreads = 128;
// per sphere: F0 (3), covering momentum (3), friction TT xx yy zz xy yz zx (6),
// torque T0 (3), covering angular momentum (3), friction TR row-major (9),
// friction RR xx yy zz xy yz zx (6)
constexpr int kAcc = 33;

// d - L floor(d / L + 1/2) for d = x - c in (-L, L): the minimum image by
// comparisons (the same value wherever |d| < L / 2 - 1, which covers every
// node a sphere of 2 a + 6 <= L can reach).
__device__ __forceinline__ double periodic_offset(double d, int L)
{
    const double h = 0.5 * (double)L;
    return d >= h ? __dadd_rn(d, -(double)L) : (d < -h ? __dadd_rn(d, (double)L) : d);
}

__device__ __forceinline__ double wrap_pos(double v, int L) { return __dadd_rn(v, -(double)L * floor(v / (double)L)); }

// v in (-L, 2L): one add or subtract (box offsets are below L).
__device__ __forceinline__ int wrap_i(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

constexpr int kFar = -1, kNear = -2;  // fluid nodes without / with a solid neighbour

// The box of B^3 nodes around a sphere starts at base = floor(c - a) - 2
// per axis; cf = c - base (FP32, in [2, 3)) places the centre in it.  One
// block works on one sphere: its first threads fill these in shared memory.
struct Box {
    int base[3];
    float cf[3];
};

__device__ __forceinline__ void box_setup(Box &b, const double c[3], double a)
{
    if (threadIdx.x < 3) {
        const int d = threadIdx.x;
        const int base = (int)floor(c[d] - a) - 2;
        b.base[d] = base;
        b.cf[d] = (float)(c[d] - (double)base);
    }
    __syncthreads();
}

// Node k of the box: lattice coordinates and offsets within the box.
__device__ __forceinline__ void box_node(const Box &b, int B, int k, const StepArgs &g, int &x, int &y, int &z,
                                         int o[3])
{
    o[0] = k % B;
    o[1] = (k / B) % B;
    o[2] = k / (B * B);
    x = wrap_i(b.base[0] + o[0], g.nx);
    y = wrap_i(b.base[1] + o[1], g.ny);
    z = wrap_i(b.base[2] + o[2], g.nz);
}

// |r - c| < a with the minimum image, the arithmetic of the definition
// written without contractions.
__device__ __forceinline__ bool inside(int x, int y, int z, const double c[3], double a, const StepArgs &g)
{
    const double dx = periodic_offset(__dadd_rn((double)x, -c[0]), g.nx);
    const double dy = periodic_offset(__dadd_rn((double)y, -c[1]), g.ny);
    const double dz = periodic_offset(__dadd_rn((double)z, -c[2]), g.nz);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 < __dmul_rn(a, a);
}

// inside() decided in FP32 where the squared distance is clearly away from
// a^2 (the FP32 error is below 1e-5 a^2 for boxes of this size), in FP64
// otherwise: the same decisions as inside(), mostly without FP64 arithmetic.
__device__ __forceinline__ bool inside_fast(const Box &b, const int o[3], int x, int y, int z, const double c[3],
                                            double a, const StepArgs &g)
{
    const float dx = (float)o[0] - b.cf[0], dy = (float)o[1] - b.cf[1], dz = (float)o[2] - b.cf[2];
    const float d2 = dx * dx + dy * dy + dz * dz, a2 = (float)(a * a);
    if (d2 < a2 * (1.0f - 1e-4f)) return true;
    if (d2 > a2 * (1.0f + 1e-4f)) return false;
    return inside(x, y, z, c, a, g);
}

__global__ void k_sph_place(int *owner, const double *pos, double a, int B, int n, StepArgs g, unsigned int *err)
{
    __shared__ Box b;
    const int p = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double c[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
    box_setup(b, c, a);
    if (p >= n || k >= B * B * B) return;
    int x, y, z, o[3];
    box_node(b, B, k, g, x, y, z, o);
    if (!inside_fast(b, o, x, y, z, c, a, g)) return;
    const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
    if (atomicCAS(owner + s, -1, p) != -1) atomicOr(err, LB_DERR_SPHERE);
}

__global__ void k_sph_half(const double *pos, const double *vel, const double *mass, double mass0, int n, double *rh,
                           float *acc, unsigned int *count, StepArgs g, unsigned int *err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) *count = 0u;  // the near-node list of this step
    if (p >= n) return;
    const double m = mass ? mass[p] : mass0;
    const int L[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) {
        const double u = vel[3 * p + d];
        if (!(fabs(u) <= 1.0)) atomicOr(err, LB_DERR_SPHERE);  // also catches NaN
        rh[3 * p + d] = m > 0.0 ? wrap_pos(__dadd_rn(pos[3 * p + d], 0.5 * u), L[d]) : pos[3 * p + d];
    }
    for (int q = 0; q < kAcc; ++q) acc[kAcc * p + q] = 0.0f;
}

__device__ __forceinline__ void cross3f(const float a[3], const float b[3], float out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

// The solid map follows the half-step centres (uncovered nodes get the
// equilibrium of the surface velocity U + Omega x rho at time t, which this
// kernel reads before any update).  om: angular velocities, or NULL.
__global__ void k_sph_map(int *owner, float *pops, const double *rh, const double *vel, const double *om, double a,
                          int B, int n, StepArgs g, float *acc, unsigned int *err)
{
    __shared__ Box b;
    const int p = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double c[3] = {rh[3 * p], rh[3 * p + 1], rh[3 * p + 2]};
    box_setup(b, c, a);
    if (p >= n || k >= B * B * B) return;
    int x, y, z, o[3];
    box_node(b, B, k, g, x, y, z, o);
    const size_t s = ((size_t)z * g.ny + y) * g.nx + x;
    const size_t P = g.pitch;
    const int old = owner[s];
    const float rv[3] = {(float)o[0] - b.cf[0], (float)o[1] - b.cf[1], (float)o[2] - b.cf[2]};
    float j[3] = {0.f, 0.f, 0.f};
    if (inside_fast(b, o, x, y, z, c, a, g)) {
        if (old == p) return;
        if (old >= 0) {  // a node passing from one sphere to another
            atomicOr(err, LB_DERR_SPHERE);
            return;
        }
#pragma unroll
        for (int i = 1; i < 19; ++i) {  // covered: its fluid momentum goes to the sphere
            const float v = pops[(size_t)i * P + s];
            if (lbd::cx(i)) j[0] += lbd::cx(i) * v;
            if (lbd::cy(i)) j[1] += lbd::cy(i) * v;
            if (lbd::cz(i)) j[2] += lbd::cz(i) * v;
        }
        owner[s] = p;
    } else if (old == p) {  // uncovered: new fluid at the surface velocity
        owner[s] = kNear;
        float u[3] = {(float)vel[3 * p], (float)vel[3 * p + 1], (float)vel[3 * p + 2]};
        if (om) {
            const float w[3] = {(float)om[3 * p], (float)om[3 * p + 1], (float)om[3 * p + 2]};
            float wr[3];
            cross3f(w, rv, wr);
            for (int d = 0; d < 3; ++d) u[d] += wr[d];
        }
        const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float cu = lbd::cx(i) * u[0] + lbd::cy(i) * u[1] + lbd::cz(i) * u[2];
            pops[(size_t)i * P + s] = lbd::weight(i) * g.rho0 * (3.0f * cu + 4.5f * cu * cu - 1.5f * u2);
        }
        for (int d = 0; d < 3; ++d) j[d] = -g.rho0 * u[d];
    } else {
        return;
    }
    for (int d = 0; d < 3; ++d) atomicAdd(acc + kAcc * p + 3 + d, j[d]);
    if (om) {
        float mom[3];
        cross3f(rv, j, mom);
        for (int d = 0; d < 3; ++d) atomicAdd(acc + kAcc * p + 15 + d, mom[d]);
    }
}

// Sums of each sphere over its boundary links (fluid node r, r + c_b solid,
// r_b = r + c_b/2, rho_b = r_b - R, g = rho_b x c_b): F0 = sum 2 n*_b c_b,
// the friction blocks 6 rho0 sum a_b (c c^T, and with ROT c g^T, g g^T) and
// with ROT the torque T0 = sum 2 n*_b g.  A block reduces its sums before one
// atomic per entry.  The fluid nodes within a + 2.5 of the centre are marked
// near (a solid neighbour of any sphere) or far on the way.
template <bool ROT>
__global__ void __launch_bounds__(kSphThreads) k_sph_links(int *owner, const float *pops, const double *rh,
                                                            double a, int B, int n, StepArgs g, float *acc,
                                                            int *list, unsigned int *count)
{
    constexpr int NV = ROT ? 27 : 9;
    __shared__ float red[kSphThreads / 32][NV];
    __shared__ Box b;
    const int p = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0f;
    const double c[3] = {rh[3 * p], rh[3 * p + 1], rh[3 * p + 2]};
    box_setup(b, c, a);
    bool add = false;  // a near node for the list of the re-update
    size_t s = 0;
    if (p < n && k < B * B * B) {
        int x, y, z, o[3];
        box_node(b, B, k, g, x, y, z, o);
        s = ((size_t)z * g.ny + y) * g.nx + x;
        const int own = owner[s];
        const float dx = (float)o[0] - b.cf[0], dy = (float)o[1] - b.cf[1], dz = (float)o[2] - b.cf[2];
        const float rf = (float)a + 2.5f;
        if (own < 0 && dx * dx + dy * dy + dz * dz > rf * rf) {
            // no node of this sphere within two lattice units: no links; the
            // mark stays (another sphere may be near, and a stale near mark
            // only costs the exact recomputation of a far node)
        } else if (own < 0) {
            bool near = false;
#pragma unroll
            for (int i = 1; i < 19; ++i) {
                const int tx = wrap_i(x + lbd::cx(i), g.nx), ty = wrap_i(y + lbd::cy(i), g.ny),
                          tz = wrap_i(z + lbd::cz(i), g.nz);
                const int ow = owner[((size_t)tz * g.ny + ty) * g.nx + tx];
                near = near || ow >= 0;
                if (ow != p) continue;
                const float nb = 2.0f * pops[(size_t)i * g.pitch + s];
                const float cb[3] = {(float)lbd::cx(i), (float)lbd::cy(i), (float)lbd::cz(i)};
                const float za = 6.0f * g.rho0 * lbd::weight(i);
                v[0] += nb * cb[0];
                v[1] += nb * cb[1];
                v[2] += nb * cb[2];
                v[3] += za * cb[0] * cb[0];
                v[4] += za * cb[1] * cb[1];
                v[5] += za * cb[2] * cb[2];
                v[6] += za * cb[0] * cb[1];
                v[7] += za * cb[1] * cb[2];
                v[8] += za * cb[2] * cb[0];
                if (ROT) {
                    const float rb[3] = {dx + 0.5f * cb[0], dy + 0.5f * cb[1], dz + 0.5f * cb[2]};
                    float gv[3];
                    cross3f(rb, cb, gv);
#pragma unroll
                    for (int d = 0; d < 3; ++d) v[9 + d] += nb * gv[d];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int d = 0; d < 3; ++d) v[12 + 3 * r + d] += za * cb[r] * gv[d];
                    v[21] += za * gv[0] * gv[0];
                    v[22] += za * gv[1] * gv[1];
                    v[23] += za * gv[2] * gv[2];
                    v[24] += za * gv[0] * gv[1];
                    v[25] += za * gv[1] * gv[2];
                    v[26] += za * gv[2] * gv[0];
                }
            }
            const int mark = near ? kNear : kFar;
            if (own != mark) owner[s] = mark;
            add = near;
        }
    }
    {  // append the near nodes, one atomic per warp (a node near two spheres
       // appears twice and is recomputed with the same value)
        const unsigned ball = __ballot_sync(0xffffffffu, add);
        if (ball) {
            const int lane = threadIdx.x & 31, leader = __ffs(ball) - 1;
            unsigned int base = 0;
            if (lane == leader) base = atomicAdd(count, (unsigned int)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (add) list[base + __popc(ball & ((1u << lane) - 1u))] = (int)s;
        }
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < NV; ++q) red[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV && p < n) {
        float t = 0.0f;
        for (int q = 0; q < kSphThreads / 32; ++q) t += red[q][threadIdx.x];
        if (t != 0.0f) {
            // F0 -> 0..2, friction TT -> 6..11, T0 -> 12..14, TR -> 18..26, RR -> 27..32
            const int q = threadIdx.x;
            const int slot = q < 3 ? q : (q < 9 ? q + 3 : (q < 12 ? q + 3 : q + 6));
            atomicAdd(acc + kAcc * p + slot, t);
        }
    }
}

// Eigen-decomposition of a symmetric N x N matrix by cyclic Jacobi rotations
// (FP32), until the off-diagonal part is below 1e-7 of the diagonal.
template <int N>
__device__ void jacobi(float A[N][N], float w[N], float V[N][N])
{
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) V[i][j] = (i == j) ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 15; ++sweep) {
        float off = 0.0f, dia = 0.0f;
#pragma unroll
        for (int p = 0; p < N; ++p) {
            dia += fabsf(A[p][p]);
#pragma unroll
            for (int q = p + 1; q < N; ++q) off += fabsf(A[p][q]);
        }
        if (!(off > 1e-7f * dia)) break;
#pragma unroll
        for (int p = 0; p < N - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) {
                if (A[p][q] == 0.0f) continue;
                const float th = (A[q][q] - A[p][p]) / (2.0f * A[p][q]);
                const float t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
                const float c = rsqrtf(t * t + 1.0f), s = t * c;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    const float vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = A[i][i];
}

// The velocity update of N components (3: translation; 6: translation and
// rotation) in the variables W = M^1/2 V, where dW/dt = -K W + G with
// K = M^-1/2 Z M^-1/2 and G = M^-1/2 F; per eigen-direction of K (kappa),
// written as increments of W so that FP32 carries only the change:
//   W' - W = (1 - e^-kappa) (G / kappa - W)                       (Eq. EOMUsol)
//   W~ - W = ((1 - e^-kappa) / kappa - 1) W + (1 - (1 - e^-kappa) / kappa) G / kappa
// (the consistency equation); a direction without links takes the limits G
// and G / 2.  V is FP64, V' = V + M^-1/2 (W' - W).
template <int N>
__device__ void velocity_update(const float Z[N][N], const float sq[N], double V[N], const float F[N], float Vt[N])
{
    float K[N][N], Q[N][N], w[N], Wf[N], G[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        Wf[i] = sq[i] * (float)V[i];
        G[i] = F[i] / sq[i];
#pragma unroll
        for (int j = 0; j < N; ++j) K[i][j] = Z[i][j] / (sq[i] * sq[j]);
    }
    jacobi<N>(K, w, Q);
    float dn[N], dt[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float we = 0.0f, ge = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            we += Q[i][k] * Wf[i];
            ge += Q[i][k] * G[i];
        }
        const float ka = w[k];
        if (ka < 1e-6f) {
            dn[k] = ge;
            dt[k] = 0.5f * ge;
        } else {
            const float e1 = -expm1f(-ka), r = e1 / ka;
            dn[k] = e1 * (ge / ka - we);
            dt[k] = (r - 1.0f) * we + (1.0f - r) * ge / ka;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float sn = 0.0f, st = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            sn += Q[i][k] * dn[k];
            st += Q[i][k] * dt[k];
        }
        Vt[i] = (float)V[i] + st / sq[i];
        V[i] += (double)(sn / sq[i]);
    }
}

// U(t+h), U~ (and with om Omega(t+h), Omega~) of each sphere; the moment of
// inertia is 2/5 m a^2.
__global__ void k_sph_update(double *vel, double *om, const double *mass, double mass0, double a, const double *force,
                             int n, const float *acc, float4 *ut, float4 *uw)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double m = mass ? mass[p] : mass0;
    const float *ac = acc + kAcc * p;
    if (!(m > 0.0)) {  // held fixed: the surface moves with U (+ Omega x rho)
        ut[p] = make_float4((float)vel[3 * p], (float)vel[3 * p + 1], (float)vel[3 * p + 2], 0.0f);
        uw[p] = om ? make_float4((float)om[3 * p], (float)om[3 * p + 1], (float)om[3 * p + 2], 0.0f)
                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const double I = 0.4 * m * a * a;
    if (om) {
        double V[6];
        float F[6], Z[6][6], sq[6], Vt[6];
        for (int d = 0; d < 3; ++d) {
            V[d] = vel[3 * p + d] + (double)ac[3 + d] / m;  // covered / uncovered nodes
            V[3 + d] = om[3 * p + d] + (double)ac[15 + d] / I;
            F[d] = ac[d] + (force ? (float)force[3 * p + d] : 0.0f);
            F[3 + d] = ac[12 + d];
            sq[d] = sqrtf((float)m);
            sq[3 + d] = sqrtf((float)I);
        }
        const float tt[3][3] = {{ac[6], ac[9], ac[11]}, {ac[9], ac[7], ac[10]}, {ac[11], ac[10], ac[8]}};
        const float rr[3][3] = {{ac[27], ac[30], ac[32]}, {ac[30], ac[28], ac[31]}, {ac[32], ac[31], ac[29]}};
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) {
                Z[r][d] = tt[r][d];
                Z[3 + r][3 + d] = rr[r][d];
                Z[r][3 + d] = ac[18 + 3 * r + d];
                Z[3 + d][r] = ac[18 + 3 * r + d];
            }
        velocity_update<6>(Z, sq, V, F, Vt);
        for (int d = 0; d < 3; ++d) {
            vel[3 * p + d] = V[d];
            om[3 * p + d] = V[3 + d];
        }
        ut[p] = make_float4(Vt[0], Vt[1], Vt[2], 0.0f);
        uw[p] = make_float4(Vt[3], Vt[4], Vt[5], 0.0f);
        return;
    }
    double V[3];
    float F[3], sq[3], Vt[3];
    for (int d = 0; d < 3; ++d) {
        V[d] = vel[3 * p + d] + (double)ac[3 + d] / m;
        F[d] = ac[d] + (force ? (float)force[3 * p + d] : 0.0f);
        sq[d] = sqrtf((float)m);
    }
    const float Z[3][3] = {{ac[6], ac[9], ac[11]}, {ac[9], ac[7], ac[10]}, {ac[11], ac[10], ac[8]}};
    velocity_update<3>(Z, sq, V, F, Vt);
    for (int d = 0; d < 3; ++d) vel[3 * p + d] = V[d];
    ut[p] = make_float4(Vt[0], Vt[1], Vt[2], 0.0f);
    uw[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__global__ void k_sph_finish(double *pos, const double *vel, const double *mass, double mass0, const double *rh,
                             int n, StepArgs g)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double m = mass ? mass[p] : mass0;
    if (!(m > 0.0)) return;
    const int L[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) pos[3 * p + d] = wrap_pos(__dadd_rn(rh[3 * p + d], 0.5 * vel[3 * p + d]), L[d]);
}

// Minimum image of d along an axis of length L (|d| < L).
__device__ __forceinline__ float image_f(float d, int L)
{
    const float h = 0.5f * (float)L;
    return d > h ? d - (float)L : (d < -h ? d + (float)L : d);
}

// Stream and collide fluid node (x, y, z) whose map entry is own (< 0): a
// population whose source node is solid (sphere o) returns from the node
// itself with the moving-wall term, n_i(r) = n*_-i(r) + 2 a_i rho0
// u_b.c_i / c_s^2 with u_b = U~_o + Omega~_o x (r_b - R_o), r_b = r - c_i / 2
// (Eqs. MBB, NodeVel; c_b = -c_i); far fluid nodes pull without looking at
// the map.  rot: the spheres rotate (uw, rh are read).
template <bool NOISE>
__device__ __forceinline__ void sphere_node(const float *__restrict__ src, float *__restrict__ dst,
                                            const float *__restrict__ ffield, const int *__restrict__ owner,
                                            const float4 *__restrict__ ut, const float4 *__restrict__ uw,
                                            const double *__restrict__ rh, bool rot, const StepArgs &a, int x, int y,
                                            int z, int own)
{
    const size_t self = ((size_t)z * a.ny + y) * a.nx + x;
    const int xm = (x == 0) ? a.nx - 1 : x - 1, xp = (x == a.nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? a.ny - 1 : y - 1, yp = (y == a.ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? a.nz - 1 : z - 1, zp = (z == a.nz - 1) ? 0 : z + 1;
    const size_t P = a.pitch;
    float n[19];
    if (own == kFar) {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
            const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
            const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
            n[i] = __ldg(src + (size_t)i * P + ((size_t)sz * a.ny + sy) * a.nx + sx);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
            const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
            const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
            const size_t t = ((size_t)sz * a.ny + sy) * a.nx + sx;
            const int o = i == 0 ? kFar : __ldg(owner + t);
            if (o >= 0) {
                const float4 v = __ldg(ut + o);
                float ub[3] = {v.x, v.y, v.z};
                if (rot) {
                    const float4 w = __ldg(uw + o);
                    const float rb[3] = {image_f((float)((double)x - 0.5 * lbd::cx(i) - rh[3 * o]), a.nx),
                                         image_f((float)((double)y - 0.5 * lbd::cy(i) - rh[3 * o + 1]), a.ny),
                                         image_f((float)((double)z - 0.5 * lbd::cz(i) - rh[3 * o + 2]), a.nz)};
                    const float wv[3] = {w.x, w.y, w.z};
                    float wr[3];
                    cross3f(wv, rb, wr);
                    for (int d = 0; d < 3; ++d) ub[d] += wr[d];
                }
                const float uc = lbd::cx(i) * ub[0] + lbd::cy(i) * ub[1] + lbd::cz(i) * ub[2];
                n[i] = __ldg(src + (size_t)lbd::opposite(i) * P + self) + 6.0f * lbd::weight(i) * a.rho0 * uc;
            } else {
                n[i] = __ldg(src + (size_t)i * P + t);
            }
        }
    }
    float fx = a.fx, fy = a.fy, fz = a.fz;
    if (ffield) {
        fx += __ldg(ffield + self);
        fy += __ldg(ffield + a.nn + self);
        fz += __ldg(ffield + 2 * a.nn + self);
    }
    float m[19], out[19];
    lbd::forward(n, m);
    collide_moments<NOISE>(m, fx, fy, fz, a, a.rk, (uint32_t)self, a.replica, out);
#pragma unroll
    for (int i = 0; i < 19; ++i) dst[(size_t)i * P + self] = out[i];
}

// The near fluid nodes (the list k_sph_links built this step), after the
// plain update of all nodes: every fluid node without a solid neighbour is
// exact from that update (solid nodes hold values nobody reads), the near
// ones are done again here with the moving bounce-back.  Grid-stride over
// the list.
template <bool NOISE>
__global__ void __launch_bounds__(kSphThreads) k_sph_near_nodes(const float *__restrict__ src, float *__restrict__ dst,
                                                                 const float *__restrict__ ffield,
                                                                 const int *__restrict__ owner,
                                                                 const float4 *__restrict__ ut,
                                                                 const float4 *__restrict__ uw, const double *rh,
                                                                 bool rot, const int *list,
                                                                 const unsigned int *count, StepArgs g)
{
    const unsigned int nl = *count;
    for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < nl; q += gridDim.x * blockDim.x) {
        const int s = list[q];
        const int x = s % g.nx, y = (s / g.nx) % g.ny, z = s / (g.nx * g.ny);
        sphere_node<NOISE>(src, dst, ffield, owner, ut, uw, rh, rot, g, x, y, z, kNear);
    }
}

int box_edge(double a) { return (int)std::ceil(2.0 * a) + 6; }

// The map as the caller sees it: sphere index or -1.
__global__ void k_sph_export(const int *owner, int *out, size_t nn)
{
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < nn; s += (size_t)gridDim.x * blockDim.x)
        out[s] = owner[s] >= 0 ? owner[s] : -1;
}

bool check_spheres(const lb_handle *h, const lb_spheres *s, const char *who)
{
    if (!s || s->n < 0 || s->n > 65535 || s->reserved != 0) {
        set_error("%s: need 0 <= n <= 65535 spheres and reserved = 0", who);
        return false;
    }
    if (s->n > 0 && (!s->pos || !s->vel || ((uintptr_t)s->pos & 7u) || ((uintptr_t)s->vel & 7u) ||
                     ((uintptr_t)s->omega & 7u))) {
        set_error("%s: pos, vel (and omega) must be 8-byte aligned device arrays", who);
        return false;
    }
    const int lmin = std::min(h->p.nx, std::min(h->p.ny, h->p.nz));
    if (!(s->radius > 0.0) || box_edge(s->radius) > lmin) {
        set_error("%s: need 0 < radius and 2 radius + 6 <= the shortest box edge (%d)", who, lmin);
        return false;
    }
    return true;
}

lb_status spheres_supported(const lb_handle *h, const char *who)
{
    if (h->p.walls || h->p.dtype != LB_F32 || h->p.equilibrium) {
        set_error("%s: spheres need a periodic box with FP32 storage and the quadratic equilibrium", who);
        return LB_EUNSUPPORTED;
    }
    return LB_OK;
}

lb_status ensure_sphere_buffers(lb_handle *h, int n, double radius)
{
    cudaError_t e = cudaSuccess;
    if (!h->sph_owner) e = cudaMalloc((void **)&h->sph_owner, h->n_nodes * sizeof(int));
    if (e == cudaSuccess && !h->sph_count) e = cudaMalloc((void **)&h->sph_count, sizeof(unsigned int));
    const int B = box_edge(radius);
    const size_t need = (size_t)n * B * B * B;  // every box node of every sphere at most once
    if (e == cudaSuccess && h->sph_list_cap < need) {
        cudaFree(h->sph_list);
        h->sph_list = nullptr;
        h->sph_list_cap = 0;
        e = cudaMalloc((void **)&h->sph_list, need * sizeof(int));
        if (e == cudaSuccess) h->sph_list_cap = need;
    }
    if (e == cudaSuccess && h->sph_cap < n) {
        cudaFree(h->sph_acc);
        cudaFree(h->sph_rh);
        cudaFree(h->sph_ut);
        cudaFree(h->sph_uw);
        h->sph_acc = nullptr;
        h->sph_rh = nullptr;
        h->sph_ut = nullptr;
        h->sph_uw = nullptr;
        h->sph_cap = 0;
        e = cudaMalloc((void **)&h->sph_acc, (size_t)n * kAcc * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->sph_rh, (size_t)n * 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->sph_ut, (size_t)n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->sph_uw, (size_t)n * sizeof(float4));
        if (e == cudaSuccess) h->sph_cap = n;
    }
    if (e != cudaSuccess) {
        set_error("spheres: device allocation failed (%s)", cudaGetErrorString(e));
        return LB_ENOMEM;
    }
    return LB_OK;
}

}  // namespace

void destroy_spheres(lb_handle *h)
{
    cudaFree(h->sph_owner);
    cudaFree(h->sph_acc);
    cudaFree(h->sph_rh);
    cudaFree(h->sph_ut);
    cudaFree(h->sph_uw);
    cudaFree(h->sph_list);
    cudaFree(h->sph_count);
    h->sph_uw = nullptr;
    h->sph_list = nullptr;
    h->sph_count = nullptr;
    h->sph_list_cap = 0;
    h->sph_owner = nullptr;
    h->sph_acc = nullptr;
    h->sph_rh = nullptr;
    h->sph_ut = nullptr;
    h->sph_cap = 0;
    h->sph_n = -1;
}

}  // namespace lbi

using namespace lbi;

extern "C" {

lb_status lb_spheres_place(lb_handle *h, const lb_spheres *s)
{
    if (!h || !check_spheres(h, s, "lb_spheres_place")) return LB_EINVAL;
    lb_status st = spheres_supported(h, "lb_spheres_place");
    if (st != LB_OK) return st;
    join_overlap(h);
    st = ensure_sphere_buffers(h, std::max(s->n, 1), s->radius);
    if (st != LB_OK) return st;
    const StepArgs g = make_args(h);
    cudaError_t e = cudaMemsetAsync(h->sph_owner, 0xff, h->n_nodes * sizeof(int), h->stream);  // all fluid
    if (e == cudaSuccess && s->n > 0) {
        const int B = box_edge(s->radius);
        const dim3 grid((unsigned)((B * B * B + kSphThreads - 1) / kSphThreads), (unsigned)s->n);
        k_sph_place<<<grid, kSphThreads, 0, h->stream>>>(h->sph_owner, s->pos, s->radius, B, s->n, g, h->d_err);
        // near / far marks around the placed spheres (the sums go to scratch)
        e = cudaMemcpyAsync(h->sph_rh, s->pos, (size_t)s->n * 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                            h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->sph_acc, 0, (size_t)s->n * kAcc * sizeof(float), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->sph_count, 0, sizeof(unsigned int), h->stream);
        if (e == cudaSuccess)
            k_sph_links<false><<<grid, kSphThreads, 0, h->stream>>>(
                h->sph_owner, static_cast<const float *>(h->pops[h->cur]), h->sph_rh, s->radius, B, s->n, g, h->sph_acc,
                h->sph_list, h->sph_count);
        h->launches += 2;
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail("lb_spheres_place", e);
    h->sph_n = s->n;
    h->sph_a = s->radius;
    return LB_OK;
}

lb_status lb_step_spheres(lb_handle *h, const lb_spheres *s)
{
    const lbi::NvtxRange range("lb_step_spheres");
    if (!h || !check_spheres(h, s, "lb_step_spheres")) return LB_EINVAL;
    lb_status st = spheres_supported(h, "lb_step_spheres");
    if (st != LB_OK) return st;
    if (h->sph_n != s->n || h->sph_a != s->radius) {
        set_error("lb_step_spheres: the spheres differ from the placed ones (call lb_spheres_place)");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (h->facc_dirty) {
        set_error("lb_step_spheres: point-particle impulses are pending; spheres and point particles are not "
                  "coupled in one step");
        return LB_EUNSUPPORTED;
    }
    const StepArgs g = make_args(h);
    float *src = static_cast<float *>(h->pops[h->cur]);
    float *dst = static_cast<float *>(h->pops[1 - h->cur]);
    const int n = s->n;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        const int B = box_edge(s->radius);
        const unsigned pb = (unsigned)((n + kSphThreads - 1) / kSphThreads);
        const dim3 grid((unsigned)((B * B * B + kSphThreads - 1) / kSphThreads), (unsigned)n);
        k_sph_half<<<pb, kSphThreads, 0, h->stream>>>(s->pos, s->vel, s->mass, s->mass0, n, h->sph_rh, h->sph_acc,
                                                      h->sph_count, g, h->d_err);
        k_sph_map<<<grid, kSphThreads, 0, h->stream>>>(h->sph_owner, src, h->sph_rh, s->vel, s->omega, s->radius, B, n,
                                                       g, h->sph_acc, h->d_err);
        if (s->omega)
            k_sph_links<true><<<grid, kSphThreads, 0, h->stream>>>(h->sph_owner, src, h->sph_rh, s->radius, B, n, g,
                                                                   h->sph_acc, h->sph_list, h->sph_count);
        else
            k_sph_links<false><<<grid, kSphThreads, 0, h->stream>>>(h->sph_owner, src, h->sph_rh, s->radius, B, n, g,
                                                                    h->sph_acc, h->sph_list, h->sph_count);
        k_sph_update<<<pb, kSphThreads, 0, h->stream>>>(s->vel, s->omega, s->mass, s->mass0, s->radius, s->force, n,
                                                        h->sph_acc, h->sph_ut, h->sph_uw);
        h->launches += 4;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {  // every node with the plain update (solid nodes get values nobody reads)
        e = launch_stream_collide_dt<0>(h, src, dst, nullptr, nullptr);
        h->launches += 1;
    }
    if (e == cudaSuccess && n > 0) {  // then the near fluid nodes with the moving bounce-back
        const unsigned grid = (unsigned)(4 * device_sm_count());
        const bool rot = s->omega != nullptr;
        if (g.kT > 0.0f)
            k_sph_near_nodes<true><<<grid, kSphThreads, 0, h->stream>>>(src, dst, h->force, h->sph_owner, h->sph_ut,
                                                                        h->sph_uw, h->sph_rh, rot, h->sph_list,
                                                                        h->sph_count, g);
        else
            k_sph_near_nodes<false><<<grid, kSphThreads, 0, h->stream>>>(src, dst, h->force, h->sph_owner, h->sph_ut,
                                                                         h->sph_uw, h->sph_rh, rot, h->sph_list,
                                                                         h->sph_count, g);
        h->launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        k_sph_finish<<<(unsigned)((n + kSphThreads - 1) / kSphThreads), kSphThreads, 0, h->stream>>>(
            s->pos, s->vel, s->mass, s->mass0, h->sph_rh, n, g);
        h->launches += 1;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail("lb_step_spheres", e);
    h->cur = 1 - h->cur;
    h->step += 1;
    return LB_OK;
}

lb_status lb_get_solid_map(lb_handle *h, int *owner_out)
{
    if (!h || !owner_out) {
        set_error("lb_get_solid_map: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = cudaSuccess;
    if (h->sph_owner && h->sph_n >= 0) {
        k_sph_export<<<(unsigned)std::min<size_t>((h->n_nodes + 255) / 256, 65535), 256, 0, h->stream>>>(
            h->sph_owner, owner_out, h->n_nodes);
        h->launches += 1;
        e = cudaGetLastError();
    } else {
        e = cudaMemsetAsync(owner_out, 0xff, h->n_nodes * sizeof(int), h->stream);
    }
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_get_solid_map", e);
}

}  // extern "C"
