// stream_collide.cuh -- fused pull-stream + MRT collision + noise + forcing.
//
// One thread per fluid node; a block covers BX consecutive x of one (y, z)
// row, so the 19 plane loads and 19 plane stores of a warp are coalesced
// (the +-x neighbours of a row are the same 32-byte sectors shifted by one
// element).  Everything between the loads and the stores stays in registers:
//   pull       n_i(r) = n*_i(r - c_i)                       Eq. (LBE)
//              (link bounce-back at solid z-planes,          Sec. 4.1 Eq. (MBB), u_b = 0)
//   moments    m_k = sum_i e_ki n_i                          Sec. 3.4 Eq. (forward), Table 1
//   velocity   j = m_1..3 + f/2, u = j / rho                 Sec. 3.7 Eq. (special_choice_momentum_density)
//   relax      m*_k = m^eq_k + gamma_k (m_k - m^eq_k) + F_k  Eq. (lco_update); Sec. 3.7 Sigma
//   noise      + sqrt(mu rho w_k) (1 - gamma_k^2)^1/2 r_k    Eqs. (stochupdaterule1), (detailedbalance1)
//   back       n*_i = a_i sum_k e_ki m*_k / w_k              Eq. (back_transformation), q = a
//   store      deviation n*_i - a_i rho0 (scaled for FP16 / BF16)
#pragma once

#include "d3q19.cuh"
#include "f32x2.cuh"
#include "lbf_internal.h"

namespace lbi {

constexpr int kBX = 128;  // threads per block along x


// Collision of one node (Sec. 3.4, 3.5, 3.7) from its pulled populations n
// (deviations n_i - a_i rho0) and the force density (fx, fy, fz) to the
// post-collision deviations out.  Physics constants come from a; the noise
// stream is Philox with round keys rk and counter (node, a.step, b, replica).
template <bool NOISE>
__device__ __forceinline__ void collide_moments(const float m[19], float fx, float fy, float fz, const StepArgs &a,
                                                const lbd::RoundKeys &rk, uint32_t node, uint32_t replica,
                                                float out[19])
{
    const float rho = a.rho0 + m[0];
    const float inv_rho = 1.0f / rho;
    const float ux = (m[1] + 0.5f * fx) * inv_rho;
    const float uy = (m[2] + 0.5f * fy) * inv_rho;
    const float uz = (m[3] + 0.5f * fz) * inv_rho;

    // ---- relaxation in moment space ----------------------------------------
    const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const float u2 = uxx + uyy + uzz;
    const float meq4 = rho * u2;
    const float meq5 = rho * (3.0f * uxx - u2);
    const float meq6 = rho * (uyy - uzz);
    const float meq7 = rho * ux * uy;
    const float meq8 = rho * uy * uz;
    const float meq9 = rho * uz * ux;
    // forcing moments of Delta'' (Sigma of Eq. (moment_two_external_force))
    const float uf = ux * fx + uy * fy + uz * fz;
    const float gs1 = 1.0f + a.g_shear;
    const float F4 = (1.0f + a.g_bulk) * uf;
    const float F5 = gs1 * (3.0f * ux * fx - uf);
    const float F6 = gs1 * (uy * fy - uz * fz);
    const float F7 = 0.5f * gs1 * (ux * fy + uy * fx);
    const float F8 = 0.5f * gs1 * (uy * fz + uz * fy);
    const float F9 = 0.5f * gs1 * (uz * fx + ux * fz);

    float M[19];  // post-collision moments divided by w_k
    M[0] = m[0];
    M[1] = 3.0f * (m[1] + fx);
    M[2] = 3.0f * (m[2] + fy);
    M[3] = 3.0f * (m[3] + fz);
    M[4] = lbd::inv_w(4) * (meq4 + a.g_bulk * (m[4] - meq4) + F4);
    M[5] = lbd::inv_w(5) * (meq5 + a.g_shear * (m[5] - meq5) + F5);
    M[6] = lbd::inv_w(6) * (meq6 + a.g_shear * (m[6] - meq6) + F6);
    M[7] = lbd::inv_w(7) * (meq7 + a.g_shear * (m[7] - meq7) + F7);
    M[8] = lbd::inv_w(8) * (meq8 + a.g_shear * (m[8] - meq8) + F8);
    M[9] = lbd::inv_w(9) * (meq9 + a.g_shear * (m[9] - meq9) + F9);
#pragma unroll
    for (int k = 10; k < 16; ++k) M[k] = lbd::inv_w(k) * (a.g_odd * m[k]);
#pragma unroll
    for (int k = 16; k < 19; ++k) M[k] = lbd::inv_w(k) * (a.g_even * m[k]);

    if (NOISE) {
        // sqrt(mu rho w_k) phi_k r_k, divided by w_k: (phi_k / sqrt(w_k)) times a
        // Gaussian of variance mu rho (the factor rides in the Box-Muller radius)
        float g[16];
        lbd::gaussians16(rk, node, a.step, 0u, replica, a.mu * (a.noise_rho0 ? a.rho0 : rho), g);
#pragma unroll
        for (int k = 4; k < 19; ++k) M[k] = fmaf(a.amp[k - 4], g[k - 4], M[k]);
    }

    lbd::backward(M, out);
}

// The same from the pulled populations n (deviations n_i - a_i rho0).
template <bool NOISE>
__device__ __forceinline__ void collide_node(const float n[19], float fx, float fy, float fz, const StepArgs &a,
                                             const lbd::RoundKeys &rk, uint32_t node, uint32_t replica,
                                             float out[19])
{
    float m[19];
    lbd::forward(n, m);
    collide_moments<NOISE>(m, fx, fy, fz, a, rk, node, replica, out);
}

// One step of a butterfly reduce-scatter over the warp: each lane keeps one
// half of its N values (the upper half if `hi`), receives the other lane's
// copy of that half and adds it, so the lanes now hold disjoint halves.
template <int N>
__device__ __forceinline__ void butterfly_half(const float *in, float *out, int offset, bool hi)
{
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const float keep = hi ? in[i + N / 2] : in[i];
        const float send = hi ? in[i] : in[i + N / 2];
        out[i] = keep + __shfl_xor_sync(0xffffffffu, send, offset);
    }
}

// Moment sums of a warp: lane l holds 38 values (m0_k + m1_k, then
// m0_k^2 + m1_k^2; zeros where valid is false), the warp needs their 38 sums.
// Five butterfly steps halve the values per lane (40 -> 20 -> 10 -> 5, padded
// to 6 -> 3, padded to 4 -> 2), each sum is formed in a fixed order, and the
// lane that ends with sum k writes it to part[warp][k].  After a
// __syncthreads the block's sums are part[0] + ... + part[kBX/32 - 1]
// (block_moment_sums_out).  Every lane of the warp calls it.
__device__ __forceinline__ void warp_moment_sums(const float m0[19], const float m1[19], bool valid,
                                                 float (*part)[38])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float a[40];
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        a[k] = m0[k] + m1[k];
        a[19 + k] = fmaf(m0[k], m0[k], m1[k] * m1[k]);
    }
    a[38] = a[39] = 0.0f;
    if (!__all_sync(0xffffffffu, valid)) {  // a warp at the end of a row
#pragma unroll
        for (int k = 0; k < 38; ++k) a[k] = valid ? a[k] : 0.0f;
    }
    float b[20], c[10], d[6], e[4], f[2];
    butterfly_half<40>(a, b, 16, lane & 16);
    butterfly_half<20>(b, c, 8, lane & 8);
    butterfly_half<10>(c, d, 4, lane & 4);
    d[5] = 0.0f;
    butterfly_half<6>(d, e, 2, lane & 2);
    e[3] = 0.0f;
    butterfly_half<4>(e, f, 1, lane & 1);
    // lane l holds, for j = 0, 1, the sum of entry k = base + b1 3 + pos of
    // the 5-entry block base = 20 b4 + 10 b3 + 5 b2, pos = 2 b0 + j (b_i the
    // bits of l); pos 3 and block entries 5 and beyond are padding
    const int base = 20 * ((lane >> 4) & 1) + 10 * ((lane >> 3) & 1) + 5 * ((lane >> 2) & 1);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int pos = 2 * (lane & 1) + j;
        const int idx = 3 * ((lane >> 1) & 1) + pos;
        const int k = base + idx;
        if (pos < 3 && idx < 5 && k < 38) part[warp][k] = f[j];
    }
}

// FP32 throughout: FP64 arithmetic is slow on this part, and a block that
// ends in a chain of FP64 adds holds its SM slot meanwhile.
__device__ __forceinline__ void block_moment_sums_out(const float (*part)[38], float *out)
{
    __syncthreads();
    if (threadIdx.x < 38) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < kBX / 32; ++w) t += part[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// The whole update of fluid node (x, y, z): pull, force, collision, store.
// SUMS: the warp's moment sums go to part (see warp_moment_sums); every
// lane calls, lanes without a node (valid false) add zeros.
template <int DT, bool NOISE, bool FIELD, bool WALLS, bool SUMS = false>
__device__ __forceinline__ void update_node(const typename lbd::Store<DT>::T *__restrict__ src,
                                            typename lbd::Store<DT>::T *__restrict__ dst,
                                            const float *__restrict__ ffield, const float *__restrict__ facc,
                                            const StepArgs &a, int x, int y, int z, bool valid = true,
                                            float (*part)[38] = nullptr)
{
    using S = lbd::Store<DT>;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    int zm, zp;
    if (WALLS) {
        zm = z - 1;
        zp = z + 1;
    } else {
        zm = (z == 0) ? nz - 1 : z - 1;
        zp = (z == nz - 1) ? 0 : z + 1;
    }
    const size_t P = a.pitch;
    const uint32_t self = (uint32_t)((z * ny + y) * nx + x);

    // ---- pull streaming --------------------------------------------------
    float n[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        bool bounce = false;
        if (WALLS && lbd::cz(i) != 0) bounce = (sz == 0) || (sz == nz - 1);
        const size_t k = bounce ? (size_t)lbd::opposite(i) * P + self
                                : (size_t)i * P + (uint32_t)((sz * ny + sy) * nx + sx);
        n[i] = in_bounds(k, 19 * P, a.err) ? S::load(src + k, a.inv_scale) : 0.0f;
    }

    // ---- force and collision -----------------------------------------------
    float fx = a.fx, fy = a.fy, fz = a.fz;
    if (FIELD) {
        if (ffield) {  // caller's field, component stride N
            fx += __ldg(ffield + self);
            fy += __ldg(ffield + a.nn + self);
            fz += __ldg(ffield + 2 * a.nn + self);
        }
        if (facc) {  // library accumulator, component stride = plane pitch
            fx += __ldg(facc + self);
            fy += __ldg(facc + P + self);
            fz += __ldg(facc + 2 * P + self);
        }
    }
    float m[19], out[19];
    lbd::forward(n, m);
    if (SUMS) {
        float none[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) none[k] = 0.0f;
        warp_moment_sums(m, none, valid, part);
    }
    if (!valid) return;
    collide_moments<NOISE>(m, fx, fy, fz, a, a.rk, self, a.replica, out);
#pragma unroll
    for (int i = 0; i < 19; ++i)
        if (in_bounds((size_t)i * P + self, 19 * P, a.err)) dst[(size_t)i * P + self] = S::pack(out[i], a.scale);
}

__device__ __forceinline__ size_t block_linear()
{
    return blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
}

// SUMS: the block also writes the moment sums of its nodes (pre-collision,
// as lb_moments defines them) to partials[block][38].
template <int DT, bool NOISE, bool FIELD, bool WALLS, bool SUMS>
__global__ void __launch_bounds__(kBX) k_stream_collide(const typename lbd::Store<DT>::T *__restrict__ src,
                                                        typename lbd::Store<DT>::T *__restrict__ dst,
                                                        const float *__restrict__ ffield,
                                                        const float *__restrict__ facc, const StepArgs a,
                                                        float *partials)
{
    const int x = blockIdx.x * kBX + threadIdx.x;
    if (SUMS) {
        __shared__ float part[kBX / 32][38];
        const bool valid = x < a.nx;  // lanes past the row load node 0 of it and store nothing
        update_node<DT, NOISE, FIELD, WALLS, true>(src, dst, ffield, facc, a, valid ? x : 0, blockIdx.y,
                                                   blockIdx.z + a.z0, valid, part);
        block_moment_sums_out(part, partials + 38 * block_linear());
    } else {
        if (x >= a.nx) return;
        update_node<DT, NOISE, FIELD, WALLS>(src, dst, ffield, facc, a, x, blockIdx.y, blockIdx.z + a.z0);
    }
}

// Node k (0 .. span^3 - 1, x fastest) of the block of nodes that an impulse
// stencil can touch around the recorded cell (bx, by, bz): [b, b + 1] per
// axis for span 2 (phi_2), [b - 1, b + 2] for span 4 (phi_3 and phi_4).
// Returns false for a node outside the fluid.
template <bool WALLS>
__device__ __forceinline__ bool patch_node(int bx, int by, int bz, int k, int span, const StepArgs &a, int &x,
                                           int &y, int &z)
{
    if (span == 3) {  // a phi_3 stencil origin: the 27 nodes of the stencil
        x = bx + k % 3;
        y = by + (k / 3) % 3;
        z = bz + k / 9;
    } else {  // a cell: its corners (span 2) or one node further on each side (span 4)
        const int sh = span == 4 ? 2 : 1, lo = span == 4 ? -1 : 0, m = span - 1;
        x = bx + lo + (k & m);
        y = by + lo + ((k >> sh) & m);
        z = bz + lo + (k >> (2 * sh));
    }
    x = x < 0 ? x + a.nx : (x >= a.nx ? x - a.nx : x);
    y = y < 0 ? y + a.ny : (y >= a.ny ? y - a.ny : y);
    if ((unsigned)x >= (unsigned)a.nx) x = ((x % a.nx) + a.nx) % a.nx;  // boxes narrower than the stencil
    if ((unsigned)y >= (unsigned)a.ny) y = ((y % a.ny) + a.ny) % a.ny;
    if (!WALLS) {
        z = z < 0 ? z + a.nz : (z >= a.nz ? z - a.nz : z);
        if ((unsigned)z >= (unsigned)a.nz) z = ((z % a.nz) + a.nz) % a.nz;
    }
    return z >= a.z0 && z < a.z1;
}

// Re-update of the nodes that received particle impulses, after an update of
// all nodes that left the impulses out (the coupling ran meanwhile): the
// span^3 nodes of each record of particle p, records[s][p] (the linear index
// of its cell at sub-step s, or of its phi_3 stencil origin: span 3), are
// updated again from the same pre-step state
// with the impulses added.  The update of a node depends only on that state, the
// forces at the node and the counter-based noise, so the result is the one a
// single update with the impulses would give.  Thread (p, q) walks p's
// distinct cells and takes nodes q, q + 8, ... of each; a node shared by several
// particles is updated once, by the thread that raises its tag to `tag`
// first (tags grow by one per patch, so the array is never cleared).
template <int DT, bool NOISE, bool WALLS>
__global__ void __launch_bounds__(kBX) k_patch_impulse_nodes(const typename lbd::Store<DT>::T *__restrict__ src,
                                                             typename lbd::Store<DT>::T *__restrict__ dst,
                                                             const float *__restrict__ ffield,
                                                             float *__restrict__ facc, const int *records,
                                                             int n, int nsub, int span, unsigned int *claim,
                                                             unsigned int tag, const StepArgs a)
{
    const int t = blockIdx.x * kBX + threadIdx.x;
    if (t >= n * 8) return;
    const int p = t >> 3, q = t & 7;
    const int nk = span * span * span;
    int prev = -1;
    for (int s = 0; s < nsub; ++s) {
        const int base = records[(size_t)s * n + p];
        if (base == prev) continue;  // same cell as the sub-step before
        prev = base;
        const int bx = base % a.nx, by = (base / a.nx) % a.ny, bz = base / (a.nx * a.ny);
        for (int e = q; e < nk; e += 8) {
            int x, y, z;
            if (!patch_node<WALLS>(bx, by, bz, e, span, a, x, y, z)) continue;  // solid node
            const size_t node = ((size_t)z * a.ny + y) * a.nx + x;
            if (atomicMax(claim + node, tag) == tag) continue;  // another thread has it
            update_node<DT, NOISE, true, WALLS>(src, dst, ffield, facc, a, x, y, z);
            // the impulses are applied: clear them for the next coupling call
            facc[node] = 0.0f;
            facc[a.pitch + node] = 0.0f;
            facc[2 * a.pitch + node] = 0.0f;
        }
    }
}

// The same for FP32 storage, by a correction of the stored result instead of
// a second update: the forces enter the collision only through u and the
// force moments of modes 1..9, and rho and the pre-collision j are
// recovered from the stored n* (mass is conserved, the stored momentum is
// j + f).  With f_b the force of the first update and f_n = f_b + the
// impulse, the stored moments change by dM_1..3 = 3 (f_n - f_b) and, for
// k = 4..9, dM_k = ((1 - gamma_k) (m^eq_k(u_n) - m^eq_k(u_b)) + F_k(u_n, f_n)
// - F_k(u_b, f_b)) / w_k; n* += backward(dM).  No pull and no noise; the
// claim makes sure each node is corrected once.  Eight blocks per SM (64 registers, no
// spills): the launch for the workload's ~1.3e5 threads fits in one wave.
template <bool WALLS>
__global__ void __launch_bounds__(kBX, 8) k_patch_impulse_nodes_f32(float *__restrict__ dst, const float *__restrict__ ffield,
                                                                 float *__restrict__ facc, const int *records, int n,
                                                                 int nsub, int span, unsigned int *claim,
                                                                 unsigned int tag, const StepArgs a)
{
    const int t = blockIdx.x * kBX + threadIdx.x;
    if (t >= n * 8) return;
    const int p = t >> 3, q = t & 7;
    const size_t P = a.pitch;
    const int nk = span * span * span;
    int prev = -1;
    for (int s = 0; s < nsub; ++s) {
        const int base = records[(size_t)s * n + p];
        if (base == prev) continue;  // same cell as the sub-step before
        prev = base;
        const int bx = base % a.nx, by = (base / a.nx) % a.ny, bz = base / (a.nx * a.ny);
        for (int e = q; e < nk; e += 8) {
            int x, y, z;
            if (!patch_node<WALLS>(bx, by, bz, e, span, a, x, y, z)) continue;  // solid node
            const size_t node = ((size_t)z * a.ny + y) * a.nx + x;
            // the claim, the impulse and the stored values are requested
            // together (one memory round trip instead of three); the values
            // are used only by the thread that wins the claim, and nothing
            // else writes this node during the kernel
            const unsigned int had = atomicMax(claim + node, tag);
            const float df[3] = {facc[node], facc[P + node], facc[2 * P + node]};
            float ns[19], m[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) ns[i] = dst[(size_t)i * P + node];
            if (had == tag) continue;  // another thread has it
            if (df[0] == 0.0f && df[1] == 0.0f && df[2] == 0.0f) continue;
            lbd::forward(ns, m);
            float fb[3] = {a.fx, a.fy, a.fz};
            if (ffield) {
                fb[0] += ffield[node];
                fb[1] += ffield[a.nn + node];
                fb[2] += ffield[2 * a.nn + node];
            }
            const float fn[3] = {fb[0] + df[0], fb[1] + df[1], fb[2] + df[2]};
            const float rho = a.rho0 + m[0];
            const float ir = 1.0f / rho;
            const float j[3] = {m[1] - fb[0], m[2] - fb[1], m[3] - fb[2]};
            float dM[19];
#pragma unroll
            for (int k = 0; k < 19; ++k) dM[k] = 0.0f;
            dM[1] = 3.0f * df[0];
            dM[2] = 3.0f * df[1];
            dM[3] = 3.0f * df[2];
            const float gs1 = 1.0f + a.g_shear;
#pragma unroll
            for (int side = 0; side < 2; ++side) {  // + (u_n, f_n), - (u_b, f_b)
                const float *f = side ? fb : fn;
                const float sg = side ? -1.0f : 1.0f;
                const float ux = (j[0] + 0.5f * f[0]) * ir, uy = (j[1] + 0.5f * f[1]) * ir, uz = (j[2] + 0.5f * f[2]) * ir;
                const float uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, u2 = uxx + uyy + uzz;
                const float uf = ux * f[0] + uy * f[1] + uz * f[2];
                dM[4] += sg * ((1.0f - a.g_bulk) * rho * u2 + (1.0f + a.g_bulk) * uf);
                dM[5] += sg * ((1.0f - a.g_shear) * rho * (3.0f * uxx - u2) + gs1 * (3.0f * ux * f[0] - uf));
                dM[6] += sg * ((1.0f - a.g_shear) * rho * (uyy - uzz) + gs1 * (uy * f[1] - uz * f[2]));
                dM[7] += sg * ((1.0f - a.g_shear) * rho * ux * uy + 0.5f * gs1 * (ux * f[1] + uy * f[0]));
                dM[8] += sg * ((1.0f - a.g_shear) * rho * uy * uz + 0.5f * gs1 * (uy * f[2] + uz * f[1]));
                dM[9] += sg * ((1.0f - a.g_shear) * rho * uz * ux + 0.5f * gs1 * (uz * f[0] + ux * f[2]));
            }
#pragma unroll
            for (int k = 4; k < 10; ++k) dM[k] *= lbd::inv_w(k);
            float dn[19];
            lbd::backward(dM, dn);
#pragma unroll
            for (int i = 0; i < 19; ++i) dst[(size_t)i * P + node] = ns[i] + dn[i];
            // the impulses are applied: clear them for the next coupling call
            facc[node] = 0.0f;
            facc[P + node] = 0.0f;
            facc[2 * P + node] = 0.0f;
        }
    }
}

// Two neighbouring nodes x0 = 2t, x0 + 1 per thread (even nx).  Both pull
// their populations from the same rows of each plane, so one address per
// plane serves both (the second is an immediate offset); planes with c_x = 0
// and all stores move the pair as one 8-byte (FP32) or 4-byte (FP16 / BF16)
// access.  Collision and noise are those of collide_node, computed for the
// two nodes at once in packed FP32 (f32x2.cuh).
template <int DT>
struct Pair;
template <>
struct Pair<0> {
    static __device__ __forceinline__ void load(const float *p, float inv, float &a, float &b)
    {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void store(float *p, float a, float b, float)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
};
template <>
struct Pair<1> {
    static __device__ __forceinline__ void load(const __half *p, float inv, float &a, float &b)
    {
        const __half2 v = __ldg(reinterpret_cast<const __half2 *>(p));
        a = __low2float(v) * inv;
        b = __high2float(v) * inv;
    }
    static __device__ __forceinline__ void store(__half *p, float a, float b, float sc)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a * sc, b * sc);
    }
};
template <>
struct Pair<2> {
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float inv, float &a, float &b)
    {
        const __nv_bfloat162 v = __ldg(reinterpret_cast<const __nv_bfloat162 *>(p));
        a = __low2float(v) * inv;
        b = __high2float(v) * inv;
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float a, float b, float sc)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a * sc, b * sc);
    }
};

// Pull streaming of nodes x0, x0 + 1 of row (y, z) (link bounce-back at solid
// z-planes) into packed pairs n (node x0 in the low halves, FP16 / BF16
// unscaled), and their force densities f0, f1 (body force + caller's field +
// library accumulator).
template <int DT, bool FIELD, bool WALLS>
__device__ __forceinline__ void load_pair(const typename lbd::Store<DT>::T *__restrict__ src,
                                          const float *__restrict__ ffield, const float *__restrict__ facc,
                                          const StepArgs &a, int x0, int y, int z, lbp::F2 n[19], float f0[3],
                                          float f1[3])
{
    using S = lbd::Store<DT>;
    using PR = Pair<DT>;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xm = (x0 == 0) ? nx - 1 : x0 - 1;       // source of node x0 for c_x = +1
    const int xp = (x0 + 2 == nx) ? 0 : x0 + 2;       // source of node x0 + 1 for c_x = -1
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    int zm, zp;
    if (WALLS) {
        zm = z - 1;
        zp = z + 1;
    } else {
        zm = (z == 0) ? nz - 1 : z - 1;
        zp = (z == nz - 1) ? 0 : z + 1;
    }
    const uint32_t P = (uint32_t)a.pitch;
    const uint32_t self = (uint32_t)((z * ny + y) * nx + x0);
    const size_t lim = 19 * (size_t)P;  // elements of a population buffer (index checks)
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        bool bounce = false;
        if (WALLS && lbd::cz(i) != 0) bounce = (sz == 0) || (sz == nz - 1);
        // stored values as loaded (FP16 / BF16: still scaled; the pair is
        // unscaled below by one packed multiply)
        float v0 = 0.0f, v1 = 0.0f;
        if (bounce) {
            const uint32_t k = (uint32_t)lbd::opposite(i) * P + self;
            if (in_bounds(k + 1, lim, a.err)) PR::load(src + k, 1.0f, v0, v1);
        } else {
            const uint32_t row = (uint32_t)i * P + (uint32_t)((sz * ny + sy) * nx);
            if (lbd::cx(i) == 0) {
                if (in_bounds(row + x0 + 1, lim, a.err)) PR::load(src + row + x0, 1.0f, v0, v1);
            } else if (lbd::cx(i) == 1) {
                if (in_bounds(row + xm, lim, a.err) && in_bounds(row + x0, lim, a.err)) {
                    v0 = S::load(src + row + xm, 1.0f);
                    v1 = S::load(src + row + x0, 1.0f);
                }
            } else {
                if (in_bounds(row + x0 + 1, lim, a.err) && in_bounds(row + xp, lim, a.err)) {
                    v0 = S::load(src + row + x0 + 1, 1.0f);
                    v1 = S::load(src + row + xp, 1.0f);
                }
            }
        }
        n[i] = DT == 0 ? lbp::f2(v0, v1) : lbp::f2(v0, v1) * lbp::f2s(a.inv_scale);
    }

    f0[0] = f1[0] = a.fx;
    f0[1] = f1[1] = a.fy;
    f0[2] = f1[2] = a.fz;
    if (FIELD) {
        if (ffield) {  // caller's field, component stride N
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                f0[d] += __ldg(ffield + d * a.nn + self);
                f1[d] += __ldg(ffield + d * a.nn + self + 1);
            }
        }
        if (facc) {  // library accumulator, component stride = plane pitch
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float u, v;
                Pair<0>::load(facc + d * (size_t)P + self, 1.0f, u, v);
                f0[d] += u;
                f1[d] += v;
            }
        }
    }
}

// Store of the packed post-collision pair (FP16 / BF16: scaled by one packed
// multiply, then rounded to nearest even).
template <int DT>
__device__ __forceinline__ void store_pair(typename lbd::Store<DT>::T *__restrict__ dst, const StepArgs &a,
                                           uint32_t self, const lbp::F2 out[19])
{
    const uint32_t P = (uint32_t)a.pitch;
    const size_t lim = 19 * (size_t)P;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float o0, o1;
        lbp::split(DT == 0 ? out[i] : out[i] * lbp::f2s(a.scale), o0, o1);
        if (in_bounds((uint32_t)i * P + self + 1, lim, a.err)) Pair<DT>::store(dst + (uint32_t)i * P + self, o0, o1, 1.0f);
    }
}

template <int DT, bool NOISE, bool FIELD, bool WALLS, bool SUMS = false>
__device__ __forceinline__ void update_pair(const typename lbd::Store<DT>::T *__restrict__ src,
                                            typename lbd::Store<DT>::T *__restrict__ dst,
                                            const float *__restrict__ ffield, const float *__restrict__ facc,
                                            const StepArgs &a, int x0, int y, int z, bool valid = true,
                                            float (*part)[38] = nullptr)
{
    const uint32_t self = (uint32_t)((z * a.ny + y) * a.nx + x0);
    lbp::F2 n[19];
    float f0[3], f1[3];
    load_pair<DT, FIELD, WALLS>(src, ffield, facc, a, x0, y, z, n, f0, f1);
    // both nodes' moments, collision, noise and back transform in packed
    // FP32 (f32x2.cuh), node x0 in the low halves
    lbp::F2 m[19], out[19];
    lbp::forward2(n, m);
    if (SUMS) {  // both nodes' moments summed before the collisions
        float m0[19], m1[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) lbp::split(m[k], m0[k], m1[k]);
        warp_moment_sums(m0, m1, valid, part);
        if (!valid) return;
    }
    lbp::collide_moments2<NOISE>(m, lbp::f2(f0[0], f1[0]), lbp::f2(f0[1], f1[1]), lbp::f2(f0[2], f1[2]), a, a.rk,
                                 self, a.replica, out);
    store_pair<DT>(dst, a, self, out);
}

template <int DT, bool NOISE, bool FIELD, bool WALLS, bool SUMS>
__global__ void __launch_bounds__(kBX) k_stream_collide2(const typename lbd::Store<DT>::T *__restrict__ src,
                                                         typename lbd::Store<DT>::T *__restrict__ dst,
                                                         const float *__restrict__ ffield,
                                                         const float *__restrict__ facc, const StepArgs a,
                                                         float *partials)
{
    const int x0 = 2 * (blockIdx.x * kBX + threadIdx.x);
    if (SUMS) {
        __shared__ float part[kBX / 32][38];
        const bool valid = x0 < a.nx;  // lanes past the row load nodes 0, 1 of it and store nothing
        update_pair<DT, NOISE, FIELD, WALLS, true>(src, dst, ffield, facc, a, valid ? x0 : 0, blockIdx.y,
                                                   blockIdx.z + a.z0, valid, part);
        block_moment_sums_out(part, partials + 38 * block_linear());
    } else {
        if (x0 >= a.nx) return;
        update_pair<DT, NOISE, FIELD, WALLS>(src, dst, ffield, facc, a, x0, blockIdx.y, blockIdx.z + a.z0);
    }
}

// Launch geometry of the stream-collide kernels: two nodes per thread when
// rows pair up and element indices fit 32 bits.
inline bool sc_paired(const lb_handle *h)
{
    return (h->p.nx % 2 == 0) && (19.0 * (double)h->pitch < 4294967296.0);
}

inline dim3 sc_grid(const lb_handle *h)
{
    const int nzf = h->p.walls ? h->p.nz - 2 : h->p.nz;
    const int nxt = sc_paired(h) ? h->p.nx / 2 : h->p.nx;
    return dim3((nxt + kBX - 1) / kBX, h->p.ny, nzf);
}

// partials != NULL: the launch also writes per-block moment sums
// (partials[block][38], block = blockIdx.x + gridDim.x (blockIdx.y + gridDim.y blockIdx.z)).
template <int DT>
cudaError_t launch_stream_collide_dt(const lb_handle *h, const void *src, void *dst, const float *facc,
                                     float *partials)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    const dim3 grid = sc_grid(h);
    const dim3 block(kBX);
    const bool noise = a.kT > 0.0f;
    const bool field = (h->force != nullptr) || (facc != nullptr);
    const bool walls = h->p.walls != 0;
    const bool paired = sc_paired(h);
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
#define LBI_SC(NZ, FL, WL)                                                                                        \
    do {                                                                                                          \
        if (partials) {                                                                                           \
            if (paired)                                                                                           \
                k_stream_collide2<DT, NZ, FL, WL, true><<<grid, block, 0, h->stream>>>(s, d, h->force, facc, a,   \
                                                                                        partials);               \
            else                                                                                                  \
                k_stream_collide<DT, NZ, FL, WL, true><<<grid, block, 0, h->stream>>>(s, d, h->force, facc, a,    \
                                                                                       partials);                \
        } else {                                                                                                  \
            if (paired)                                                                                           \
                k_stream_collide2<DT, NZ, FL, WL, false><<<grid, block, 0, h->stream>>>(s, d, h->force, facc, a,  \
                                                                                         nullptr);               \
            else                                                                                                  \
                k_stream_collide<DT, NZ, FL, WL, false><<<grid, block, 0, h->stream>>>(s, d, h->force, facc, a,   \
                                                                                        nullptr);                \
        }                                                                                                         \
    } while (0)
    if (noise) {
        if (field) {
            if (walls) LBI_SC(true, true, true); else LBI_SC(true, true, false);
        } else {
            if (walls) LBI_SC(true, false, true); else LBI_SC(true, false, false);
        }
    } else {
        if (field) {
            if (walls) LBI_SC(false, true, true); else LBI_SC(false, true, false);
        } else {
            if (walls) LBI_SC(false, false, true); else LBI_SC(false, false, false);
        }
    }
#undef LBI_SC
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_patch_dt(const lb_handle *h, const void *src, void *dst, float *facc, const int *records,
                            int n, int nsub, int span, unsigned int *claim, unsigned int tag)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    if (n <= 0 || nsub <= 0) return cudaSuccess;
    const unsigned int blocks = (unsigned int)(((size_t)n * 8 + kBX - 1) / kBX);
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
    const bool noise = a.kT > 0.0f, walls = h->p.walls != 0;
    if (DT == 0) {  // FP32: correct the stored result in place
        float *d32 = reinterpret_cast<float *>(dst);
        if (walls)
            k_patch_impulse_nodes_f32<true><<<blocks, kBX, 0, h->stream>>>(d32, h->force, facc, records, n, nsub, span,
                                                                          claim, tag, a);
        else
            k_patch_impulse_nodes_f32<false><<<blocks, kBX, 0, h->stream>>>(d32, h->force, facc, records, n, nsub,
                                                                           span, claim, tag, a);
        return cudaGetLastError();
    }
#define LBI_PATCH(NZ, WL) \
    k_patch_impulse_nodes<DT, NZ, WL><<<blocks, kBX, 0, h->stream>>>(s, d, h->force, facc, records, n, nsub, span, claim, \
                                                     tag, a)
    if (noise) {
        if (walls) LBI_PATCH(true, true); else LBI_PATCH(true, false);
    } else {
        if (walls) LBI_PATCH(false, true); else LBI_PATCH(false, false);
    }
#undef LBI_PATCH
    return cudaGetLastError();
}

}  // namespace lbi
