// exp_eq.cu -- the stream-collide update with the exponential equilibrium of
// Sec. 3.6, Eq. (equildist_lagrange): the populations that maximise the
// entropy of Eq. (boltzmann_entropy_function) at given mass and momentum,
// n^eq_i = rho a_i exp(lambda.c_i) / Z, Z = sum_i a_i exp(lambda.c_i), with
// lambda the root of sum_i a_i c_i exp(lambda.c_i) / Z = u.  The standard
// equilibrium of Eq. (original_equil_distrib) is its expansion to O(u^2);
// this one also has parts on the kinetic modes (O(u^3)), which the
// relaxation keeps.  Everything else is the collision of
// stream_collide.cuh: the same moments, eigenvalues, forcing and noise.
// Rows of even length take two nodes per thread with the arithmetic in packed
// FP32 (f32x2.cuh), as the quadratic update does.
//
// lambda comes from two Newton steps in FP32 from the first-order value
// lambda = 3u (the Jacobian is the covariance of c under the weights); the
// start is off by O(u^2) relative and each step squares that, so two steps
// reach FP32 rounding for |u| up to ~0.15.  With
// x_i = exp(lambda.c_i) - 1 and s = sum_i a_i x_i the deviation from the
// reference state is n^eq_i - a_i rho0 = a_i (delta rho + rho (x_i - s) /
// (1 + s)): no difference of nearly equal numbers.
#include "stream_collide.cuh"

namespace lbi {

namespace {

// x_i = exp(lambda.c_i) - 1 for the 18 moving directions from three
// expm1 values: with e_d = exp(+-lambda_d) - 1 (exp(-a) - 1 = -x / (1 + x)
// for x = exp(a) - 1) and (1 + x)(1 + e) - 1 = x + e + x e over the (one or
// two) non-zero components of c_i.
__device__ __forceinline__ void exp_dirs(const float l[3], float x[19])
{
    float ep[3], em[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ep[d] = expm1f(l[d]);
        em[d] = -ep[d] / (1.0f + ep[d]);
    }
    x[0] = 0.0f;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int c3[3] = {lbd::cx(i), lbd::cy(i), lbd::cz(i)};
        float xi = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (c3[d] != 0) {
                const float e = c3[d] > 0 ? ep[d] : em[d];
                xi = xi + e + xi * e;
            }
        x[i] = xi;
    }
}

// Deviation moments meq[k] of n^eq - a rho0 (Table 1 transform).
__device__ __forceinline__ void exp_eq_moments(float drho, float rho, float ux, float uy, float uz, float meq[19])
{
    float l[3] = {3.0f * ux, 3.0f * uy, 3.0f * uz};
    const float u[3] = {ux, uy, uz};
    float x[19];
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        float s = 0.0f, m[3] = {0.f, 0.f, 0.f}, C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        exp_dirs(l, x);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const float cx = lbd::cx(i), cy = lbd::cy(i), cz = lbd::cz(i);
            const float xi = x[i];
            const float w = lbd::weight(i) * xi;
            s += w;
            m[0] += w * cx;
            m[1] += w * cy;
            m[2] += w * cz;
            C[0] += w * cx * cx;
            C[1] += w * cy * cy;
            C[2] += w * cz * cz;
            C[3] += w * cx * cy;
            C[4] += w * cy * cz;
            C[5] += w * cz * cx;
        }
        const float iz = 1.0f / (1.0f + s);
        for (int d = 0; d < 3; ++d) m[d] *= iz;
        // covariance (1/3 I + sum a c c x) / Z - m m^T
        const float axx = (1.0f / 3.0f + C[0]) * iz - m[0] * m[0], ayy = (1.0f / 3.0f + C[1]) * iz - m[1] * m[1];
        const float azz = (1.0f / 3.0f + C[2]) * iz - m[2] * m[2], axy = C[3] * iz - m[0] * m[1];
        const float ayz = C[4] * iz - m[1] * m[2], azx = C[5] * iz - m[2] * m[0];
        const float r[3] = {u[0] - m[0], u[1] - m[1], u[2] - m[2]};
        // Cramer's rule on the symmetric 3x3 system
        const float c00 = ayy * azz - ayz * ayz, c01 = azx * ayz - axy * azz, c02 = axy * ayz - azx * ayy;
        const float det = axx * c00 + axy * c01 + azx * c02;
        const float c11 = axx * azz - azx * azx, c12 = axy * azx - axx * ayz, c22 = axx * ayy - axy * axy;
        const float id = 1.0f / det;
        l[0] += id * (c00 * r[0] + c01 * r[1] + c02 * r[2]);
        l[1] += id * (c01 * r[0] + c11 * r[1] + c12 * r[2]);
        l[2] += id * (c02 * r[0] + c12 * r[1] + c22 * r[2]);
    }
    float s = 0.0f;
    exp_dirs(l, x);
#pragma unroll
    for (int i = 1; i < 19; ++i) s += lbd::weight(i) * x[i];
    const float g = rho / (1.0f + s);
    float d[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) d[i] = lbd::weight(i) * (drho + g * (x[i] - s));
    lbd::forward(d, meq);
}

// The collision of collide_moments() with the moments of the exponential
// equilibrium in place of the quadratic ones (all non-conserved modes).
template <bool NOISE>
__device__ __forceinline__ void collide_exp(const float m[19], float fx, float fy, float fz, const StepArgs &a,
                                            uint32_t node, float out[19])
{
    const float rho = a.rho0 + m[0];
    const float inv_rho = 1.0f / rho;
    const float ux = (m[1] + 0.5f * fx) * inv_rho;
    const float uy = (m[2] + 0.5f * fy) * inv_rho;
    const float uz = (m[3] + 0.5f * fz) * inv_rho;
    float meq[19];
    exp_eq_moments(m[0], rho, ux, uy, uz, meq);
    const float uf = ux * fx + uy * fy + uz * fz;
    const float gs1 = 1.0f + a.g_shear;
    const float F[6] = {(1.0f + a.g_bulk) * uf,           gs1 * (3.0f * ux * fx - uf),
                        gs1 * (uy * fy - uz * fz),          0.5f * gs1 * (ux * fy + uy * fx),
                        0.5f * gs1 * (uy * fz + uz * fy),   0.5f * gs1 * (uz * fx + ux * fz)};
    float M[19];
    M[0] = m[0];
    M[1] = 3.0f * (m[1] + fx);
    M[2] = 3.0f * (m[2] + fy);
    M[3] = 3.0f * (m[3] + fz);
    M[4] = lbd::inv_w(4) * (meq[4] + a.g_bulk * (m[4] - meq[4]) + F[0]);
#pragma unroll
    for (int k = 5; k < 10; ++k) M[k] = lbd::inv_w(k) * (meq[k] + a.g_shear * (m[k] - meq[k]) + F[k - 4]);
#pragma unroll
    for (int k = 10; k < 16; ++k) M[k] = lbd::inv_w(k) * (meq[k] + a.g_odd * (m[k] - meq[k]));
#pragma unroll
    for (int k = 16; k < 19; ++k) M[k] = lbd::inv_w(k) * (meq[k] + a.g_even * (m[k] - meq[k]));
    if (NOISE) {
        float g[16];
        lbd::gaussians16(a.rk, node, a.step, 0u, a.replica, a.mu * (a.noise_rho0 ? a.rho0 : rho), g);
#pragma unroll
        for (int k = 4; k < 19; ++k) M[k] = fmaf(a.amp[k - 4], g[k - 4], M[k]);
    }
    lbd::backward(M, out);
}

// One node per thread: pull (link bounce-back at the walls), force, the
// collision above, store.  Grid (ceil(nx / 128), ny, fluid planes).
template <int DT, bool NOISE, bool WALLS>
__global__ void __launch_bounds__(128) k_stream_collide_exp(const typename lbd::Store<DT>::T *__restrict__ src,
                                                             typename lbd::Store<DT>::T *__restrict__ dst,
                                                             const float *__restrict__ ffield,
                                                             const float *__restrict__ facc, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const int x = blockIdx.x * 128 + threadIdx.x, y = blockIdx.y, z = blockIdx.z + a.z0;
    if (x >= a.nx) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int xm = (x == 0) ? nx - 1 : x - 1, xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1, yp = (y == ny - 1) ? 0 : y + 1;
    const int zm = WALLS ? z - 1 : ((z == 0) ? nz - 1 : z - 1);
    const int zp = WALLS ? z + 1 : ((z == nz - 1) ? 0 : z + 1);
    const size_t P = a.pitch;
    const size_t self = ((size_t)z * ny + y) * nx + x;
    float n[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
        const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
        const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
        const bool bounce = WALLS && lbd::cz(i) != 0 && (sz == 0 || sz == nz - 1);
        const size_t off = bounce ? (size_t)lbd::opposite(i) * P + self
                                  : (size_t)i * P + ((size_t)sz * ny + sy) * nx + sx;
        n[i] = S::load(src + off, a.inv_scale);
    }
    float fx = a.fx, fy = a.fy, fz = a.fz;
    if (ffield) {
        fx += __ldg(ffield + self);
        fy += __ldg(ffield + a.nn + self);
        fz += __ldg(ffield + 2 * a.nn + self);
    }
    if (facc) {
        fx += __ldg(facc + self);
        fy += __ldg(facc + P + self);
        fz += __ldg(facc + 2 * P + self);
    }
    float m[19], out[19];
    lbd::forward(n, m);
    collide_exp<NOISE>(m, fx, fy, fz, a, (uint32_t)self, out);
#pragma unroll
    for (int i = 0; i < 19; ++i) dst[(size_t)i * P + self] = S::pack(out[i], a.scale);
}

// ---- the same for two neighbouring nodes in packed FP32 (f32x2.cuh) ------
using lbp::F2;

__device__ __forceinline__ F2 rcp2(F2 v)
{
    float l, h;
    lbp::split(v, l, h);
    return lbp::f2(__frcp_rn(l), __frcp_rn(h));
}

// x_i = exp(lambda.c_i) - 1 for both nodes (exp_dirs, the expm1 per half).
__device__ __forceinline__ void exp_dirs2(const F2 l[3], F2 x[19])
{
    F2 ep[3], em[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float lo, hi;
        lbp::split(l[d], lo, hi);
        ep[d] = lbp::f2(expm1f(lo), expm1f(hi));
        em[d] = (lbp::f2s(0.0f) - ep[d]) * rcp2(lbp::f2s(1.0f) + ep[d]);
    }
    x[0] = lbp::f2s(0.0f);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int c3[3] = {lbd::cx(i), lbd::cy(i), lbd::cz(i)};
        F2 xi = lbp::f2s(0.0f);
        bool first = true;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (c3[d] != 0) {
                const F2 e = c3[d] > 0 ? ep[d] : em[d];
                xi = first ? e : lbp::fma2(xi, e, xi + e);  // (1 + x)(1 + e) - 1
                first = false;
            }
        x[i] = xi;
    }
}

// Deviation moments meq of n^eq - a rho0 for both nodes (exp_eq_moments).
__device__ __forceinline__ void exp_eq_moments2(F2 drho, F2 rho, F2 ux, F2 uy, F2 uz, F2 meq[19])
{
    const F2 three = lbp::f2s(3.0f), third = lbp::f2s(1.0f / 3.0f);
    F2 l[3] = {ux * three, uy * three, uz * three};
    const F2 u[3] = {ux, uy, uz};
    F2 x[19];
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        F2 sm = lbp::f2s(0.0f), m[3], C[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) m[k] = lbp::f2s(0.0f);
#pragma unroll
        for (int k = 0; k < 6; ++k) C[k] = lbp::f2s(0.0f);
        exp_dirs2(l, x);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const int cx = lbd::cx(i), cy = lbd::cy(i), cz = lbd::cz(i);
            const F2 w = x[i] * lbd::weight(i);
            sm = sm + w;
            if (cx) m[0] = cx > 0 ? m[0] + w : m[0] - w;
            if (cy) m[1] = cy > 0 ? m[1] + w : m[1] - w;
            if (cz) m[2] = cz > 0 ? m[2] + w : m[2] - w;
            if (cx) C[0] = C[0] + w;
            if (cy) C[1] = C[1] + w;
            if (cz) C[2] = C[2] + w;
            if (cx && cy) C[3] = cx * cy > 0 ? C[3] + w : C[3] - w;
            if (cy && cz) C[4] = cy * cz > 0 ? C[4] + w : C[4] - w;
            if (cz && cx) C[5] = cz * cx > 0 ? C[5] + w : C[5] - w;
        }
        const F2 iz = rcp2(lbp::f2s(1.0f) + sm);
#pragma unroll
        for (int d = 0; d < 3; ++d) m[d] = m[d] * iz;
        // covariance (1/3 I + sum a c c x) / Z - m m^T
        const F2 axx = (third + C[0]) * iz - m[0] * m[0], ayy = (third + C[1]) * iz - m[1] * m[1];
        const F2 azz = (third + C[2]) * iz - m[2] * m[2], axy = C[3] * iz - m[0] * m[1];
        const F2 ayz = C[4] * iz - m[1] * m[2], azx = C[5] * iz - m[2] * m[0];
        const F2 r[3] = {u[0] - m[0], u[1] - m[1], u[2] - m[2]};
        // Cramer's rule on the symmetric 3x3 system
        const F2 c00 = ayy * azz - ayz * ayz, c01 = azx * ayz - axy * azz, c02 = axy * ayz - azx * ayy;
        const F2 det = axx * c00 + axy * c01 + azx * c02;
        const F2 c11 = axx * azz - azx * azx, c12 = axy * azx - axx * ayz, c22 = axx * ayy - axy * axy;
        const F2 id = rcp2(det);
        l[0] = lbp::fma2(id, c00 * r[0] + c01 * r[1] + c02 * r[2], l[0]);
        l[1] = lbp::fma2(id, c01 * r[0] + c11 * r[1] + c12 * r[2], l[1]);
        l[2] = lbp::fma2(id, c02 * r[0] + c12 * r[1] + c22 * r[2], l[2]);
    }
    F2 sm = lbp::f2s(0.0f);
    exp_dirs2(l, x);
#pragma unroll
    for (int i = 1; i < 19; ++i) sm = lbp::fma2(x[i], lbd::weight(i), sm);
    const F2 g = rho * rcp2(lbp::f2s(1.0f) + sm);
    F2 d[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) d[i] = lbp::fma2(g, x[i] - sm, drho) * lbd::weight(i);
    lbp::forward2(d, meq);
}

// collide_exp for both nodes (packed FP32; the noise as in collide_moments2).
template <bool NOISE>
__device__ __forceinline__ void collide_exp2(const F2 m[19], F2 fx, F2 fy, F2 fz, const StepArgs &a, uint32_t node0,
                                             F2 out[19])
{
    const F2 half = lbp::f2s(0.5f), three = lbp::f2s(3.0f);
    const F2 rho = lbp::f2s(a.rho0) + m[0];
    const F2 inv_rho = rcp2(rho);
    const F2 ux = lbp::fma2(half, fx, m[1]) * inv_rho;
    const F2 uy = lbp::fma2(half, fy, m[2]) * inv_rho;
    const F2 uz = lbp::fma2(half, fz, m[3]) * inv_rho;
    F2 meq[19];
    exp_eq_moments2(m[0], rho, ux, uy, uz, meq);
    const F2 uf = ux * fx + uy * fy + uz * fz;
    const F2 gs1 = lbp::f2s(1.0f + a.g_shear), hgs1 = lbp::f2s(0.5f * (1.0f + a.g_shear));
    const F2 F[6] = {lbp::f2s(1.0f + a.g_bulk) * uf, gs1 * (ux * fx * three - uf), gs1 * (uy * fy - uz * fz),
                     hgs1 * (ux * fy + uy * fx),      hgs1 * (uy * fz + uz * fy),   hgs1 * (uz * fx + ux * fz)};
    F2 M[19];
    M[0] = m[0];
    M[1] = (m[1] + fx) * three;
    M[2] = (m[2] + fy) * three;
    M[3] = (m[3] + fz) * three;
    M[4] = lbp::fma2(lbp::f2s(a.g_bulk), m[4] - meq[4], meq[4] + F[0]) * lbd::inv_w(4);
#pragma unroll
    for (int k = 5; k < 10; ++k) M[k] = lbp::fma2(lbp::f2s(a.g_shear), m[k] - meq[k], meq[k] + F[k - 4]) * lbd::inv_w(k);
#pragma unroll
    for (int k = 10; k < 16; ++k) M[k] = lbp::fma2(lbp::f2s(a.g_odd), m[k] - meq[k], meq[k]) * lbd::inv_w(k);
#pragma unroll
    for (int k = 16; k < 19; ++k) M[k] = lbp::fma2(lbp::f2s(a.g_even), m[k] - meq[k], meq[k]) * lbd::inv_w(k);
    if (NOISE) {
        const F2 var = a.noise_rho0 ? lbp::f2s(a.mu * a.rho0) : rho * a.mu;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const lbd::U4 r0 = lbd::philox10(lbd::U4{node0, a.step, (uint32_t)b, a.replica}, a.rk);
            const lbd::U4 r1 = lbd::philox10(lbd::U4{node0 + 1u, a.step, (uint32_t)b, a.replica}, a.rk);
            F2 g[4];
            lbp::box_muller2(r0.x, r0.y, r1.x, r1.y, g[0], g[1], var);
            lbp::box_muller2(r0.z, r0.w, r1.z, r1.w, g[2], g[3], var);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = 4 + 4 * b + j;
                if (k < 19) M[k] = lbp::fma2(g[j], a.amp[k - 4], M[k]);
            }
        }
    }
    lbp::backward2(M, out);
}

// Two nodes per thread (even nx): the pull and store of k_stream_collide2,
// the exponential collision in packed FP32.  Grid (ceil(nx / 256), ny, fluid planes).
template <int DT, bool NOISE, bool WALLS>
__global__ void __launch_bounds__(128) k_stream_collide_exp2(const typename lbd::Store<DT>::T *__restrict__ src,
                                                              typename lbd::Store<DT>::T *__restrict__ dst,
                                                              const float *__restrict__ ffield,
                                                              const float *__restrict__ facc, const StepArgs a)
{
    const int x0 = 2 * (blockIdx.x * 128 + threadIdx.x), y = blockIdx.y, z = blockIdx.z + a.z0;
    if (x0 >= a.nx) return;
    F2 n[19], m[19], out[19];
    float f0[3], f1[3];
    load_pair<DT, true, WALLS>(src, ffield, facc, a, x0, y, z, n, f0, f1);
    lbp::forward2(n, m);
    const uint32_t self = (uint32_t)((z * a.ny + y) * a.nx + x0);
    collide_exp2<NOISE>(m, lbp::f2(f0[0], f1[0]), lbp::f2(f0[1], f1[1]), lbp::f2(f0[2], f1[2]), a, self, out);
    store_pair<DT>(dst, a, self, out);
}

template <int DT>
cudaError_t launch_exp_dt(const lb_handle *h, const void *src, void *dst, const float *facc)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
    const bool noise = a.kT > 0.0f, walls = h->p.walls != 0;
    if (sc_paired(h)) {  // two nodes per thread, packed FP32
        const dim3 grid((unsigned)((a.nx / 2 + 127) / 128), (unsigned)a.ny, (unsigned)(a.z1 - a.z0));
#define LBI_EXP2(NZ, WL) k_stream_collide_exp2<DT, NZ, WL><<<grid, 128, 0, h->stream>>>(s, d, h->force, facc, a)
        if (noise) {
            if (walls) LBI_EXP2(true, true); else LBI_EXP2(true, false);
        } else {
            if (walls) LBI_EXP2(false, true); else LBI_EXP2(false, false);
        }
#undef LBI_EXP2
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((a.nx + 127) / 128), (unsigned)a.ny, (unsigned)(a.z1 - a.z0));
#define LBI_EXP(NZ, WL) k_stream_collide_exp<DT, NZ, WL><<<grid, 128, 0, h->stream>>>(s, d, h->force, facc, a)
    if (noise) {
        if (walls) LBI_EXP(true, true); else LBI_EXP(true, false);
    } else {
        if (walls) LBI_EXP(false, true); else LBI_EXP(false, false);
    }
#undef LBI_EXP
    return cudaGetLastError();
}

}  // namespace

// One stream-collide launch of a handle whose lb_params.equilibrium selects
// the exponential form.
cudaError_t launch_stream_collide_exp(const lb_handle *h, const void *src, void *dst, const float *facc)
{
    switch (h->p.dtype) {
    case LB_F32: return launch_exp_dt<0>(h, src, dst, facc);
    case LB_F16: return launch_exp_dt<1>(h, src, dst, facc);
    default: return launch_exp_dt<2>(h, src, dst, facc);
    }
}

}  // namespace lbi
