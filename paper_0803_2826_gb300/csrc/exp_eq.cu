// exp_eq.cu -- the stream-collide update with the exponential equilibrium of
// Sec. 3.6, Eq. (equildist_lagrange): the populations that maximise the
// entropy of Eq. (boltzmann_entropy_function) at given mass and momentum,
// n^eq_i = rho a_i exp(lambda.c_i) / Z, Z = sum_i a_i exp(lambda.c_i), with
// lambda the root of sum_i a_i c_i exp(lambda.c_i) / Z = u.  The standard
// equilibrium of Eq. (original_equil_distrib) is its expansion to O(u^2);
// this one also has parts on the kinetic modes (O(u^3)), which the
// relaxation keeps.  Everything else is the collision of
// stream_collide.cuh: the same moments, eigenvalues, forcing and noise.
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

template <int DT>
cudaError_t launch_exp_dt(const lb_handle *h, const void *src, void *dst, const float *facc)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    const dim3 grid((unsigned)((a.nx + 127) / 128), (unsigned)a.ny, (unsigned)(a.z1 - a.z0));
    const T *s = static_cast<const T *>(src);
    T *d = static_cast<T *>(dst);
    const bool noise = a.kT > 0.0f, walls = h->p.walls != 0;
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
