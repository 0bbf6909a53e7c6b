// adjoint.cu -- reverse mode of the deterministic (kT = 0) stream-collide
// step, the kinetic-energy loss seed, and a checkpointed driver.
//
// One forward step maps the stored state S_t to S_{t+1} = C(pull(S_t), f).
// Its adjoint, derived here in moment space (Table 1 basis, q = a):
//   back transform  n* = B m*,  B = diag(a) E^T diag(1/w)
//                   -> mu*_k = (1/w_k) sum_i e_ki a_i lambda_i
//   relaxation      m*_0 = m_0, m*_a = m_a + f_a (a = 1..3),
//                   m*_k = (1 - g_k) rho P_k(u) + g_k m_k + F_k(u, f) (k = 4..9),
//                   m*_k = g_k m_k (k >= 10), with rho = rho0 + m_0,
//                   u = (m_1..3 + f/2) / rho   (Sec. 3.4 Eq. (lco_update),
//                   Sec. 3.7 Eqs. (special_choice_momentum_density),
//                   (moment_two_external_force))
//   forward         m = E n -> dL/dn_i = sum_k e_ki mu_k
//   pull            n_i(r) = S_i(r - c_i) (or S_opp(i)(r) at a wall)
//                   -> lambda_t is the push of dL/dn back to those entries;
//                   every fluid entry receives exactly one value, so the
//                   push is a plain store.
// P_k are the equilibrium stress polynomials (u^2, 3ux^2 - u^2, uy^2 - uz^2,
// ux uy, uy uz, uz ux) and F_k the force moments of Sigma.
#include <cmath>
#include <vector>

#include "d3q19.cuh"
#include "lbf_internal.h"

namespace lbi {

template <int DT>
cudaError_t launch_stream_collide_dt(const lb_handle *h, const void *src, void *dst, const float *facc, float *partials);

namespace {

constexpr int kAdjBX = 128;

template <bool WALLS>
__device__ __forceinline__ void neighbours(int x, int y, int z, const StepArgs &a, int &xm, int &xp, int &ym, int &yp,
                                           int &zm, int &zp)
{
    xm = (x == 0) ? a.nx - 1 : x - 1;
    xp = (x == a.nx - 1) ? 0 : x + 1;
    ym = (y == 0) ? a.ny - 1 : y - 1;
    yp = (y == a.ny - 1) ? 0 : y + 1;
    if (WALLS) {
        zm = z - 1;
        zp = z + 1;
    } else {
        zm = (z == 0) ? a.nz - 1 : z - 1;
        zp = (z == a.nz - 1) ? 0 : z + 1;
    }
}

// Source entry of the pull for direction i at node (x, y, z): returns the
// plane and the node index; at a wall the link bounces back to the node itself.
template <bool WALLS>
__device__ __forceinline__ void pull_source(int i, int x, int y, int z, int xm, int xp, int ym, int yp, int zm, int zp,
                                            const StepArgs &a, int &plane, uint32_t &node)
{
    const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
    const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
    const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
    const bool bounce = WALLS && lbd::cz(i) != 0 && (sz == 0 || sz == a.nz - 1);
    if (bounce) {
        plane = lbd::opposite(i);
        node = (uint32_t)((z * a.ny + y) * a.nx + x);
    } else {
        plane = i;
        node = (uint32_t)((sz * a.ny + sy) * a.nx + sx);
    }
}

template <int DT, bool WALLS>
__global__ void __launch_bounds__(kAdjBX)
    k_adjoint_step(const typename lbd::Store<DT>::T *__restrict__ state, const float *__restrict__ lam_in,
                   float *__restrict__ lam_out, const float *__restrict__ ffield, const float *__restrict__ impulse,
                   float *grad_f, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const int x = blockIdx.x * kAdjBX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y;
    const int z = blockIdx.z + a.z0;
    int xm, xp, ym, yp, zm, zp;
    neighbours<WALLS>(x, y, z, a, xm, xp, ym, yp, zm, zp);
    const size_t P = a.pitch;
    const uint32_t self = (uint32_t)((z * a.ny + y) * a.nx + x);

    // forward quantities at this node
    float n[19];
    int plane[19];
    uint32_t src[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        pull_source<WALLS>(i, x, y, z, xm, xp, ym, yp, zm, zp, a, plane[i], src[i]);
        n[i] = S::load(state + (size_t)plane[i] * P + src[i], a.inv_scale);
    }
    float m[19];
    lbd::forward(n, m);
    float f[3] = {a.fx, a.fy, a.fz};
    if (ffield) {
        f[0] += ffield[self];
        f[1] += ffield[a.nn + self];
        f[2] += ffield[2 * a.nn + self];
    }
    if (impulse) {  // particle impulses of the step ([3][pitch])
        f[0] += impulse[self];
        f[1] += impulse[P + self];
        f[2] += impulse[2 * P + self];
    }
    const float rho = a.rho0 + m[0];
    const float ir = 1.0f / rho;
    const float u[3] = {(m[1] + 0.5f * f[0]) * ir, (m[2] + 0.5f * f[1]) * ir, (m[3] + 0.5f * f[2]) * ir};

    // adjoint of the back transform
    float al[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) al[i] = lbd::weight(i) * __ldg(lam_in + (size_t)i * P + self);
    float mus[19];
    lbd::forward(al, mus);
#pragma unroll
    for (int k = 0; k < 19; ++k) mus[k] *= lbd::inv_w(k);

    // adjoint of the relaxation, the equilibrium and the force moments
    const float gs = a.g_shear, gv = a.g_bulk;
    const float cs = 1.0f + gs, cv = 1.0f + gv;
    const float ux = u[0], uy = u[1], uz = u[2];
    const float u2 = ux * ux + uy * uy + uz * uz;
    const float Pk[6] = {u2, 3.0f * ux * ux - u2, uy * uy - uz * uz, ux * uy, uy * uz, uz * ux};
    const float gk[6] = {gv, gs, gs, gs, gs, gs};
    // dP_k/du rows
    const float dP[6][3] = {{2.0f * ux, 2.0f * uy, 2.0f * uz},
                            {4.0f * ux, -2.0f * uy, -2.0f * uz},
                            {0.0f, 2.0f * uy, -2.0f * uz},
                            {uy, ux, 0.0f},
                            {0.0f, uz, uy},
                            {uz, 0.0f, ux}};
    // dF_k/du rows (F4 = cv u.f, F5 = cs (3 ux fx - u.f), F6 = cs (uy fy - uz fz),
    // F7 = cs/2 (ux fy + uy fx), F8 = cs/2 (uy fz + uz fy), F9 = cs/2 (uz fx + ux fz))
    const float dFu[6][3] = {{cv * f[0], cv * f[1], cv * f[2]},
                             {2.0f * cs * f[0], -cs * f[1], -cs * f[2]},
                             {0.0f, cs * f[1], -cs * f[2]},
                             {0.5f * cs * f[1], 0.5f * cs * f[0], 0.0f},
                             {0.0f, 0.5f * cs * f[2], 0.5f * cs * f[1]},
                             {0.5f * cs * f[2], 0.0f, 0.5f * cs * f[0]}};
    // dF_k/df rows: the same expressions with u and f exchanged
    const float dFf[6][3] = {{cv * ux, cv * uy, cv * uz},
                             {2.0f * cs * ux, -cs * uy, -cs * uz},
                             {0.0f, cs * uy, -cs * uz},
                             {0.5f * cs * uy, 0.5f * cs * ux, 0.0f},
                             {0.0f, 0.5f * cs * uz, 0.5f * cs * uy},
                             {0.5f * cs * uz, 0.0f, 0.5f * cs * ux}};
    float rbar = 0.0f, ubar[3] = {0.f, 0.f, 0.f}, fbar[3] = {mus[1], mus[2], mus[3]};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float mk = mus[4 + q];
        const float one_g = 1.0f - gk[q];
        rbar += mk * one_g * Pk[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            ubar[d] += mk * (one_g * rho * dP[q][d] + dFu[q][d]);
            fbar[d] += mk * dFf[q][d];
        }
    }
    float mu[19];
    mu[0] = mus[0] + rbar - (ubar[0] * ux + ubar[1] * uy + ubar[2] * uz) * ir;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        mu[1 + d] = mus[1 + d] + ubar[d] * ir;
        fbar[d] += 0.5f * ubar[d] * ir;
    }
    mu[4] = gv * mus[4];
#pragma unroll
    for (int k = 5; k < 10; ++k) mu[k] = gs * mus[k];
#pragma unroll
    for (int k = 10; k < 16; ++k) mu[k] = a.g_odd * mus[k];
#pragma unroll
    for (int k = 16; k < 19; ++k) mu[k] = a.g_even * mus[k];

    // dL/dn_i = sum_k e_ki mu_k = backward(mu)_i / a_i, pushed to the pull sources
    float dn[19];
    lbd::backward(mu, dn);
#pragma unroll
    for (int i = 0; i < 19; ++i) lam_out[(size_t)plane[i] * P + src[i]] = dn[i] * (1.0f / lbd::weight(i));
    if (grad_f) {
        grad_f[self] += fbar[0];
        grad_f[a.nn + self] += fbar[1];
        grad_f[2 * a.nn + self] += fbar[2];
    }
}

// lambda_T for L = 1/2 sum_{box} |j|^2 / rho: dL/dn_i = u.c_i - u^2/2 inside
// the box, 0 elsewhere (every fluid entry is written); dL/df += u/2.
template <int DT, bool WALLS>
__global__ void __launch_bounds__(kAdjBX)
    k_adjoint_seed(const typename lbd::Store<DT>::T *__restrict__ state, float *__restrict__ lam_out,
                   const float *__restrict__ ffield, float *grad_f, double *loss, int3 lo, int3 hi, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const int x = blockIdx.x * kAdjBX + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z + a.z0;
    float Lloc = 0.0f;
    if (x < a.nx) {
        int xm, xp, ym, yp, zm, zp;
        neighbours<WALLS>(x, y, z, a, xm, xp, ym, yp, zm, zp);
        const size_t P = a.pitch;
        const uint32_t self = (uint32_t)((z * a.ny + y) * a.nx + x);
        const bool inside = x >= lo.x && x < hi.x && y >= lo.y && y < hi.y && z >= lo.z && z < hi.z;
        float n[19];
        int plane[19];
        uint32_t src[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            pull_source<WALLS>(i, x, y, z, xm, xp, ym, yp, zm, zp, a, plane[i], src[i]);
            n[i] = inside ? S::load(state + (size_t)plane[i] * P + src[i], a.inv_scale) : 0.0f;
        }
        float dn[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) dn[i] = 0.0f;
        if (inside) {
            float m[19];
            lbd::forward(n, m);
            float f[3] = {a.fx, a.fy, a.fz};
            if (ffield) {
                f[0] += ffield[self];
                f[1] += ffield[a.nn + self];
                f[2] += ffield[2 * a.nn + self];
            }
            const float rho = a.rho0 + m[0];
            const float j[3] = {m[1] + 0.5f * f[0], m[2] + 0.5f * f[1], m[3] + 0.5f * f[2]};
            const float u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
            const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            Lloc = 0.5f * (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / rho;
#pragma unroll
            for (int i = 0; i < 19; ++i) dn[i] = u[0] * lbd::cx(i) + u[1] * lbd::cy(i) + u[2] * lbd::cz(i) - 0.5f * u2;
            if (grad_f) {
                grad_f[self] += 0.5f * u[0];
                grad_f[a.nn + self] += 0.5f * u[1];
                grad_f[2 * a.nn + self] += 0.5f * u[2];
            }
        }
#pragma unroll
        for (int i = 0; i < 19; ++i) lam_out[(size_t)plane[i] * P + src[i]] = dn[i];
    }
    // loss: warp reduction, one double atomic per warp
    double v = (double)Lloc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(loss, v);
}

template <int DT>
cudaError_t launch_adjoint_dt(const lb_handle *h, const void *state, const float *lam_in, float *lam_out,
                              float *grad_f, const float *impulse)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    dim3 grid((a.nx + kAdjBX - 1) / kAdjBX, a.ny, a.z1 - a.z0);
    const T *s = static_cast<const T *>(state);
    if (h->p.walls)
        k_adjoint_step<DT, true><<<grid, kAdjBX, 0, h->stream>>>(s, lam_in, lam_out, h->force, impulse, grad_f, a);
    else
        k_adjoint_step<DT, false><<<grid, kAdjBX, 0, h->stream>>>(s, lam_in, lam_out, h->force, impulse, grad_f, a);
    return cudaGetLastError();
}

// dL/du at the nodes (lam_u, [3][pitch], set by the coupling reverse pass)
// into dL/dstate through u = (sum n c + f/2) / rho of the pulled populations:
// d u_d / d n_i = (c_id - u_d) / rho, added at the stored entry each n_i is
// pulled from; d u_d / d f_d = 1 / (2 rho) into grad_f ([3][N]).  lam_u is
// zeroed on the way, so it is clean for the next call.
template <int DT, bool WALLS>
__global__ void __launch_bounds__(kAdjBX)
    k_lambda_u_to_pops(const typename lbd::Store<DT>::T *__restrict__ state, float *lam_u, float *lam_out,
                       const float *__restrict__ ffield, const float *__restrict__ impulse, float *grad_f,
                       const StepArgs a)
{
    using S = lbd::Store<DT>;
    const int x = blockIdx.x * kAdjBX + threadIdx.x;
    if (x >= a.nx) return;
    const int y = blockIdx.y;
    const int z = blockIdx.z + a.z0;
    const size_t P = a.pitch;
    const uint32_t self = (uint32_t)((z * a.ny + y) * a.nx + x);
    const float lu[3] = {lam_u[self], lam_u[P + self], lam_u[2 * P + self]};
    if (lu[0] == 0.0f && lu[1] == 0.0f && lu[2] == 0.0f) return;
    lam_u[self] = lam_u[P + self] = lam_u[2 * P + self] = 0.0f;
    int xm, xp, ym, yp, zm, zp;
    neighbours<WALLS>(x, y, z, a, xm, xp, ym, yp, zm, zp);
    float n[19];
    int plane[19];
    uint32_t src[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        pull_source<WALLS>(i, x, y, z, xm, xp, ym, yp, zm, zp, a, plane[i], src[i]);
        n[i] = S::load(state + (size_t)plane[i] * P + src[i], a.inv_scale);
    }
    float m[19];
    lbd::forward(n, m);
    // the velocity the forward coupling interpolated: f = body force + field
    // (the particle impulses of the step are not part of it)
    float f[3] = {a.fx, a.fy, a.fz};
    if (ffield) {
        f[0] += ffield[self];
        f[1] += ffield[a.nn + self];
        f[2] += ffield[2 * a.nn + self];
    }
    (void)impulse;
    const float rho = a.rho0 + m[0];
    const float ir = 1.0f / rho;
    const float u[3] = {(m[1] + 0.5f * f[0]) * ir, (m[2] + 0.5f * f[1]) * ir, (m[3] + 0.5f * f[2]) * ir};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float v = lu[0] * ((float)lbd::cx(i) - u[0]) + lu[1] * ((float)lbd::cy(i) - u[1]) +
                        lu[2] * ((float)lbd::cz(i) - u[2]);
        atomicAdd(lam_out + (size_t)plane[i] * P + src[i], v * ir);
    }
    if (grad_f) {
#pragma unroll
        for (int d = 0; d < 3; ++d) grad_f[d * a.nn + self] += 0.5f * lu[d] * ir;
    }
}

template <int DT>
cudaError_t launch_lambda_u_dt(const lb_handle *h, const void *state, float *lam_u, float *lam_out, float *grad_f)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    dim3 grid((a.nx + kAdjBX - 1) / kAdjBX, a.ny, a.z1 - a.z0);
    const T *s = static_cast<const T *>(state);
    if (h->p.walls)
        k_lambda_u_to_pops<DT, true><<<grid, kAdjBX, 0, h->stream>>>(s, lam_u, lam_out, h->force, nullptr, grad_f, a);
    else
        k_lambda_u_to_pops<DT, false><<<grid, kAdjBX, 0, h->stream>>>(s, lam_u, lam_out, h->force, nullptr, grad_f, a);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_seed_dt(const lb_handle *h, const void *state, float *lam_out, float *grad_f, double *loss,
                           int3 lo, int3 hi)
{
    using T = typename lbd::Store<DT>::T;
    const StepArgs a = make_args(h);
    dim3 grid((a.nx + kAdjBX - 1) / kAdjBX, a.ny, a.z1 - a.z0);
    const T *s = static_cast<const T *>(state);
    if (h->p.walls)
        k_adjoint_seed<DT, true><<<grid, kAdjBX, 0, h->stream>>>(s, lam_out, h->force, grad_f, loss, lo, hi, a);
    else
        k_adjoint_seed<DT, false><<<grid, kAdjBX, 0, h->stream>>>(s, lam_out, h->force, grad_f, loss, lo, hi, a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const lb_handle *h, const void *state, const float *lam_in, float *lam_out, float *grad_f,
                           const float *impulse = nullptr)
{
    switch (h->p.dtype) {
    case LB_F32: return launch_adjoint_dt<0>(h, state, lam_in, lam_out, grad_f, impulse);
    case LB_F16: return launch_adjoint_dt<1>(h, state, lam_in, lam_out, grad_f, impulse);
    default: return launch_adjoint_dt<2>(h, state, lam_in, lam_out, grad_f, impulse);
    }
}

cudaError_t launch_lambda_u(const lb_handle *h, const void *state, float *lam_u, float *lam_out, float *grad_f)
{
    switch (h->p.dtype) {
    case LB_F32: return launch_lambda_u_dt<0>(h, state, lam_u, lam_out, grad_f);
    case LB_F16: return launch_lambda_u_dt<1>(h, state, lam_u, lam_out, grad_f);
    default: return launch_lambda_u_dt<2>(h, state, lam_u, lam_out, grad_f);
    }
}

// a += b over n floats
__global__ void k_axpy1(float *a, const float *b, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

cudaError_t launch_seed(const lb_handle *h, const void *state, float *lam_out, float *grad_f, double *loss, int3 lo,
                        int3 hi)
{
    switch (h->p.dtype) {
    case LB_F32: return launch_seed_dt<0>(h, state, lam_out, grad_f, loss, lo, hi);
    case LB_F16: return launch_seed_dt<1>(h, state, lam_out, grad_f, loss, lo, hi);
    default: return launch_seed_dt<2>(h, state, lam_out, grad_f, loss, lo, hi);
    }
}

cudaError_t step_from(lb_handle *h, const void *src, void *dst, uint32_t step, const float *impulse = nullptr)
{
    const uint32_t saved = h->step;
    h->step = step;
    cudaError_t e;
    switch (h->p.dtype) {
    case LB_F32:
        e = h->p.equilibrium ? launch_stream_collide_exp(h, src, dst, impulse)
                             : launch_stream_collide_dt<0>(h, src, dst, impulse, nullptr);
        break;
    case LB_F16:
        e = h->p.equilibrium ? launch_stream_collide_exp(h, src, dst, impulse)
                             : launch_stream_collide_dt<1>(h, src, dst, impulse, nullptr);
        break;
    default:
        e = h->p.equilibrium ? launch_stream_collide_exp(h, src, dst, impulse)
                             : launch_stream_collide_dt<2>(h, src, dst, impulse, nullptr);
        break;
    }
    h->step = saved;
    return e;
}

bool check_adjoint_handle(const lb_handle *h, const char *who)
{
    if (!h) {
        set_error("%s: handle is NULL", who);
        return false;
    }
    if (h->p.kT != 0.0) {
        set_error("%s: the adjoint is defined for deterministic runs (kT = 0)", who);
        return false;
    }
    if (h->p.equilibrium) {
        set_error("%s: the adjoint is derived for the quadratic equilibrium", who);
        return false;
    }
    return true;
}

bool box_ok(const lb_handle *h, const int lo[3], const int hi[3])
{
    const int L[3] = {h->p.nx, h->p.ny, h->p.nz};
    for (int d = 0; d < 3; ++d)
        if (lo[d] < 0 || hi[d] > L[d] || lo[d] > hi[d]) return false;
    return true;
}

// Carve `count` blocks of `bytes` each (256-byte aligned) from the handle's
// arena, growing it first if needed (the only allocation of the reverse-mode
// drivers; a grown arena replaces the old one, whose contents are dropped).
struct Carver {
    size_t need = 0;
    std::vector<std::pair<void **, size_t>> req;
    void add(void **p, size_t bytes)
    {
        req.push_back({p, need});
        need += (bytes + 255) & ~(size_t)255;
    }
    cudaError_t place(lb_handle *h)
    {
        if (h->arena_bytes < need) {
            cudaError_t e = cudaStreamSynchronize(h->stream);  // the old arena may still be in use
            if (e != cudaSuccess) return e;
            cudaFree(h->arena);
            h->arena = nullptr;
            h->arena_bytes = 0;
            e = cudaMalloc((void **)&h->arena, need);
            if (e != cudaSuccess) {
                h->arena = nullptr;
                return e;
            }
            h->arena_bytes = need;
        }
        for (auto &r : req) *r.first = h->arena + r.second;
        return cudaSuccess;
    }
};

}  // namespace
}  // namespace lbi

using namespace lbi;

extern "C" {

lb_status lb_step_from(lb_handle *h, const void *src, void *dst, uint32_t step)
{
    if (!h || !src || !dst || src == dst) {
        set_error("lb_step_from: need a handle and two distinct buffers");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = step_from(h, src, dst, step);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_step_from", e);
}

lb_status lb_adjoint_step(lb_handle *h, const void *state, const float *lambda_in, float *lambda_out,
                          float *grad_force)
{
    if (!check_adjoint_handle(h, "lb_adjoint_step")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (!state || !lambda_in || !lambda_out || lambda_in == lambda_out) {
        set_error("lb_adjoint_step: need a state and two distinct adjoint buffers");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = launch_adjoint(h, state, lambda_in, lambda_out, grad_force);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_step", e);
}

lb_status lb_adjoint_seed_kinetic(lb_handle *h, const void *state, const int lo[3], const int hi[3], float *lambda_out,
                                  float *grad_force, double *loss)
{
    if (!h || !state || !lo || !hi || !lambda_out || !loss) {
        set_error("lb_adjoint_seed_kinetic: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (!box_ok(h, lo, hi)) {
        set_error("lb_adjoint_seed_kinetic: sub-box outside the lattice");
        return LB_EINVAL;
    }
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = launch_seed(h, state, lambda_out, grad_force, loss, make_int3(lo[0], lo[1], lo[2]),
                        make_int3(hi[0], hi[1], hi[2]));
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_seed_kinetic", e);
}

// Arena layout of the uncoupled reverse pass: nseg checkpoints, K - 1
// segment states, two adjoint buffers.
struct KineticBuffers {
    std::vector<void *> ckpt, seg;
    float *lam[2] = {nullptr, nullptr};
    float *gseed = nullptr;  // dL/df of the loss itself (j = sum n c + f/2), [3][N]
};

static cudaError_t kinetic_buffers(lb_handle *h, int nsteps, int K, KineticBuffers &b)
{
    const int nseg = (nsteps + K - 1) / K;
    const size_t pop_bytes = 19 * h->pitch * h->elem;
    const size_t lam_bytes = 19 * h->pitch * sizeof(float);
    b.ckpt.assign(nseg, nullptr);
    b.seg.assign(K, nullptr);
    Carver c;
    for (int s = 0; s < nseg; ++s) c.add(&b.ckpt[s], pop_bytes);
    for (int k = 1; k < K; ++k) c.add(&b.seg[k], pop_bytes);
    for (int q = 0; q < 2; ++q) c.add((void **)&b.lam[q], lam_bytes);
    c.add((void **)&b.gseed, 3 * h->n_nodes * sizeof(float));
    return c.place(h);
}

lb_status lb_adjoint_forward(lb_handle *h, int nsteps, int checkpoint_every, const int lo[3], const int hi[3],
                             double *loss)
{
    const NvtxRange range("lb_adjoint_forward");
    if (!check_adjoint_handle(h, "lb_adjoint_forward")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (nsteps < 1 || checkpoint_every < 1 || !lo || !hi || !loss || !box_ok(h, lo, hi)) {
        set_error("lb_adjoint_forward: need nsteps >= 1, checkpoint_every >= 1, a valid sub-box and a loss");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (h->facc_dirty) {
        set_error("lb_adjoint_forward: pending particle impulses are not differentiated");
        return LB_EUNSUPPORTED;
    }
    const int K = std::min(checkpoint_every, nsteps);
    KineticBuffers b;
    cudaError_t e = kinetic_buffers(h, nsteps, K, b);
    if (e != cudaSuccess) {
        set_error("lb_adjoint_forward: checkpoint allocation failed (%s)", cudaGetErrorString(e));
        return LB_ENOMEM;
    }
    h->adj_ready = 0;
    const size_t pop_bytes = 19 * h->pitch * h->elem;
    const uint32_t step0 = h->step;
    for (int t = 0; t < nsteps && e == cudaSuccess; ++t) {
        if (t % K == 0) e = cudaMemcpyAsync(b.ckpt[t / K], h->pops[h->cur], pop_bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && lb_step(h, 1) != LB_OK) e = cudaErrorLaunchFailure;
    }
    // the loss and its seed lambda_T = dL/dstate at the final state (first
    // adjoint buffer) with its own dL/df (gseed), for lb_adjoint_backward
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.gseed, 0, 3 * h->n_nodes * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.lam[0], 0, 19 * h->pitch * sizeof(float), h->stream);
    if (e == cudaSuccess)
        e = launch_seed(h, h->pops[h->cur], b.lam[0], b.gseed, loss, make_int3(lo[0], lo[1], lo[2]),
                        make_int3(hi[0], hi[1], hi[2]));
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail("lb_adjoint_forward", e);
    h->adj_ready = 1;
    h->adj_nsteps = nsteps;
    h->adj_K = K;
    h->adj_step0 = step0;
    return LB_OK;
}

lb_status lb_adjoint_backward(lb_handle *h, float *grad_force)
{
    const NvtxRange range("lb_adjoint_backward");
    if (!check_adjoint_handle(h, "lb_adjoint_backward")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (!grad_force) {
        set_error("lb_adjoint_backward: grad_force is NULL");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (!h->adj_ready) {
        set_error("lb_adjoint_backward: no lb_adjoint_forward run to reverse");
        return LB_EINVAL;
    }
    const int nsteps = h->adj_nsteps, K = h->adj_K;
    const int nseg = (nsteps + K - 1) / K;
    KineticBuffers b;
    cudaError_t e = kinetic_buffers(h, nsteps, K, b);  // the forward's layout: no allocation
    if (e != cudaSuccess) return cuda_fail("lb_adjoint_backward", e);
    const size_t lam_bytes = 19 * h->pitch * sizeof(float);
    e = cudaMemsetAsync(b.lam[1], 0, lam_bytes, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad_force, b.gseed, 3 * h->n_nodes * sizeof(float), cudaMemcpyDeviceToDevice,
                            h->stream);
    int cur = 0;
    for (int s = nseg - 1; s >= 0 && e == cudaSuccess; --s) {
        const int t0 = s * K, t1 = std::min(nsteps, t0 + K);
        b.seg[0] = b.ckpt[s];
        for (int t = t0; t < t1 - 1 && e == cudaSuccess; ++t) {
            e = step_from(h, b.seg[t - t0], b.seg[t - t0 + 1], h->adj_step0 + (uint32_t)t);
            h->launches += 1;
        }
        for (int t = t1 - 1; t >= t0 && e == cudaSuccess; --t) {
            e = launch_adjoint(h, b.seg[t - t0], b.lam[cur], b.lam[1 - cur], grad_force);
            h->launches += 1;
            cur = 1 - cur;
        }
    }
    h->adj_ready = 0;  // the adjoint buffers were consumed
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_backward", e);
}

lb_status lb_adjoint_kinetic(lb_handle *h, int nsteps, int checkpoint_every, const int lo[3], const int hi[3],
                             float *grad_force, double *loss)
{
    if (!grad_force) {
        set_error("lb_adjoint_kinetic: grad_force is NULL");
        return LB_EINVAL;
    }
    lb_status st = lb_adjoint_forward(h, nsteps, checkpoint_every, lo, hi, loss);
    if (st != LB_OK) return st;
    return lb_adjoint_backward(h, grad_force);
}


lb_status lb_adjoint_step_impulse(lb_handle *h, const void *state, const float *impulse, const float *lambda_in,
                                  float *lambda_out, float *grad_force)
{
    if (!check_adjoint_handle(h, "lb_adjoint_step_impulse")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (!state || !lambda_in || !lambda_out || lambda_in == lambda_out) {
        set_error("lb_adjoint_step_impulse: need a state and two distinct adjoint buffers");
        return LB_EINVAL;
    }
    join_overlap(h);
    cudaError_t e = launch_adjoint(h, state, lambda_in, lambda_out, grad_force, impulse);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_step_impulse", e);
}

lb_status lb_adjoint_couple(lb_handle *h, const void *state, const lb_particles *start, const lb_couple_params *cp,
                            const float *lambda_facc, float *lambda_pos, float *lambda_mom, float *lambda_pops,
                            float *grad_force)
{
    if (!check_adjoint_handle(h, "lb_adjoint_couple")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (!state || !start || !cp || !lambda_facc || !lambda_pops ||
        (start->n > 0 && (!lambda_pos || !lambda_mom))) {
        set_error("lb_adjoint_couple: NULL argument");
        return LB_EINVAL;
    }
    join_overlap(h);
    if (!h->lam_u) {
        cudaError_t e = cudaMalloc((void **)&h->lam_u, 3 * h->pitch * sizeof(float));
        if (e == cudaSuccess) e = cudaMemsetAsync(h->lam_u, 0, 3 * h->pitch * sizeof(float), h->stream);
        if (e != cudaSuccess) {
            set_error("lb_adjoint_couple: scratch allocation failed (%s)", cudaGetErrorString(e));
            return LB_ENOMEM;
        }
    }
    lb_status st = couple_adjoint(h, state, start, cp, lambda_facc, lambda_pos, lambda_mom, h->lam_u);
    if (st != LB_OK || start->n == 0) return st;
    cudaError_t e = launch_lambda_u(h, state, h->lam_u, lambda_pops, grad_force);
    h->launches += 1;
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_couple", e);
}

lb_status lb_adjoint_kinetic_coupled(lb_handle *h, const lb_particles *parts, const lb_couple_params *cp, int nsteps,
                                     int checkpoint_every, const int lo[3], const int hi[3], float *grad_force,
                                     float *grad_pos, float *grad_mom, double *loss)
{
    const NvtxRange range("lb_adjoint_kinetic_coupled");
    if (!check_adjoint_handle(h, "lb_adjoint_kinetic_coupled")) return h ? LB_EUNSUPPORTED : LB_EINVAL;
    if (!parts || !cp || nsteps < 1 || checkpoint_every < 1 || !lo || !hi || !grad_force || !loss ||
        !box_ok(h, lo, hi) || (parts->n > 0 && (!grad_pos || !grad_mom))) {
        set_error("lb_adjoint_kinetic_coupled: need particles, nsteps >= 1, checkpoint_every >= 1, a valid "
                  "sub-box and outputs");
        return LB_EINVAL;
    }
    if (!adjoint_couple_ok(h, parts, cp, "lb_adjoint_kinetic_coupled")) return LB_EUNSUPPORTED;
    join_overlap(h);
    if (h->facc_dirty) {
        set_error("lb_adjoint_kinetic_coupled: pending particle impulses (call lb_step first)");
        return LB_EUNSUPPORTED;
    }
    lb_couple_params c1 = *cp;
    c1.flags &= ~LB_COUPLE_OVERLAP;
    const int n = parts->n;
    const int K = std::min(checkpoint_every, nsteps);
    const int nseg = (nsteps + K - 1) / K;
    const size_t pop_bytes = 19 * h->pitch * h->elem;
    const size_t lam_bytes = 19 * h->pitch * sizeof(float);
    const size_t facc_bytes = 3 * h->pitch * sizeof(float);
    const size_t grad_bytes = 3 * h->n_nodes * sizeof(float);
    const size_t pos_bytes = (size_t)n * 3 * sizeof(double), mom_bytes = (size_t)n * 3 * sizeof(float);
    std::vector<void *> ckpt(nseg, nullptr), seg(K, nullptr);
    std::vector<double *> cpos(nseg, nullptr), spos(K + 1, nullptr);  // particles before step k of a segment
    std::vector<float *> cmom(nseg, nullptr), smom(K + 1, nullptr), sfacc(K, nullptr);
    float *lam[2] = {nullptr, nullptr};
    float *gstep = nullptr;
    cudaError_t e = cudaSuccess;
    {
        // all temporaries from the handle's arena (allocated once, reused)
        Carver c;
        for (int s = 0; s < nseg; ++s) {
            c.add(&ckpt[s], pop_bytes);
            if (n) c.add((void **)&cpos[s], pos_bytes);
            if (n) c.add((void **)&cmom[s], mom_bytes);
        }
        for (int k = 0; k <= K; ++k) {
            if (k > 0 && k < K) c.add(&seg[k], pop_bytes);
            if (n) c.add((void **)&spos[k], pos_bytes);
            if (n) c.add((void **)&smom[k], mom_bytes);
            if (k < K) c.add((void **)&sfacc[k], facc_bytes);
        }
        for (int b = 0; b < 2; ++b) c.add((void **)&lam[b], lam_bytes);
        c.add((void **)&gstep, grad_bytes);
        e = c.place(h);
    }
    h->adj_ready = 0;  // the arena now holds this call's buffers
    if (e != cudaSuccess) {
        set_error("lb_adjoint_kinetic_coupled: checkpoint allocation failed (%s)", cudaGetErrorString(e));
        return LB_ENOMEM;
    }
    const uint32_t step0 = h->step;
    // forward pass: populations and particle state checkpointed every K steps
    for (int t = 0; t < nsteps && e == cudaSuccess; ++t) {
        if (t % K == 0) {
            e = cudaMemcpyAsync(ckpt[t / K], h->pops[h->cur], pop_bytes, cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess && n)
                e = cudaMemcpyAsync(cpos[t / K], parts->pos, pos_bytes, cudaMemcpyDeviceToDevice, h->stream);
            if (e == cudaSuccess && n)
                e = cudaMemcpyAsync(cmom[t / K], parts->mom, mom_bytes, cudaMemcpyDeviceToDevice, h->stream);
        }
        lb_status st = (e == cudaSuccess) ? couple_particles(h, parts, &c1) : LB_ECUDA;
        if (st == LB_OK) st = lb_step(h, 1);
        if (st != LB_OK) {
            return st;
        }
    }
    // the last step applied its impulses: clear them now, so the recompute
    // below can reuse the stencil records
    if (e == cudaSuccess) e = clear_particle_forces(h);
    h->facc_stale = 0;
    int cur = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(lam[0], 0, lam_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam[1], 0, lam_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad_force, 0, grad_bytes, h->stream);
    if (e == cudaSuccess && n) e = cudaMemsetAsync(grad_pos, 0, (size_t)n * 3 * sizeof(float), h->stream);
    if (e == cudaSuccess && n) e = cudaMemsetAsync(grad_mom, 0, (size_t)n * 3 * sizeof(float), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = launch_seed(h, h->pops[h->cur], lam[cur], grad_force, loss, make_int3(lo[0], lo[1], lo[2]),
                        make_int3(hi[0], hi[1], hi[2]));
    h->launches += 1;
    for (int sgi = nseg - 1; sgi >= 0 && e == cudaSuccess; --sgi) {
        const int t0 = sgi * K, t1 = std::min(nsteps, t0 + K);
        seg[0] = ckpt[sgi];
        // recompute the segment: populations, the particle state before each
        // step and each step's impulses
        if (n) e = cudaMemcpyAsync(spos[0], cpos[sgi], pos_bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(smom[0], cmom[sgi], mom_bytes, cudaMemcpyDeviceToDevice, h->stream);
        for (int t = t0; t < t1 && e == cudaSuccess; ++t) {
            const int k = t - t0;
            if (n) {  // the coupling updates in place: run it on a copy in slot k + 1
                e = cudaMemcpyAsync(spos[k + 1], spos[k], pos_bytes, cudaMemcpyDeviceToDevice, h->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(smom[k + 1], smom[k], mom_bytes, cudaMemcpyDeviceToDevice, h->stream);
                lb_particles pk = *parts;
                pk.pos = spos[k + 1];
                pk.mom = smom[k + 1];
                if (e == cudaSuccess && couple_on(h, seg[k], &pk, &c1, sfacc[k]) != LB_OK) e = cudaErrorLaunchFailure;
            } else {
                e = cudaMemsetAsync(sfacc[k], 0, facc_bytes, h->stream);
            }
            if (e == cudaSuccess && t + 1 < t1) {
                e = step_from(h, seg[k], seg[k + 1], step0 + (uint32_t)t, sfacc[k]);
                h->launches += 1;
            }
        }
        // reverse through the segment
        for (int t = t1 - 1; t >= t0 && e == cudaSuccess; --t) {
            const int k = t - t0;
            e = cudaMemsetAsync(gstep, 0, grad_bytes, h->stream);
            if (e == cudaSuccess) e = launch_adjoint(h, seg[k], lam[cur], lam[1 - cur], gstep, sfacc[k]);
            if (e == cudaSuccess) {
                const size_t cnt = 3 * h->n_nodes;
                k_axpy1<<<(unsigned int)std::min<size_t>((cnt + 255) / 256, 4096), 256, 0, h->stream>>>(grad_force,
                                                                                                      gstep, cnt);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && n) {
                lb_particles pk = *parts;
                pk.pos = spos[k];
                pk.mom = smom[k];
                if (lb_adjoint_couple(h, seg[k], &pk, &c1, gstep, grad_pos, grad_mom, lam[1 - cur], grad_force) !=
                    LB_OK)
                    e = cudaErrorLaunchFailure;
            }
            h->launches += 2;
            cur = 1 - cur;
        }
    }
    return e == cudaSuccess ? LB_OK : cuda_fail("lb_adjoint_kinetic_coupled", e);
}

}  // extern "C"
