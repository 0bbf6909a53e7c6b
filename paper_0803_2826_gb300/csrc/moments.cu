// moments.cu -- state initialisation / conversion and the hydrodynamic
// moments of the pre-collision state.
//
//   init        n^eq(rho, u) of Eq. (original_equil_distrib), in FP64, stored
//               as deviations n - a rho0 in the storage format
//   moments     rho = m_0, j = m_1..3 + f/2, pi from m_0, m_4..m_9
//               (Sec. 3.4 Eqs. (hmodes_beg)-(hmodes_end); Sec. 3.7 for j)
//   sums        sum over fluid nodes of dm_k and dm_k^2 with a deterministic
//               two-pass reduction (block partials in scratch, then one
//               block adds the partials in block order)
#include <cstdio>

#include "d3q19.cuh"
#include "lbf_internal.h"

namespace lbi {

namespace {

__device__ __forceinline__ void node_xyz(size_t s, int nx, int ny, int &x, int &y, int &z)
{
    const size_t row = s / (size_t)nx;
    x = (int)(s - row * (size_t)nx);
    z = (int)(row / (size_t)ny);
    y = (int)(row - (size_t)z * (size_t)ny);
}

template <int DT>
__global__ void k_init_equilibrium(typename lbd::Store<DT>::T *dst, const double *rho, const double *u,
                                   const StepArgs a)
{
    using S = lbd::Store<DT>;
    const size_t N = a.nn;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N;
         s += (size_t)gridDim.x * blockDim.x) {
        const double r = rho ? rho[s] : (double)a.rho0;
        const double ux = u ? u[s] : 0.0, uy = u ? u[N + s] : 0.0, uz = u ? u[2 * N + s] : 0.0;
        const double u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double ai = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            const double cu = ux * lbd::cx(i) + uy * lbd::cy(i) + uz * lbd::cz(i);
            const double dev = ai * (r - (double)a.rho0) + ai * r * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
            dst[(size_t)i * a.pitch + s] = S::pack((float)dev, a.scale);
        }
    }
}

template <int DT>
__global__ void k_set_populations(typename lbd::Store<DT>::T *dst, const double *n, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const size_t N = a.nn;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N;
         s += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double ai = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            const double dev = n[(size_t)i * N + s] - ai * (double)a.rho0;
            dst[(size_t)i * a.pitch + s] = S::pack((float)dev, a.scale);
        }
    }
}

template <int DT>
__global__ void k_get_populations(const typename lbd::Store<DT>::T *src, double *n, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const size_t N = a.nn;
    const size_t plane = (size_t)a.nx * a.ny;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N;
         s += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(s / plane);
        const bool solid = z < a.z0 || z >= a.z1;  // wall nodes hold no state: the rest state
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double ai = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            const float dev = solid ? 0.0f : S::cvt(src[(size_t)i * a.pitch + s], a.inv_scale);
            n[(size_t)i * N + s] = ai * (double)a.rho0 + (double)dev;
        }
    }
}

constexpr int kRedThreads = 256;

template <int DT>
__global__ void __launch_bounds__(kRedThreads)
    k_moments(const typename lbd::Store<DT>::T *__restrict__ src, const float *__restrict__ ffield, float *rho_out,
              float *j_out, float *pi_out, double *partials, const StepArgs a)
{
    using S = lbd::Store<DT>;
    const size_t N = a.nn;
    const bool walls = a.z0 > 0;
    // per-thread partial sums in FP32 (a thread sees ~N / grid nodes); the
    // block and grid levels add in FP64
    float acc[2 * 19];
#pragma unroll
    for (int k = 0; k < 38; ++k) acc[k] = 0.0f;

    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N;
         s += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(s, a.nx, a.ny, x, y, z);
        if (z < a.z0 || z >= a.z1) {  // solid wall plane
            if (rho_out) rho_out[s] = a.rho0;
            if (j_out) for (int d = 0; d < 3; ++d) j_out[d * N + s] = 0.0f;
            if (pi_out) for (int c = 0; c < 6; ++c) pi_out[c * N + s] = 0.0f;
            continue;
        }
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
        float n[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int sx = lbd::cx(i) == 1 ? xm : (lbd::cx(i) == -1 ? xp : x);
            const int sy = lbd::cy(i) == 1 ? ym : (lbd::cy(i) == -1 ? yp : y);
            const int sz = lbd::cz(i) == 1 ? zm : (lbd::cz(i) == -1 ? zp : z);
            const bool bounce = walls && lbd::cz(i) != 0 && (sz == 0 || sz == a.nz - 1);
            const size_t off = bounce ? ((size_t)lbd::opposite(i) * a.pitch + s)
                                      : ((size_t)i * a.pitch + ((size_t)sz * a.ny + sy) * a.nx + sx);
            n[i] = S::cvt(src[off], a.inv_scale);
        }
        float m[19];
        lbd::forward(n, m);
        const float rho = a.rho0 + m[0];
        if (rho_out) rho_out[s] = rho;
        if (j_out) {
            float fx = a.fx, fy = a.fy, fz = a.fz;
            if (ffield) {
                fx += ffield[s];
                fy += ffield[N + s];
                fz += ffield[2 * N + s];
            }
            j_out[s] = m[1] + 0.5f * fx;
            j_out[N + s] = m[2] + 0.5f * fy;
            j_out[2 * N + s] = m[3] + 0.5f * fz;
        }
        if (pi_out) {
            pi_out[s] = (rho + m[4] + m[5]) * (1.0f / 3.0f);
            pi_out[N + s] = (2.0f * rho + 2.0f * m[4] - m[5] + 3.0f * m[6]) * (1.0f / 6.0f);
            pi_out[2 * N + s] = (2.0f * rho + 2.0f * m[4] - m[5] - 3.0f * m[6]) * (1.0f / 6.0f);
            pi_out[3 * N + s] = m[7];
            pi_out[4 * N + s] = m[8];
            pi_out[5 * N + s] = m[9];
        }
        if (partials) {
#pragma unroll
            for (int k = 0; k < 19; ++k) {
                acc[k] += m[k];
                acc[19 + k] = fmaf(m[k], m[k], acc[19 + k]);
            }
        }
    }
    if (!partials) return;

    // block reduction in a fixed order: warp shuffles, then warps in order
    __shared__ double red[kRedThreads / 32][38];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 38; ++k) {
        double v = (double)acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 38) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 38 + threadIdx.x] = v;
    }
}

__global__ void k_sum_partials(const double *partials, int nblocks, double *sums, unsigned int *err)
{
    const int k = threadIdx.x;
    if (k >= 38) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * 38 + k];
    sums[k] = v;
    if (!isfinite(v)) atomicOr(err, LB_DERR_NONFINITE);
}

int grid_for(size_t N, int cap)
{
    size_t g = (N + kRedThreads - 1) / kRedThreads;
    if (g > (size_t)cap) g = (size_t)cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

#define LBI_DT_SWITCH(DTV, CALL)                  \
    switch (DTV) {                                \
    case LB_F32: { constexpr int DT = 0; CALL; } break;  \
    case LB_F16: { constexpr int DT = 1; CALL; } break;  \
    default: { constexpr int DT = 2; CALL; } break;      \
    }

cudaError_t launch_init_equilibrium(const lb_handle *h, void *dst, const double *rho, const double *u)
{
    const StepArgs a = make_args(h);
    const int g = grid_for(a.nn, 8 * device_sm_count());
    LBI_DT_SWITCH(h->p.dtype,
                  (k_init_equilibrium<DT><<<g, kRedThreads, 0, h->stream>>>(
                      static_cast<typename lbd::Store<DT>::T *>(dst), rho, u, a)));
    return cudaGetLastError();
}

cudaError_t launch_set_populations(const lb_handle *h, void *dst, const double *n)
{
    const StepArgs a = make_args(h);
    const int g = grid_for(a.nn, 8 * device_sm_count());
    LBI_DT_SWITCH(h->p.dtype, (k_set_populations<DT><<<g, kRedThreads, 0, h->stream>>>(
                                  static_cast<typename lbd::Store<DT>::T *>(dst), n, a)));
    return cudaGetLastError();
}

cudaError_t launch_get_populations(const lb_handle *h, const void *src, double *n)
{
    const StepArgs a = make_args(h);
    const int g = grid_for(a.nn, 8 * device_sm_count());
    LBI_DT_SWITCH(h->p.dtype, (k_get_populations<DT><<<g, kRedThreads, 0, h->stream>>>(
                                  static_cast<const typename lbd::Store<DT>::T *>(src), n, a)));
    return cudaGetLastError();
}

cudaError_t launch_moments(const lb_handle *h, const void *src, float *rho, float *j, float *pi, double *sums)
{
    const StepArgs a = make_args(h);
    const int g = grid_for(a.nn, h->red_blocks);
    double *partials = sums ? h->d_partials : nullptr;
    LBI_DT_SWITCH(h->p.dtype, (k_moments<DT><<<g, kRedThreads, 0, h->stream>>>(
                                  static_cast<const typename lbd::Store<DT>::T *>(src), h->force, rho, j,
                                  pi, partials, a)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !sums) return e;
    k_sum_partials<<<1, 64, 0, h->stream>>>(h->d_partials, g, sums, h->d_err);
    return cudaGetLastError();
}

}  // namespace lbi
