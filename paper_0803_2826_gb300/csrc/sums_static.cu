// sums_static.cu -- lb_moment_sums_static: the global moment sums of
// lb_moments, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application whose device memory
// is entirely reserved up front by another framework's pool, or a monitoring
// loop that must never block on, or fail in, an allocation in the middle of
// a long run.  They cannot create an lb_handle either (lb_create allocates
// its reduction scratch), so this entry point takes the population buffer and
// the parameters directly and allocates nothing.  Its reduction scratch is the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cuda.h>
#include <mutex>

#include "d3q19.cuh"
#include "lbf_internal.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticMaxBlocks = 4096;                 // scratch rows
constexpr size_t kStaticChunk = 65536;                 // nodes per block
constexpr size_t kStaticMaxNodes = kStaticChunk * kStaticMaxBlocks;  // 2^28 nodes

// Block partial sums: kStaticMaxBlocks x LB_NSUMS doubles (1.2 MiB).  Every
// call overwrites the rows it uses before the final pass reads them.
static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks * LB_NSUMS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;

// The array's device address, per device, together with the unique id of
// the context it was looked up in: after cudaDeviceReset (or under another
// context) the address of the old context is no longer valid, so a changed
// id repeats the lookup.
struct ScratchAddr {
    unsigned long long ctx_id;
    double *ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// Unique id of the calling thread's current context, through the driver
// entry points the runtime exposes (no link against the driver library).
// Returns false when there is no current context or the driver lacks the
// calls.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        resolved = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Block b reduces nodes [b * chunk, min(N, (b + 1) * chunk)) of the
// pre-collision state: dm_k = sum_i e_ki (n_i - a_i rho0) and dm_k^2 over fluid
// nodes, the same quantities as lb_moments' sums (Table 1 basis).
template <int DT>
__global__ void __launch_bounds__(kStaticThreads)
    k_sums_static(const typename lbd::Store<DT>::T *__restrict__ src, double *partials, lbi::StepArgs a)
{
    using S = lbd::Store<DT>;
    const size_t N = a.nn;
    const bool walls = a.z0 > 0;
    const size_t begin = (size_t)blockIdx.x * kStaticChunk;
    const size_t end = begin + kStaticChunk < N ? begin + kStaticChunk : N;
    float acc[2 * 19];
#pragma unroll
    for (int k = 0; k < 38; ++k) acc[k] = 0.0f;
    for (size_t s = begin + threadIdx.x; s < end; s += kStaticThreads) {
        const size_t row = s / (size_t)a.nx;
        const int x = (int)(s - row * (size_t)a.nx);
        const int z = (int)(row / (size_t)a.ny);
        const int y = (int)(row - (size_t)z * (size_t)a.ny);
        if (z < a.z0 || z >= a.z1) continue;
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
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            acc[k] += m[k];
            acc[19 + k] = fmaf(m[k], m[k], acc[19 + k]);
        }
    }
    __shared__ double red[kStaticThreads / 32][38];
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
        for (int w = 0; w < kStaticThreads / 32; ++w) v += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 38 + threadIdx.x] = v;
    }
}

__global__ void k_sums_static_final(const double *partials, int nblocks, double *sums)
{
    const int k = threadIdx.x;
    if (k >= 38) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * 38 + k];
    sums[k] = v;
}

// Device address of the static scratch on the current device, looked up on
// the first call in a context (once per device while its context lives).
lb_status static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbi::cuda_fail("lb_moment_sums_static (cudaGetDevice)", e);
    if (dev < 0 || dev >= kMaxDevices) {
        lbi::set_error("lb_moment_sums_static: device %d beyond the %d supported", dev, kMaxDevices);
        return LB_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    ScratchAddr &c = g_scratch[dev];
    if (!c.ptr || !have_id || c.ctx_id != id) {
        double *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_static_partials);
        if (e != cudaSuccess) return lbi::cuda_fail("lb_moment_sums_static (cudaGetSymbolAddress)", e);
        if (!ptr) {
            lbi::set_error("lb_moment_sums_static: cudaGetSymbolAddress returned a null address");
            return LB_ECUDA;
        }
        // the lookup made the device's primary context current if none was
        unsigned long long id2 = 0;
        c.ctx_id = current_context_id(&id2) ? id2 : 0;
        c.ptr = ptr;
    }
    *out = c.ptr;
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_moment_sums_static(const lb_params *p, const void *pops, double *sums, void *stream)
{
    if (!p || !pops || !sums) {
        lbi::set_error("lb_moment_sums_static: NULL argument");
        return LB_EINVAL;
    }
    const size_t pitch = lb_plane_pitch(p);  // also validates the parameters
    if (pitch == 0) return LB_EINVAL;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    if (N > kStaticMaxNodes) {
        lbi::set_error("lb_moment_sums_static: %zu nodes exceed the static scratch limit of %zu nodes", N,
                       kStaticMaxNodes);
        return LB_EINVAL;
    }
    double *partials = nullptr;
    lb_status st = static_scratch(&partials);
    if (st != LB_OK) return st;
    // the handle-free equivalent of make_args for the fields the kernel reads
    lb_handle tmp{};
    tmp.p = *p;
    tmp.n_nodes = N;
    tmp.pitch = pitch;
    const lbi::StepArgs a = lbi::make_args(&tmp);
    const int blocks = (int)((N + kStaticChunk - 1) / kStaticChunk);
    cudaStream_t s = (cudaStream_t)stream;
    switch (p->dtype) {
    case LB_F32:
        k_sums_static<0><<<blocks, kStaticThreads, 0, s>>>(static_cast<const float *>(pops), partials, a);
        break;
    case LB_F16:
        k_sums_static<1><<<blocks, kStaticThreads, 0, s>>>(static_cast<const __half *>(pops), partials, a);
        break;
    default:
        k_sums_static<2><<<blocks, kStaticThreads, 0, s>>>(static_cast<const __nv_bfloat16 *>(pops), partials, a);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lbi::cuda_fail("lb_moment_sums_static", e);
    k_sums_static_final<<<1, 64, 0, s>>>(partials, blocks, sums);
    e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : lbi::cuda_fail("lb_moment_sums_static", e);
}
