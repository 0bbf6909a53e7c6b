// noise.cu -- exposes the kernels' Philox4x32-10 words and Box-Muller
// Gaussians (the noise source of Sec. 3.5 and Sec. 4.5) for verification.
#include "d3q19.cuh"
#include "lbf_internal.h"

namespace {

__global__ void k_noise_words(uint32_t k0, uint32_t k1, uint32_t replica, uint32_t step, uint32_t domain,
                              uint32_t index0, int count, int nblocks, uint32_t *words, float *gauss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    for (int b = 0; b < nblocks; ++b) {
        const lbd::U4 r = lbd::philox10(lbd::U4{index0 + (uint32_t)q, step, (domain << 8) | (uint32_t)b, replica}, k0, k1);
        const size_t o = ((size_t)q * nblocks + b) * 4;
        words[o] = r.x;
        words[o + 1] = r.y;
        words[o + 2] = r.z;
        words[o + 3] = r.w;
        if (gauss) {
            lbd::box_muller(r.x, r.y, gauss[o], gauss[o + 1]);
            lbd::box_muller(r.z, r.w, gauss[o + 2], gauss[o + 3]);
        }
    }
}

__global__ void k_box_muller(const uint32_t *words, int npairs, float *gauss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    lbd::box_muller(words[2 * q], words[2 * q + 1], gauss[2 * q], gauss[2 * q + 1]);
}

}  // namespace

extern "C" lb_status lb_box_muller(const uint32_t *words, int npairs, float *gauss, void *stream)
{
    if (npairs < 0 || (npairs > 0 && (!words || !gauss))) {
        lbi::set_error("lb_box_muller: need npairs >= 0 and both buffers");
        return LB_EINVAL;
    }
    if (npairs == 0) return LB_OK;
    const int threads = 256;
    k_box_muller<<<(npairs + threads - 1) / threads, threads, 0, (cudaStream_t)stream>>>(words, npairs, gauss);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : lbi::cuda_fail("lb_box_muller", e);
}

extern "C" lb_status lb_noise_words(uint64_t seed, uint32_t replica, uint32_t step, uint32_t domain,
                                    uint32_t index0, int count, int nblocks, uint32_t *words, float *gauss,
                                    void *stream)
{
    if (count < 0 || nblocks < 1 || nblocks > 4 || (count > 0 && !words)) {
        lbi::set_error("lb_noise_words: need count >= 0, 1 <= nblocks <= 4 and a words buffer");
        return LB_EINVAL;
    }
    if (count == 0) return LB_OK;
    const int threads = 128;
    k_noise_words<<<(count + threads - 1) / threads, threads, 0, (cudaStream_t)stream>>>(
        (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), replica, step, domain, index0, count, nblocks,
        words, gauss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : lbi::cuda_fail("lb_noise_words", e);
}
