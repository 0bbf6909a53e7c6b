// step_sums.cu -- the moment sums of lb_step_sums: the stream-collide
// launch of the step writes one row of 38 partial sums per block (the
// pre-collision moments of its nodes, Sec. 3.4 Table 1, and their squares);
// passes of a fixed-order row reduction turn them into the 38 sums, so the
// result does not depend on scheduling.  The arithmetic is FP32 with Kahan
// compensation (FP64 arithmetic is slow on this part); the result is stored
// as FP64.
#include "stream_collide.cuh"

namespace lbi {

namespace {

constexpr int kRows = 8;           // rows summed side by side in a block
constexpr int kRowsPerBlock = 256; // rows one block reduces to one

struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// out[b][k] = sum over rows r of block b of in[r][k], r in
// [b kRowsPerBlock, (b + 1) kRowsPerBlock) and below nrows; thread (j, k)
// takes rows j, j + kRows, ... of the block, then the kRows values are added
// in order.  Contiguous threads read contiguous row entries.  The last pass
// (one block) writes FP64.
__global__ void __launch_bounds__(38 * kRows) k_reduce_rows(const float *in, size_t nrows, float *out,
                                                             double *final_out, unsigned int *err)
{
    __shared__ float part[kRows][38];
    const int k = threadIdx.x % 38, j = threadIdx.x / 38;
    const size_t r0 = (size_t)blockIdx.x * kRowsPerBlock;
    constexpr int kPer = kRowsPerBlock / kRows;
    float x[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {  // all loads first, then the adds in row order
        const size_t r = r0 + j + (size_t)q * kRows;
        x[q] = r < nrows ? in[r * 38 + k] : 0.0f;
    }
    Kahan v;
#pragma unroll
    for (int q = 0; q < kPer; ++q) v.add(x[q]);
    part[j][k] = v.s;
    __syncthreads();
    if (j == 0) {
        Kahan t;
#pragma unroll
        for (int q = 0; q < kRows; ++q) t.add(part[q][k]);
        if (final_out) {
            final_out[k] = (double)t.s;
            if (!isfinite(t.s)) atomicOr(err, LB_DERR_NONFINITE);
        } else {
            out[(size_t)blockIdx.x * 38 + k] = t.s;
        }
    }
}

}  // namespace

size_t sc_block_count(const lb_handle *h)
{
    const dim3 g = sc_grid(h);
    return (size_t)g.x * g.y * g.z;
}

size_t step_sums_scratch(size_t nblocks)
{
    size_t rows = nblocks, total = 0;
    do {
        rows = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
        total += rows;
    } while (rows > 1);
    return total * 38;
}

// partials: [nblocks][38]; scratch: step_sums_scratch(nblocks) floats.
cudaError_t reduce_step_sums(const lb_handle *h, const float *partials, size_t nblocks, float *scratch,
                             double *sums)
{
    const float *in = partials;
    size_t rows = nblocks;
    float *buf = scratch;
    do {
        const size_t out_rows = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
        const bool last = out_rows == 1;
        k_reduce_rows<<<(unsigned int)out_rows, 38 * kRows, 0, h->stream>>>(in, rows, buf, last ? sums : nullptr,
                                                                            h->d_err);
        in = buf;
        buf += out_rows * 38;
        rows = out_rows;
    } while (rows > 1);
    return cudaGetLastError();
}

}  // namespace lbi
