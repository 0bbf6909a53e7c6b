// d3q19.cuh -- device-side lattice algebra for the fluctuating D3Q19 update.
//
// Velocity order (library convention): 0 rest; 1 +x, 2 -x, 3 +y, 4 -y,
// 5 +z, 6 -z; 7 (1,1,0), 8 (1,-1,0), 9 (-1,1,0), 10 (-1,-1,0), 11 (0,1,1),
// 12 (0,1,-1), 13 (0,-1,1), 14 (0,-1,-1), 15 (1,0,1), 16 (1,0,-1),
// 17 (-1,0,1), 18 (-1,0,-1).  Opposite pairs: (1,2) (3,4) (5,6) (7,10)
// (8,9) (11,14) (12,13) (15,18) (16,17).
//
// The moment transform of Sec. 3.4 (Table 1, q = a) is written out in
// even/odd form: for an opposite pair (i, i') the even moments (0, 4..9,
// 16..18) see only n_i + n_i' and the odd ones (1..3, 10..15) only
// n_i - n_i'.  All basis entries are small integers, so the forward
// transform is additions only and the back transform
// n_i = a_i sum_k e_ki m_k / w_k (Eq. (back_transformation)) needs one scale
// per mode plus additions.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbd {

// Weights a^{c_i} (Sec. 3.3) and norms w_k (Table 1).
constexpr float kA0 = 1.0f / 3.0f;
constexpr float kA1 = 1.0f / 18.0f;
constexpr float kA2 = 1.0f / 36.0f;

__host__ __device__ constexpr float weight(int i) { return i == 0 ? kA0 : (i <= 6 ? kA1 : kA2); }

// 1 / w_k.
__host__ __device__ constexpr float inv_w(int k)
{
    return k == 0 ? 1.0f
         : k <= 3 ? 3.0f
         : k == 4 ? 1.5f
         : k == 5 ? 0.75f
         : k == 6 ? 2.25f
         : k <= 9 ? 9.0f
         : k <= 12 ? 1.5f
         : k <= 15 ? 4.5f
         : k == 16 ? 0.5f
         : k == 17 ? 0.75f
         : 2.25f;
}

// sqrt(1 / w_k)
__host__ __device__ constexpr float sqrt_inv_w(int k)
{
    return k == 0 ? 1.0f
         : k <= 3 ? 1.7320508075688772f
         : k == 4 ? 1.2247448713915890f
         : k == 5 ? 0.8660254037844386f
         : k == 6 ? 1.5f
         : k <= 9 ? 3.0f
         : k <= 12 ? 1.2247448713915890f
         : k <= 15 ? 2.1213203435596424f
         : k == 16 ? 0.7071067811865476f
         : k == 17 ? 0.8660254037844386f
         : 1.5f;
}

// w_k
__host__ __device__ constexpr float norm_w(int k)
{
    return k == 0 ? 1.0f
         : k <= 3 ? (1.0f / 3.0f)
         : k == 4 ? (2.0f / 3.0f)
         : k == 5 ? (4.0f / 3.0f)
         : k == 6 ? (4.0f / 9.0f)
         : k <= 9 ? (1.0f / 9.0f)
         : k <= 12 ? (2.0f / 3.0f)
         : k <= 15 ? (2.0f / 9.0f)
         : k == 16 ? 2.0f
         : k == 17 ? (4.0f / 3.0f)
         : (4.0f / 9.0f);
}

// Lattice velocity components as compile-time functions of i.
__host__ __device__ constexpr int cx(int i)
{
    return (i == 1 || i == 7 || i == 8 || i == 15 || i == 16) ? 1
         : (i == 2 || i == 9 || i == 10 || i == 17 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i)
{
    return (i == 3 || i == 7 || i == 9 || i == 11 || i == 12) ? 1
         : (i == 4 || i == 8 || i == 10 || i == 13 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i)
{
    return (i == 5 || i == 11 || i == 13 || i == 15 || i == 17) ? 1
         : (i == 6 || i == 12 || i == 14 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int opposite(int i)
{
    return i == 0 ? 0
         : i <= 6 ? (i % 2 == 1 ? i + 1 : i - 1)
         : i == 7 ? 10 : i == 8 ? 9 : i == 9 ? 8 : i == 10 ? 7
         : i == 11 ? 14 : i == 12 ? 13 : i == 13 ? 12 : i == 14 ? 11
         : i == 15 ? 18 : i == 16 ? 17 : i == 17 ? 16 : 15;
}

// Forward transform m_k = sum_i e_ki n_i (Eq. (forward)).
__device__ __forceinline__ void forward(const float n[19], float m[19])
{
    // even (pair sums) and odd (pair differences) parts
    const float sx = n[1] + n[2], sy = n[3] + n[4], sz = n[5] + n[6];
    const float sa = n[7] + n[10], sb = n[8] + n[9];     // (1,1,0), (1,-1,0)
    const float sc = n[11] + n[14], sd = n[12] + n[13];  // (0,1,1), (0,1,-1)
    const float se = n[15] + n[18], sg = n[16] + n[17];  // (1,0,1), (1,0,-1)
    const float dx = n[1] - n[2], dy = n[3] - n[4], dz = n[5] - n[6];
    const float pa = n[7] - n[10], pb = n[8] - n[9];
    const float pc = n[11] - n[14], pd = n[12] - n[13];
    const float pe = n[15] - n[18], pg = n[16] - n[17];

    const float A = sx + sy + sz;
    const float Dxy = sa + sb, Dyz = sc + sd, Dxz = se + sg;
    const float D = Dxy + Dyz + Dxz;
    const float t5 = Dxy - 2.0f * Dyz + Dxz;
    const float t6 = Dxy - Dxz;
    const float syz = sy + sz;
    m[0] = n[0] + A + D;
    m[4] = D - n[0];
    m[5] = 2.0f * sx - syz + t5;
    m[6] = sy - sz + t6;
    m[7] = sa - sb;
    m[8] = sc - sd;
    m[9] = se - sg;
    m[16] = n[0] - 2.0f * A + D;
    m[17] = syz - 2.0f * sx + t5;
    m[18] = sz - sy + t6;

    const float Px = pa + pb, Qx = pe + pg;
    const float Py = pa - pb, Qy = pc + pd;
    const float Pz = pc - pd, Qz = pe - pg;
    const float hx = Px + Qx, hy = Py + Qy, hz = Pz + Qz;
    m[1] = dx + hx;
    m[2] = dy + hy;
    m[3] = dz + hz;
    m[10] = hx - 2.0f * dx;
    m[11] = hy - 2.0f * dy;
    m[12] = hz - 2.0f * dz;
    m[13] = Px - Qx;
    m[14] = Qy - Py;
    m[15] = Qz - Pz;
}

// Back transform n_i = a_i sum_k e_ki M_k with M_k = m_k / w_k already scaled.
__device__ __forceinline__ void backward(const float M[19], float n[19])
{
    // rest
    n[0] = kA0 * (M[0] - M[4] + M[16]);
    // axes: even part E, odd part O; n_+ = a (E + O), n_- = a (E - O)
    {
        const float base = M[0] - 2.0f * M[16];
        const float Ex = base + 2.0f * M[5] - 2.0f * M[17];
        const float Ox = M[1] - 2.0f * M[10];
        const float Eyz = base - M[5] + M[17];
        const float Ey = Eyz + M[6] - M[18];
        const float Ez = Eyz - M[6] + M[18];
        const float Oy = M[2] - 2.0f * M[11];
        const float Oz = M[3] - 2.0f * M[12];
        n[1] = kA1 * (Ex + Ox);
        n[2] = kA1 * (Ex - Ox);
        n[3] = kA1 * (Ey + Oy);
        n[4] = kA1 * (Ey - Oy);
        n[5] = kA1 * (Ez + Oz);
        n[6] = kA1 * (Ez - Oz);
    }
    // diagonals
    {
        const float base = M[0] + M[4] + M[16];
        // xy plane
        const float Exy = base + M[5] + M[6] + M[17] + M[18];
        const float E7 = Exy + M[7], E8 = Exy - M[7];
        const float oxy1 = M[1] + M[10] + M[13];  // x-odd part seen from the xy plane
        const float oxy2 = M[2] + M[11] - M[14];  // y-odd part seen from the xy plane
        const float O7 = oxy1 + oxy2, O8 = oxy1 - oxy2;
        n[7] = kA2 * (E7 + O7);
        n[10] = kA2 * (E7 - O7);
        n[8] = kA2 * (E8 + O8);
        n[9] = kA2 * (E8 - O8);
        // yz plane
        const float Eyz = base - 2.0f * M[5] - 2.0f * M[17];
        const float E11 = Eyz + M[8], E12 = Eyz - M[8];
        const float oyz2 = M[2] + M[11] + M[14];  // y-odd part seen from the yz plane
        const float oyz3 = M[3] + M[12] - M[15];  // z-odd part seen from the yz plane
        const float O11 = oyz2 + oyz3, O12 = oyz2 - oyz3;
        n[11] = kA2 * (E11 + O11);
        n[14] = kA2 * (E11 - O11);
        n[12] = kA2 * (E12 + O12);
        n[13] = kA2 * (E12 - O12);
        // xz plane
        const float Exz = base + M[5] - M[6] + M[17] - M[18];
        const float E15 = Exz + M[9], E16 = Exz - M[9];
        const float oxz1 = M[1] + M[10] - M[13];  // x-odd part seen from the xz plane
        const float oxz3 = M[3] + M[12] + M[15];  // z-odd part seen from the xz plane
        const float O15 = oxz1 + oxz3, O16 = oxz1 - oxz3;
        n[15] = kA2 * (E15 + O15);
        n[18] = kA2 * (E15 - O15);
        n[16] = kA2 * (E16 + O16);
        n[17] = kA2 * (E16 - O16);
    }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): multipliers 0xD2511F53, 0xCD9E8D57,
// key increments 0x9E3779B9, 0xBB67AE85, ten rounds.  The 64-bit product
// gives both halves of each multiply in one instruction.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__host__ __device__ __forceinline__ void philox_round(U4 &c, uint32_t k0, uint32_t k1)
{
    const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c.x;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c.z;
    c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
}

// Key schedule computed in the loop (particle kernels: one call per thread).
__host__ __device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Round keys precomputed on the host (kernel parameters, so every XOR with a
// key reads the constant bank).
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ __forceinline__ U4 philox10(U4 c, const RoundKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) philox_round(c, rk.k0[r], rk.k1[r]);
    return c;
}

inline RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

// Uniform in (0,1): (2 (x >> 9) + 1) 2^-24.  The top 23 bits become the
// mantissa of a float in [1, 2); subtracting 1 - 2^-24 is exact (Sterbenz)
// and yields the odd multiple of 2^-24, so no integer-to-float conversion.
__device__ __forceinline__ float uniform01(uint32_t x)
{
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.99999994039535522f;
}

// -2 ln v for a uniform v = (2k + 1) 2^-24 given with d = 1 - v (both
// exact), without branches: the hardware log2 (absolute error below 2^-22.6
// on [0.5, 2], 2 ulp elsewhere) where d >= 2^-5, so |ln v| >= 0.031; below
// that, where an absolute error would be large against ln v, the Taylor
// series -ln(1 - d) = d + d^2/2 + ... + d^6/6 (remainder < 2^-32 relative).
__device__ __forceinline__ float neg2log(float v, float d)
{
    const float lg = -1.3862943611198906f * __log2f(v);  // -2 ln 2 log2 v
    float t = fmaf(d, 1.0f / 6.0f, 0.2f);
    t = fmaf(d, t, 0.25f);
    t = fmaf(d, t, 1.0f / 3.0f);
    t = fmaf(d, t, 0.5f);
    t = fmaf(d, t, 1.0f);
    const float s = (2.0f * d) * t;
    return d < 0.03125f ? s : lg;
}

// Box-Muller pair from two raw words: sqrt(-2 ln v1) (cos, sin)(2 pi v2).
// The angle is centred, 2 pi v2 = pi + 2 pi (v2 - 1/2) with v2 - 1/2 exact,
// so the hardware sine / cosine see an argument in (-pi, pi), where their
// absolute error is below 2^-21; cos and sin of the shifted angle change sign.
// With var != 1 the pair has variance var (the radius is sqrt(-2 ln v1 var)).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &g0, float &g1, float var = 1.0f)
{
    const float v1 = uniform01(a);
    const float d1 = 1.0f - v1;  // exact for v1 >= 1/2, the only range where it is used
    const float w = uniform01(b) - 0.5f;
    const float L = neg2log(v1, d1) * var;  // -2 ln v1 >= 2^-23
    const float r = L * rsqrtf(L);
    float s, c;
    __sincosf(6.283185307179586f * w, &s, &c);
    g0 = -r * c;
    g1 = -r * s;
}

// Sixteen Gaussians of variance var for counter word 0, step, domain,
// replica: Philox blocks b = 0..3 with counter (w0, step, domain<<8 | b, replica).
__device__ __forceinline__ void gaussians16(const RoundKeys &rk, uint32_t w0, uint32_t step, uint32_t domain,
                                            uint32_t replica, float var, float g[16])
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const U4 r = philox10(U4{w0, step, (domain << 8) | (uint32_t)b, replica}, rk);
        box_muller(r.x, r.y, g[4 * b + 0], g[4 * b + 1], var);
        box_muller(r.z, r.w, g[4 * b + 2], g[4 * b + 3], var);
    }
}

// ---------------------------------------------------------------------------
// Population storage: FP32 deviations, or deviations * scale in FP16 / BF16.
// ---------------------------------------------------------------------------
template <int DT>
struct Store;

template <>
struct Store<0> {
    using T = float;
    static __device__ __forceinline__ float load(const T *p, float /*inv_scale*/) { return __ldg(p); }
    static __device__ __forceinline__ float cvt(T v, float /*inv_scale*/) { return v; }
    static __device__ __forceinline__ T pack(float x, float /*scale*/) { return x; }
};

template <>
struct Store<1> {
    using T = __half;
    static __device__ __forceinline__ float load(const T *p, float inv_scale)
    {
        return __half2float(__ldg(p)) * inv_scale;
    }
    static __device__ __forceinline__ float cvt(T v, float inv_scale) { return __half2float(v) * inv_scale; }
    static __device__ __forceinline__ T pack(float x, float scale) { return __float2half_rn(x * scale); }
};

template <>
struct Store<2> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const T *p, float inv_scale)
    {
        return __bfloat162float(__ldg(p)) * inv_scale;
    }
    static __device__ __forceinline__ float cvt(T v, float inv_scale)
    {
        return __bfloat162float(v) * inv_scale;
    }
    static __device__ __forceinline__ T pack(float x, float scale) { return __float2bfloat16_rn(x * scale); }
};

}  // namespace lbd
