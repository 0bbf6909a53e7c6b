// f32x2.cuh -- the collision of two neighbouring nodes at once in Blackwell's
// packed FP32 arithmetic (add / sub / mul / fma .rn.f32x2: one instruction
// computes the same IEEE operation on the two 32-bit halves of a 64-bit
// register pair).
//
// The paired stream-collide kernels hold nodes x0 and x0 + 1 of a row in
// every thread and do the same arithmetic on both; here the two values of a
// quantity travel as one F2 (low half: node x0, high half: node x0 + 1), so
// the moment transform (Table 1, Eq. forward), the relaxation and forcing
// (Eq. lco_update, Sec. 3.7 Sigma), the Box-Muller scaling of the noise
// (Sec. 3.5) and the back transform (Eq. back_transformation) issue one
// instruction per operation for the pair instead of two.  Operations without
// a packed form (reciprocal, log2, rsqrt, sine / cosine, the Philox integer
// rounds, compares) run per half.  Every packed operation rounds each half
// exactly as the scalar operation would, so the results are those of
// d3q19.cuh / stream_collide.cuh's scalar code up to which multiply-adds the
// compiler fuses there.
#pragma once

#include <cstdint>

#include "d3q19.cuh"
#include "step_args.h"

namespace lbp {

struct F2 {
    unsigned long long v;
};

__device__ __forceinline__ F2 f2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ F2 f2s(float c) { return f2(c, c); }
__device__ __forceinline__ void split(F2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ float lo(F2 a)
{
    float l, h;
    split(a, l, h);
    return l;
}
__device__ __forceinline__ float hi(F2 a)
{
    float l, h;
    split(a, l, h);
    return h;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
// a * b + c, rounded once per half
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
__device__ __forceinline__ F2 fma2(F2 a, float b, F2 c) { return fma2(a, f2s(b), c); }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * f2s(b); }

// Forward transform m_k = sum_i e_ki n_i (Eq. forward, Table 1) of both nodes:
// the even / odd factorisation of lbd::forward.
__device__ __forceinline__ void forward2(const F2 n[19], F2 m[19])
{
    const F2 sx = n[1] + n[2], sy = n[3] + n[4], sz = n[5] + n[6];
    const F2 sa = n[7] + n[10], sb = n[8] + n[9];
    const F2 sc = n[11] + n[14], sd = n[12] + n[13];
    const F2 se = n[15] + n[18], sg = n[16] + n[17];
    const F2 dx = n[1] - n[2], dy = n[3] - n[4], dz = n[5] - n[6];
    const F2 pa = n[7] - n[10], pb = n[8] - n[9];
    const F2 pc = n[11] - n[14], pd = n[12] - n[13];
    const F2 pe = n[15] - n[18], pg = n[16] - n[17];

    const F2 A = sx + sy + sz;
    const F2 Dxy = sa + sb, Dyz = sc + sd, Dxz = se + sg;
    const F2 D = Dxy + Dyz + Dxz;
    const F2 t5 = (Dxy + Dxz) - (Dyz + Dyz);
    const F2 t6 = Dxy - Dxz;
    const F2 syz = sy + sz;
    const F2 sx2 = sx + sx;
    m[0] = n[0] + A + D;
    m[4] = D - n[0];
    m[5] = sx2 - syz + t5;
    m[6] = sy - sz + t6;
    m[7] = sa - sb;
    m[8] = sc - sd;
    m[9] = se - sg;
    m[16] = n[0] - (A + A) + D;
    m[17] = syz - sx2 + t5;
    m[18] = sz - sy + t6;

    const F2 Px = pa + pb, Qx = pe + pg;
    const F2 Py = pa - pb, Qy = pc + pd;
    const F2 Pz = pc - pd, Qz = pe - pg;
    const F2 hx = Px + Qx, hy = Py + Qy, hz = Pz + Qz;
    m[1] = dx + hx;
    m[2] = dy + hy;
    m[3] = dz + hz;
    m[10] = hx - (dx + dx);
    m[11] = hy - (dy + dy);
    m[12] = hz - (dz + dz);
    m[13] = Px - Qx;
    m[14] = Qy - Py;
    m[15] = Qz - Pz;
}

// Back transform n_i = a_i sum_k e_ki M_k (M_k = m_k / w_k) of both nodes:
// lbd::backward in packed form.
__device__ __forceinline__ void backward2(const F2 M[19], F2 n[19])
{
    const F2 A0 = f2s(lbd::kA0), A1 = f2s(lbd::kA1), A2 = f2s(lbd::kA2);
    const F2 M5x2 = M[5] + M[5], M16x2 = M[16] + M[16], M17x2 = M[17] + M[17];
    n[0] = A0 * (M[0] - M[4] + M[16]);
    {
        const F2 base = M[0] - M16x2;
        const F2 Ex = base + M5x2 - M17x2;
        const F2 Ox = M[1] - (M[10] + M[10]);
        const F2 Eyz = base - M[5] + M[17];
        const F2 Ey = Eyz + M[6] - M[18];
        const F2 Ez = Eyz - M[6] + M[18];
        const F2 Oy = M[2] - (M[11] + M[11]);
        const F2 Oz = M[3] - (M[12] + M[12]);
        n[1] = A1 * (Ex + Ox);
        n[2] = A1 * (Ex - Ox);
        n[3] = A1 * (Ey + Oy);
        n[4] = A1 * (Ey - Oy);
        n[5] = A1 * (Ez + Oz);
        n[6] = A1 * (Ez - Oz);
    }
    {
        const F2 base = M[0] + M[4] + M[16];
        const F2 Exy = base + M[5] + M[6] + M[17] + M[18];
        const F2 E7 = Exy + M[7], E8 = Exy - M[7];
        const F2 oxy1 = M[1] + M[10] + M[13];
        const F2 oxy2 = M[2] + M[11] - M[14];
        const F2 O7 = oxy1 + oxy2, O8 = oxy1 - oxy2;
        n[7] = A2 * (E7 + O7);
        n[10] = A2 * (E7 - O7);
        n[8] = A2 * (E8 + O8);
        n[9] = A2 * (E8 - O8);
        const F2 Eyz = base - M5x2 - M17x2;
        const F2 E11 = Eyz + M[8], E12 = Eyz - M[8];
        const F2 oyz2 = M[2] + M[11] + M[14];
        const F2 oyz3 = M[3] + M[12] - M[15];
        const F2 O11 = oyz2 + oyz3, O12 = oyz2 - oyz3;
        n[11] = A2 * (E11 + O11);
        n[14] = A2 * (E11 - O11);
        n[12] = A2 * (E12 + O12);
        n[13] = A2 * (E12 - O12);
        const F2 Exz = base + M[5] - M[6] + M[17] - M[18];
        const F2 E15 = Exz + M[9], E16 = Exz - M[9];
        const F2 oxz1 = M[1] + M[10] - M[13];
        const F2 oxz3 = M[3] + M[12] + M[15];
        const F2 O15 = oxz1 + oxz3, O16 = oxz1 - oxz3;
        n[15] = A2 * (E15 + O15);
        n[18] = A2 * (E15 - O15);
        n[16] = A2 * (E16 + O16);
        n[17] = A2 * (E16 - O16);
    }
}

// Box-Muller pairs of the two nodes (words (a0, b0) of node x0, (a1, b1) of
// node x0 + 1): the map of lbd::box_muller -- uniforms (2 (w >> 9) + 1) 2^-24
// from the mantissa bits, -2 ln v1 from the hardware log2 or the series near
// 1, the radius sqrt(-2 ln v1 var) as L rsqrt(L), the centred angle -- with
// the FP32 arithmetic packed and the special functions per half.
__device__ __forceinline__ void box_muller2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, F2 &g0, F2 &g1,
                                            F2 var)
{
    const F2 off = f2s(0.99999994039535522f);
    const F2 v1 = f2(__uint_as_float(0x3F800000u | (a0 >> 9)), __uint_as_float(0x3F800000u | (a1 >> 9))) - off;
    const F2 d1 = f2s(1.0f) - v1;
    const F2 w = (f2(__uint_as_float(0x3F800000u | (b0 >> 9)), __uint_as_float(0x3F800000u | (b1 >> 9))) - off) -
                 f2s(0.5f);
    float v1l, v1h, d1l, d1h;
    split(v1, v1l, v1h);
    split(d1, d1l, d1h);
    const F2 lg = f2(__log2f(v1l), __log2f(v1h)) * f2s(-1.3862943611198906f);
    F2 t = fma2(d1, f2s(1.0f / 6.0f), f2s(0.2f));
    t = fma2(d1, t, f2s(0.25f));
    t = fma2(d1, t, f2s(1.0f / 3.0f));
    t = fma2(d1, t, f2s(0.5f));
    t = fma2(d1, t, f2s(1.0f));
    const F2 ser = (d1 + d1) * t;
    float sl, sh, ll, lh;
    split(ser, sl, sh);
    split(lg, ll, lh);
    const F2 L = f2(d1l < 0.03125f ? sl : ll, d1h < 0.03125f ? sh : lh) * var;
    float Ll, Lh;
    split(L, Ll, Lh);
    const F2 nr = L * f2(-rsqrtf(Ll), -rsqrtf(Lh));  // -sqrt(L)
    const F2 ang = w * f2s(6.283185307179586f);
    float al, ah, s0, c0, s1, c1;
    split(ang, al, ah);
    __sincosf(al, &s0, &c0);
    __sincosf(ah, &s1, &c1);
    g0 = nr * f2(c0, c1);
    g1 = nr * f2(s0, s1);
}

// Where collide_moments2 takes its Philox round keys: ParamKeys reads the
// precomputed keys of one seed (kernel parameters: constant-bank operands);
// RunningKeys forms round r's keys as key + r W from the two key words (two
// adds a round, but only two registers: for kernels whose key is data, e.g.
// one per replica, and which would otherwise hold all twenty).  pair() runs
// the two nodes' counter blocks.
struct ParamKeys {
    const lbd::RoundKeys &rk;
    __device__ __forceinline__ void pair(const lbd::U4 &c0, const lbd::U4 &c1, lbd::U4 &r0, lbd::U4 &r1) const
    {
        r0 = lbd::philox10(c0, rk);
        r1 = lbd::philox10(c1, rk);
    }
};
struct RunningKeys {
    uint32_t k0, k1;
    __device__ __forceinline__ void pair(const lbd::U4 &c0, const lbd::U4 &c1, lbd::U4 &r0, lbd::U4 &r1) const
    {
        r0 = c0;
        r1 = c1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint32_t q0 = k0 + (uint32_t)r * lbd::kPhiloxW0, q1 = k1 + (uint32_t)r * lbd::kPhiloxW1;
            lbd::philox_round(r0, q0, q1);
            lbd::philox_round(r1, q0, q1);
        }
    }
};

// Collision of nodes node0, node0 + 1 (Sec. 3.4, 3.5, 3.7) from their
// moments m and force densities (fx, fy, fz) to the post-collision
// deviations out: lbi::collide_moments of each node, paired.
template <bool NOISE, class Keys>
__device__ __forceinline__ void collide_moments2k(const F2 m[19], F2 fx, F2 fy, F2 fz, const lbi::StepArgs &a,
                                                  const Keys &keys, uint32_t node0, uint32_t replica, F2 out[19])
{
    const F2 half = f2s(0.5f), three = f2s(3.0f);
    const F2 rho = f2s(a.rho0) + m[0];
    float rl, rh;
    split(rho, rl, rh);
    const F2 inv_rho = f2(__frcp_rn(rl), __frcp_rn(rh));
    const F2 ux = fma2(half, fx, m[1]) * inv_rho;
    const F2 uy = fma2(half, fy, m[2]) * inv_rho;
    const F2 uz = fma2(half, fz, m[3]) * inv_rho;

    const F2 uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const F2 u2 = uxx + uyy + uzz;
    const F2 meq4 = rho * u2;
    const F2 meq5 = rho * (uxx * three - u2);
    const F2 meq6 = rho * (uyy - uzz);
    const F2 ruy = rho * uy;
    const F2 meq7 = ruy * ux;
    const F2 meq8 = ruy * uz;
    const F2 meq9 = rho * uz * ux;
    const F2 uf = ux * fx + uy * fy + uz * fz;
    const F2 gs1 = f2s(1.0f + a.g_shear);
    const F2 hgs1 = f2s(0.5f * (1.0f + a.g_shear));
    const F2 F4 = f2s(1.0f + a.g_bulk) * uf;
    const F2 F5 = gs1 * (ux * fx * three - uf);
    const F2 F6 = gs1 * (uy * fy - uz * fz);
    const F2 F7 = hgs1 * (ux * fy + uy * fx);
    const F2 F8 = hgs1 * (uy * fz + uz * fy);
    const F2 F9 = hgs1 * (uz * fx + ux * fz);

    const F2 gb = f2s(a.g_bulk), gsh = f2s(a.g_shear);
    F2 M[19];
    M[0] = m[0];
    M[1] = (m[1] + fx) * three;
    M[2] = (m[2] + fy) * three;
    M[3] = (m[3] + fz) * three;
    M[4] = fma2(gb, m[4] - meq4, meq4 + F4) * lbd::inv_w(4);
    M[5] = fma2(gsh, m[5] - meq5, meq5 + F5) * lbd::inv_w(5);
    M[6] = fma2(gsh, m[6] - meq6, meq6 + F6) * lbd::inv_w(6);
    M[7] = fma2(gsh, m[7] - meq7, meq7 + F7) * lbd::inv_w(7);
    M[8] = fma2(gsh, m[8] - meq8, meq8 + F8) * lbd::inv_w(8);
    M[9] = fma2(gsh, m[9] - meq9, meq9 + F9) * lbd::inv_w(9);
    const F2 godd = f2s(a.g_odd), geven = f2s(a.g_even);
#pragma unroll
    for (int k = 10; k < 16; ++k) M[k] = m[k] * godd * lbd::inv_w(k);
#pragma unroll
    for (int k = 16; k < 19; ++k) M[k] = m[k] * geven * lbd::inv_w(k);

    if (NOISE) {
        // sqrt(mu rho w_k) phi_k r_k / w_k: (phi_k / sqrt(w_k)) times a Gaussian
        // of variance mu rho; the four Gaussians of each Philox block go into
        // their modes at once (r_4 .. r_18 = Gaussians 0 .. 14)
        const F2 var = a.noise_rho0 ? f2s(a.mu * a.rho0) : rho * a.mu;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            lbd::U4 r0, r1;
            keys.pair(lbd::U4{node0, a.step, (uint32_t)b, replica}, lbd::U4{node0 + 1u, a.step, (uint32_t)b, replica},
                      r0, r1);
            F2 g[4];
            box_muller2(r0.x, r0.y, r1.x, r1.y, g[0], g[1], var);
            box_muller2(r0.z, r0.w, r1.z, r1.w, g[2], g[3], var);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = 4 + 4 * b + j;
                if (k < 19) M[k] = fma2(g[j], a.amp[k - 4], M[k]);
            }
        }
    }

    backward2(M, out);
}

template <bool NOISE>
__device__ __forceinline__ void collide_moments2(const F2 m[19], F2 fx, F2 fy, F2 fz, const lbi::StepArgs &a,
                                                 const lbd::RoundKeys &rk, uint32_t node0, uint32_t replica,
                                                 F2 out[19])
{
    collide_moments2k<NOISE>(m, fx, fy, fz, a, ParamKeys{rk}, node0, replica, out);
}

}  // namespace lbp
