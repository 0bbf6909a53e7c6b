// step_args.h -- the constants every update kernel receives by value (a
// kernel's view of the handle: geometry, relaxation, noise and force).
#pragma once

#include <cstddef>
#include <cstdint>

#include "d3q19.cuh"
#include "lbfluct.h"

namespace lbi {

// Geometry and physics constants a kernel launch needs, in FP32 where the
// kernels compute in FP32.
struct StepArgs {
    int nx, ny, nz;
    int z0, z1;            // fluid z-range [z0, z1)
    size_t pitch;          // elements per population plane
    size_t nn;             // nodes nx*ny*nz (component stride of caller fields)
    float rho0;
    float kT;
    float mu;              // kT / c_s^2
    float g_shear, g_bulk, g_odd, g_even;
    float phi_shear, phi_bulk, phi_odd, phi_even;  // sqrt(1 - gamma^2)
    float amp[15];         // noise of mode k = 4..18 per unit sqrt(mu rho): phi_k / sqrt(w_k)
    float fx, fy, fz;      // uniform body force
    float scale, inv_scale;  // storage scale of FP16/BF16 deviations
    int noise_rho0;
    uint32_t key0, key1;   // Philox key (seed)
    uint32_t replica;
    uint32_t step;
    lbd::RoundKeys rk;     // Philox round keys of (key0, key1)
    unsigned int *err;     // device error word (index checks of LB_DEBUG_BOUNDS builds)
};

// Index checks of a library built with -DLB_DEBUG_BOUNDS: the element index i
// of an access to an array of n elements is tested first; outside, the error
// word gets LB_DERR_BOUNDS and the caller skips the access.  In ordinary
// builds the test is the constant true and costs nothing.
#ifdef LB_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(size_t i, size_t n, unsigned int *err)
{
    if (i < n) return true;
    if (err) atomicOr(err, LB_DERR_BOUNDS);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(size_t, size_t, unsigned int *) { return true; }
#endif

}  // namespace lbi
