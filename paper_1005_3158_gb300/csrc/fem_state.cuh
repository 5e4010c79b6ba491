// Device helpers shared by the kernel translation units of libfem (the step
// kernels in fem_kernels.cu, the state I/O and energy kernels in fem_io.cu):
// the checked build's index test, deterministic warp and block sums, the
// conversions between the stored state (E, or T in the apparent-capacity
// formulation) and T or E, and the grid size of the grid-stride kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fem_device.cuh"
#include "fem_internal.h"

// Checked build (FEM_CHECKED): every shared-memory slot, partial, mirror and
// node index is tested before use; a failure sets kErrBadIndex in the
// device error flag (reported by the next synchronising call) and skips the
// access.  The release build compiles the tests out.
#ifdef FEM_CHECKED
#define FEM_IN(i, n, err) fem::index_ok((int64_t)(i), (int64_t)(n), (err))
#else
#define FEM_IN(i, n, err) true
#endif

namespace fem {

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of K doubles per thread; result valid in thread 0.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K])
{
    __shared__ double red[NT / 32][K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; w++) s += red[w][k];
            v[k] = s;
        }
    }
}

// Node state access: the state is E (enthalpy formulation) or T
// (apparent-capacity formulation, v.is_T); these convert with the node's
// capacities and phase-change range.
template <typename real>
__device__ __forceinline__ real state_T(const StateView<real> &v, int64_t i)
{
    const real s = v.E(i);
    return v.is_T ? s : temperature_of(s, v.C[i], v.Lc[i], v.ph[i], v.ranges);
}
template <typename real>
__device__ __forceinline__ real state_E(const StateView<real> &v, int64_t i)
{
    const real s = v.E(i);
    return v.is_T ? enthalpy_of(s, v.C[i], v.Lc[i], v.ph[i], v.ranges) : s;
}
template <typename real>
__device__ __forceinline__ void state_set_T(const StateView<real> &v, int64_t i, real T)
{
    v.E(i) = v.is_T ? T : enthalpy_of(T, v.C[i], v.Lc[i], v.ph[i], v.ranges);
}
template <typename real>
__device__ __forceinline__ void state_set_E(const StateView<real> &v, int64_t i, real E)
{
    v.E(i) = v.is_T ? temperature_of(E, v.C[i], v.Lc[i], v.ph[i], v.ranges) : E;
}

#ifdef FEM_CHECKED
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int *err)
{
    const bool ok = i >= 0 && i < n;
    if (!ok && err) atomicOr(err, kErrBadIndex);
    return ok;
}
#endif

// Grid of a grid-stride kernel over n items: one thread per item, at most
// 64 CTAs per SM of a 152-SM GB300.
inline int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

}  // namespace fem
