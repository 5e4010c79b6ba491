// fem_energy_sums_noalloc: the FP64 energy sums of a nodal state held in
// caller-provided device memory, computed without allocating anything.
//
// It is the allocation-free variant of the library's energy reduction
// (per-CTA partial sums followed by one final CTA).  The per-CTA partials
// live in a file-scope static device array instead of memory from
// cudaMalloc; see include/fem.h for who needs this and for the limits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "fem.h"
#include "fem_device.cuh"
#include "fem_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kNodesPerCta = 8192;      // fixed: the sum order does not depend on the GPU
constexpr int64_t kMaxCtas = 16384;
constexpr int64_t kMaxNodes = kNodesPerCta * kMaxCtas;  // 134,217,728 nodes

// Scratch: one (sum E, latent) pair per CTA.  Every GPU that loads the
// library holds these 256 KiB until the process exits.  All calls share it.
static __device__ __align__(256) double g_noalloc_partials[2 * kMaxCtas];

__device__ __forceinline__ double warp_total(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// CTA b sums nodes [b*kNodesPerCta, (b+1)*kNodesPerCta) into partials[2b..2b+1]
// (every slot it owns is overwritten, so nothing needs clearing first).
template <typename real>
__global__ void __launch_bounds__(kThreads) k_noalloc_partials(
    const real *__restrict__ E, const real *__restrict__ C, const real *__restrict__ Lc,
    const uint8_t *__restrict__ ph, const real *__restrict__ ranges, int64_t n,
    double *__restrict__ partials)
{
    __shared__ double red[kThreads / 32][2];
    const int64_t i0 = (int64_t)blockIdx.x * kNodesPerCta;
    const int64_t i1 = i0 + kNodesPerCta < n ? i0 + kNodesPerCta : n;
    double u = 0.0, lat = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kThreads) {
        u += (double)E[i];
        lat += fem::latent_of(E[i], C[i], Lc[i], ph[i], ranges);
    }
    u = warp_total(u);
    lat = warp_total(lat);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[warp][0] = u; red[warp][1] = lat; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0, sl = 0.0;
        for (int w = 0; w < kThreads / 32; w++) { su += red[w][0]; sl += red[w][1]; }
        partials[2 * blockIdx.x] = su;
        partials[2 * blockIdx.x + 1] = sl;
    }
}

// One CTA: out[0..1] = sums of the n_ctas partial pairs (fixed order).
__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double *__restrict__ partials,
                                                            int64_t n_ctas, double *__restrict__ out)
{
    __shared__ double red[kThreads / 32][2];
    double u = 0.0, lat = 0.0;
    for (int64_t b = threadIdx.x; b < n_ctas; b += kThreads) {
        u += partials[2 * b];
        lat += partials[2 * b + 1];
    }
    u = warp_total(u);
    lat = warp_total(lat);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[warp][0] = u; red[warp][1] = lat; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0, sl = 0.0;
        for (int w = 0; w < kThreads / 32; w++) { su += red[w][0]; sl += red[w][1]; }
        out[0] = su;
        out[1] = sl;
    }
}

fem_status fail(fem_status st, const char *msg)
{
    fem::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" fem_status fem_energy_sums_noalloc(fem_precision prec, const void *E, const void *C,
                                              const void *Lc, const uint8_t *phase,
                                              const void *ranges, int64_t n_nodes, double *out,
                                              void *cuda_stream)
{
    char msg[256];
    if (prec != FEM_FP64 && prec != FEM_FP32) return fail(FEM_EINVAL, "unknown precision");
    if (!E || !C || !Lc || !phase || !ranges || !out)
        return fail(FEM_EINVAL, "NULL device pointer argument");
    if (n_nodes <= 0 || n_nodes > kMaxNodes) {
        snprintf(msg, sizeof msg,
                 "n_nodes = %lld is outside [1, %lld], the capacity of the static scratch",
                 (long long)n_nodes, (long long)kMaxNodes);
        return fail(FEM_EINVAL, msg);
    }
    // The scratch's device address is looked up on every call, with the
    // caller's device current: it belongs to the current context's copy of
    // the module, which a context reset (cudaDeviceReset) replaces, so an
    // address kept from an earlier call could be stale.  The lookup
    // allocates nothing.
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch failed: %s",
                 cudaGetErrorString(e));
        return fail(FEM_ECUDA, msg);
    }
    double *scratch = (double *)p;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t n_ctas = (n_nodes + kNodesPerCta - 1) / kNodesPerCta;
    if (prec == FEM_FP32)
        k_noalloc_partials<float><<<(unsigned)n_ctas, kThreads, 0, st>>>(
            (const float *)E, (const float *)C, (const float *)Lc, phase, (const float *)ranges,
            n_nodes, scratch);
    else
        k_noalloc_partials<double><<<(unsigned)n_ctas, kThreads, 0, st>>>(
            (const double *)E, (const double *)C, (const double *)Lc, phase,
            (const double *)ranges, n_nodes, scratch);
    k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, n_ctas, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "kernel launch failed: %s", cudaGetErrorString(e));
        return fail(FEM_ECUDA, msg);
    }
    fem::set_last_error("");
    return FEM_OK;
}
